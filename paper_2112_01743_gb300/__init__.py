"""GB300 (sm_103a) CPAA PageRank: CUDA kernels behind a C ABI (include/cpaa.h)
and a thin ctypes binding with the same names.

The binding does argument marshalling only; every step of the method runs in
the library's kernels.  Importing the binding fails loudly when libcpaa.so has
not been built (``__graft_entry__.build()`` or ``python -m
paper_2112_01743_gb300.build``).
"""
from .cpaa import *  # noqa: F401,F403
from .cpaa import __all__  # noqa: F401
