"""Plain FP64 CPU oracle for CPAA PageRank (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import anything from this package.  It shares no code with the CUDA library
in ``paper_2112_01743_gb300`` and never imports it; the GPU path never imports
this package.
"""
