"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package holds only input generation: graphs as symmetric CSR arrays and
personalization vectors.  It contains none of the PageRank arithmetic, and it
imports neither the oracle nor the CUDA library.
"""
from .graphs import (chung_lu, grid_deleted, star, cycle, complete, complete_bipartite,
                     path, circulant, random_small, all_graphs, from_edges, shuffled, with_self_loops, Csr)
from .vectors import uniform_p, seed_vectors, seed_dense

__all__ = ["chung_lu", "grid_deleted", "star", "cycle", "complete", "complete_bipartite",
           "path", "circulant", "random_small", "all_graphs", "from_edges", "shuffled", "with_self_loops", "Csr",
           "uniform_p", "seed_vectors", "seed_dense"]
