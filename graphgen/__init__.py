"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA tests/benchmarks.

This package generates inputs only and holds none of the method's arithmetic:
  * R-MAT power-law graphs (symmetrised, self-loops and duplicates removed, 0/1 pattern,
    int32 column indices) -- the stand-in for the paper's graph datasets (Section 4,
    Table "graphs"), which are not available;
  * graphs with closed-form spectra (cycle, complete, star, hypercube, disjoint unions);
  * directed graphs (directed R-MAT and families with closed-form singular values) for the
    SVD path;
  * seeded N(0, 1) and U[0, 1) dense blocks.
"""
from .graphs import (CSR, rmat, cycle, complete, star, hypercube, path, erdos_renyi,
                     disjoint_union, from_edges, normal_block, uniform_block, build, directed_cycle, out_star,
                     transitive_tournament, complete_bipartite_directed)

__all__ = ["CSR", "rmat", "cycle", "complete", "star", "hypercube", "path", "erdos_renyi",
           "disjoint_union", "from_edges", "normal_block", "uniform_block", "build", "directed_cycle", "out_star",
           "transitive_tournament", "complete_bipartite_directed"]
