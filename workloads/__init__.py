"""Seeded synthetic inputs shaped like the paper's workloads.

This package draws random numbers and assembles input matrices. It holds none of
the factorization method's arithmetic (no objective, gradient, step or line
search), so both the CPU oracle's tests and the CUDA path may use it.
"""
from .generators import (  # noqa: F401
    planted_dense,
    uniform_init,
    gmm_knn_graph,
    gmm_points,
    chung_lu_csr,
    uneven_batch,
    Csr,
)
