"""Named synthetic workloads (seeded): the shapes, sizes and value distributions of
the paper's experiments at the scale the GPU path is measured on."""
from __future__ import annotations

import math

import numpy as np

from .generators import planted_dense, uniform_init


def dense_planted_8192(r: int = 64, batch: int = 1, n: int = 8192):
    """n = 8192 planted problem: W0 ~ U[0,1]^(n x r), A = W0 W0^T + E with E symmetric
    |N(0, 0.05^2)|; starts U[0, sqrt(mean(A)/r)] per restart j (seed 3000 + r + j).
    Returns (A float64, [W_start_j])."""
    A, _ = planted_dense(n, r, 0.05, seed=2000 + r)
    upper = math.sqrt(A.mean() / r)
    starts = [uniform_init(n, r, upper, seed=3000 + r + j) for j in range(batch)]
    return A, starts


def dense_planted_500():
    """n = 500, r = 10 planted problem with |N(0, 0.01^2)| noise (the parity workload)."""
    A, _ = planted_dense(500, 10, 0.01, seed=1000)
    return A, [uniform_init(500, 10, math.sqrt(A.mean() / 10), seed=1001)]
