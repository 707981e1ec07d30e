"""Randomized eigen-sketch of the LAI approximation (oracle side).

TEST INFRASTRUCTURE ONLY.

Sec. 2.3 (Eq. (8)): for a random sketch S (n x l) take the thin QR factorization
V S = Q R and the small eigendecomposition Q^T V Q = P E P^T; then
V ~ U E U^T with U = Q P.  Readings where the paper is silent: S is standard
normal (Philox stream), ``power_iters`` subspace iterations Q <- qr(V Q) are
applied before forming Q^T V Q, the small matrix is symmetrised, and the ``k``
eigenpairs of largest |eigenvalue| are kept with their signs.
"""
from __future__ import annotations

import numpy as np

from .philox import philox_gaussian


def lai_sketch(apply_V, n: int, k: int, oversample: int, power_iters: int, seed: int):
    """Return (U, lam): U n x k with orthonormal columns, lam the k eigenvalues.

    ``apply_V(X)`` returns V @ X for an n x m array X (library matmul or a sparse
    product).  QR and the symmetric eigensolver are numpy's (library routines).
    """
    ell = k + oversample
    if ell > n:
        raise ValueError("k + oversample must not exceed n")
    S = philox_gaussian(n, ell, seed)
    Q, _ = np.linalg.qr(apply_V(S))
    for _ in range(power_iters):
        Q, _ = np.linalg.qr(apply_V(Q))
    T = Q.T @ apply_V(Q)
    T = 0.5 * (T + T.T)
    lam, P = np.linalg.eigh(T)
    order = np.argsort(-np.abs(lam), kind="stable")[:k]
    return Q @ P[:, order], lam[order]
