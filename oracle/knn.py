"""FP64 oracle of the graph pre-processing for Graph-SNMPBB and of the clustering scores.

TEST INFRASTRUCTURE ONLY.

* kNN similarity graph (Sec. 2.2 builds Graph-SNMPBB on a similarity graph of the data; the
  recipe here is the clustering workload's): the k nearest other points of each point by
  squared Euclidean distance (ties: lower index first), the self-tuning scale s_i = distance to
  the ``sigma_rank``-th neighbour, S_ij = exp(-d_ij^2 / (s_i s_j)) on the kNN pairs, symmetrised
  as max(S, S^T), degrees d_i = sum_j S_ij and A^ = D^-1/2 S D^-1/2.  Distances are evaluated
  by their definition sum_t (x_it - x_jt)^2 in FP64.
* Clustering scores of Sec. 4 (the paper reports accuracy and ARI): the contingency table of
  two labelings; the adjusted Rand index of Hubert and Arabie from that table; the accuracy
  of the best one-to-one matching of predicted to true labels (an assignment problem, solved
  by scipy's routine).
"""
from __future__ import annotations

import numpy as np


def knn_graph(X, k: int, sigma_rank: int):
    """Returns (nbr [n, k], d2 [n, k], S [n, n] symmetrised, deg [n], A_hat [n, n]); dense
    outputs, for the small test sizes."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    D2 = np.empty((n, n))
    for i in range(n):
        diff = X - X[i]
        D2[i] = np.sum(diff * diff, axis=1)
    np.fill_diagonal(D2, np.inf)
    nbr = np.argsort(D2, axis=1, kind="stable")[:, :k]
    d2 = np.take_along_axis(D2, nbr, axis=1)
    s = np.sqrt(d2[:, sigma_rank - 1])
    S = np.zeros((n, n))
    for i in range(n):
        for t in range(k):
            j = nbr[i, t]
            S[i, j] = np.exp(-d2[i, t] / (s[i] * s[j]))
    S = np.maximum(S, S.T)
    deg = S.sum(axis=1)
    inv = 1.0 / np.sqrt(deg)
    A_hat = (inv[:, None] * S) * inv[None, :]
    return nbr, d2, S, deg, A_hat


def contingency(truth, pred, k_true: int, k_pred: int) -> np.ndarray:
    """Table T[a, b] = #{i : truth_i = a, pred_i = b}."""
    T = np.zeros((k_true, k_pred), dtype=np.int64)
    np.add.at(T, (np.asarray(truth), np.asarray(pred)), 1)
    return T


def adjusted_rand_index(T) -> float:
    """Hubert-Arabie adjusted Rand index of a contingency table: (index - expected) /
    (max - expected) with index = sum_ab C(T_ab, 2), expected = sum_a C(a_a, 2) sum_b C(b_b, 2) /
    C(n, 2), max = (sum_a C(a_a, 2) + sum_b C(b_b, 2)) / 2, a and b the row and column sums."""
    T = np.asarray(T, dtype=np.float64)
    comb = lambda x: x * (x - 1.0) / 2.0  # noqa: E731
    n = T.sum()
    idx = comb(T).sum()
    sa = comb(T.sum(axis=1)).sum()
    sb = comb(T.sum(axis=0)).sum()
    exp = sa * sb / comb(n)
    mx = 0.5 * (sa + sb)
    return float((idx - exp) / (mx - exp)) if mx != exp else 1.0


def matched_accuracy(T) -> float:
    """Fraction of points whose predicted label, mapped by the best one-to-one matching of
    predicted to true labels, equals the true label."""
    from scipy.optimize import linear_sum_assignment

    T = np.asarray(T)
    r, c = linear_sum_assignment(-T)
    return float(T[r, c].sum() / T.sum())
