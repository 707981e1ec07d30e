"""Seeded input generators.

Every generator takes an integer seed and returns numpy arrays (float64 unless
stated).  The recipes follow the synthetic workloads used to exercise symmetric
NMF: planted dense factorizations (the synthetic experiment of the paper's
Sec. 4.2, with added symmetric noise), a k-nearest-neighbour similarity graph of a
Gaussian mixture (the graph-clustering pre-processing of Sec. 2.2 and Sec. 4.1),
a Chung-Lu power-law graph (a stand-in for large sparse symmetric matrices) and a
batch of uneven planted problems.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Csr:
    """Compressed sparse row matrix (int32 row pointers / column indices)."""

    n: int
    rowptr: np.ndarray  # int32, n+1
    colidx: np.ndarray  # int32, nnz
    values: np.ndarray  # float64 or float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        out[rows, self.colidx] = self.values
        return out


def _sym_abs_normal(n: int, sigma: float, g: np.random.Generator) -> np.ndarray:
    """Symmetric matrix with iid |N(0, sigma^2)| entries on and above the diagonal."""
    U = np.abs(g.normal(0.0, sigma, size=(n, n)))
    E = np.triu(U)
    return E + np.triu(E, 1).T


def planted_dense(n: int, r: int, sigma: float = 0.01, seed: int = 0,
                  rel_noise: float | None = None):
    """A = W0 W0^T + E with W0 ~ U[0,1]^(n x r) and E symmetric |N(0, sigma^2)|.

    With ``rel_noise`` set, E is rescaled so that ||E||_F = rel_noise * ||W0 W0^T||_F.
    Returns (A, W0), both float64.
    """
    g = np.random.default_rng(seed)
    W0 = g.random((n, r))
    P = W0 @ W0.T
    E = _sym_abs_normal(n, 1.0 if rel_noise is not None else sigma, g)
    if rel_noise is not None:
        E *= rel_noise * np.linalg.norm(P) / max(np.linalg.norm(E), 1e-300)
    A = P + E
    return A, W0


def uniform_init(n: int, cols: int, upper: float, seed: int) -> np.ndarray:
    """Initial factor with iid U[0, upper] entries (n x cols, float64)."""
    g = np.random.default_rng(seed)
    return g.random((n, cols)) * upper


def gmm_points(n: int, d: int, comps: int, seed: int):
    """The Gaussian-mixture points of gmm_knn_graph (same seeded draws): ``comps`` equally
    weighted components in R^d, means ~ N(0, 4 I), unit covariance.  Returns (X float32 n x d,
    labels)."""
    g = np.random.default_rng(seed)
    labels = g.integers(0, comps, size=n)
    means = g.normal(0.0, 2.0, size=(comps, d))
    X = (means[labels] + g.normal(size=(n, d))).astype(np.float32)
    return X, labels


def gmm_knn_graph(n: int = 20000, d: int = 64, comps: int = 20, k: int = 10,
                  sigma_rank: int = 7, seed: int = 3000, chunk: int = 2048):
    """k-nearest-neighbour Gaussian similarity graph of a Gaussian mixture.

    Points: ``comps`` equally weighted components in R^d, means ~ N(0, 4 I), unit
    covariance.  For each point the k nearest other points are kept; the
    similarity is S_ij = exp(-d_ij^2 / (s_i s_j)) with s_i the distance to the
    ``sigma_rank``-th neighbour (self-tuning scale); S is symmetrised as
    max(S, S^T).  Returns (A_hat, L, labels, S) where A_hat = D^-1/2 S D^-1/2 and
    L = D - S as Csr matrices (D = diag of row sums of S).
    """
    g = np.random.default_rng(seed)
    labels = g.integers(0, comps, size=n)
    means = g.normal(0.0, 2.0, size=(comps, d))
    X = (means[labels] + g.normal(size=(n, d))).astype(np.float32)
    sq = np.einsum("ij,ij->i", X, X)
    nbr = np.empty((n, k), dtype=np.int64)
    nd2 = np.empty((n, k), dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d2 = sq[s:e, None] + sq[None, :] - 2.0 * (X[s:e] @ X.T)
        d2[np.arange(e - s), np.arange(s, e)] = np.inf  # exclude self
        part = np.argpartition(d2, k, axis=1)[:, :k]
        pd = np.take_along_axis(d2, part, axis=1)
        order = np.argsort(pd, axis=1, kind="stable")
        nbr[s:e] = np.take_along_axis(part, order, axis=1)
        nd2[s:e] = np.maximum(np.take_along_axis(pd, order, axis=1), 0.0)
    scale = np.sqrt(nd2[:, sigma_rank - 1])
    rows = np.repeat(np.arange(n), k)
    cols = nbr.ravel()
    vals = np.exp(-nd2.ravel() / (scale[rows] * scale[cols]))
    # symmetrise with max(S, S^T): take the max over duplicate (i,j) in the union
    r2 = np.concatenate([rows, cols])
    c2 = np.concatenate([cols, rows])
    v2 = np.concatenate([vals, vals])
    key = r2 * n + c2
    order = np.lexsort((-v2, key))
    key, v2 = key[order], v2[order]
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key, v2 = key[first], v2[first]
    rr, cc = key // n, key % n
    deg = np.bincount(rr, weights=v2, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rr, minlength=n), out=rowptr[1:])
    dis = 1.0 / np.sqrt(deg)
    S = Csr(n, rowptr.astype(np.int32), cc.astype(np.int32), v2)
    A_hat = Csr(n, S.rowptr, S.colidx, v2 * dis[rr] * dis[cc])
    # L = D - S, diagonal inserted in column order
    lr = np.concatenate([rr, np.arange(n)])
    lc = np.concatenate([cc, np.arange(n)])
    lv = np.concatenate([-v2, deg])
    o = np.lexsort((lc, lr))
    lr, lc, lv = lr[o], lc[o], lv[o]
    lptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(lr, minlength=n), out=lptr[1:])
    L = Csr(n, lptr.astype(np.int32), lc.astype(np.int32), lv)
    return A_hat, L, labels, S


def chung_lu_csr(n: int = 2_000_000, exponent: float = 2.1, mean_degree: float = 16.0,
                 seed: int = 4000) -> Csr:
    """Symmetric Chung-Lu power-law graph with U(0,1] edge weights.

    Expected degrees w_i proportional to (i + i0)^(-1/(exponent-1)), scaled to the
    requested mean degree, with i0 chosen so that the largest expected degree is
    sqrt(sum w) (every pair probability w_i w_j / sum w then stays <= 1).  Edges are
    drawn as sum(w)/2 independent endpoint pairs, each endpoint chosen with
    probability proportional to w; self loops and repeated pairs are dropped (the
    usual fast approximation of Chung-Lu sampling).  Both triangles are stored.
    """
    g = np.random.default_rng(seed)
    a = 1.0 / (exponent - 1.0)
    total = mean_degree * n
    wmax = np.sqrt(total)
    # choose i0 with wmax / mean = (i0)^-a / mean_{i}((i+i0)^-a) by bisection on log i0
    idx = np.arange(n, dtype=np.float64)

    def ratio(i0):
        w = (idx + i0) ** (-a)
        return (w[0] / w.mean()) * mean_degree

    lo, hi = 1e-3, float(n)
    for _ in range(60):
        mid = np.sqrt(lo * hi)
        if ratio(mid) > wmax:
            lo = mid
        else:
            hi = mid
    w = (idx + hi) ** (-a)
    w *= total / w.sum()
    m = int(total / 2)
    p = w / w.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    i = np.searchsorted(cdf, g.random(m), side="right").astype(np.int64)
    j = np.searchsorted(cdf, g.random(m), side="right").astype(np.int64)
    np.minimum(i, n - 1, out=i)
    np.minimum(j, n - 1, out=j)
    keep = i != j
    i, j = i[keep], j[keep]
    lo_, hi_ = np.minimum(i, j), np.maximum(i, j)
    key = np.unique(lo_ * n + hi_)
    lo_, hi_ = key // n, key % n
    vals = 1.0 - g.random(len(key))  # U(0,1]
    rr = np.concatenate([lo_, hi_])
    cc = np.concatenate([hi_, lo_])
    vv = np.concatenate([vals, vals])
    o = np.lexsort((cc, rr))
    rr, cc, vv = rr[o], cc[o], vv[o]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rr, minlength=n), out=rowptr[1:])
    return Csr(n, rowptr.astype(np.int32), cc.astype(np.int32), vv)


def uneven_batch(count: int = 256, n_range=(64, 2048), r_range=(4, 32),
                 rel_noise: float = 0.01, seed: int = 5000):
    """A batch of independent planted problems of uneven size.

    Problem p uses seed ``seed + p``: n ~ U{n_range}, r ~ U{r_range},
    A = W0 W0^T + E with ||E||_F = rel_noise ||W0 W0^T||_F.
    Returns a list of (A, W0, r).
    """
    g = np.random.default_rng(seed)
    ns = g.integers(n_range[0], n_range[1] + 1, size=count)
    rs = g.integers(r_range[0], r_range[1] + 1, size=count)
    out = []
    for p in range(count):
        A, W0 = planted_dense(int(ns[p]), int(rs[p]), seed=seed + 1 + p, rel_noise=rel_noise)
        out.append((A, W0, int(rs[p])))
    return out
