"""GPU kNN similarity graph, cluster assignment and clustering scores against the FP64 oracle
(oracle/knn.py), through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S
from oracle import knn as OK
from workloads import gmm_points

pytestmark = pytest.mark.gpu


def _clean_rows(X, k, rel_gap=1e-5):
    """Rows whose k-th and (k+1)-th nearest distances are apart by more than rel_gap (an FP32
    evaluation cannot reorder their neighbour sets)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    clean = np.ones(n, dtype=bool)
    for i in range(n):
        d = np.sum((X - X[i]) ** 2, axis=1)
        d[i] = np.inf
        p = np.sort(d)[: k + 1]
        clean[i] = (p[k] - p[k - 1]) > rel_gap * p[k]
    return clean


def _dense_from_csr(rp, ci, v, n):
    M = np.zeros((n, n))
    for i in range(n):
        M[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return M


@pytest.mark.parametrize("n,d,comps,k,sr", [(700, 16, 5, 10, 7), (257, 3, 4, 32, 32), (130, 40, 3, 1, 1)])
def test_knn_graph_vs_oracle(n, d, comps, k, sr):
    import torch
    X, _ = gmm_points(n, d, comps, seed=41 + n)
    Xd = torch.tensor(X, device="cuda:0")
    rp, ci, ah, sv, dg = S.snmf_knn_graph(Xd, k=k, sigma_rank=sr)
    torch.cuda.synchronize()
    rp, ci, ah, sv, dg = (t.cpu().numpy() for t in (rp, ci, ah, sv, dg))
    # CSR well-formed: columns strictly ascending per row, no self loops
    assert rp[0] == 0 and np.all(np.diff(rp) >= k)
    for i in range(n):
        c = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and not np.any(c == i)
    _, _, So, do, Ao = OK.knn_graph(X.astype(np.float64), k, sr)
    Sg = _dense_from_csr(rp, ci, sv, n)
    Ag = _dense_from_csr(rp, ci, ah, n)
    # symmetric pattern and values (max(S, S^T) is symmetric bit for bit)
    assert np.array_equal(Sg, Sg.T)
    clean = _clean_rows(X, k)
    pat_g, pat_o = Sg > 0, So > 0
    bad = np.argwhere(pat_g != pat_o)
    for i, j in bad:
        assert not (clean[i] and clean[j]), f"pattern differs at ({i}, {j}) between two clean rows"
    both = clean[:, None] & clean[None, :]
    # FP32 distances and exp: |dS| <= 1e-5 on entries of clean rows; degrees relative 1e-5
    assert np.max(np.abs(Sg - So)[both]) < 1e-5
    union = pat_g | pat_o
    rows = clean & np.array([bool(np.all(clean[union[i]])) for i in range(n)])
    assert rows.sum() > 0.5 * n
    np.testing.assert_allclose(dg[rows], do[rows], rtol=1e-5)
    assert np.max(np.abs(Ag - Ao)[rows][:, rows]) < 1e-5


def test_knn_graph_rejects_bad_arguments():
    import torch
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda:0")
    for k, sr in [(0, 1), (10, 1), (33, 1), (3, 4), (3, 0)]:
        with pytest.raises(S.SnmfError):
            S.snmf_knn_graph(X, k=k, sigma_rank=sr)


def test_cluster_scores_vs_oracle():
    import torch
    g = np.random.default_rng(5)
    n, kt, kp = 5001, 7, 9
    truth = g.integers(0, kt, size=n).astype(np.int32)
    pred = np.where(g.random(n) < 0.7, truth, g.integers(0, kp, size=n)).astype(np.int32)
    T, ari, acc = S.snmf_cluster_scores(torch.tensor(truth, device="cuda:0"), torch.tensor(pred, device="cuda:0"),
                                        kt, kp)
    To = OK.contingency(truth, pred, kt, kp)
    assert np.array_equal(T, To)
    assert abs(ari - OK.adjusted_rand_index(To)) < 1e-12
    assert abs(acc - OK.matched_accuracy(To)) < 1e-12
    bad = torch.tensor(np.append(pred[:-1], kp).astype(np.int32), device="cuda:0")
    with pytest.raises(S.SnmfError):
        S.snmf_cluster_scores(torch.tensor(truth, device="cuda:0"), bad, kt, kp)


@pytest.mark.parametrize("kt,kp", [(1, 1), (3, 5), (6, 2), (20, 20)])
def test_matching_accuracy_shapes(kt, kp):
    import torch
    g = np.random.default_rng(kt * 31 + kp)
    n = 999
    truth = g.integers(0, kt, size=n).astype(np.int32)
    pred = g.integers(0, kp, size=n).astype(np.int32)
    T, ari, acc = S.snmf_cluster_scores(torch.tensor(truth, device="cuda:0"), torch.tensor(pred, device="cuda:0"),
                                        kt, kp)
    To = OK.contingency(truth, pred, kt, kp)
    assert abs(acc - OK.matched_accuracy(To)) < 1e-12
    assert abs(ari - OK.adjusted_rand_index(To)) < 1e-12


def test_graph_clustering_end_to_end():
    """kNN graph of a Gaussian mixture on the GPU, SymNMF of A^ with the paper's graph term,
    labels by argmax of H, scores on the GPU: the scores equal the oracle's scores of the same
    labels, and the clusters are recovered."""
    import torch
    n, d, comps = 1500, 32, 5
    X, labels = gmm_points(n, d, comps, seed=77)
    Xd = torch.tensor(X, device="cuda:0")
    rp, ci, ah, _, _ = S.snmf_knn_graph(Xd, k=10, sigma_rank=7)
    o = S.snmf_default_options(precision=S.SNMF_F32, batch=4, max_iter=400, seed=3)
    h = S.snmf_create(S.csr_matrix(n, rp, ci, ah), comps, o)
    try:
        S.snmf_set_graph_reg(h, None, 0.1)
        st, _ = S.snmf_solve(h)
        per = S.snmf_restart_stats(h, o.batch)
        best = int(np.argmin(per["residual"]))
        lab = S.snmf_cluster_assign(h, best, n)
        torch.cuda.synchronize()
        with pytest.raises(S.SnmfError):
            S.snmf_cluster_assign(h, o.batch, n)
    finally:
        S.snmf_destroy(h)
    truth = torch.tensor(labels.astype(np.int32), device="cuda:0")
    T, ari, acc = S.snmf_cluster_scores(truth, lab, comps, comps)
    To = OK.contingency(labels, lab.cpu().numpy(), comps, comps)
    assert np.array_equal(T, To)
    assert abs(ari - OK.adjusted_rand_index(To)) < 1e-12
    assert abs(acc - OK.matched_accuracy(To)) < 1e-12
    assert acc > 0.9 and ari > 0.8


def test_knn_graph_rejects_duplicate_points_and_nan():
    import torch
    X, _ = gmm_points(64, 4, 2, seed=9)
    Xd = torch.tensor(np.repeat(X[:8], 8, axis=0), device="cuda:0")  # 8 copies of each point
    with pytest.raises(S.SnmfError):
        S.snmf_knn_graph(Xd, k=10, sigma_rank=7)  # s_i = 0
    Xn = X.copy()
    Xn[5, 2] = np.nan
    with pytest.raises(S.SnmfError):
        S.snmf_knn_graph(torch.tensor(Xn, device="cuda:0"), k=10, sigma_rank=7)
