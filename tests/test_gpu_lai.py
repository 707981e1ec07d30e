"""LAI-SNMPBB (Sec. 2.3) on the GPU against the oracle's own sketch (same Philox
Gaussian stream): the sketched operator U E U^T, and the solve on it."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_02887_gb300.snmf as S
from workloads import chung_lu_csr, planted_dense, uniform_init

from gpu_helpers import gpu_solve, rel

pytestmark = pytest.mark.gpu


def _apply_lai(h, X, dev, torch, dtype):
    Xt = torch.tensor(X, dtype=dtype, device=dev)
    Yt = torch.empty_like(Xt)
    xax = S.snmf_apply(h, Xt, Yt, X.shape[1])
    return Yt.cpu().numpy().astype(np.float64), xax


def test_lai_operator_matches_oracle_fp64():
    import torch
    dev = torch.device("cuda:0")
    n, rank = 600, 10
    A, _ = planted_dense(n, rank, 0.01, seed=4101)  # rank-10 signal + small noise: clear gap after 10
    k, p, q, seed = 10, 6, 2, 4102
    Uo, lo = O.lai_sketch(lambda X: A @ X, n, k, p, q, seed)
    op = O.LaiOperator(Uo, lo)
    X = uniform_init(n, k, 1.0, 4103)
    h = S.snmf_create(S.dense_matrix(torch.tensor(A, device=dev)), k, S.snmf_default_options(precision=S.SNMF_F64))
    try:
        S.snmf_lai_sketch(h, k, p, q, seed)
        Y, xax = _apply_lai(h, X, dev, torch, torch.float64)
    finally:
        S.snmf_destroy(h)
    ref = O.apply_A(op, X)
    assert rel(Y, ref) <= 1e-9, rel(Y, ref)
    assert abs(xax - float(np.sum(X * ref))) <= 1e-9 * abs(xax)
    # and the sketch reproduces A on its dominant subspace
    assert rel(Y, A @ X) <= 0.02


def test_lai_penalty_solve_matches_oracle_fp64():
    n, r = 500, 8
    A, _ = planted_dense(n, r, 0.01, seed=4201)
    k, p, q, seed = 8, 6, 2, 4202
    Uo, lo = O.lai_sketch(lambda X: A @ X, n, k, p, q, seed)
    W0 = uniform_init(n, r, math.sqrt(A.mean() / r), 4203)
    opts = O.Options(max_iter=6, tol=0.0, memory=10, objective="closed", lambda_sym=0.01 * np.linalg.norm(A))
    Wo, Ho, _ = O.snmpbb_penalty(O.LaiOperator(Uo, lo), W0, W0, opts)
    W, H, _, _, _ = gpu_solve(A, W0, r, W0, lai=(k, p, q, seed), max_iter=6, tol=0.0)
    # the sketch reproduces the oracle's operator to about 2e-14 (CholeskyQR and the Jacobi
    # eigensolver against numpy's); the iterates measure <= 6e-13 over these 6 iterations, and
    # the oracle moves its W by the size of a perturbation of U (1e-12 -> 1.1e-12 after 6)
    assert rel(W, Wo) <= 1e-11 and rel(H, Ho) <= 1e-11, (rel(W, Wo), rel(H, Ho))


def test_lai_sketch_csr_fp32_power_law():
    import scipy.sparse as sp
    import torch
    dev = torch.device("cuda:0")
    G = chung_lu_csr(n=20000, mean_degree=16, seed=4301)
    Asp = sp.csr_matrix((G.values, G.colidx, G.rowptr), shape=(G.n, G.n))
    k, p, q, seed = 16, 8, 2, 4302
    Uo, lo = O.lai_sketch(lambda X: Asp @ X, G.n, k, p, q, seed)
    X = uniform_init(G.n, 4, 1.0, 4303)
    rp = torch.tensor(G.rowptr, device=dev)
    ci = torch.tensor(G.colidx, device=dev)
    va = torch.tensor(G.values, dtype=torch.float32, device=dev)
    h = S.snmf_create(S.csr_matrix(G.n, rp, ci, va), 4, S.snmf_default_options(precision=S.SNMF_F32))
    try:
        S.snmf_lai_sketch(h, k, p, q, seed)
        Y, _ = _apply_lai(h, X, dev, torch, torch.float32)
    finally:
        S.snmf_destroy(h)
    ref = O.apply_A(O.LaiOperator(Uo, lo), X)
    assert rel(Y, ref) <= 2e-3, rel(Y, ref)


def test_lai_rejects_bad_sizes():
    import torch
    dev = torch.device("cuda:0")
    A = torch.eye(50, dtype=torch.float64, device=dev)
    h = S.snmf_create(S.dense_matrix(A), 2, S.snmf_default_options(precision=S.SNMF_F64))
    try:
        with pytest.raises(S.SnmfError):
            S.snmf_lai_sketch(h, 40, 20, 1, 1)   # k + p > n
        with pytest.raises(S.SnmfError):
            S.snmf_lai_sketch(h, 0, 4, 1, 1)
    finally:
        S.snmf_destroy(h)


def test_svd_start_matches_oracle_fp64():
    """SVD start (Sec. 4.1 guideline (4)) from the device eigen-sketch: on a planted A with a
    wide spectral gap after r (noise 1e-3) two power iterations make the sketch's top-r
    eigenvectors exact to rounding, so W_0 = |U E^1/2| equals oracle.svd_init (numpy's SVD); on
    a noisier A it equals |U| |lambda|^1/2 of the oracle's own sketch (same Philox stream);
    W_0 = Ht_0 in every restart's columns; a solve from it converges."""
    import torch
    dev = torch.device("cuda:0")
    n, r, b = 300, 5, 2
    A_exact, _ = planted_dense(n, r, 1e-3, seed=4301)
    W_ref, H_ref = O.svd_init(A_exact, r)
    assert np.allclose(W_ref, H_ref, atol=1e-10)
    A_noisy, _ = planted_dense(n, r, 0.05, seed=4302)
    Uo, lo = O.lai_sketch(lambda X: A_noisy @ X, n, r, 6, 2, 4303)
    W_sk = np.abs(Uo) * np.sqrt(np.abs(lo))[None, :]
    for A, ref, seed, tol in ((A_exact, W_ref, 4304, 1e-8), (A_noisy, W_sk, 4303, 1e-9)):
        h = S.snmf_create(S.dense_matrix(torch.tensor(A, device=dev)), r,
                          S.snmf_default_options(precision=S.SNMF_F64, batch=b, max_iter=500, tol=1e-4))
        try:
            W = torch.zeros((n, r * b), dtype=torch.float64, device=dev)
            H = torch.zeros_like(W)
            S.snmf_svd_init(h, W, H, oversample=6, power_iters=2, seed=seed)
            Wn = W.cpu().numpy()
            assert np.array_equal(Wn, H.cpu().numpy())
            for j in range(b):
                assert rel(Wn[:, j * r:(j + 1) * r], ref) <= tol, (j, rel(Wn[:, j * r:(j + 1) * r], ref))
            st, stats = S.snmf_solve(h, W, H)
            assert st == S.SNMF_OK and stats["pg_rel"] <= 1e-4
        finally:
            S.snmf_destroy(h)
