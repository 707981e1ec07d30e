"""Uneven batch (SNMF_DENSE_BATCH) through the C ABI: each problem of a batch against the
FP64 oracle run on that problem alone."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_02887_gb300.snmf as S
from workloads import planted_dense, uniform_init

from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def make_problems(specs, noise=0.01):
    """specs: (n, r, seed) -> lists of A_p and W0_p (planted, init U[0, sqrt(mean A / r)])."""
    As, Ws = [], []
    for n, r, s in specs:
        A, _ = planted_dense(n, r, noise, seed=s)
        As.append(A)
        Ws.append(uniform_init(n, r, math.sqrt(A.mean() / r), seed=s + 1))
    return As, Ws


def batch_solve(As, Ws, precision, weights=None, **opt):
    import torch
    dev = torch.device("cuda:0")
    tdt = torch.float64 if precision == S.SNMF_F64 else torch.float32
    ns = [a.shape[0] for a in As]
    rs = [w.shape[1] for w in Ws]
    vals = torch.tensor(np.concatenate([a.ravel() for a in As]), dtype=tdt, device=dev)
    W = torch.tensor(np.concatenate([w.ravel() for w in Ws]), dtype=tdt, device=dev)
    H = W.clone()
    o = S.snmf_default_options(precision=precision, **opt)
    h = S.snmf_create(S.dense_batch_matrix(vals, ns, rs), 0, o, mlp_weights=weights)
    try:
        st, stats = S.snmf_solve(h, W, H)
        per = S.snmf_restart_stats(h, len(As))
    finally:
        S.snmf_destroy(h)
    Wn, Hn = W.cpu().numpy().astype(np.float64), H.cpu().numpy().astype(np.float64)
    out_W, out_H, off = [], [], 0
    for n, r in zip(ns, rs):
        out_W.append(Wn[off:off + n * r].reshape(n, r))
        out_H.append(Hn[off:off + n * r].reshape(n, r))
        off += n * r
    return out_W, out_H, st, stats, per


SPECS = [(37, 3, 11), (130, 7, 13), (64, 5, 15), (257, 12, 17), (3, 1, 19), (200, 64, 21), (97, 1, 23)]


def test_batch_fp64_matches_oracle_per_problem():
    """Ragged row tiles and Gram chunks (n = 37, 130, 257), n = 3 with r = 1, r = 64; the
    problems' items are interleaved in one launch per step."""
    As, Ws = make_problems(SPECS)
    for iters in (1, 8):
        W, H, _, stats, per = batch_solve(As, Ws, S.SNMF_F64, max_iter=iters, tol=0.0)
        for p, (A, W0) in enumerate(zip(As, Ws)):
            Wo, Ho, _ = O.snmpbb_penalty(A, W0, W0, O.Options(max_iter=iters, tol=0.0, memory=10, objective="closed"))
            e = max(rel(W[p], Wo), rel(H[p], Ho))
            assert e <= 1e-10, (iters, p, e)
            assert per["iters"][p] == iters


def test_batch_fp32_converges_like_oracle():
    g = np.random.default_rng(5)
    specs = [(int(g.integers(64, 600)), int(g.integers(4, 33)), 300 + 2 * p) for p in range(8)]
    As, Ws = make_problems(specs)
    W, H, st, stats, per = batch_solve(As, Ws, S.SNMF_F32, max_iter=3000, tol=1e-4)
    assert st == S.SNMF_OK, stats
    for p, (A, W0) in enumerate(zip(As, Ws)):
        _, _, info = O.snmpbb_penalty(A, W0, W0, O.Options(max_iter=3000, tol=1e-4, memory=10))
        assert per["pg_rel"][p] <= 1e-4
        assert abs(per["residual"][p] - info["residual"]) <= 1e-3, (p, per["residual"][p], info["residual"])
        # the reported residual is the true one of the returned factors, up to the FP32
        # cancellation of ||A||^2 - 2 <W, A Ht> + <W^T W, Ht^T Ht>: an error of ~1e-7 ||A||^2
        # in the sum moves the residual by ~1e-7 / (2 res)
        res = np.linalg.norm(A - W[p] @ H[p].T) / np.linalg.norm(A)
        assert abs(res - per["residual"][p]) <= max(1e-5, 2e-7 / res), (p, res, per["residual"][p])


def test_batch_bf16_reaches_oracle_residual():
    g = np.random.default_rng(6)
    specs = [(int(g.integers(128, 700)), int(g.integers(4, 33)), 500 + 2 * p) for p in range(6)]
    As, Ws = make_problems(specs)
    W, H, st, stats, per = batch_solve(As, Ws, S.SNMF_BF16, max_iter=3000, tol=1e-4)
    for p, (A, W0) in enumerate(zip(As, Ws)):
        _, _, info = O.snmpbb_penalty(A, W0, W0, O.Options(max_iter=3000, tol=1e-4, memory=10))
        res = np.linalg.norm(A - W[p] @ H[p].T) / np.linalg.norm(A)  # against the true A
        assert per["pg_rel"][p] <= 1e-4
        assert abs(res - info["residual"]) <= 1e-3, (p, res, info["residual"])


def test_batch_zero_iterations_and_zero_weight_controller():
    As, Ws = make_problems(SPECS[:4])
    W, H, _, _, per = batch_solve(As, Ws, S.SNMF_F64, max_iter=0, tol=0.0)
    for p in range(4):
        assert np.array_equal(W[p], Ws[p]) and np.array_equal(H[p], Ws[p])
    Wp, Hp, _, _, _ = batch_solve(As, Ws, S.SNMF_F32, max_iter=12, tol=0.0)
    Wl, Hl, _, sl, _ = batch_solve(As, Ws, S.SNMF_F32, max_iter=12, tol=0.0, step_controller=1,
                                   weights=np.zeros(S.SNMF_MLP_NPARAMS, np.float32))
    for p in range(4):
        assert np.array_equal(Wp[p], Wl[p]) and np.array_equal(Hp[p], Hl[p])
    assert sl["ctl_proposals"] > 0


def test_batch_bf16_product_through_final_evaluation():
    """max_iter = 0: the final evaluation's residual comes from the grouped tensor-core
    product <W, A~ Ht> (A~ = BF16(A)); it must equal the residual computed in FP64 from the
    BF16-rounded A for every problem size class (ragged 128-row tiles, r = 1..64)."""
    import torch
    As, Ws = make_problems(SPECS + [(1000, 33, 31), (129, 16, 33)])
    W, H, _, _, per = batch_solve(As, Ws, S.SNMF_BF16, max_iter=0, tol=0.0)
    for p, (A, W0) in enumerate(zip(As, Ws)):
        Ab = torch.tensor(A, dtype=torch.float32).to(torch.bfloat16).double().numpy()
        W32 = W0.astype(np.float32).astype(np.float64)
        res = np.linalg.norm(Ab - W32 @ W32.T) / np.linalg.norm(Ab)
        assert abs(per["residual"][p] - res) <= 1e-5 * max(1.0, res), (p, per["residual"][p], res)
