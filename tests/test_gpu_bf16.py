"""BF16 A on the tensor-core product: the product against an exact emulation of the
stored operands, and the reduced-precision solve against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_02887_gb300.snmf as S
from workloads import planted_dense, uniform_init

from gpu_helpers import gpu_solve, rel

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round-to-nearest-even to bfloat16 (returned as float32 values)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("n,cols", [(256, 64), (1000, 10), (700, 300), (8192, 64), (130, 16)])
def test_bf16_product_matches_emulated_operands(n, cols):
    import torch
    dev = torch.device("cuda:0")
    g = np.random.default_rng(n * 7 + cols)
    B = g.random((n, n), dtype=np.float32)
    A = (B + B.T).astype(np.float32)
    X = g.random((n, cols), dtype=np.float32)
    At = bf16_round(A).astype(np.float64)
    Xh = bf16_round(X)
    Xl = bf16_round(X.astype(np.float32) - Xh)
    ref = At @ (Xh.astype(np.float64) + Xl.astype(np.float64))
    r, b = (cols, 1) if cols <= 256 else (cols // 2, 2)   # N > 256 as two restarts
    h = S.snmf_create(S.dense_matrix(torch.tensor(A, device=dev)), r,
                      S.snmf_default_options(precision=S.SNMF_BF16, batch=b))
    try:
        Xt = torch.tensor(X, device=dev)
        Yt = torch.empty_like(Xt)
        xax = S.snmf_apply(h, Xt, Yt, cols)
    finally:
        S.snmf_destroy(h)
    Y = Yt.cpu().numpy().astype(np.float64)
    # The tensor core accumulates in FP32 without round-to-nearest, so long sums of
    # nonnegative terms drift low (measured -5.7e-6 relative at n = 8192, a uniform
    # rescaling of A rather than noise): bound by 3e-5 at these n.
    assert rel(Y, ref) <= 3e-5, rel(Y, ref)
    assert np.max(np.abs(Y - ref) / np.maximum(np.abs(ref), 1e-30)) <= 3e-5
    # the split makes the product see X to ~2^-17: error vs the unrounded X stays small
    assert rel(Y, At @ X.astype(np.float64)) <= 4e-5
    assert abs(xax - float(np.sum(X * ref))) <= 1e-5 * abs(xax)


def test_bf16_solve_reaches_oracle_residual():
    A, _ = planted_dense(500, 10, 0.01, seed=1000)
    W0 = uniform_init(500, 10, math.sqrt(A.mean() / 10), seed=1001)
    Wo, Ho, info = O.snmpbb_penalty(A, W0, W0, O.Options(max_iter=500, tol=1e-4, memory=10, objective="closed"))
    W, H, st, stats, _ = gpu_solve(A, W0, 10, W0, precision=S.SNMF_BF16, max_iter=500, tol=1e-4)
    res_true = float(np.linalg.norm(A - W @ H.T) / np.linalg.norm(A))  # against the FP64 A
    assert st == S.SNMF_OK, stats
    assert stats["pg_rel"] <= 1e-4
    assert abs(res_true - info["residual"]) <= 1e-3, (res_true, info["residual"])


def test_bf16_batched_restarts_match_single():
    """Restarts sharing A in one wide product give the same iterates as solving them
    one by one (the product columns are independent)."""
    A, _ = planted_dense(384, 8, 0.01, seed=77)
    Ws = [uniform_init(384, 8, math.sqrt(A.mean() / 8), seed=700 + j) for j in range(3)]
    Wb, Hb, _, _, _ = gpu_solve(A, np.concatenate(Ws, 1), 8, np.concatenate(Ws, 1), precision=S.SNMF_BF16,
                                batch=3, max_iter=3, tol=0.0)
    for j in range(3):
        W1, H1, _, _, _ = gpu_solve(A, Ws[j], 8, Ws[j], precision=S.SNMF_BF16, max_iter=3, tol=0.0)
        assert rel(Wb[:, 8 * j:8 * (j + 1)], W1) <= 1e-5


def test_bf16_reported_residual_is_the_stored_operators():
    """The final evaluation's closed-form residual (||A~||^2 - 2 <W, A~ Ht> + <W^T W, Ht^T Ht>)
    must equal the residual of the returned factors against the stored BF16 A~, computed
    here in FP64, to FP32 accuracy, for long K (n = 4096) and several restarts."""
    import torch
    n, r, b = 4096, 64, 4
    A, _ = planted_dense(n, r, 0.05, seed=77)
    W0 = np.concatenate([uniform_init(n, r, math.sqrt(A.mean() / r), seed=78 + j) for j in range(b)], 1)
    W, H, st, stats, per = gpu_solve(A, W0, r, W0, precision=S.SNMF_BF16, max_iter=60, tol=1e-4, batch=b)
    Ab = torch.tensor(A, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    for j in range(b):
        sl = slice(j * r, (j + 1) * r)
        res = np.linalg.norm(Ab - W[:, sl] @ H[:, sl].T) / np.linalg.norm(Ab)
        # FP32 cancellation floor: ~1e-7 ||A||^2 in res^2
        assert abs(per["residual"][j] - res) <= max(1e-5, 2e-7 / res), (j, per["residual"][j], res)
