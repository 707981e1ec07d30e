"""Failure detection at the boundary, injected on the host: a NaN in A, malformed CSR
arrays (host and device resident), and a device wait bound so short that the tensor-core
product's bounded waits run out.  No GPU is faulted: the checks reject bad input before
any product runs, and a wait that runs out makes the kernel record an error code, drain
its in-flight copies and return, after which the same handle works again."""
import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S
from workloads import planted_dense

from gpu_helpers import rel
from test_gpu_bf16 import bf16_round

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch, torch.device("cuda:0")


def test_nan_in_dense_a_is_numeric_error():
    torch, dev = _dev()
    A, _ = planted_dense(200, 4, 0.01, seed=5)
    A[17, 3] = np.nan
    A[3, 17] = np.nan
    for prec in (S.SNMF_F32, S.SNMF_BF16):
        with pytest.raises(S.SnmfError) as e:
            S.snmf_create(S.dense_matrix(torch.tensor(A, dtype=torch.float32, device=dev)), 4,
                          S.snmf_default_options(precision=prec))
        assert e.value.status == S.SNMF_ERR_NUMERIC
    with pytest.raises(S.SnmfError) as e:  # host-resident A
        S.snmf_create(S.dense_matrix(A), 4, S.snmf_default_options(precision=S.SNMF_F64))
    assert e.value.status == S.SNMF_ERR_NUMERIC


def _csr(n=50, seed=3):
    g = np.random.default_rng(seed)
    D = g.random((n, n))
    D = np.where(D > 0.8, D, 0.0)
    D = D + D.T
    rows, cols = np.nonzero(D)
    rp = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return rp, cols.astype(np.int32), D[rows, cols].astype(np.float32)


def _malformed():
    rp, ci, va = _csr()
    n = len(rp) - 1
    bad_col = ci.copy()
    bad_col[len(ci) // 2] = n            # column index out of range
    neg_col = ci.copy()
    neg_col[3] = -1
    bad_rp = rp.copy()
    bad_rp[10], bad_rp[11] = bad_rp[11], bad_rp[10] - 1   # decreasing row pointer
    short_rp = rp.copy()
    short_rp[-1] -= 1                    # rowptr[n] != nnz
    return n, va, [(rp, bad_col), (rp, neg_col), (bad_rp, ci), (short_rp, ci)]


@pytest.mark.parametrize("where", ["host", "device"])
def test_malformed_csr_is_rejected(where):
    torch, dev = _dev()
    n, va, cases = _malformed()
    for rp, ci in cases:
        if where == "host":
            m = S.csr_matrix(n, rp, ci, va)
        else:
            m = S.csr_matrix(n, torch.tensor(rp, device=dev), torch.tensor(ci, device=dev),
                             torch.tensor(va, device=dev))
        with pytest.raises(S.SnmfError) as e:
            S.snmf_create(m, 3, S.snmf_default_options())
        assert e.value.status == S.SNMF_ERR_ARG, (where, e.value)
    # a well-formed matrix passes and a malformed Laplacian is rejected the same way
    rp, ci, _ = _csr()
    keep = (torch.tensor(rp, device=dev), torch.tensor(ci, device=dev), torch.tensor(va, device=dev))
    h = S.snmf_create(S.csr_matrix(n, *keep), 3, S.snmf_default_options())
    try:
        for lrp, lci in cases:
            Lm = S.csr_matrix(n, lrp, lci, va) if where == "host" else S.csr_matrix(
                n, torch.tensor(lrp, device=dev), torch.tensor(lci, device=dev), torch.tensor(va, device=dev))
            with pytest.raises(S.SnmfError) as e:
                S.snmf_set_graph_reg(h, Lm, 0.1)
            assert e.value.status == S.SNMF_ERR_ARG
    finally:
        S.snmf_destroy(h)


def test_forced_wait_timeout_then_recovery():
    """A bound of 1 clock cycle on the device waits: the tensor-core product's waits run
    out, the call returns SNMF_ERR_TIMEOUT (a product and a solve), and after the bound is
    restored the same handle's product equals the exact emulation of the stored operands."""
    torch, dev = _dev()
    n, cols = 4096, 64
    g = np.random.default_rng(11)
    B = g.random((n, n), dtype=np.float32)
    A = (B + B.T).astype(np.float32)
    X = g.random((n, cols), dtype=np.float32)
    h = S.snmf_create(S.dense_matrix(torch.tensor(A, device=dev)), cols,
                      S.snmf_default_options(precision=S.SNMF_BF16, max_iter=3, tol=0.0))
    try:
        Xt = torch.tensor(X, device=dev)
        Yt = torch.empty_like(Xt)
        S.snmf_set_timeout(h, 1)
        with pytest.raises(S.SnmfError) as e:
            S.snmf_apply(h, Xt, Yt, cols)
        assert e.value.status == S.SNMF_ERR_TIMEOUT
        W = Xt.clone()
        H = Xt.clone()
        with pytest.raises(S.SnmfError) as e:
            S.snmf_solve(h, W, H)
        assert e.value.status == S.SNMF_ERR_TIMEOUT
        S.snmf_set_timeout(h, 0)  # the default bound again
        for _ in range(2):
            Yt.fill_(float("nan"))
            xax = S.snmf_apply(h, Xt, Yt, cols)
            At = bf16_round(A).astype(np.float64)
            Xh = bf16_round(X)
            ref = At @ (Xh.astype(np.float64) + bf16_round(X - Xh).astype(np.float64))
            Y = Yt.cpu().numpy().astype(np.float64)
            assert rel(Y, ref) <= 3e-5
            assert abs(xax - float(np.sum(X * ref))) <= 1e-5 * abs(xax)
        st, stats = S.snmf_solve(h, W.copy_(Xt), H.copy_(Xt))
        assert st in (S.SNMF_OK, S.SNMF_NOT_CONVERGED) and stats["iters"] == 3
    finally:
        S.snmf_destroy(h)
    with pytest.raises(S.SnmfError):
        S.snmf_set_timeout(None, 5)
