"""The allocation-free product entry point against the handle-based one.

Some callers cannot call cudaMalloc after start-up (they reserve all memory once,
or their memory belongs to another allocator); snmf_apply_dense_noalloc serves
them from a fixed device array.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S

pytestmark = pytest.mark.gpu


def _handle_product(A, X):
    import torch
    h = S.snmf_create(S.dense_matrix(A), X.shape[1], S.snmf_default_options(
        precision=S.SNMF_F64 if A.dtype == torch.float64 else S.SNMF_F32))
    try:
        Y = torch.empty_like(X)
        xax = S.snmf_apply(h, X, Y, X.shape[1])
    finally:
        S.snmf_destroy(h)
    return Y, xax


@pytest.mark.parametrize("dtype,n,cols,tol", [("float64", 1000, 24, 1e-13), ("float32", 2048, 64, 1e-6),
                                              ("float32", 333, 5, 1e-6)])
def test_noalloc_matches_handle_product_twice(dtype, n, cols, tol):
    import torch
    dev = torch.device("cuda:0")
    g = np.random.default_rng(n + cols)
    B = g.random((n, n))
    tdt = getattr(torch, dtype)
    A = torch.tensor(B + B.T, dtype=tdt, device=dev)
    X = torch.tensor(g.random((n, cols)), dtype=tdt, device=dev)
    Yref, xref = _handle_product(A, X)
    outs = []
    for _ in range(2):  # two calls in a row share the scratch array
        Y = torch.full_like(X, float("nan"))
        xax = S.snmf_apply_dense_noalloc(A, X, Y)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(Y - Yref) / torch.linalg.norm(Yref))
        assert err <= tol, err
        assert abs(xax - xref) <= tol * abs(xref)
        outs.append(Y.clone())
    assert torch.equal(outs[0], outs[1])


def test_noalloc_rejects_oversize():
    import torch
    dev = torch.device("cuda:0")
    n = 16384
    cols = S.NOALLOC_MAX_SLICE_PAIR_BYTES // (2 * n * 4) + 1
    A = torch.zeros((8, 8), dtype=torch.float32, device=dev)
    A_big = torch.empty((n, n), dtype=torch.float32, device=dev)
    X = torch.zeros((n, cols), dtype=torch.float32, device=dev)
    with pytest.raises(S.SnmfError):
        S.snmf_apply_dense_noalloc(A_big, X, torch.empty_like(X))
    with pytest.raises(S.SnmfError):  # lda < n
        S.snmf_apply_dense_noalloc(A[:, :4].contiguous(), X[:8], torch.empty_like(X[:8]))
