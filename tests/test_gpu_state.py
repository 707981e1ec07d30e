"""Checkpoint and exact restart (snmf_get_state / snmf_set_state) and the per-iteration
statistics ring: a solve of k outer iterations, exported and resumed for m more, reproduces a
solve of k + m iterations bit for bit (the penalty blocks restart their BB memory and
nonmonotone reference at every block, so the exported scalars are the whole state)."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_02887_gb300.snmf as S
from workloads import planted_dense, uniform_init

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,form", [(S.SNMF_F64, S.SNMF_PENALTY), (S.SNMF_F32, S.SNMF_PENALTY),
                                       (S.SNMF_F64, S.SNMF_NAIVE)])
def test_resume_reproduces_the_continuous_solve(prec, form):
    import torch
    dev = torch.device("cuda:0")
    n, r, b, k, m = 500, 10, 2, 7, 5
    A, _ = planted_dense(n, r, 0.01, seed=1000)
    W0 = np.concatenate([uniform_init(n, r, math.sqrt(A.mean() / r), seed=1001 + j) for j in range(b)], 1)
    tdt = torch.float64 if prec == S.SNMF_F64 else torch.float32
    At = torch.tensor(A, dtype=tdt, device=dev)
    o = S.snmf_default_options(precision=prec, formulation=form, batch=b, max_iter=k + m, tol=0.0, nonmonotone_M=10)
    h = S.snmf_create(S.dense_matrix(At), r, o)
    try:
        Wc = torch.tensor(W0, dtype=tdt, device=dev)
        Hc = Wc.clone()
        st, stats = S.snmf_solve(h, Wc, Hc)                      # k + m in one solve
        assert stats["iters"] == k + m
        ring, cnt = S.snmf_stats_ring(h, b)
    finally:
        S.snmf_destroy(h)
    o1 = S.snmf_default_options(precision=prec, formulation=form, batch=b, max_iter=k, tol=0.0, nonmonotone_M=10)
    h1 = S.snmf_create(S.dense_matrix(At), r, o1)
    try:
        W = torch.tensor(W0, dtype=tdt, device=dev)
        H = W.clone()
        S.snmf_solve(h1, W, H)                                   # k ...
        blob = S.snmf_get_state(h1)
    finally:
        S.snmf_destroy(h1)
    h2 = S.snmf_create(S.dense_matrix(At), r, o)                 # ... and m more on another handle
    try:
        S.snmf_set_state(h2, blob)
        st2, stats2 = S.snmf_solve(h2, W, H)
        per2 = S.snmf_restart_stats(h2, b)
    finally:
        S.snmf_destroy(h2)
    assert stats2["iters"] == k + m and all(int(x) == k + m for x in per2["iters"])
    assert torch.equal(W, Wc) and torch.equal(H, Hc)
    # statistics ring: one record per outer iteration 0 .. k + m, relative projected gradient 1 at 0
    assert cnt == k + m + 1
    for j in range(b):
        its = ring[j, :cnt, 0]
        assert np.array_equal(its, np.arange(k + m + 1))
        assert ring[j, 0, 1] == pytest.approx(1.0, rel=1e-12)
        assert np.all(ring[j, :cnt, 1] > 0) and ring[j, cnt - 1, 1] < ring[j, 0, 1]
        assert np.all(ring[j, cnt:, 0] == -1.0)
        assert np.all(ring[j, :cnt - 1, 7] == 1.0) and ring[j, cnt - 1, 7] == 0.0  # stopped at the limit


def test_ring_marks_the_tolerance_stop():
    """A restart that meets the tolerance stops there: iteration count below the limit, its
    last ring record carries the stop flag and the relative gradient at or under tol."""
    import torch
    dev = torch.device("cuda:0")
    A, _ = planted_dense(300, 6, 0.01, seed=31)
    At = torch.tensor(A, device=dev)
    tol = 1e-3
    o = S.snmf_default_options(precision=S.SNMF_F64, batch=2, max_iter=2000, tol=tol)
    h = S.snmf_create(S.dense_matrix(At), 6, o)
    try:
        W = torch.tensor(np.concatenate([uniform_init(300, 6, math.sqrt(A.mean() / 6), seed=32 + j)
                                         for j in range(2)], 1), device=dev)
        st, stats = S.snmf_solve(h, W, W.clone())
        per = S.snmf_restart_stats(h, 2)
        ring, cnt = S.snmf_stats_ring(h, 2)
    finally:
        S.snmf_destroy(h)
    assert st == S.SNMF_OK and stats["converged"] == 1
    for j in range(2):
        it = int(per["iters"][j])
        assert 0 < it < 2000
        c = min(it + 1, 256)
        last = ring[j, c - 1]
        assert last[0] == it and last[7] == 0.0 and last[1] <= tol
        assert np.all(ring[j, :c - 1, 7] == 1.0) and np.all(ring[j, :c - 1, 1] > tol)


def test_state_blob_checks():
    import torch
    dev = torch.device("cuda:0")
    A, _ = planted_dense(200, 4, 0.01, seed=7)
    At = torch.tensor(A, device=dev)
    h = S.snmf_create(S.dense_matrix(At), 4, S.snmf_default_options(precision=S.SNMF_F64, max_iter=3, tol=0.0))
    h2 = S.snmf_create(S.dense_matrix(At), 3, S.snmf_default_options(precision=S.SNMF_F64, max_iter=3, tol=0.0))
    try:
        with pytest.raises(S.SnmfError):
            S.snmf_get_state(h)                                  # no solve yet
        W = torch.tensor(uniform_init(200, 4, 0.1, seed=8), device=dev)
        S.snmf_solve(h, W, W.clone())
        blob = S.snmf_get_state(h)
        with pytest.raises(S.SnmfError):
            S.snmf_set_state(h2, blob)                           # another rank
        with pytest.raises(S.SnmfError):
            S.snmf_set_state(h, bytes(len(blob)))                    # not a state blob
        with pytest.raises(S.SnmfError):
            S.snmf_set_state(h, blob[:-8])                       # truncated
        S.snmf_set_state(h, blob)
        S.snmf_set_state(h, None)                                # dropped again
    finally:
        S.snmf_destroy(h)
        S.snmf_destroy(h2)
