"""The N > 1 host logic of bench.py on CPU: two gloo ranks take disjoint restart sets and
problem sets, and the whole-job time is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = bench.rank_restarts(3, rank)
        t = bench.max_over_ranks(10.0 + rank, world)
        seeds = torch.tensor([bench.uneven_seed(rank)], dtype=torch.int64)
        gathered = [torch.zeros_like(seeds) for _ in range(world)]
        dist.all_gather(gathered, seeds)
        out[rank] = (mine, t, [int(g.item()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_max():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    r0, r1 = res[0], res[1]
    assert set(r0[0]).isdisjoint(r1[0]) and sorted(r0[0] + r1[0]) == list(range(6))
    assert r0[1] == r1[1] == 11.0
    assert len(set(r0[2])) == 2 and r0[2] == r1[2]


def _shard_main(rank, world, port, out):
    """Row-partitioned A X, Gram and inner products of one problem on two gloo ranks, the
    local compute done with numpy (standing in for the GPU kernels on each rank)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2606_02887_gb300 import rowshard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, N = 203, 12
        g = np.random.default_rng(7)
        B = g.random((n, n))
        A = B + B.T
        X = g.random((n, N))
        lo, hi = rowshard.row_ranges(n, world)[rank]
        A_rows = torch.tensor(A[lo:hi])
        X_loc = torch.tensor(X[lo:hi])
        Y_loc = rowshard.sharded_product(A_rows, X_loc, rank, world, n, lambda a, x: a @ x)
        G = rowshard.sharded_gram(X_loc, lambda x: x.T @ x)
        d = rowshard.sharded_dots([float((X_loc * Y_loc).sum()), float((X_loc * X_loc).sum())])
        out[rank] = (lo, hi, Y_loc.numpy(), G.numpy(), d.numpy())
    finally:
        dist.destroy_process_group()


def test_row_partition_matches_single_rank():
    import numpy as np

    from paper_2606_02887_gb300.rowshard import row_ranges
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    n, N = 203, 12
    g = np.random.default_rng(7)
    B = g.random((n, n))
    A = B + B.T
    X = g.random((n, N))
    Y = np.concatenate([res[k][2] for k in range(world)], axis=0)
    assert [(res[k][0], res[k][1]) for k in range(world)] == row_ranges(n, world)
    assert np.allclose(Y, A @ X, rtol=1e-12)
    for k in range(world):
        assert np.allclose(res[k][3], X.T @ X, rtol=1e-12)
        assert np.allclose(res[k][4], [np.sum(X * (A @ X)), np.sum(X * X)], rtol=1e-12)
    assert row_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]


def _outer_main(rank, world, port, out):
    """One outer iteration of SNMPBB (the W block, then the H block, Alg. 1 each) with the rows
    of A, W and Ht split over two gloo ranks.  A rank holds only its rows.  The exchanges are the
    row partition's: X_fix all-gathered for each block's product, the Grams all-reduced, and
    every inner product of Alg. 1 taken as a local partial plus one all-reduce.  The oracle's
    own Algorithm 1 (nmpbb) runs on each rank with those callables, numpy standing in for the
    GPU kernels."""
    import math

    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle.snmpbb as OS
    from paper_2606_02887_gb300 import rowshard
    from workloads import planted_dense, uniform_init
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, r = 157, 5
        A, _ = planted_dense(n, r, 0.01, seed=91)
        W0 = uniform_init(n, r, math.sqrt(A.mean() / r), 92)
        opts = OS.Options(memory=10, objective="closed", max_iter=1, tol=0.0)
        lo, hi = rowshard.row_ranges(n, world)[rank]
        A_rows = torch.tensor(A[lo:hi])
        del A  # from here on this rank sees its rows of A only
        OS.inner = lambda X, Y: float(rowshard.sharded_dots([float(np.sum(X * Y))])[0])
        nA2 = float(rowshard.sharded_dots([float((A_rows * A_rows).sum())])[0])
        lam = 0.01 * math.sqrt(nA2)

        def gram(X):
            return rowshard.sharded_gram(torch.tensor(X), lambda x: x.T @ x).numpy()

        def block(X_loc, Fix_loc):
            B = rowshard.sharded_product(A_rows, torch.tensor(Fix_loc), rank, world, n, lambda a, x: a @ x).numpy()
            G = gram(Fix_loc)
            rho = OS.spectral_norm(G, opts.power_iters)

            def fobj(X):
                s = rowshard.sharded_dots([float(np.sum(X * B)), float(np.sum((X - Fix_loc) ** 2))]).numpy()
                return 0.5 * nA2 - s[0] + 0.5 * float(np.sum(gram(X) * G)) + 0.5 * lam * s[1]

            def fgrad(X):
                return X @ G - B + lam * X - lam * Fix_loc

            Xn, _, _ = OS.nmpbb(fobj, fgrad, X_loc, lambda X: rho, opts.inner_iters, opts)
            return Xn

        W_loc = block(W0[lo:hi], W0[lo:hi].copy())
        Ht_loc = block(W0[lo:hi].copy(), W_loc)
        out[rank] = (lo, hi, W_loc, Ht_loc, lam)
    finally:
        dist.destroy_process_group()


def test_row_partition_runs_an_outer_iteration_of_the_oracle():
    import math

    import numpy as np

    import oracle.snmpbb as OS
    from workloads import planted_dense, uniform_init
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_outer_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    n, r = 157, 5
    A, _ = planted_dense(n, r, 0.01, seed=91)
    W0 = uniform_init(n, r, math.sqrt(A.mean() / r), 92)
    W, Ht, info = OS.snmpbb_penalty(A, W0, W0, OS.Options(memory=10, objective="closed", max_iter=1, tol=0.0))
    Wd = np.concatenate([res[k][2] for k in range(world)], axis=0)
    Hd = np.concatenate([res[k][3] for k in range(world)], axis=0)
    assert abs(res[0][4] - info["lam"]) <= 1e-14 * info["lam"]
    assert np.linalg.norm(Wd - W) <= 1e-10 * np.linalg.norm(W)
    assert np.linalg.norm(Hd - Ht) <= 1e-10 * np.linalg.norm(Ht)
    assert not np.allclose(W, W0)  # the iteration moved
