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
