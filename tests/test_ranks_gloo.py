"""Multi-rank host logic on CPU: two gloo processes on 127.0.0.1.

The path shards by scene and exchanges no data; what runs across ranks is the
barrier around the timed region, the maximum of the per-rank times and the sum
of the per-rank work.  These tests run that logic with world size 2.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_03451_gb300 import ranks as RK


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        RK.barrier()
        # rank r "took" 1 + 2 r seconds for 10 (r + 1) units of work
        t = RK.max_over_ranks(1.0 + 2.0 * rank)
        units = RK.sum_over_ranks(10.0 * (rank + 1))
        shard = list(RK.scene_shard(7, rank, world))
        seeds = RK.rank_seeds(rank)
        RK.barrier()
        out.put((rank, t, units, shard, seeds))
    finally:
        dist.destroy_process_group()


def test_two_rank_reductions_and_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, units, shard, seeds in res:
        assert t == 3.0                      # the slowest rank's time on every rank
        assert units == 30.0                 # work of both ranks
        assert RK.job_throughput(units, t) == 10.0
    shards = [r[3] for r in res]
    assert shards[0] + shards[1] == list(range(7))      # disjoint, complete, in order
    assert abs(len(shards[0]) - len(shards[1])) <= 1
    assert res[0][4] != res[1][4]                       # every rank fits its own room


def test_single_process_identity():
    assert not dist.is_initialized()
    assert RK.max_over_ranks(2.5) == 2.5
    assert RK.sum_over_ranks(4.0) == 4.0
    RK.barrier()


@pytest.mark.parametrize("n,world", [(0, 3), (5, 1), (32, 8), (3, 4), (33, 8)])
def test_scene_shard_partition(n, world):
    got = [i for r in range(world) for i in RK.scene_shard(n, r, world)]
    assert got == list(range(n))
    sizes = [len(RK.scene_shard(n, r, world)) for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_scene_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        RK.scene_shard(4, 2, 2)
    with pytest.raises(ValueError):
        RK.job_throughput(1.0, 0.0)
