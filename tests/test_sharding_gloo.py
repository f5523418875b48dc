"""The multi-rank path of the batched workload on CPU: two gloo ranks split
the 256 seeded problems with sharding.shard, each sees the same partition,
the loads are balanced, and the max-over-ranks time reduction the benchmark
uses gives the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2411_03501_gb300 import workloads as W
from paper_2411_03501_gb300.sharding import estimated_cost, shard


def test_shard_is_a_balanced_partition():
    costs = [estimated_cost(p[0]) for p in W.batched(256)]
    for world in (1, 2, 3, 4, 8):
        parts = shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(256))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= (sum(costs) / world) * 1.05 + max(costs)
    with pytest.raises(ValueError):
        shard(costs, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [estimated_cost(p[0]) for p in W.batched(256)]
        mine = shard(costs, world)[rank]
        # every rank reports its share; rank 0 checks the union
        sizes = [None] * world
        dist.all_gather_object(sizes, mine)
        # the benchmark's timing: max over ranks of each rank's time
        t = torch.tensor([10.0 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        units = torch.tensor([float(len(mine))], dtype=torch.float64)
        dist.all_reduce(units, op=dist.ReduceOp.SUM)
        if rank == 0:
            q.put((sizes, float(t.item()), float(units.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_split_the_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    sizes, tmax, units = q.get(timeout=100)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(i for part in sizes for i in part) == list(range(256))
    assert set(sizes[0]).isdisjoint(sizes[1])
    assert tmax == 11.0
    assert units == 256.0
