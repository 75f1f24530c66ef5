"""World-size-2 gloo checks (CPU) of the multi-GPU plumbing bench.py uses:
replicas time the same step and the slowest rank sets the job time; the
batched instances are sharded by rank with no exchange of data."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_max = bench.max_over_ranks(10.0 + rank, world)
    total = bench.sum_over_ranks(rank + 1, world)
    mine = bench.shard(512, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, t_max, total, gathered))
    dist.destroy_process_group()


def test_replicas_and_instance_shards_gloo():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, total, gathered in res:
        assert t_max == 11.0  # the slowest rank
        assert total == 3.0
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(512))  # every instance exactly once
        assert set(gathered[0]).isdisjoint(gathered[1])


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
