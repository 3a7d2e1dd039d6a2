"""Host logic of the multi-GPU bench on CPU: two gloo ranks.

The batched workload shards problems across ranks with no collective on the
data path; the only exchanges are the barrier around the timed region and the
max-over-ranks reduction of the elapsed time.  Both are checked here without a
GPU (gloo backend, world size 2, rendezvous on 127.0.0.1).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, count, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = list(bench.shard_indices(count, rank, world))
    bench.barrier(world)
    worst = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    dist.destroy_process_group()
    q.put((rank, mine, worst, gathered))


def test_two_rank_sharding_and_max_time():
    world, count = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, count, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, worst, gathered in results:
        assert mine == list(range(rank * count, (rank + 1) * count))
        # the shards are disjoint and cover the world * count problems
        allp = sorted(i for part in gathered for i in part)
        assert allp == list(range(world * count))
        # every rank reports the slowest rank's time
        assert worst == 1.5 + (world - 1)


def test_single_rank_needs_no_process_group():
    import bench
    assert list(bench.shard_indices(4, 0, 1)) == [0, 1, 2, 3]
    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    bench.barrier(1)
