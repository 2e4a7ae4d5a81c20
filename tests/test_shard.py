"""Sharding the batched form over ranks (bench.py --workload batch with N
ranks): the partition of the problems and the max-over-ranks timing, the
latter with world_size-2 gloo process groups on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2003_04930_gb300 import graphs, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_of_the_512_problem_batch(world):
    specs = graphs.batch_specs(512)
    costs = [shard.batch_cost(n, om) for n, om, seed in specs]
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(512))                   # every problem once
    assert all(p == sorted(p) for p in parts)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= sum(costs) / world + max(costs) + 1e-6 * sum(costs)
    # deterministic: every rank computes the same partition
    assert parts == shard.partition(costs, world)


def test_partition_small_cases():
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([5.0], 3) == [[0], [], []]
    # longest first, to the least loaded rank, ties to the lowest rank
    assert shard.partition([3.0, 3.0, 2.0, 2.0, 2.0], 2) == [[0, 2, 4], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_batch_cost_grows_with_size_and_weak_dissipation():
    assert shard.batch_cost(200, 0.5) > shard.batch_cost(100, 0.5)
    assert shard.batch_cost(100, 0.1) > shard.batch_cost(100, 0.9)


def _rank(rank, world, port, totals, steps, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.shard_time(totals[rank], steps, dist, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_shard_time_is_max_over_ranks():
    totals, steps, world = (4.0, 9.0), 3, 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, 29731, totals, steps, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (3.0, 9.0)


def test_shard_time_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.shard_time(6.0, 3) == (2.0, 6.0)
