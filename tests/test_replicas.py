"""The multi-GPU path of bench.py is replicas (one independent solve stream
per rank, no collective on the data path): ranks agree on the slowest rank's
timed total (max over ranks) and report the time per solve over the solves of
all ranks. Checked here with world_size-2 gloo process groups on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, totals, steps, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, total = bench.replica_time(totals[rank], steps, dist, torch.device("cpu"))
        out[rank] = (value, total)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("totals", [(3.0, 5.0), (7.5, 2.5)])
def test_replica_time_is_max_over_ranks(totals):
    steps, world = 3, 2
    port = 29500 + int(totals[0] * 10) % 400
    out = mp.get_context("spawn").Manager().dict()  # no fork of this (threaded) process
    mp.spawn(_rank, args=(world, port, totals, steps, out), nprocs=world, join=True)
    want = max(totals)
    for r in range(world):
        value, total = out[r]
        assert total == want
        assert value == want / (steps * world)


def test_replica_time_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_time(6.0, 3) == (2.0, 6.0)
