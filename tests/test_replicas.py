"""The multi-process benchmark path on CPU: two gloo ranks (no GPU) time independent replicas; the job time is
the slowest rank's and the throughput counts every rank's units (bench.replica_throughput)."""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.replica_throughput(100.0 + 50.0 * rank, units_per_rank=1000, steps=4, world=world)
        out[rank] = (ms, value)
    finally:
        td.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_throughput_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    slowest = 100.0 + 50.0 * (world - 1)
    for r in range(world):
        ms, value = out[r]
        assert ms == slowest
        assert value == pytest.approx(1000 * world * 4 / (slowest / 1e3))


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_throughput(250.0, units_per_rank=10, steps=2, world=1)
    assert ms == 250.0 and value == pytest.approx(10 * 2 / 0.25)
