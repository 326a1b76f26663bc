"""The multi-GPU form is independent replicas (no collective on the data
path): bench.py gives every rank its own Philox key and reports the units of
all ranks over the slowest rank's time.  Checked here with two gloo ranks on
the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 2.0 + rank  # rank 1 is the slow one
        t = bench.job_time(elapsed, dist, "cpu")
        out[rank] = (bench.replica_seed(rank), t, bench.job_throughput(1000, world, 5, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_and_throughput():
    import torch.multiprocessing as mp
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world  # distinct Philox keys: no packet is traced twice
    for r in range(world):
        assert out[r][1] == pytest.approx(3.0)  # the slowest rank's time, on every rank
        assert out[r][2] == pytest.approx(1000 * 2 * 5 / 3.0)


def test_single_process_time_is_its_own():
    import bench
    assert bench.job_time(1.5) == 1.5
    assert bench.job_throughput(10, 1, 3, 1.5) == pytest.approx(20.0)
