"""Multi-process forms, checked with two gloo ranks on the CPU.  bench.py runs
independent replicas (no collective on the data path): every rank has its
own Philox key, and the units of all ranks are reported over the slowest
rank's time.  The paper's task split (Sect. 5.2) gives every rank a packet
range of one run and sums the tables: with the oracle tracing each rank's
range, the summed tables equal one oracle run over every packet."""
import os
import socket

import numpy as np

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


def _task_rank(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    from paper_1705_04702_gb300 import tasks
    from paper_1705_04702_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = W.torus_problem(n=16, nlambda=4, packet_scale=2e-5, npx=8)
        first, count = tasks.packet_share(prob.npk, rank, world)
        # the oracle takes one range for all wavelengths: trace each wavelength's own range
        parts = [oracle.trace(prob.with_packets(np.where(np.arange(prob.wl.n) == j, prob.npk, 0).astype(np.uint64)),
                              int(first[j]), int(first[j] + count[j])) for j in range(prob.wl.n)]
        tabs = [sum(p["absorbed"] for p in parts), sum(p["images_flat"] for p in parts), sum(p["sed"] for p in parts),
                sum(p["ledger"] for p in parts)]
        out[rank] = [t.copy() for t in tasks.sum_tables(tabs, dist)]
    finally:
        dist.destroy_process_group()


def test_task_split_tables_sum_to_the_whole_run():
    import torch.multiprocessing as mp
    import oracle
    from paper_1705_04702_gb300 import tasks
    from paper_1705_04702_gb300 import workloads as W
    oracle.build()
    prob = W.torus_problem(n=16, nlambda=4, packet_scale=2e-5, npx=8)
    shares = [tasks.packet_share(prob.npk, r, 3) for r in range(3)]
    assert np.array_equal(sum(c for _, c in shares), prob.npk)
    assert np.array_equal(shares[1][0], shares[0][0] + shares[0][1])
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_task_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    full = oracle.trace(prob)
    for r in range(world):
        a, img, sed, led = out[r]
        np.testing.assert_allclose(a, full["absorbed"], rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(img, full["images_flat"], rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(sed, full["sed"], rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(led, full["ledger"], rtol=1e-12, atol=1e-300)
