"""Whole-job figures of the benchmark's replica mode (`bench.py --gpus N`):
every rank solves its own copy of the workload, and the reported throughput
is the units of all ranks over the slowest rank's time.  Checked with two
gloo ranks on the CPU (the aggregation has no GPU-specific step)."""

import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 100 + 50 r ms for 1000 * (r + 1) units
        t, u = bench.replica_totals(100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
        out.put((rank, t, u))
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max time over ranks, sum of units, the same on every rank
    assert got == [(0, 150.0, 3000.0), (1, 150.0, 3000.0)]


def test_replica_totals_alone():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_totals(12.5, 7, "cpu") == (12.5, 7.0)
