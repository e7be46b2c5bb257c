"""Host logic of bench.py's multi-GPU form (replicas, no data-path
collective): the time reported is the slowest rank's, and the whole-job
throughput counts every rank's solves.  Two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")
        out[rank] = (ms, bench.whole_job_ms_per_solve(ms, 3, 12, world))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, per_solve = out[r]
        assert ms == 150.0
        assert per_solve == pytest.approx(150.0 / (3 * 12 * 2))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.whole_job_ms_per_solve(42.0, 2, 3, 1) == 7.0
