"""The benchmark's multi-rank host logic on CPU: two gloo ranks, each with
its own replica, reduce their timings to the max and report the whole-job
value (replicas only: no data-path collective)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 150.0][rank]
    ms = bench.max_over_ranks(ms_local, torch.device("cpu"), world)
    out[rank] = (ms, bench.aggregate_value(1000, 10, world, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_aggregate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms, v = out[r]
        assert ms == 150.0
        assert v == pytest.approx(1000 * 10 * 2 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.aggregate_value(100, 4, 1, 2000.0) == pytest.approx(200.0)
