"""The host side of bench.py's multi-GPU (replica) runs on CPU: two gloo
ranks take the slowest rank's time and the whole-job rate the way the NCCL
ranks do on the GPUs."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 * (rank + 1)                  # rank 1 is the slower one
        t = bench.reduce_over_ranks(local_ms, dist)
        total = bench.reduce_over_ranks(rank + 1, dist, op="sum")
        rate = bench.whole_job_rate(4096, 5, t / 1e3, world)
        out[rank] = (t, total, rate)
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_rate():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        t, total, rate = out[r]
        assert t == 20.0 and total == 3.0
        assert rate == pytest.approx(world * 4096 * 5 / 0.020)


def test_single_process_has_no_group():
    assert bench.reduce_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(100, 2, 0.5, 1) == 400.0
