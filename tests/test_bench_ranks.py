"""The benchmark's multi-GPU path on CPU: replicas (one per rank, no exchange step)
timed by the slowest rank, whole-job throughput summed over the ranks, and the
reference arm running on rank 0 only.  Two gloo ranks stand in for two GPUs."""
import argparse
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T_local = 1.0 + rank          # rank 1 is the slow replica
    T = bench.max_over_ranks(T_local, world, "cpu")
    dist.barrier()
    out[rank] = (T, bench.job_rate(world, 1000.0, T))
    dist.destroy_process_group()


def test_replicas_time_is_the_slowest_rank_and_rate_sums_the_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1] == (2.0, 1000.0)   # 2 ranks x 1000 units in 2 s


def test_single_rank_is_untouched():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(1, 100.0, 2.0) == 50.0


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=2, warmup=3, n=1000, gpus=2)
    assert bench.run_reference(args) == 0      # returns at once, no oracle work
