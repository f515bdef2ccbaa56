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


def _shard_rank(rank, world, port, sizes, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.assign_units(sizes, world)[rank]          # no communication
    got = bench.gather_ranks({"rank": rank, "mine": mine}, world)
    out[rank] = got
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_scenes_are_dealt_out_to_ranks_disjoint_and_complete(world):
    """Batched scenes and served requests are dealt out by body count with no
    communication: every rank computes the same assignment, the rank sets are
    disjoint, their union is every scene, and the body counts differ by at most the
    largest scene."""
    import workloads
    sizes = [int(n) for n in workloads.batch_parameters(64, 3, 500, 50_000)[0]]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_rank, args=(world, _free_port(), sizes, out), nprocs=world,
                       join=True, start_method="spawn")
    views = [out[r] for r in range(world)]
    assert all(v == views[0] for v in views)            # every rank sees the same split
    sets = [set(e["mine"]) for e in views[0]]
    assert [e["rank"] for e in views[0]] == list(range(world))
    assert sum(len(x) for x in sets) == len(sizes)
    assert set().union(*sets) == set(range(len(sizes)))
    loads = [sum(sizes[i] for i in x) for x in sets]
    assert max(loads) - min(loads) <= max(sizes)


def test_single_rank_takes_every_scene():
    assert bench.assign_units([4, 9, 1], 1) == [[0, 1, 2]]
    assert bench.gather_ranks({"a": 1}, 1) == [{"a": 1}]
