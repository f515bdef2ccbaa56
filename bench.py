#!/usr/bin/env python3
"""Benchmark of the GB300 DEM hot path on its headline workload.

Workload: isotropic compaction of one million polydisperse spheres -- radii
log-normal (median 1 mm, sigma 0.25, clipped to [0.5, 2] mm), seeded loose
periodic cloud at solid fraction 0.30, same linear frictional law as the
deposition case (E = 5e7 Pa, rho = 2600, ks/kn = 0.25, friction 30 deg),
damping 0.2, gravity off, dt = 0.5 p-wave step, 5000 steps; the cell shrinks at
the constant diagonal velocity gradient that brings the fraction to 0.62 at
the last step.  A bench "step" is one DEM time step (contact pass, gather +
integration, cell update, and the collider whenever a body has used up its
sweep margin).  The timed window is the LAST `--steps` steps of the 5000-step
job (earlier steps run untimed first), so a short window measures the densest,
most contact-heavy part of the job.

Arms:
  default            CUDA path through the C ABI, inputs resident in HBM
  --impl reference   the FP64 CPU oracle on this host's cores (a bounded sample)

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the scene (the path has no exchange step: replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

JOB_STEPS = 5000
N_BODIES = 1_000_000
PHI0, PHI1 = 0.30, 0.62
METRIC = "body-steps/s & contact-updates/s (1M spheres); served p50/p99 at fixed accuracy"
UNIT = "body-steps/s"
WORKLOAD = "periodic isotropic compaction, 1M log-normal spheres, phi 0.30->0.62 over 5000 steps"

# Algorithmic bytes of the contact kernel (per table row per launch), from its operand list:
#   every row:     pair int2 (8) + cell shift (4) + Fs/kn word (32) + 2 x position/radius (64)
#   real rows add: normal/ks (32) + tan(phi) (8) + 2 x (velocity 32 + spin 32) (128)
#                  + writes Fs/kn, normal/ks, F/d1, M/d2 (4 x 32 = 128)
ROW_BYTES_ALL = 8 + 4 + 32 + 64
ROW_BYTES_REAL = 32 + 8 + 128 + 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


_WL = {}


def make_workload(n):
    import workloads
    if n not in _WL:
        _WL[n] = workloads.compaction(n=n, seed=1, phi0=PHI0, phi_target=PHI1, variant="b",
                                      steps=JOB_STEPS)
    return _WL[n]


def velgrad_for(dt):
    import workloads
    g = workloads.compaction_rate(PHI0, PHI1, JOB_STEPS, dt)
    return np.diag([g, g, g])


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# body-steps the reference arm may spend (about a minute of single-thread oracle time)
REF_BUDGET = 6e7


def run_reference(args):
    """FP64 CPU oracle on the host cores.  Each step is a bounded sample of the workload:
    the same compaction with fewer spheres (same radius law, fraction and loading), sized
    so that warm-up + timed steps stay near REF_BUDGET body-steps."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_ref = int(max(2000, min(args.n, REF_BUDGET / max(1, args.steps + args.warmup))))
    args = argparse.Namespace(**{**vars(args), "n": n_ref})
    w = make_workload(args.n)
    orc = oracle.OracleScene.from_workload(w)
    dt = orc.clock()[2]
    orc.set_velgrad(velgrad_for(dt))
    per_step = []
    for _ in range(args.warmup):
        orc.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        orc.step(1)
        per_step.append(time.perf_counter() - t)
    T = time.perf_counter() - t0
    value = args.n * args.steps / T
    st = orc.stats()
    sample = (f"oracle, one thread, from the seeded initial cloud: {args.warmup} untimed + "
              f"{args.steps} timed steps of the same compaction with {args.n} spheres "
              f"(the first steps of the job)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "n_bodies": args.n, "sample": "initial steps"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "contacts_at_end": st["n_contacts"]}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(n, seconds_hint=20.0):
    """Time the oracle (as it stands, single thread) on the first steps of the same job."""
    import oracle
    oracle.build()
    w = make_workload(n)   # cached: the same cloud the GPU arm ran
    orc = oracle.OracleScene.from_workload(w)
    dt = orc.clock()[2]
    orc.set_velgrad(velgrad_for(dt))
    orc.step(1)   # first contact pass (untimed)
    t0 = time.perf_counter()
    k = 0
    while True:
        orc.step(1)
        k += 1
        el = time.perf_counter() - t0
        if el > seconds_hint or k >= 50:
            break
    return {"value": n * k / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} oracle steps (after 1 untimed) of the {n}-sphere compaction from "
                      f"the seeded initial cloud, {el:.1f} s single-threaded"}


def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
        __graft_entry__.build()
    from paper_2301_00611_gb300 import Scene

    w = make_workload(args.n)
    stream = torch.cuda.current_stream()
    scene = Scene.from_workload(w, capacity_bodies=args.n)
    dt = scene.dt()
    L = velgrad_for(dt)
    scene.set_cell_velgrad(L)
    K, W = args.steps, args.warmup
    prelude = max(0, JOB_STEPS - W - K)
    if prelude:
        scene.step(prelude)
    scene.step(W)
    st0 = scene.stats()
    scene.set_timing(True)
    t_before = scene.timing()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        scene.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tm = scene.timing()
    st1 = scene.stats()
    launches = tm["kernel_launches"] - t_before
    T = ms / 1e3
    if world > 1:
        tt = torch.tensor([T], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        T = float(tt.item())
    value = world * args.n * K / T
    mean_real = 0.5 * (st0["n_contacts"] + st1["n_contacts"])
    contact_updates = world * mean_real * K / T
    rows_per_s = world * tm["rows_processed"] / T

    # dominant kernel: the fused contact kernel
    peak, peak_kind = _peaks()
    avg_ms = tm["contact_ms"] / max(1, tm["contact_launches"])
    rows_avg = tm["rows_processed"] / max(1, tm["contact_launches"])
    bytes_avg = ROW_BYTES_ALL * rows_avg + ROW_BYTES_REAL * mean_real
    achieved = bytes_avg / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    share = {k: tm[k] / max(1e-9, ms) for k in ("contact_ms", "integrate_ms", "cell_ms",
                                                "collider_ms")}
    clocks = clk.summary()

    # end to end: host arrays in, the whole job through the public API, state out
    e2e = None
    if not args.no_e2e:
        scene.close()
        torch.cuda.synchronize()
        pos_out = np.empty((args.n, 3))
        vel_out = np.empty((args.n, 3))
        t0 = time.perf_counter()
        s2 = Scene.from_workload(w, capacity_bodies=args.n)
        s2.set_cell_velgrad(velgrad_for(s2.dt()))
        s2.step(JOB_STEPS)
        s2.get_state_into(pos=pos_out, vel=vel_out)
        torch.cuda.synchronize()
        T2 = time.perf_counter() - t0
        s2.close()
        h2d = args.n * (3 * 8 + 8 + 4 + 3 * 8)   # pos, radius, material, (zero) velocity
        d2h = args.n * 2 * 3 * 8
        e2e = {"value": world * args.n * JOB_STEPS / T2, "unit": UNIT,
               "h2d_bytes_per_step": h2d / JOB_STEPS, "d2h_bytes_per_step": d2h / JOB_STEPS,
               "note": "whole 5000-step job through the C ABI from host arrays: scene creation, "
                       "upload, stepping, state download"}
    else:
        scene.close()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_sample(args.n, args.cpu_seconds)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "n_bodies": args.n, "job_steps": JOB_STEPS,
                       "timed_window": f"last {K} steps (prelude {prelude} + warm-up {W} untimed)",
                       "dt": dt, "l2": "working set > L2 (bodies ~200 MB + contact table)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "contact_updates_per_s": contact_updates,
            "candidate_rows_per_s": rows_per_s,
            "contacts": {"start": st0["n_contacts"], "end": st1["n_contacts"],
                         "candidates_end": st1["n_candidates"],
                         "packing_fraction_end": st1["packing_fraction"]},
            "phase_share": share,
            "collider_runs": tm["collider_runs"],
            "gpu_launches": launches,
            "clocks": clocks,
            "roofline": {"bound": "hbm", "kernel": "contact (fused geometry + law)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_kind": peak_kind, "avg_launch_ms": avg_ms,
                         "bytes_per_launch": bytes_avg},
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=JOB_STEPS - 5)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_BODIES)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
