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
import hashlib
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
# Algorithmic FP64 flops of the contact law per row (periodic cell, diagonal H; add, mul,
# div, sqrt = 1, fused multiply-add = 2), counted from the operations of sections
# 2.1.2-2.1.4 as the oracle writes them: image shift 3, branch 6, |d|^2 5, threshold 2
# (every row = 16); real rows add l, n, pen 5, image velocity 6, n- x n 9, twist 13,
# frame rotation of Fs 24, ratchet-free v12 28, perpendicular part 11, increment 9,
# Fn and Coulomb test 8, F 6, torque arms 13 (= 132 more, 148 in all).
ROW_FLOPS_ALL = 16
ROW_FLOPS_REAL = 132
# FP64 peak of GB300 from its unit counts: 152 SMs x 2 FP64 FMA per clock x 2 flops at the
# 2070 MHz maximum clock (a probe measured 1.194 TFLOP/s, 95% of it).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


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


def max_over_ranks(T, world, device):
    """The slowest replica's time: the whole job ends when its last rank does."""
    if world <= 1:
        return T
    import torch
    tt = torch.tensor([T], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def job_rate(world, units_per_rank, T):
    """Whole-job throughput of `world` replicas that each processed units_per_rank in
    the slowest replica's time T."""
    return world * units_per_rank / T


def assign_units(sizes, world):
    """Whole scenes to ranks with no communication (replicas only: scenes never
    interact): largest first, each to the rank with the fewest bodies so far (ties to
    the lower rank).  Returns one sorted index list per rank; together they hold every
    scene exactly once."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(o) for o in out]


def gather_ranks(obj, world):
    """Every rank's object, in rank order (one entry without torch.distributed)."""
    if world <= 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out


# body-steps the reference arm may spend (about a minute of single-thread
# oracle time at the dense window's coordination)
REF_BUDGET = 4e6
# coordination number of the timed window (the last steps of the 1M compaction: 2.62M
# real contacts on 1M spheres), the density of contacts the reference arm's sample has
REF_Z_WINDOW = 5.24
# the reference sample's time step relative to the workload's: its spheres overlap by
# some 10-20% of their radii (inflated radii reach the window's coordination), so at
# the workload's step they would fly apart within the sample; the oracle's work per
# step does not depend on dt
REF_DT_SCALE = 1e-2


def dense_inflation(z_target, n_probe=20000):
    """Radius factor f that gives the 1M compaction's loose cloud (solid fraction 0.30,
    the same radius law) the coordination z_target: bisection on a smaller cloud of the
    same generator, pairs counted by the oracle's brute-force-checked grid search."""
    import oracle
    import workloads
    w = workloads.compaction(n=n_probe, seed=11, phi0=PHI0, phi_target=PHI1, variant="b",
                             steps=JOB_STEPS)
    lo, hi = 1.0, 1.6
    for _ in range(30):
        f = 0.5 * (lo + hi)
        i, j, c = oracle.pairs(w.pos, w.radius * f, periodic=True, H=w.cell)
        z = 2.0 * len(i) / n_probe
        lo, hi = (f, hi) if z < z_target else (lo, f)
    return 0.5 * (lo + hi)


def run_reference(args):
    """The FP64 CPU oracle on the host cores, on a bounded sample of the timed window's
    work.  The GPU arm times the last steps of the compaction, a packing near solid
    fraction 0.62 with coordination ~5.2; without the library the oracle cannot reach
    that state, so the sample is the job's seeded loose cloud with its radii inflated
    until the coordination matches (each timed step then computes as many contacts per
    sphere as a window step), and fewer spheres so that warm-up + timed steps stay near
    REF_BUDGET body-steps.  It reports the contact counts it actually met."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_ref = int(max(2000, min(args.n, REF_BUDGET / max(1, args.steps + args.warmup))))
    f = dense_inflation(REF_Z_WINDOW)
    w = make_workload(n_ref)
    import copy
    w = copy.copy(w)
    w.radius = w.radius * f
    orc = oracle.OracleScene.from_workload(w)
    dt = orc.clock()[2] * REF_DT_SCALE
    orc.set_dt(dt)
    orc.set_velgrad(velgrad_for(dt))
    for _ in range(args.warmup):
        orc.step(1)
    c0 = orc.stats()["n_contacts"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(1)
    T = time.perf_counter() - t0
    c1 = orc.stats()["n_contacts"]
    value = n_ref * args.steps / T
    sample = (f"oracle, one thread: {args.warmup} untimed + {args.steps} timed steps of the "
              f"compaction's seeded loose cloud with {n_ref} spheres, radii x {f:.4f} so that "
              f"the coordination is the timed window's ({REF_Z_WINDOW}): {c0} contacts at the "
              f"first timed step, {c1} at the last (Z {2 * c0 / n_ref:.2f} -> "
              f"{2 * c1 / n_ref:.2f}); time step x {REF_DT_SCALE} so that the overlaps stay "
              f"put")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "n_bodies": n_ref,
                       "sample": "dense window (inflated loose cloud at the window's Z)",
                       "contacts_per_sphere": c0 / n_ref},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "contact_updates_per_s": 0.5 * (c0 + c1) * args.steps / T}
    print(json.dumps(line), flush=True)
    return 0


def export_window_start(scene):
    """State, contact history, cell, clock and step of a scene, read through the C ABI
    (the CPU baseline starts the oracle from it)."""
    it, t = scene.clock()
    return {"state": scene.state(force=False), "contacts": scene.contacts(),
            "cell": scene.cell(), "clock": (it, t), "dt": scene.dt()}


def cpu_baseline_sample(w, start, seconds_hint=20.0, max_steps=50):
    """Time the oracle (as it stands, single thread) on the timed window itself: it is
    seeded with the GPU scene's state, contact history, cell and clock at the first
    timed step and runs the same steps until about seconds_hint have passed."""
    import oracle
    oracle.build()
    orc = oracle.OracleScene.from_workload(w, dt=start["dt"])
    st = start["state"]
    orc.set_state(pos=st["pos"], vel=st["vel"], angvel=st["angvel"], ori=st["ori"])
    c = start["contacts"]
    orc.set_contacts(c["id1"], c["id2"], c["c"], c["fs"], c["normal"], c["phys"])
    cl = start["cell"]
    orc.set_cell(H=cl["H"], velgrad=cl["velgrad"], prev_velgrad=cl["prev_velgrad"],
                 prev_H=cl["prev_H"])
    orc.set_clock(*start["clock"])
    c_start = len(c["id1"])
    t0 = time.perf_counter()
    k = 0
    while True:
        orc.step(1)
        k += 1
        el = time.perf_counter() - t0
        if el > seconds_hint or k >= max_steps:
            break
    c_end = orc.stats()["n_contacts"]
    n = w.n
    return {"value": n * k / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "contact_updates_per_s": 0.5 * (c_start + c_end) * k / el,
            "sample": f"the first {k} steps of the timed window (from step {start['clock'][0]}: "
                      f"the GPU scene's state, contact history and cell imported into the "
                      f"oracle), {n} spheres, {c_start} real contacts at the start and {c_end} "
                      f"at the end, {el:.1f} s single-threaded"}


def tune_shape(Scene, w, args, precision):
    """Launch shapes for the timed scene: dem_autotune on a separate copy of the job
    advanced to mid-compaction (a contact network like the timed window's).  Launch
    shapes change no result, so the timed trajectory is the same whichever is picked."""
    from paper_2301_00611_gb300 import DEM_MIXED, DEM_FP64
    fixed = getattr(args, "shape_" + precision, None)
    if fixed:   # a given shape (to profile the variant a tuned run picked)
        cb, cps, ib, deg = (int(v) for v in fixed.split(","))
        return {"contact_block": cb, "contact_blocks_per_sm": cps, "integrate_block": ib,
                "degree_order": deg}
    if args.no_autotune:
        return None
    prec = DEM_MIXED if precision == "mixed" else DEM_FP64
    s = Scene.from_workload(w, capacity_bodies=args.n, precision=prec)
    s.set_cell_velgrad(velgrad_for(s.dt()))
    s.step(TUNE_AT)
    shape = s.autotune(steps_per_trial=TUNE_STEPS)
    s.close()
    return shape


def _run_window(Scene, w, prec, shape, velgrad, K, W, world, local, timing, capture_start):
    """The job on a fresh scene up to its last K steps, then those K steps timed with
    CUDA events (with or without the per-kernel events of dem_set_timing)."""
    import torch
    stream = torch.cuda.current_stream()
    scene = Scene.from_workload(w, capacity_bodies=w.n, precision=prec)
    if shape:
        scene.set_tuning(**shape)
    dt = scene.dt()
    scene.set_cell_velgrad(velgrad(dt))
    prelude = max(0, JOB_STEPS - W - K)
    if prelude:
        scene.step(prelude)
    scene.step(W)
    st0 = scene.stats()
    start = export_window_start(scene) if capture_start else None
    scene.set_timing(timing)
    t_before = scene.timing()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # an NVTX range around the timed steps, so that a profiler can take exactly them
    # (ncu --nvtx --nvtx-include "<precision>_window/"); no cost without a profiler
    rng = ("mixed" if prec == 1 else "fp64") + ("_window_events" if timing else "_window")
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push(rng)
        e0.record(stream)
        scene.step(K)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tm = scene.timing()
    st1 = scene.stats()
    scene.close()
    return {"ms": ms, "dt": dt, "prelude": prelude, "tm": tm, "st0": st0, "st1": st1,
            "launches": tm["kernel_launches"] - t_before, "clocks": clk.summary(),
            "start": start}


def _time_window(Scene, w, args, precision, world, local, shape=None, capture_start=False,
                 velgrad=velgrad_for, K=None):
    """Run the job to its timed window and time its last K steps; returns the
    measurements (and, with capture_start, the scene's state at the first timed step).
    The job runs twice: the value comes from a run without per-kernel CUDA events (they
    cost the step some 2-5%), the per-kernel times and phase shares from a second run of
    the same job (the same trajectory: every run of a scene is bitwise reproducible)
    with the events on."""
    from paper_2301_00611_gb300 import DEM_MIXED, DEM_FP64
    prec = DEM_MIXED if precision == "mixed" else DEM_FP64
    K = args.steps if K is None else K
    W = args.warmup
    plain = _run_window(Scene, w, prec, shape, velgrad, K, W, world, local, False, capture_start)
    timed = _run_window(Scene, w, prec, shape, velgrad, K, W, world, local, True, False)
    ms, tm = plain["ms"], timed["tm"]
    st0, st1 = plain["st0"], plain["st1"]
    T = max_over_ranks(ms / 1e3, world, "cuda")
    mean_real = 0.5 * (st0["n_contacts"] + st1["n_contacts"])
    avg_ms = tm["contact_ms"] / max(1, tm["contact_launches"])
    rows_avg = tm["rows_processed"] / max(1, tm["contact_launches"])
    return {"T": T, "ms": ms, "ms_timed": timed["ms"], "dt": plain["dt"],
            "prelude": plain["prelude"], "tm": tm, "st0": st0, "st1": st1,
            "mean_real": mean_real, "avg_ms": avg_ms, "rows_avg": rows_avg, "K": K,
            "launches": plain["launches"], "clocks": plain["clocks"], "start": plain["start"]}


# Algorithmic bytes of the mixed-precision contact kernel (per row), from its operand list:
#   every row:     pair 8 + cell shift 4 + reference branch/kn 16 + squared reference gap 4
#                  + two FP32 offsets 32 = 64
#   real rows add: FP64 shear history 32 + normal/ks 16 + two FP32 velocity/spin 64
#                  + writes history 32, normal 16, F/d1 16, M/d2 16 = 192
ROW_BYTES_ALL_MIXED = 64
ROW_BYTES_REAL_MIXED = 192
TUNE_AT = 4500      # step of the job at which the launch shapes are tuned (the dense end,
                    # where most of the step time is spent)
TUNE_STEPS = 10     # timed steps per autotune trial

# Algorithmic cost of the integrator per body and per real contact (each real contact is
# summed by both of its bodies), counted from its operand lists and operations:
#   FP64, per body: reads x, v, w, m/I, orientation, reference position (6 x 32 B), the
#     CSR offsets and order (12 B), flags (1 B); writes x, v, w, orientation (4 x 32 B)
#     = 333 B; per real contact: two 64 B row outputs + one down-list entry = 132 B.
#     Flops per body (add/mul 1, fused multiply-add 2): damping and leapfrog of force and
#     torque 42, fluctuation velocity 6, homoDeform 15, position 6, orientation 45,
#     displacement bound 15, per-body constants 2 = 131; per real contact 2 x 9 = 18.
#   mixed, per body: FP32 mirrors and FP64 records read (vw 32, offset 16, reference
#     16 + 32, m/I 16, orientation 16, x v w 96, CSR 8, flags 1) = 233 B, written
#     (x v w 96, vw 32, offset 16, orientation 16) = 160 B; per real contact two 32 B
#     row outputs + one down-list entry = 68 B.
INT_BYTES_BODY, INT_BYTES_REAL = 333, 132
INT_FLOPS_BODY, INT_FLOPS_REAL = 131, 18
INT_BYTES_BODY_MIXED, INT_BYTES_REAL_MIXED = 393, 68


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the step
# kernels, from one ncu capture of this workload's timed window (the last 30 steps,
# taken through the NVTX ranges the window is marked with; the profile under profiles/
# gives the command): the mean of the captured working launches, which process `rows`
# candidate rows and about `real` real contacts each.  A figure describes the
# kernel sources whose digest is stored with it and is reported as null for any other
# build (the integrator's include the collider, which sets the body order it runs in).
KERNEL_SOURCES = {"contact": {"fp64": ("contact.cu", "dem_internal.cuh"),
                              "mixed": ("contact_mixed.cu", "dem_internal.cuh")},
                  "integrate": {"fp64": ("integrate.cu", "collider.cu", "dem_internal.cuh"),
                                "mixed": ("integrate.cu", "collider.cu", "dem_internal.cuh")}}
TRAFFIC_PROFILE = "profiles/dram_traffic_compaction_1m.md"
TRAFFIC = {
    ("fp64", "contact"): {"bytes": 809.1e6, "rows": 4654436, "real": 2592000, "step": 4975,
                          "digest": "d2a67f79426e6fc6"},
    ("fp64", "integrate"): {"bytes": 639.9e6, "rows": 4654436, "real": 2592000, "step": 4975,
                            "digest": "397853ded890a3d6"},
    ("mixed", "contact"): {"bytes": 611.1e6, "rows": 4654436, "real": 2591000, "step": 4975,
                           "digest": "ccbf9b2d833aaeda"},
    ("mixed", "integrate"): {"bytes": 528.1e6, "rows": 4654436, "real": 2591000, "step": 4975,
                             "digest": "397853ded890a3d6"},
}


def kernel_digest(name, precision):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name][precision]:
        with open(os.path.join(ROOT, "paper_2301_00611_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(precision, name, algorithmic_at):
    t = TRAFFIC.get((precision, name))
    if not t or t["digest"] != kernel_digest(name, precision):
        return None, None
    note = (f"ncu DRAM bytes per launch in the last 30 steps of the job ({t['rows']} rows, "
            f"{t['real']} real contacts; the algorithmic bytes of such a launch are "
            f"{algorithmic_at(t['rows'], t['real']):.4g}); {TRAFFIC_PROFILE}")
    return t["bytes"], note


# The method's own algorithmic bytes (what a contact and a body must move per
# step, independent of this implementation's layout): 244 B read + 120 B written per
# real contact in the contact pass, 470 B per real contact and 180 B per body per step.
METHOD_CONTACT_BYTES = 364
METHOD_STEP_CONTACT_BYTES, METHOD_STEP_BODY_BYTES = 470, 180


def _kernel_rooflines(res, precision, n, peak, peak_kind, traffic=True, fp64_peak=None):
    """Roofline of the contact and integrator kernels of one timed window: achieved
    algorithmic flops (FP64, FP64-pipe bound) or bytes (mixed, HBM bound) per launch over
    the kernel's average launch time from its CUDA events.  FP64 kernels divide by the
    FP64 rate measured in this run (fp64_peak, TFLOP/s; the figure derived from unit
    counts and clock is reported beside it), and carry their HBM fractions both for this
    implementation's operand bytes and for the method's per-contact bytes."""
    tm, real = res["tm"], res["mean_real"]
    c_ms = res["avg_ms"]
    i_ms = tm["integrate_ms"] / max(1, tm["integrate_launches"])
    out = {}
    if precision == "fp64":
        pk = fp64_peak if fp64_peak else FP64_PEAK_TFLOPS
        pk_kind = ("measured (FP64 FMA-chain probe dem_measure_fp64_peak, this run)"
                   if fp64_peak else "derived from unit counts and clock (FP64 FMA pipe)")
        cf = ROW_FLOPS_ALL * res["rows_avg"] + ROW_FLOPS_REAL * real
        cb = ROW_BYTES_ALL * res["rows_avg"] + ROW_BYTES_REAL * real
        if_ = INT_FLOPS_BODY * n + INT_FLOPS_REAL * real
        ib = INT_BYTES_BODY * n + INT_BYTES_REAL * real
        for name, ms, fl, by in (("contact", c_ms, cf, cb), ("integrate", i_ms, if_, ib)):
            tf = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
            gb = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
            out[name] = {"bound": "alu", "achieved": tf, "peak": pk,
                         "unit": "TFLOP/s", "frac": tf / pk, "traffic": None,
                         "peak_kind": pk_kind, "derived_peak": FP64_PEAK_TFLOPS,
                         "frac_of_derived": tf / FP64_PEAK_TFLOPS,
                         "avg_launch_ms": ms, "flops_per_launch": fl,
                         "hbm": {"achieved_gbs": gb, "peak_gbs": peak, "frac": gb / peak,
                                 "peak_kind": peak_kind, "bytes_per_launch": by}}
        sb = METHOD_CONTACT_BYTES * real
        sg = sb / (c_ms / 1e3) / 1e9 if c_ms > 0 else 0.0
        out["contact"]["hbm_method_bytes"] = {"bytes_per_launch": sb, "achieved_gbs": sg,
                                              "frac": sg / peak, "peak_kind": peak_kind}
    else:
        cb = ROW_BYTES_ALL_MIXED * res["rows_avg"] + ROW_BYTES_REAL_MIXED * real
        ib = INT_BYTES_BODY_MIXED * n + INT_BYTES_REAL_MIXED * real
        for name, ms, by in (("contact", c_ms, cb), ("integrate", i_ms, ib)):
            gb = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
            out[name] = {"bound": "hbm", "achieved": gb, "peak": peak, "unit": "GB/s",
                         "frac": gb / peak, "traffic": None, "peak_kind": peak_kind,
                         "avg_launch_ms": ms, "bytes_per_launch": by}
    if precision == "fp64":
        alg = {"contact": lambda r, c: ROW_BYTES_ALL * r + ROW_BYTES_REAL * c,
               "integrate": lambda r, c: INT_BYTES_BODY * n + INT_BYTES_REAL * c}
    else:
        alg = {"contact": lambda r, c: ROW_BYTES_ALL_MIXED * r + ROW_BYTES_REAL_MIXED * c,
               "integrate": lambda r, c: INT_BYTES_BODY_MIXED * n + INT_BYTES_REAL_MIXED * c}
    for name, o in out.items():
        if not traffic:   # the stored DRAM figures belong to the 1M compaction
            continue
        tb, note = _traffic(precision, name, alg[name])
        o["traffic"] = tb
        if note:
            o["traffic_note"] = note
    share = {"contact": tm["contact_ms"], "integrate": tm["integrate_ms"]}
    dom = max(share, key=share.get)
    line = dict(out[dom])
    line["kernel"] = dom + (" (fused geometry + law)" if dom == "contact" else
                            " (fixed-order gather + damped leapfrog)") + \
        (", FP64" if precision == "fp64" else ", mixed")
    return line, out


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
    from paper_2301_00611_gb300.dem import measure_fp64_peak

    w = make_workload(args.n)
    K, W = args.steps, args.warmup
    peak, peak_kind = _peaks()
    fp64_peak = measure_fp64_peak()
    shape64 = tune_shape(Scene, w, args, "fp64")
    res = _time_window(Scene, w, args, "fp64", world, local, shape64,
                       capture_start=(rank == 0 and not args.no_cpu_baseline))
    mixed = None
    if args.precision in ("both", "mixed"):
        shape32 = tune_shape(Scene, w, args, "mixed")
        mixed = _time_window(Scene, w, args, "mixed", world, local, shape32)
        mixed["shape"] = shape32

    T, ms, tm = res["T"], res["ms"], res["tm"]
    value = job_rate(world, args.n * K, T)
    contact_updates = world * res["mean_real"] * K / T
    rows_per_s = world * tm["rows_processed"] / T
    share = {k: tm[k] / max(1e-9, res["ms_timed"]) for k in ("contact_ms", "integrate_ms",
                                                              "cell_ms", "collider_ms")}
    rl64, rk64 = _kernel_rooflines(res, "fp64", args.n, peak, peak_kind, fp64_peak=fp64_peak)
    # the whole step against the method's algorithmic bytes (N 180 B + C 470 B per step)
    step_bytes = METHOD_STEP_BODY_BYTES * args.n + METHOD_STEP_CONTACT_BYTES * res["mean_real"]
    step_gbs = step_bytes / (ms / K / 1e3) / 1e9
    mixed_line = None
    if mixed is not None:
        mrl, mrk = _kernel_rooflines(mixed, "mixed", args.n, peak, peak_kind)
        mixed_line = {
            "value": world * args.n * K / mixed["T"], "unit": UNIT,
            "ms_per_step": mixed["ms"] / K,
            "dtype": "mixed: f32 contact geometry/law, f64 shear history, integration and "
                     "reductions",
            "contact_updates_per_s": world * mixed["mean_real"] * K / mixed["T"],
            "phase_share": {k: mixed["tm"][k] / max(1e-9, mixed["ms_timed"])
                            for k in ("contact_ms", "integrate_ms", "cell_ms", "collider_ms")},
            "collider_runs": mixed["tm"]["collider_runs"], "gpu_launches": mixed["launches"],
            "launch_shape": mixed["shape"],
            "clocks": mixed["clocks"],
            "contacts": {"start": mixed["st0"]["n_contacts"], "end": mixed["st1"]["n_contacts"]},
            "roofline": mrl,
            "roofline_kernels": mrk,
        }

    # end to end: host arrays in, the whole job through the public API, state out
    e2e = None
    if not args.no_e2e:
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
               "note": "whole 5000-step FP64 job through the C ABI from host arrays: scene "
                       "creation, upload, stepping, state download"}

    # the batched sweep and the served stream: whole scenes dealt out to the ranks
    batched = None if args.no_batch else run_batch_measure(args, world, rank)
    served = None if args.no_serve else run_served_measure(args, world, rank)
    triax = config_1a = None
    if rank == 0 and not args.no_extra:
        config_1a = compaction_1a_measure(args, Scene, peak, peak_kind, fp64_peak)
        triax = triax_measure(args, TRIAX_HEADLINE_N, None)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_sample(w, res["start"], args.cpu_seconds)
        st0, st1 = res["st0"], res["st1"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "n_bodies": args.n, "job_steps": JOB_STEPS,
                       "timed_window": f"last {K} steps (prelude {res['prelude']} + warm-up {W} "
                                       f"untimed)",
                       "dt": res["dt"], "l2": "working set > L2 (bodies ~200 MB + contact table)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "contact_updates_per_s": contact_updates,
            "candidate_rows_per_s": rows_per_s,
            "contacts": {"start": st0["n_contacts"], "end": st1["n_contacts"],
                         "candidates_end": st1["n_candidates"],
                         "packing_fraction_end": st1["packing_fraction"]},
            "phase_share": share,
            "timing_note": "value and ms_per_step: the window run without per-kernel CUDA "
                           "events; phase shares, collider runs and the kernels' launch "
                           "times (roofline): a second run of the same job with the events "
                           "on (ms_per_step_instrumented)",
            "ms_per_step_instrumented": res["ms_timed"] / K,
            "step_hbm_method_bytes": {"bytes_per_step": step_bytes, "achieved_gbs": step_gbs,
                                      "frac": step_gbs / peak, "peak_kind": peak_kind},
            "fp64_peak_tflops": {"measured": fp64_peak, "derived": FP64_PEAK_TFLOPS},
            "collider_runs": tm["collider_runs"],
            "gpu_launches": res["launches"],
            "launch_shape": shape64,
            "clocks": res["clocks"],
            "roofline": rl64,
            "roofline_kernels": rk64,
            "mixed": mixed_line,
            "batched": batched,
            "served": served,
            "config_1a": config_1a,
            "triax": triax,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batched sweep
BATCH_SCENES = 512
BATCH_STEPS = 2000
BATCH_TUNE_STEPS = 4   # timed steps per autotune trial (the trials are real steps)


def _sync():
    import torch
    torch.cuda.synchronize()


def _batch_scene(Scene, ws, precision):
    g = Scene(capacity_bodies=sum(w.n for w in ws), precision=precision, dt=1.0)
    g.set_material(0, 1000.0, 1e6, 0.25, 0.5)
    subs = [g.add_workload(w, material_base=1 + k) for k, w in enumerate(ws)]
    return g, subs


def _stat_errors(pairs, ns):
    """Per-scene errors of (test, reference) statistics pairs: kinetic energy relative to
    the reference's final value and to the reference run's peak (the scale of a
    deposition that has settled to rest), coordination relative (and against one contact,
    2/N, its resolution), packing fraction relative."""
    ke = np.array([abs(a["kinetic_energy"] / b["kinetic_energy"] - 1) for a, b in pairs])
    ke_pk = np.array([abs(a["kinetic_energy"] - b["kinetic_energy"]) / b["ke_peak"]
                      for a, b in pairs])
    zr = np.array([abs(a["coordination"] - b["coordination"]) / max(b["coordination"], 2.0 / n)
                   for (a, b), n in zip(pairs, ns)])
    zc = np.array([abs(a["coordination"] - b["coordination"]) * n / 2.0
                   for (a, b), n in zip(pairs, ns)])
    ph = np.array([abs(a["packing_fraction"] / b["packing_fraction"] - 1) for a, b in pairs])
    worst = int(np.argmax(ke))
    return {"kinetic_energy_rel_median": float(np.median(ke)),
            "kinetic_energy_rel_p90": float(np.percentile(ke, 90)),
            "kinetic_energy_rel_max": float(ke.max()),
            "scenes_within_1e-3_kinetic_energy": float(np.mean(ke <= 1e-3)),
            "kinetic_energy_rel_to_peak_max": float(ke_pk.max()),
            "kinetic_energy_rel_to_peak_p90": float(np.percentile(ke_pk, 90)),
            "scenes_within_1e-3_kinetic_energy_rel_to_peak": float(np.mean(ke_pk <= 1e-3)),
            "coordination_rel_max": float(zr.max()),
            "coordination_contacts_differing_max": float(zc.max()),
            "scenes_within_1e-3_coordination_or_one_contact": float(np.mean(
                (zr <= 1e-3) | (zc <= 1.0 + 1e-9))),
            "packing_fraction_rel_max": float(ph.max()),
            "worst_kinetic_energy_scene": {"n": int(ns[worst]),
                                           "kinetic_energy_rel": float(ke[worst]),
                                           "rel_to_peak": float(ke_pk[worst])}}


def _plain_run(Scene, w, steps, precision, dt=None, velgrad=None, chunk=500, state=False,
               nudge=False):
    """The plain one-scene-at-a-time path: a fresh scene stepped `steps` times (in
    chunks, recording the peak kinetic energy at the chunk ends); returns its final
    statistics with "ke_peak", and its state if asked.  nudge: every coordinate moved
    by one ulp first (the rounding-level perturbation that measures how far the
    dynamics alone carry a difference of the size FP64 rounding makes)."""
    if nudge:
        import copy
        w = copy.copy(w)
        w.pos = np.nextafter(w.pos, np.inf)
    sc = Scene.from_workload(w, precision=precision, dt=dt)
    if velgrad is not None:
        sc.set_cell_velgrad(velgrad)
    done, peak = 0, 0.0
    while done < steps:
        k = min(chunk, steps - done)
        sc.step(k)
        done += k
        st = sc.stats()
        peak = max(peak, st["kinetic_energy"])
    st["ke_peak"] = peak
    out = (st, sc.state(force=False)) if state else st
    sc.close()
    return out


def run_batch_measure(args, world=1, rank=0):
    """The batched deposition sweep: every scene a sub-scene of one device scene
    (mixed precision, one launch per kernel per step for all of them, launch shapes
    from dem_autotune in the first steps), against the plain FP64 path running the
    same scenes one at a time.  The same batch in FP64 shows the batching itself
    changes nothing: its states are compared bit for bit with the plain runs'.  Under
    several ranks the scenes are dealt out by body count (assign_units), each rank runs
    its share, and the rates are whole-machine (scene-steps of all ranks over the
    slowest rank's time).  Returns the measurement dict (rank 0; None elsewhere)."""
    import workloads
    from paper_2301_00611_gb300 import DEM_FP64, DEM_MIXED, Scene
    ws_all = workloads.batch_depositions(args.batch_scenes, 3, steps=BATCH_STEPS)
    mine = assign_units([w.n for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in mine]
    out = {}
    for label, prec in (("mixed", DEM_MIXED), ("fp64", DEM_FP64)):
        g, subs = _batch_scene(Scene, ws, prec)
        _sync()
        t0 = time.perf_counter()
        shape = g.autotune(steps_per_trial=BATCH_TUNE_STEPS)   # 11 trials of 5 real steps
        done = g.subscene(subs[0])["iter"]
        _sync()
        t_tune = time.perf_counter() - t0
        t0 = time.perf_counter()
        g.step(BATCH_STEPS - done)
        _sync()
        t_batch = time.perf_counter() - t0
        out[label] = {"T": t_batch, "timed": BATCH_STEPS - done, "tune_steps": done,
                      "tune_s": t_tune, "shape": shape,
                      "stats": [g.subscene_stats(q) for q in subs],
                      "states": [g.subscene_state(q) for q in subs] if label == "fp64" else None}
        g.close()
    # plain FP64, one scene at a time (the same full 2000-step jobs)
    t_plain = 0.0
    plain_stats, same = [], 0
    step = max(1, args.batch_plain_every)
    idx = list(range(0, len(ws), step))
    for i in idx:
        _sync()
        t0 = time.perf_counter()
        st, state = _plain_run(Scene, ws[i], BATCH_STEPS, DEM_FP64, state=True)
        _sync()
        t_plain += time.perf_counter() - t0
        plain_stats.append(st)
        b = out["fp64"]["states"][i]
        same += all(np.array_equal(b[k], state[k]) for k in ("pos", "vel", "angvel", "ori"))
    # the chaos floor: the plain FP64 path against itself with every coordinate moved by
    # one ulp, on every 8th scene
    ulp_idx = list(range(0, len(idx), 8))
    pairs_ulp = [(_plain_run(Scene, ws[idx[j]], BATCH_STEPS, DEM_FP64, nudge=True),
                  plain_stats[j]) for j in ulp_idx]
    mx, fp = out["mixed"], out["fp64"]
    local = {"n_scenes": len(ws), "bodies": sum(w.n for w in ws), "T_mixed": mx["T"],
             "pairs_ulp": pairs_ulp, "ns_ulp": [ws[idx[j]].n for j in ulp_idx],
             "T_fp64": fp["T"], "timed_mixed": mx["timed"], "timed_fp64": fp["timed"],
             "t_plain": t_plain, "plain_scenes": len(idx), "same": same,
             "pairs_mixed": [(mx["stats"][i], p) for i, p in zip(idx, plain_stats)],
             "pairs_fp64": [(fp["stats"][i], p) for i, p in zip(idx, plain_stats)],
             "ns": [ws[i].n for i in idx], "tune_steps": mx["tune_steps"],
             "tune_s": mx["tune_s"], "shape": mx["shape"], "shape64": fp["shape"]}
    allr = gather_ranks(local, world)
    if rank != 0:
        return None
    T_mx = max(r["T_mixed"] for r in allr)
    T_fp = max(r["T_fp64"] for r in allr)
    T_pl = max(r["t_plain"] for r in allr)
    n_sc = sum(r["n_scenes"] for r in allr)
    nsum = sum(r["bodies"] for r in allr)
    batched = sum(r["n_scenes"] * r["timed_mixed"] for r in allr) / T_mx
    plain = sum(r["plain_scenes"] for r in allr) * BATCH_STEPS / T_pl
    pm = [p for r in allr for p in r["pairs_mixed"]]
    pf = [p for r in allr for p in r["pairs_fp64"]]
    ns = [n for r in allr for n in r["ns"]]
    compared = sum(r["plain_scenes"] for r in allr)
    return {
        "workload": f"{n_sc} gravity depositions, sizes log-uniform [500, 50000] "
                    f"({nsum} spheres), friction U[0.2, 0.7] rad, E log-uniform [1e6, 1e8] Pa, "
                    f"{BATCH_STEPS} steps each",
        "value": batched, "unit": "scene-steps/s",
        "body_steps_per_s": nsum * allr[0]["timed_mixed"] / T_mx,
        "timed_steps": allr[0]["timed_mixed"], "tuning_steps": allr[0]["tune_steps"],
        "tuning_seconds": allr[0]["tune_s"], "launch_shape": allr[0]["shape"],
        "ranks": world, "scenes_per_rank": [r["n_scenes"] for r in allr],
        "batched_fp64": {"value": sum(r["n_scenes"] * r["timed_fp64"] for r in allr) / T_fp,
                         "unit": "scene-steps/s", "launch_shape": allr[0]["shape64"],
                         "states_bitwise_equal_to_plain": f"{sum(r['same'] for r in allr)} of "
                                                          f"{compared}"},
        "plain_fp64_one_at_a_time": {"value": plain, "unit": "scene-steps/s",
                                     "scenes_timed": compared,
                                     "note": "stepped in chunks of 500 with a statistics read "
                                             "at each chunk end (the peak kinetic energy)"},
        "speedup_vs_plain": batched / plain,
        "accuracy_vs_plain_fp64": {"batched_mixed": _stat_errors(pm, ns),
                                   "batched_fp64": _stat_errors(pf, ns),
                                   "scenes_compared": compared,
                                   "chaos_floor_fp64_one_ulp": _stat_errors(
                                       [p for r in allr for p in r["pairs_ulp"]],
                                       [n for r in allr for n in r["ns_ulp"]]),
                                   "chaos_floor_note": "the plain FP64 path against itself "
                                   "with every coordinate moved by one ulp, every 8th scene: "
                                   "how far the dynamics alone carry a rounding-level "
                                   "difference over the same steps"},
        "dtype": "mixed (batched) vs f64 (plain)",
    }


SERVED_REQUESTS = 100


def served_requests():
    import workloads
    return workloads.serving_requests(SERVED_REQUESTS, 4, 200.0, nmin=1000, nmax=50_000,
                                      smin=500, smax=2000)


def _served_velgrad(rq, w, dt):
    import workloads
    if not w.periodic:
        return None
    return workloads.compaction_rate(0.30, 0.62, rq["steps"], dt) * np.eye(3)


def run_served_measure(args, world=1, rank=0):
    """A short served stream through the library's request server (dem_server_*, mixed
    precision): Poisson arrivals (200/s), spheres log-uniform [1000, 50000], step
    budgets U[500, 2000], depositions and periodic compactions mixed.  Requests are
    submitted in real time at their arrival; latency is completion - arrival.  Beside
    it: the plain FP64 one-scene-at-a-time path as a FIFO queue over the same arrivals
    (measured service times), and the served results' statistics against the plain
    FP64 ones.  Under several ranks each rank serves its share of the requests (dealt
    out by body count)."""
    from paper_2301_00611_gb300 import DEM_FP64, DEM_MIXED, Scene
    from paper_2301_00611_gb300 import serve
    import workloads
    reqs_all = served_requests()
    mine = assign_units([r["n"] for r in reqs_all], world)[rank]
    reqs = [reqs_all[i] for i in mine]
    built = {rq["id"]: workloads.request_workload(rq) for rq in reqs}
    _sync()
    results, summary, wall = serve.serve_stream(reqs, lambda rq: built[rq["id"]], 0, DEM_MIXED,
                                                args.tick_steps, _served_velgrad)
    lat = [results[rq["id"]]["latency"] for rq in reqs]
    # plain FP64 FIFO over the same arrivals
    t_free, plain_lat, busy, pairs, ns = 0.0, [], 0.0, [], []
    for rq in sorted(reqs, key=lambda r: r["arrival"]):
        w = built[rq["id"]]
        dt = serve.pwave_dt(w)
        _sync()
        t0 = time.perf_counter()
        st = _plain_run(Scene, w, rq["steps"], DEM_FP64, dt=dt,
                        velgrad=_served_velgrad(rq, w, dt))
        _sync()
        svc = time.perf_counter() - t0
        busy += svc
        start = max(t_free, rq["arrival"])
        t_free = start + svc
        plain_lat.append(t_free - rq["arrival"])
        pairs.append((results[rq["id"]]["stats"], st))
        ns.append(w.n)
    # chaos floor: the plain FP64 path against itself, coordinates moved by one ulp
    pairs_ulp, ns_ulp = [], []
    by_id = {rq["id"]: k for k, rq in enumerate(sorted(reqs, key=lambda r: r["arrival"]))}
    for rq in reqs[::2]:
        w = built[rq["id"]]
        dt = serve.pwave_dt(w)
        pairs_ulp.append((_plain_run(Scene, w, rq["steps"], DEM_FP64, dt=dt,
                                     velgrad=_served_velgrad(rq, w, dt), nudge=True),
                          pairs[by_id[rq["id"]]][1]))
        ns_ulp.append(w.n)
    scene_steps = sum(rq["steps"] for rq in reqs)
    local = {"lat": lat, "plain_lat": plain_lat, "wall": wall, "busy": busy,
             "scene_steps": scene_steps, "body_steps": summary["body_steps"],
             "pairs": pairs, "ns": ns, "max_resident": summary["max_resident"],
             "pairs_ulp": pairs_ulp, "ns_ulp": ns_ulp,
             "conc": summary["concurrency_mean"], "device_bytes": summary["device_bytes"],
             "conc_hist": summary["concurrency_hist"],
             "budget": summary["budget_bytes"], "rows_per_body": summary["rows_per_body"]}
    allr = gather_ranks(local, world)
    if rank != 0:
        return None
    lat = [x for r in allr for x in r["lat"]]
    plain_lat = [x for r in allr for x in r["plain_lat"]]
    wall = max(r["wall"] for r in allr)
    busy = max(r["busy"] for r in allr)
    ss = sum(r["scene_steps"] for r in allr)
    return {"workload": f"{len(reqs_all)} requests, Poisson 200/s, spheres log-uniform "
                        "[1000, 50000], steps U[500, 2000], deposition/compaction mix",
            "p50_s": serve.percentile(lat, 50), "p99_s": serve.percentile(lat, 99),
            "scene_steps_per_s": ss / wall,
            "body_steps_per_s": sum(r["body_steps"] for r in allr) / wall, "wall_s": wall,
            "concurrency_mean": allr[0]["conc"], "concurrency_max": allr[0]["max_resident"],
            "concurrency_hist": _conc_hist(allr[0]["conc_hist"]),
            "admission": {"budget_bytes": allr[0]["budget"],
                          "device_bytes_max": allr[0]["device_bytes"],
                          "rows_per_body_estimate": allr[0]["rows_per_body"]},
            "dtype": "mixed", "ranks": world,
            "plain_fp64_fifo": {"p50_s": serve.percentile(plain_lat, 50),
                                "p99_s": serve.percentile(plain_lat, 99),
                                "scene_steps_per_s": ss / busy, "dtype": "f64"},
            "accuracy_vs_plain_fp64": _stat_errors([p for r in allr for p in r["pairs"]],
                                                   [n for r in allr for n in r["ns"]]),
            "chaos_floor_fp64_one_ulp": _stat_errors([p for r in allr for p in r["pairs_ulp"]],
                                                     [n for r in allr for n in r["ns_ulp"]])}


def _conc_hist(hist):
    """The server's ticks by resident requests, keyed by the bins' ranges."""
    from paper_2301_00611_gb300.dem import CONCURRENCY_BIN_EDGES as edges
    out, lo = {}, 1
    for hi, n in zip(edges, hist):
        out[str(lo) if hi == lo else (f"{lo}-{hi}" if hi else f">{lo - 1}")] = n
        lo = (hi or lo) + 1
    return out


def run_serve(args):
    """Serving (config 4): a Poisson stream of deposition / compaction requests (spheres
    log-uniform [1000, 200000], steps U[500, 5000]) replayed in real time against the
    library's request server (dem_server_*, mixed precision, admission by device
    footprint within --serve-budget-gb), then the same requests through the plain FP64
    one-scene-at-a-time path as a FIFO queue over the same arrivals."""
    import multiprocessing as mp
    import workloads
    reqs = workloads.serving_requests(args.requests, 4, args.rate)
    # the requests' scenes are built client-side before the clock starts, in a spawned
    # process pool created before this process touches the GPU
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        built = dict(zip([r["id"] for r in reqs], pool.map(workloads.request_workload, reqs)))
    import torch
    from paper_2301_00611_gb300 import DEM_FP64, DEM_MIXED, Scene
    from paper_2301_00611_gb300 import serve
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    budget = int(args.serve_budget_gb * 2 ** 30)
    results, summary, wall = serve.serve_stream(reqs, lambda rq: built[rq["id"]], budget,
                                                DEM_MIXED, args.tick_steps, _served_velgrad)
    lat = [r["latency"] for r in results.values()]
    t_free, plain_lat, busy = 0.0, [], 0.0
    for rq in sorted(reqs, key=lambda r: r["arrival"]):
        w = built[rq["id"]]
        dt = serve.pwave_dt(w)
        _sync()
        t0 = time.perf_counter()
        serve.run_alone(w, rq["steps"], DEM_FP64, _served_velgrad(rq, w, dt), dt=dt)
        _sync()
        svc = time.perf_counter() - t0
        busy += svc
        start = max(t_free, rq["arrival"])
        t_free = start + svc
        plain_lat.append(t_free - rq["arrival"])
    scene_steps = sum(rq["steps"] for rq in reqs)
    line = {
        "metric": "served p50/p99 latency and scene-steps/s (Poisson request stream)",
        "value": serve.percentile(lat, 99), "unit": "s (p99 latency)",
        "higher_is_better": False, "n_gpus": 1, "data": "synthetic (seeded)",
        "config": {"workload": f"{len(reqs)} requests, Poisson {args.rate}/s, spheres "
                               "log-uniform [1000, 200000], steps U[500, 5000], "
                               "deposition/compaction mix",
                   "budget_bytes": summary["budget_bytes"], "tick_steps": args.tick_steps},
        "served": {"p50_s": serve.percentile(lat, 50), "p99_s": serve.percentile(lat, 99),
                   "scene_steps_per_s": scene_steps / wall, "wall_s": wall,
                   "body_steps_per_s": summary["body_steps"] / wall,
                   "concurrency_mean": summary["concurrency_mean"],
                   "concurrency_max": summary["max_resident"], "ticks": summary["ticks"],
                   "concurrency_hist": _conc_hist(summary["concurrency_hist"]),
                   "device_bytes_max": summary["device_bytes"],
                   "rows_per_body_estimate": summary["rows_per_body"], "dtype": "mixed"},
        "plain_fp64_fifo": {"p50_s": serve.percentile(plain_lat, 50),
                            "p99_s": serve.percentile(plain_lat, 99),
                            "scene_steps_per_s": scene_steps / busy, "dtype": "f64"},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- triaxial loading

TRIAX_N = 4_000_000
# the triaxial case folded into the headline line: the same loading at one million
# spheres (seeding the four-million-sphere cloud alone takes about a minute on the host)
TRIAX_HEADLINE_N = 1_000_000
TRIAX_LOAD_STEPS = 10_000
TRIAX_WORKLOAD = ("triaxial loading of a dense periodic packing: {n} spheres, radii uniform "
                  "[0.8, 1.2] mm, friction 0.5 rad, 1% axial strain per 10,000 steps, lateral "
                  "stresses held by the cell servo, 10,000 loading steps")


def run_triax(args):
    n = args.n if args.n is not None else TRIAX_N
    print(json.dumps(triax_measure(args, n, args.steps)), flush=True)
    return 0


def triax_measure(args, n, steps=None):
    """The four-million-sphere triaxial case in mixed precision.  Untimed preparation: a
    seeded loose cloud (solid fraction 0.3) compacted isotropically over 3000 steps and
    relaxed for 300; the lateral stress it reaches becomes the servo's goal.  Loading:
    axial strain rate 1e-6 per step, lateral stresses held by the stress servo (every 5
    steps), 10,000 steps of which the launch shapes are tuned on real steps near the
    start and the last K are timed with CUDA events."""
    import torch
    import workloads
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_00611_gb300 import Scene, DEM_MIXED
    peak, peak_kind = _peaks()
    w = workloads.periodic_cloud(n, 2, phi=0.3, rmin=0.8e-3, rmax=1.2e-3, friction=0.5)
    s = Scene.from_workload(w, precision=DEM_MIXED)
    dt = s.dt()
    rate = workloads.compaction_rate(0.3, 0.64, 3000, dt)
    s.set_cell_velgrad(np.diag([rate, rate, rate]))
    s.step(3000)
    s.set_cell_velgrad(np.zeros((3, 3)))
    s.step(300)
    st = s.stats()
    lateral = float(np.mean(np.diag(st["stress"])[:2]))
    axial = -0.01 / (10000 * dt)
    s.set_triax([lateral, lateral, axial], 0b011, [10 * abs(axial)] * 3, 0.25, 5)
    it0 = s.clock()[0]
    H_load = s.cell()["H"]
    s.step(20)
    if args.shape_mixed:
        cb, cps, ib, deg = (int(v) for v in args.shape_mixed.split(","))
        shape = {"contact_block": cb, "contact_blocks_per_sm": cps, "integrate_block": ib,
                 "degree_order": deg}
        s.set_tuning(**shape)
    elif args.no_autotune:
        shape = None
    else:
        shape = s.autotune(steps_per_trial=TUNE_STEPS)
    W = args.warmup
    done = s.clock()[0] - it0
    K = TRIAX_LOAD_STEPS - done - W if steps is None else steps
    s.step(W)
    st0 = s.stats()
    s.set_timing(True)
    t_before = s.timing()["kernel_launches"]
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        s.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tm = s.timing()
    st1 = s.stats()
    sig = np.diag(st1["stress"])
    H = s.cell()["H"]
    s.close()
    res = {"tm": tm, "mean_real": 0.5 * (st0["n_contacts"] + st1["n_contacts"]),
           "avg_ms": tm["contact_ms"] / max(1, tm["contact_launches"]),
           "rows_avg": tm["rows_processed"] / max(1, tm["contact_launches"])}
    rl, rk = _kernel_rooflines(res, "mixed", n, peak, peak_kind, traffic=False)
    T = ms / 1e3
    line = {
        "metric": f"body-steps/s ({n}-sphere triaxial loading, mixed precision)",
        "value": n * K / T, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed: f32 contact geometry/law, f64 shear history, integration and "
                 "reductions",
        "data": "synthetic (seeded)",
        "config": {"workload": TRIAX_WORKLOAD.format(n=n), "n_bodies": n, "dt": dt,
                   "timed_window": f"last {K} of the {done + W + K} loading steps "
                                   f"({done} tuning/settling and {W} warm-up untimed)",
                   "preparation": "compaction 0.3 -> dense over 3000 steps, 300 steps of "
                                  "relaxation (untimed)",
                   "packing_fraction_at_load": st["packing_fraction"],
                   "l2": f"working set > L2 (bodies ~{n * 200 / 1e9:.1f} GB + contact table)",
                   "parallelism": "single GPU"},
        "contact_updates_per_s": res["mean_real"] * K / T,
        "candidate_rows_per_s": tm["rows_processed"] / T,
        "contacts": {"start": st0["n_contacts"], "end": st1["n_contacts"]},
        "servo": {"lateral_goal": lateral, "lateral_end": [float(sig[0]), float(sig[1])],
                  "axial_strain_end": float(H[2, 2] / H_load[2, 2] - 1.0)},
        "phase_share": {k: tm[k] / max(1e-9, ms) for k in ("contact_ms", "integrate_ms",
                                                           "cell_ms", "collider_ms")},
        "collider_runs": tm["collider_runs"],
        "gpu_launches": tm["kernel_launches"] - t_before,
        "launch_shape": shape,
        "clocks": clk.summary(),
        "roofline": rl,
        "roofline_kernels": rk,
    }
    return line


def compaction_1a_measure(args, Scene, peak, peak_kind, fp64_peak):
    """Config "1a": the 1M compaction at the stated strain rate, 1e-2 per second (the
    cell barely moves in 5000 steps: the packing stays a loose cloud near 0.30), FP64;
    every step after the warm-up is timed."""
    w = make_workload(N_BODIES)   # the same seeded cloud; only the loading differs
    rate = -1e-2
    res = _time_window(Scene, w, args, "fp64", 1, 0, None,
                       velgrad=lambda dt: np.diag([rate, rate, rate]),
                       K=JOB_STEPS - args.warmup)
    rl, _ = _kernel_rooflines(res, "fp64", w.n, peak, peak_kind, traffic=False,
                              fp64_peak=fp64_peak)
    K = res["K"]
    return {"workload": f"periodic isotropic compaction at the stated strain rate 1e-2/s, "
                        f"1M log-normal spheres, 5000 steps (FP64)",
            "value": w.n * K / res["T"], "unit": UNIT, "ms_per_step": res["ms"] / K,
            "timed_window": f"last {K} steps after {args.warmup} warm-up",
            "contacts": {"start": res["st0"]["n_contacts"], "end": res["st1"]["n_contacts"]},
            "packing_fraction_end": res["st1"]["packing_fraction"],
            "contact_updates_per_s": res["mean_real"] * K / res["T"],
            "collider_runs": res["tm"]["collider_runs"], "clocks": res["clocks"],
            "roofline": rl}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the rest of the job after the warm-up)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="spheres (default: 1M; 4M in the triaxial mode)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of dem_autotune's")
    ap.add_argument("--shape-fp64", default=None,
                    help="launch shape 'contact_block,blocks_per_sm,integrate_block,degree_order' "
                         "of the FP64 run instead of the autotuner's")
    ap.add_argument("--shape-mixed", default=None, help="the same for the mixed run")
    ap.add_argument("--mode", default="headline",
                    choices=["headline", "batch", "serve", "triax"])
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched deposition sweep out of the headline line")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the served request stream out of the headline line")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave the 4M triaxial loading and config 1a out of the headline line")
    ap.add_argument("--batch-scenes", type=int, default=BATCH_SCENES)
    ap.add_argument("--batch-plain-every", type=int, default=1,
                    help="time the plain FP64 path on every k-th scene of the sweep")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0,
                    help="device-memory budget of the serve mode's resident requests")
    ap.add_argument("--tick-steps", type=int, default=200)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.mode == "triax" and args.impl == "ours":
        return run_triax(args)
    if args.n is None:
        args.n = N_BODIES
    if args.steps is None:
        args.steps = JOB_STEPS - args.warmup
    if args.impl == "reference":   # the oracle on the headline workload, whatever the mode
        return run_reference(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "batch":
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps({"metric": "batched deposition sweep", **run_batch_measure(args)}),
              flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
