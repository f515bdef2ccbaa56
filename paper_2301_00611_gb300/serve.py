"""Serving helpers over the library's request server (``dem_server_*``).

The server itself -- admission by device footprint, ticks, retirement, latency
accounting -- runs in the C++ library (``csrc/server_sched.h``, ``csrc/server.cu``)
on its own worker thread; ``Server`` in ``dem.py`` marshals its calls.  This module
adds what a client of it does: replay a request stream in real time (each request
submitted when the wall clock passes its arrival), collect every result, and the
plain one-scene-at-a-time path it is compared against.

The paper has no serving layer; this is the batching/serving pattern applied to
its hot path.
"""
from __future__ import annotations

import time

import numpy as np

from .dem import DEM_FP64, DEM_MIXED, Scene, Server


def pwave_dt(w, factor=None):
    """The workload's step: dt_factor x min r sqrt(rho / E) over its spheres (the
    p-wave critical step of utils.PWaveTimeStep).  Passing the same explicit dt to the
    served and the alone run makes their clocks identical by construction."""
    rho = np.array([m.density for m in w.materials])[w.mat_id]
    E = np.array([m.young for m in w.materials])[w.mat_id]
    f = w.dt_factor if factor is None else factor
    return float(f * np.min(w.radius * np.sqrt(rho / E)))


def percentile(values, p):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, p))


def serve_stream(requests, make_workload, budget_bytes=0, precision=DEM_MIXED, tick_steps=200,
                 velgrad_for=None, keep_state=False, time_scale=1.0, explicit_dt=True):
    """Replay a request stream in real time against a new server: request k is
    submitted when the wall clock passes requests[k]["arrival"] x time_scale seconds
    after the start.  make_workload(rq) -> workload; velgrad_for(rq, w, dt) -> 3x3 or
    None.  Returns (results by request id, server summary, wall seconds); a result
    holds the request's latency (completion - submission, measured by the server),
    its statistics and, with keep_state, its final state."""
    order = sorted(requests, key=lambda r: r["arrival"])
    built = [(rq, make_workload(rq)) for rq in order]
    tickets = {}
    with Server(precision=precision, budget_bytes=budget_bytes, tick_steps=tick_steps) as srv:
        t0 = time.perf_counter()
        for rq, w in built:
            delay = rq["arrival"] * time_scale - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            dt = pwave_dt(w) if explicit_dt else 0.0
            vg = velgrad_for(rq, w, dt) if velgrad_for else None
            tickets[rq["id"]] = srv.submit(w, rq["steps"], velgrad=vg, keep_state=keep_state,
                                           dt=dt)
        results = {}
        for rid, t in tickets.items():
            srv.wait(t)
            results[rid] = srv.result(t, state=keep_state)
            srv.release(t)
        wall = time.perf_counter() - t0
        summary = srv.stats()
    return results, summary, wall


def run_alone(w, steps, precision=DEM_FP64, velgrad=None, dt=None, state=False):
    """The one-scene-at-a-time path: a fresh scene, `steps` steps; its statistics (and
    its final state with state=True)."""
    s = Scene.from_workload(w, precision=precision, dt=dt)
    if velgrad is not None:
        s.set_cell_velgrad(velgrad)
    s.step(steps)
    st = s.stats()
    out = (st, s.state(force=False)) if state else st
    s.close()
    return out


__all__ = ["Server", "serve_stream", "run_alone", "percentile", "pwave_dt", "DEM_FP64",
           "DEM_MIXED"]
