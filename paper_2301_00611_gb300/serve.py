"""Continuous-batching DEM server over the C ABI.

Requests (a scene and a step budget) are admitted as sub-scenes of one device
scene while its body budget has room, advanced together by the same launches tick
by tick (one ``dem_step`` per tick for every resident scene), and retired when
their budget is spent: the final state and statistics are copied to the host and
the sub-scene is removed, which frees room for the requests still waiting.  Scene
state never leaves the device between ticks.  A tick is the smallest remaining
budget among the resident scenes, capped by ``tick_steps``, so no scene overshoots
its budget and a finished scene leaves at the end of the tick it finished in.

The paper has no serving layer; this is the batching/serving pattern applied to
its hot path.  All stepping runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from .dem import DEM_FP64, DEM_MIXED, Scene

MATERIAL_SLOTS = 4000   # material ids handed to resident scenes (library limit 4096)


@dataclass
class Result:
    """Outcome of one request."""
    rid: int
    n: int
    steps: int
    arrival: float          # seconds since the server started
    admitted: float
    finished: float
    stats: dict
    state: dict | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Resident:
    rid: int
    sub: int
    n: int
    steps: int
    left: int
    arrival: float
    admitted: float
    mat_base: int
    mat_count: int
    keep_state: bool


@dataclass
class Server:
    """capacity_bodies: spheres resident at once (the device footprint budget: bodies
    and, through the contact table, their contacts).  precision: DEM_MIXED or DEM_FP64.
    tick_steps: upper bound of the steps between two admission points."""
    capacity_bodies: int
    precision: int = DEM_MIXED
    tick_steps: int = 200
    keep_state: bool = False
    scene: object = None    # a Scene-like object (tests pass a host fake); default: a new Scene
    _scene: Scene = field(init=False, repr=False)
    _waiting: list = field(default_factory=list, init=False, repr=False)
    _resident: list = field(default_factory=list, init=False, repr=False)
    _free_mats: list = field(default_factory=list, init=False, repr=False)
    results: list = field(default_factory=list, init=False)
    resident_bodies: int = field(default=0, init=False)
    scene_steps: int = field(default=0, init=False)
    body_steps: int = field(default=0, init=False)
    ticks: int = field(default=0, init=False)
    concurrency: list = field(default_factory=list, init=False)

    def __post_init__(self):
        # sub-scene 0 is an empty placeholder: every request becomes its own sub-scene
        if self.scene is None:
            self.scene = Scene(capacity_bodies=self.capacity_bodies, precision=self.precision,
                               dt=1.0)
        self._scene = self.scene
        self._scene.set_material(0, 1000.0, 1e6, 0.25, 0.5)
        self._free_mats = [(1, MATERIAL_SLOTS - 1)]
        self._t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self._t0

    # --- material ids (each resident scene gets its own range)
    def _alloc_mats(self, k):
        for i, (a, m) in enumerate(self._free_mats):
            if m >= k:
                self._free_mats[i] = (a + k, m - k)
                return a
        raise RuntimeError("material table exhausted")

    def _free_mat_range(self, a, k):
        self._free_mats.append((a, k))
        self._free_mats.sort()
        merged = []
        for s, m in self._free_mats:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + m)
            elif m > 0:
                merged.append((s, m))
        self._free_mats = merged

    # --- requests
    def submit(self, rid, workload, steps, arrival=None, velgrad=None, keep_state=None):
        """Queue a request: `workload` (a workloads.Workload) advanced by `steps` steps.
        velgrad: callable dt -> 3x3 velocity gradient of a periodic scene (or None)."""
        if workload.n > self.capacity_bodies:
            raise ValueError("request larger than the server's body budget")
        self._waiting.append((rid, workload, int(steps), self.now() if arrival is None else arrival,
                              velgrad, self.keep_state if keep_state is None else keep_state))

    def _admit(self):
        """Admit waiting requests in arrival order while they fit (first come, first
        served: a request that does not fit blocks those behind it, so none starves)."""
        admitted = False
        while self._waiting:
            rid, w, steps, arrival, velgrad, keep = self._waiting[0]
            if self.resident_bodies + w.n > self.capacity_bodies:
                break
            self._waiting.pop(0)
            base = self._alloc_mats(len(w.materials))
            sub = self._scene.add_workload(w, material_base=base)
            if velgrad is not None:
                dt = self._scene.subscene(sub)["dt"]
                self._scene.set_subscene_velgrad(sub, velgrad(dt))
            self._resident.append(_Resident(rid, sub, w.n, steps, steps, arrival, self.now(),
                                            base, len(w.materials), keep))
            self.resident_bodies += w.n
            admitted = True
        return admitted

    def _retire(self):
        done = [r for r in self._resident if r.left == 0]
        # read every finished scene before removing any (a removal changes the layout
        # until the next step)
        out = [(r, self._scene.subscene_stats(r.sub),
                self._scene.subscene_state(r.sub) if r.keep_state else None) for r in done]
        t = self.now()
        for r, st, state in out:
            self._scene.remove_subscene(r.sub)
            self._free_mat_range(r.mat_base, r.mat_count)
            self.resident_bodies -= r.n
            self.results.append(Result(r.rid, r.n, r.steps, r.arrival, r.admitted, t, st, state))
        self._resident = [r for r in self._resident if r.left > 0]

    def tick(self):
        """Admit what fits, advance every resident scene by one tick, retire the
        finished ones.  Returns the number of steps advanced (0 when idle)."""
        self._admit()
        if not self._resident:
            return 0
        k = min(self.tick_steps, min(r.left for r in self._resident))
        self._scene.step(k)
        self.ticks += 1
        self.concurrency.append(len(self._resident))
        for r in self._resident:
            r.left -= k
            self.scene_steps += k
            self.body_steps += k * r.n
        self._retire()
        return k

    @property
    def idle(self):
        return not self._waiting and not self._resident

    def close(self):
        self._scene.close()


def percentile(values, p):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, p))


def serve_stream(requests, make_workload, capacity_bodies, precision=DEM_MIXED, tick_steps=200,
                 velgrad_for=None, keep_state=False, time_scale=1.0, scene=None):
    """Replay a request stream in real time: each request is submitted when the wall
    clock passes its arrival (times scaled by time_scale), the server ticks in
    between.  Returns (server, wall seconds)."""
    srv = Server(capacity_bodies, precision, tick_steps, keep_state, scene)
    order = sorted(requests, key=lambda r: r["arrival"])
    i = 0
    t0 = srv.now()
    while i < len(order) or not srv.idle:
        now = srv.now() - t0
        while i < len(order) and order[i]["arrival"] * time_scale <= now:
            rq = order[i]
            w = make_workload(rq)
            vg = velgrad_for(rq, w) if velgrad_for else None
            srv.submit(rq["id"], w, rq["steps"], arrival=t0 + rq["arrival"] * time_scale,
                       velgrad=vg)
            i += 1
        if srv.tick() == 0 and i < len(order):
            wait = order[i]["arrival"] * time_scale - (srv.now() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
    return srv, srv.now() - t0


def run_alone(w, steps, precision=DEM_FP64, velgrad=None):
    """The one-scene-at-a-time path: a fresh scene, `steps` steps, its statistics."""
    s = Scene.from_workload(w, precision=precision)
    if velgrad is not None:
        s.set_cell_velgrad(velgrad(s.dt()))
    s.step(steps)
    st = s.stats()
    s.close()
    return st


__all__ = ["Server", "Result", "serve_stream", "run_alone", "percentile", "DEM_FP64",
           "DEM_MIXED"]
