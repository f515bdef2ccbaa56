"""Seeded synthetic inputs shared by the DEM oracle, the CUDA path, the tests and the bench.

This module holds input generation only -- sphere clouds, radius
distributions and the material/loading parameters of each workload -- and
none of the method's arithmetic (no contact law, no integrator, no time-step
rule).  Both sides of every parity comparison take their inputs from here.

Workloads (the Yade text's tutorial setups, scaled; every one is synthetic):

* ``deposition``  -- gravity deposition in a walled box (the loose-cloud and
  box setup of the Yade tutorial; ``utils.aabbWalls`` around a
  ``SpherePack.makeCloud`` cloud).
* ``compaction``  -- loose periodic cloud under isotropic compaction by a
  constant cell velocity gradient (section 2.1.6, ``Cell.velGrad``).
* ``periodic_cloud`` / ``box_cloud`` -- small clouds for parity tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "rsa.c")
_LIB = os.path.join(_HERE, "librsa.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the placement helper with gcc (no FMA contraction, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.wl_rsa_place.restype = ctypes.c_int
        lib.wl_rsa_place.argtypes = [ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_long, ctypes.c_void_p]
        lib.wl_uniform.restype = None
        lib.wl_uniform.argtypes = [ctypes.c_long, ctypes.c_uint64, ctypes.c_void_p]
        _lib = lib
    return _lib


def uniform(n: int, seed: int) -> np.ndarray:
    """n uniform [0,1) doubles from splitmix64(seed): identical on every platform."""
    out = np.empty(int(n), dtype=np.float64)
    if n:
        _load().wl_uniform(int(n), int(seed) & (2**64 - 1), out.ctypes.data)
    return out


def rsa_place(radius: np.ndarray, lo, hi, periodic: bool, seed: int,
              max_attempts: int = 200000) -> np.ndarray:
    """Random sequential placement of non-overlapping spheres (makeCloud-like)."""
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    pos = np.zeros((radius.size, 3), dtype=np.float64)
    rc = _load().wl_rsa_place(radius.size, radius.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                              int(bool(periodic)), int(seed) & (2**64 - 1), int(max_attempts),
                              pos.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"rsa_place failed (code {rc}): cloud too dense for the box")
    return pos


@dataclass
class Material:
    density: float
    young: float
    poisson: float          # ks/kn ratio (ElastMat.poisson)
    friction: float         # friction angle [rad]


@dataclass
class Workload:
    """One seeded scene: geometry, materials and loading; no derived physics."""
    name: str
    pos: np.ndarray                      # (n,3) float64
    radius: np.ndarray                   # (n,)  float64
    mat_id: np.ndarray                   # (n,)  int32
    materials: list
    periodic: bool
    cell: np.ndarray                     # (3,3) column base vectors (periodic only)
    box_lo: np.ndarray
    box_hi: np.ndarray
    wall_mask: int                       # bit 2*axis + side: 6 axis-aligned walls
    gravity: np.ndarray
    damping: float
    dt_factor: float                     # dt = dt_factor * p-wave critical step
    steps: int
    velgrad: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    vel: np.ndarray | None = None
    angvel: np.ndarray | None = None
    note: str = ""

    @property
    def n(self) -> int:
        return int(self.radius.size)


def _lognormal_clipped(n, median, sigma, lo, hi, seed):
    rng = np.random.default_rng(seed)
    r = rng.lognormal(mean=np.log(median), sigma=sigma, size=n)
    return np.clip(r, lo, hi)


def deposition(n: int = 1000, seed: int = 0, box=(0.3, 0.3, 0.6), rmin=0.009, rmax=0.011,
               density=2600.0, young=5e7, poisson=0.25, friction=np.deg2rad(30.0),
               damping=0.2, steps=2000) -> Workload:
    """Gravity deposition: n spheres, radii U[rmin,rmax], random non-overlapping cloud in a
    walled box (6 walls on the box faces), g = -9.81 z, dt = 0.5 p-wave step."""
    u = uniform(n, seed * 7919 + 1)
    radius = rmin + u * (rmax - rmin)
    lo = np.zeros(3)
    hi = np.asarray(box, dtype=np.float64)
    pos = rsa_place(radius, lo, hi, periodic=False, seed=seed * 104729 + 3)
    return Workload(name=f"deposition_n{n}_s{seed}", pos=pos, radius=radius,
                    mat_id=np.zeros(n, dtype=np.int32),
                    materials=[Material(density, young, poisson, friction)],
                    periodic=False, cell=np.diag(hi), box_lo=lo, box_hi=hi, wall_mask=0x3F,
                    gravity=np.array([0.0, 0.0, -9.81]), damping=damping, dt_factor=0.5,
                    steps=steps)


def compaction_rate(phi0: float, phi1: float, steps: int, dt: float) -> float:
    """Diagonal velocity-gradient entry g such that (1+g*dt)^(3*steps) = phi0/phi1
    (the cell volume ratio needed to take the solid fraction from phi0 to phi1).
    Loading-path parameter of the workload, not part of the method."""
    return ((phi0 / phi1) ** (1.0 / (3.0 * steps)) - 1.0) / dt


def compaction(n: int = 1_000_000, seed: int = 1, phi0: float = 0.3, phi_target: float = 0.62,
               variant: str = "b", steps: int = 5000, density=2600.0, young=5e7, poisson=0.25,
               friction=np.deg2rad(30.0), damping=0.2, median=1e-3, sigma=0.25,
               rclip=(0.5e-3, 2e-3)) -> Workload:
    """Isotropic compaction of a loose periodic cloud.

    Radii log-normal (median 1 mm, sigma 0.25, clipped to [0.5, 2] mm), random
    non-overlapping cloud at solid fraction phi0 in a periodic cube, g = 0,
    damping 0.2.  Variant "a": strain rate 1e-2 per unit time (as stated; the
    fraction barely moves in 5000 steps).  Variant "b": the constant rate that
    brings the fraction to phi_target at the last step (set by the caller once
    dt is known: ``velgrad`` is left zero and ``note`` says so).
    """
    radius = _lognormal_clipped(n, median, sigma, rclip[0], rclip[1], seed * 7919 + 11)
    vs = float(np.sum(4.0 / 3.0 * np.pi * radius ** 3))
    L = (vs / phi0) ** (1.0 / 3.0)
    lo = np.zeros(3)
    hi = np.full(3, L)
    pos = rsa_place(radius, lo, hi, periodic=True, seed=seed * 104729 + 13)
    vg = np.zeros((3, 3))
    if variant == "a":
        vg = -1e-2 * np.eye(3)
    return Workload(name=f"compaction{variant}_n{n}_s{seed}", pos=pos, radius=radius,
                    mat_id=np.zeros(n, dtype=np.int32),
                    materials=[Material(density, young, poisson, friction)],
                    periodic=True, cell=np.diag(hi), box_lo=lo, box_hi=hi, wall_mask=0,
                    gravity=np.zeros(3), damping=damping, dt_factor=0.5, steps=steps,
                    velgrad=vg, note=f"phi0={phi0} phi_target={phi_target} variant={variant}")


def periodic_cloud(n: int, seed: int, phi: float = 0.3, rmin=0.8e-3, rmax=1.2e-3,
                   friction=0.5, young=5e7, density=2600.0, poisson=0.25, damping=0.2,
                   vel_scale=0.0, angvel_scale=0.0, inflate=1.0) -> Workload:
    """Small periodic cloud with uniform radii and optional random velocities (parity tests).
    ``inflate`` > 1 scales every radius after placement, so that neighbours overlap and the
    first step already has a contact network."""
    u = uniform(n, seed * 31 + 5)
    radius = rmin + u * (rmax - rmin)
    vs = float(np.sum(4.0 / 3.0 * np.pi * radius ** 3))
    L = (vs / phi) ** (1.0 / 3.0)
    lo = np.zeros(3)
    hi = np.full(3, L)
    pos = rsa_place(radius, lo, hi, periodic=True, seed=seed * 7 + 17)
    radius = radius * inflate
    vel = angvel = None
    if vel_scale:
        vel = (uniform(3 * n, seed * 13 + 19).reshape(n, 3) - 0.5) * 2 * vel_scale
    if angvel_scale:
        angvel = (uniform(3 * n, seed * 17 + 23).reshape(n, 3) - 0.5) * 2 * angvel_scale
    return Workload(name=f"pcloud_n{n}_s{seed}", pos=pos, radius=radius,
                    mat_id=np.zeros(n, dtype=np.int32),
                    materials=[Material(density, young, poisson, friction)],
                    periodic=True, cell=np.diag(hi), box_lo=lo, box_hi=hi, wall_mask=0,
                    gravity=np.zeros(3), damping=damping, dt_factor=0.5, steps=0,
                    vel=vel, angvel=angvel)


def box_cloud(n: int, seed: int, phi: float = 0.2, rmin=0.8e-3, rmax=1.2e-3, aspect=(1, 1, 2),
              friction=0.5, young=5e7, density=2600.0, poisson=0.25, damping=0.2,
              gravity=(0.0, 0.0, -9.81), wall_mask=0x3F, vel_scale=0.0, angvel_scale=0.0,
              two_materials=False, inflate=1.0) -> Workload:
    """Small walled-box cloud (parity tests); optionally two materials assigned at random.
    ``inflate`` > 1 scales every radius after placement (overlapping neighbours and, near the
    faces, sphere-wall overlaps)."""
    u = uniform(n, seed * 31 + 7)
    radius = rmin + u * (rmax - rmin)
    vs = float(np.sum(4.0 / 3.0 * np.pi * radius ** 3))
    a = np.asarray(aspect, dtype=np.float64)
    s = (vs / phi / np.prod(a)) ** (1.0 / 3.0)
    lo = np.zeros(3)
    hi = a * s
    pos = rsa_place(radius, lo, hi, periodic=False, seed=seed * 7 + 29)
    radius = radius * inflate
    mats = [Material(density, young, poisson, friction)]
    mat_id = np.zeros(n, dtype=np.int32)
    if two_materials:
        mats.append(Material(1.5 * density, 2.0 * young, 0.3, 0.7 * friction))
        mat_id = (uniform(n, seed * 41 + 3) < 0.5).astype(np.int32)
    vel = angvel = None
    if vel_scale:
        vel = (uniform(3 * n, seed * 13 + 31).reshape(n, 3) - 0.5) * 2 * vel_scale
    if angvel_scale:
        angvel = (uniform(3 * n, seed * 17 + 37).reshape(n, 3) - 0.5) * 2 * angvel_scale
    return Workload(name=f"bcloud_n{n}_s{seed}", pos=pos, radius=radius, mat_id=mat_id,
                    materials=mats, periodic=False, cell=np.diag(hi), box_lo=lo, box_hi=hi,
                    wall_mask=wall_mask, gravity=np.asarray(gravity, dtype=np.float64),
                    damping=damping, dt_factor=0.5, steps=0, vel=vel, angvel=angvel)


def scaled_deposition(n: int, seed: int, friction: float, young: float, rmin=0.009, rmax=0.011,
                      solid_fraction=0.078, aspect=(1.0, 1.0, 2.0), density=2600.0,
                      poisson=0.25, damping=0.2, steps=2000) -> Workload:
    """Gravity deposition with the box scaled to n: aspect 1:1:2 and the solid fraction
    of the 1000-sphere deposition (7.8%), so every scene is that one at another size."""
    u = uniform(n, seed * 7919 + 17)
    radius = rmin + u * (rmax - rmin)
    vs = float(np.sum(4.0 / 3.0 * np.pi * radius ** 3))
    a = np.asarray(aspect, dtype=np.float64)
    side = (vs / solid_fraction / float(np.prod(a))) ** (1.0 / 3.0)
    hi = side * a
    lo = np.zeros(3)
    pos = rsa_place(radius, lo, hi, periodic=False, seed=seed * 104729 + 19)
    return Workload(name=f"deposition_n{n}_s{seed}", pos=pos, radius=radius,
                    mat_id=np.zeros(n, dtype=np.int32),
                    materials=[Material(density, young, poisson, friction)],
                    periodic=False, cell=np.diag(hi), box_lo=lo, box_hi=hi, wall_mask=0x3F,
                    gravity=np.array([0.0, 0.0, -9.81]), damping=damping, dt_factor=0.5,
                    steps=steps)


def batch_parameters(n_scenes: int = 512, seed: int = 3, nmin: int = 500, nmax: int = 50_000):
    """Per-scene sizes and materials of the batched deposition sweep: sphere counts
    log-uniform in [nmin, nmax], friction angle uniform in [0.2, 0.7] rad, Young's
    modulus log-uniform in [1e6, 1e8] Pa (one splitmix64 stream per quantity)."""
    u = uniform(3 * n_scenes, seed * 7919 + 23).reshape(3, n_scenes)
    n = np.floor(np.exp(np.log(nmin) + u[0] * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    friction = 0.2 + 0.5 * u[1]
    young = np.exp(np.log(1e6) + u[2] * (np.log(1e8) - np.log(1e6)))
    return n, friction, young


def batch_depositions(n_scenes: int = 512, seed: int = 3, nmin: int = 500, nmax: int = 50_000,
                      steps: int = 2000) -> list:
    """The batched sweep: one scaled deposition per scene (see batch_parameters)."""
    n, fr, E = batch_parameters(n_scenes, seed, nmin, nmax)
    return [scaled_deposition(int(n[k]), seed * 100003 + k, float(fr[k]), float(E[k]), steps=steps)
            for k in range(n_scenes)]


def serving_requests(n_requests: int = 2000, seed: int = 4, rate: float = 200.0,
                     nmin: int = 1000, nmax: int = 200_000, smin: int = 500, smax: int = 5000):
    """Request stream of the serving workload: Poisson arrivals (exponential gaps of
    mean 1/rate), sphere counts log-uniform in [nmin, nmax], step budgets uniform in
    [smin, smax], kind alternating at random between a scaled gravity deposition and a
    periodic compaction, friction angle U[0.2, 0.7] rad, Young's modulus
    log-uniform [1e6, 1e8] Pa.  Returns a list of dicts (no spheres yet: a request's
    scene is built by request_workload when it is submitted)."""
    u = uniform(6 * n_requests, seed * 7919 + 29).reshape(6, n_requests)
    gaps = -np.log1p(-u[0]) / rate
    t = np.cumsum(gaps) - gaps[0]
    n = np.floor(np.exp(np.log(nmin) + u[1] * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    steps = (smin + np.floor(u[2] * (smax - smin + 1))).astype(np.int64)
    kind = np.where(u[3] < 0.5, "deposition", "compaction")
    fr = 0.2 + 0.5 * u[4]
    E = np.exp(np.log(1e6) + u[5] * (np.log(1e8) - np.log(1e6)))
    return [{"id": k, "arrival": float(t[k]), "n": int(n[k]), "steps": int(steps[k]),
             "kind": str(kind[k]), "friction": float(fr[k]), "young": float(E[k]),
             "seed": seed * 1000003 + k} for k in range(n_requests)]


def request_workload(req: dict) -> Workload:
    """The scene of one serving request: a scaled deposition, or a periodic compaction
    from solid fraction 0.3 toward 0.62 over its step budget (log-normal radii as in
    the 1M-sphere compaction; the caller sets the rate once dt is known)."""
    if req["kind"] == "deposition":
        return scaled_deposition(req["n"], req["seed"], req["friction"], req["young"],
                                 steps=req["steps"])
    return compaction(n=req["n"], seed=req["seed"], steps=req["steps"], young=req["young"],
                      friction=req["friction"])
