"""ctypes binding of ``libdem.so`` (declared in ``include/dem.h``).

Argument marshalling only: every step of the DEM path runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library is missing or cannot
be loaded, every call raises.  Names follow the C ABI (``dem_step`` ->
``Scene.step`` and so on).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdem.so")

DEM_OK = 0
DEM_LAW_LINEAR = 0
DEM_LAW_HERTZ_MINDLIN = 1
STATUS_NAMES = {
    0: "DEM_OK", 1: "DEM_ERR_INVALID_ARG", 2: "DEM_ERR_OUT_OF_RANGE", 3: "DEM_ERR_OOM",
    4: "DEM_ERR_CAPACITY", 5: "DEM_ERR_NONFINITE", 6: "DEM_ERR_GEOMETRY", 7: "DEM_ERR_TIMEOUT",
    8: "DEM_ERR_CUDA", 9: "DEM_ERR_STATE", 10: "DEM_ERR_UNSUPPORTED",
}
DEM_FP64 = 0
DEM_MIXED = 1


class DemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SceneDesc(ctypes.Structure):
    _fields_ = [
        ("periodic", ctypes.c_int),
        ("cell_h", ctypes.c_double * 9),
        ("box_lo", ctypes.c_double * 3),
        ("box_hi", ctypes.c_double * 3),
        ("wall_mask", ctypes.c_int),
        ("gravity", ctypes.c_double * 3),
        ("damping", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("verlet_dist", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("capacity_bodies", ctypes.c_longlong),
        ("capacity_contacts", ctypes.c_longlong),
        ("cuda_stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
    ]


class SubsceneDesc(ctypes.Structure):
    _fields_ = [
        ("periodic", ctypes.c_int),
        ("cell_h", ctypes.c_double * 9),
        ("box_lo", ctypes.c_double * 3),
        ("box_hi", ctypes.c_double * 3),
        ("wall_mask", ctypes.c_int),
        ("wall_material", ctypes.c_int),
        ("gravity", ctypes.c_double * 3),
        ("damping", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("verlet_dist", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iter", ctypes.c_longlong),
        ("time", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("n_bodies", ctypes.c_longlong),
        ("n_contacts", ctypes.c_longlong),
        ("n_wall_contacts", ctypes.c_longlong),
        ("n_candidates", ctypes.c_longlong),
        ("n_rebuilds", ctypes.c_longlong),
        ("kinetic_energy", ctypes.c_double),
        ("unbalanced_force", ctypes.c_double),
        ("coordination", ctypes.c_double),
        ("packing_fraction", ctypes.c_double),
        ("stress", ctypes.c_double * 9),
    ]


class Timing(ctypes.Structure):
    _fields_ = [
        ("contact_ms", ctypes.c_double),
        ("integrate_ms", ctypes.c_double),
        ("cell_ms", ctypes.c_double),
        ("collider_ms", ctypes.c_double),
        ("contact_launches", ctypes.c_longlong),
        ("integrate_launches", ctypes.c_longlong),
        ("cell_launches", ctypes.c_longlong),
        ("collider_runs", ctypes.c_longlong),
        ("rows_processed", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
    ]


class ServerDesc(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("budget_bytes", ctypes.c_longlong),
        ("tick_steps", ctypes.c_longlong),
        ("rows_per_body", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("scene", SubsceneDesc),
        ("n_materials", ctypes.c_int),
        ("materials", ctypes.c_void_p),
        ("n", ctypes.c_longlong),
        ("pos", ctypes.c_void_p),
        ("radius", ctypes.c_void_p),
        ("mat_id", ctypes.c_void_p),
        ("vel", ctypes.c_void_p),
        ("angvel", ctypes.c_void_p),
        ("velgrad", ctypes.c_void_p),
        ("nsteps", ctypes.c_longlong),
        ("keep_state", ctypes.c_int),
    ]


class RequestResult(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_longlong),
        ("n", ctypes.c_longlong),
        ("nsteps", ctypes.c_longlong),
        ("iter", ctypes.c_longlong),
        ("time", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("latency", ctypes.c_double),
        ("stats", Stats),
    ]


class ServerSummary(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "submitted", "completed", "failed", "waiting", "resident", "resident_bodies",
        "max_resident", "ticks", "scene_steps", "body_steps", "budget_bytes",
        "resident_bytes_est", "device_bytes")] + [(k, ctypes.c_double) for k in (
        "rows_per_body", "wall_s", "busy_s", "latency_p50", "latency_p99", "latency_max",
        "latency_mean", "concurrency_mean")] + [("concurrency_hist", ctypes.c_longlong * 8)]

# upper edges of ServerSummary.concurrency_hist's bins (the last bin is open)
CONCURRENCY_BIN_EDGES = (1, 2, 4, 8, 16, 32, 64, None)


# C ABI: name -> (restype, argtypes)
_P = ctypes.c_void_p
class Tuning(ctypes.Structure):
    _fields_ = [
        ("contact_block", ctypes.c_int),
        ("contact_blocks_per_sm", ctypes.c_int),
        ("integrate_block", ctypes.c_int),
        ("degree_order", ctypes.c_int),
        ("step_graphs", ctypes.c_int),
    ]


_SIGS = {
    "dem_scene_desc_init": (None, [_P]),
    "dem_scene_create": (ctypes.c_int, [_P, _P]),
    "dem_scene_destroy": (None, [_P]),
    "dem_set_material": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double]),
    "dem_add_spheres": (ctypes.c_int, [_P, ctypes.c_longlong, _P, _P, _P, _P, _P, _P, _P]),
    "dem_set_dt": (ctypes.c_int, [_P, ctypes.c_double]),
    "dem_get_dt": (ctypes.c_int, [_P, _P]),
    "dem_set_cell_velgrad": (ctypes.c_int, [_P, _P]),
    "dem_set_triax": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int]),
    "dem_step": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "dem_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "dem_set_state": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dem_get_cell": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dem_set_cell": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dem_get_clock": (ctypes.c_int, [_P, _P, _P]),
    "dem_set_clock": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_double]),
    "dem_count_contacts": (ctypes.c_int, [_P, _P]),
    "dem_get_contacts": (ctypes.c_int, [_P, ctypes.c_longlong, _P, _P, _P, _P, _P, _P, _P, _P,
                                        _P, _P]),
    "dem_set_contacts": (ctypes.c_int, [_P, ctypes.c_longlong, _P, _P, _P, _P, _P, _P]),
    "dem_get_stats": (ctypes.c_int, [_P, _P]),
    "dem_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "dem_get_timing": (ctypes.c_int, [_P, _P]),
    "dem_set_tuning": (ctypes.c_int, [_P, _P]),
    "dem_subscene_desc_init": (None, [_P]),
    "dem_add_subscene": (ctypes.c_int, [_P, _P, _P]),
    "dem_add_spheres_to": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong, _P, _P, _P, _P, _P,
                                          _P, _P]),
    "dem_remove_subscene": (ctypes.c_int, [_P, ctypes.c_int]),
    "dem_get_subscene": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "dem_get_subscene_stats": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "dem_set_subscene_velgrad": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "dem_flip_cell": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "dem_set_density_scaling": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "dem_set_peri3d": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_longlong, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _P, _P, _P]),
    "dem_get_peri3d": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dem_get_density_scaling": (ctypes.c_int, [_P, _P]),
    "dem_num_bodies": (ctypes.c_int, [_P, _P]),
    "dem_get_micro": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "dem_get_body_stress": (ctypes.c_int, [_P, _P]),
    "dem_set_law": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "dem_set_timestepper": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double]),
    "dem_get_state_range": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_longlong, _P, _P, _P,
                                           _P]),
    "dem_get_tuning": (ctypes.c_int, [_P, _P]),
    "dem_autotune": (ctypes.c_int, [_P, ctypes.c_longlong, _P]),
    "dem_find_pairs": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, _P,
                                      ctypes.c_double, ctypes.c_longlong, _P, _P, _P, _P, _P]),
    "dem_find_pairs_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, _P,
                                              ctypes.c_double, ctypes.c_longlong, _P, _P, _P, _P,
                                              _P]),
    "dem_server_desc_init": (None, [_P]),
    "dem_server_create": (ctypes.c_int, [_P, _P]),
    "dem_server_destroy": (None, [_P]),
    "dem_request_init": (None, [_P]),
    "dem_server_submit": (ctypes.c_int, [_P, _P, _P]),
    "dem_server_poll": (ctypes.c_int, [_P, ctypes.c_longlong, _P]),
    "dem_server_wait": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_double]),
    "dem_server_result": (ctypes.c_int, [_P, ctypes.c_longlong, _P, _P, _P, _P, _P]),
    "dem_server_release": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "dem_server_stats": (ctypes.c_int, [_P, _P]),
    "dem_server_last_error": (ctypes.c_char_p, [_P]),
    "dem_measure_fp64_peak": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _P, _P]),
    "dem_last_error": (ctypes.c_char_p, [_P]),
    "dem_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdem.so (fails loudly: there is no fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Scene:
    """One DEM scene on the GPU (a handle of the C ABI)."""

    def __init__(self, periodic=False, cell=None, box_lo=(0, 0, 0), box_hi=(1, 1, 1),
                 wall_mask=0, gravity=(0, 0, 0), damping=0.2, dt=0.0, verlet_dist=-0.5,
                 precision=DEM_FP64, capacity_bodies=0, capacity_contacts=0, stream=None,
                 device=-1, use_torch_stream=True):
        self._lib = load_library()
        d = SceneDesc()
        self._lib.dem_scene_desc_init(ctypes.byref(d))
        d.periodic = int(bool(periodic))
        H = np.eye(3) if cell is None else np.asarray(cell, dtype=np.float64).reshape(3, 3)
        for q in range(9):
            d.cell_h[q] = float(H.flat[q])
        for k in range(3):
            d.box_lo[k] = float(box_lo[k])
            d.box_hi[k] = float(box_hi[k])
            d.gravity[k] = float(gravity[k])
        d.wall_mask = int(wall_mask)
        d.damping = float(damping)
        d.dt = float(dt)
        d.verlet_dist = float(verlet_dist)
        d.precision = int(precision)
        d.capacity_bodies = int(capacity_bodies)
        d.capacity_contacts = int(capacity_contacts)
        if stream is None and use_torch_stream:
            stream = _current_stream()
        d.cuda_stream = stream
        d.device = int(device)
        h = ctypes.c_void_p()
        rc = self._lib.dem_scene_create(ctypes.byref(d), ctypes.byref(h))
        if rc != DEM_OK:
            raise DemError(rc, self._lib.dem_last_error(None).decode())
        self._h = h
        self.periodic = bool(periodic)
        self.desc = d

    @classmethod
    def from_workload(cls, w, dt=None, **kw):
        s = cls(periodic=w.periodic, cell=w.cell, box_lo=w.box_lo, box_hi=w.box_hi,
                wall_mask=w.wall_mask, gravity=w.gravity, damping=w.damping, **kw)
        for k, m in enumerate(w.materials):
            s.set_material(k, m.density, m.young, m.poisson, m.friction)
        s.add_spheres(w.pos, w.radius, w.mat_id, w.vel, w.angvel)
        if dt is not None:
            s.set_dt(dt)
        if w.periodic and np.any(w.velgrad):
            s.set_cell_velgrad(w.velgrad)
        return s

    def _check(self, rc):
        if rc != DEM_OK:
            raise DemError(rc, self._lib.dem_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dem_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- scene construction
    def set_material(self, mat_id, density, young, poisson, friction_angle):
        self._check(self._lib.dem_set_material(self._h, int(mat_id), float(density), float(young),
                                               float(poisson), float(friction_angle)))

    def add_spheres(self, pos, radius, mat_id=None, vel=None, angvel=None, fixed=None):
        pos = _f64(pos, (-1, 3))
        radius = _f64(radius)
        mat = None if mat_id is None else np.ascontiguousarray(mat_id, dtype=np.int32)
        vel = _f64(vel, (-1, 3))
        angvel = _f64(angvel, (-1, 3))
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        first = ctypes.c_longlong()
        self._check(self._lib.dem_add_spheres(self._h, radius.size, _ptr(pos), _ptr(radius),
                                              _ptr(mat), _ptr(vel), _ptr(angvel), _ptr(fx),
                                              ctypes.byref(first)))
        return first.value

    def set_dt(self, dt):
        self._check(self._lib.dem_set_dt(self._h, float(dt)))

    def dt(self):
        v = ctypes.c_double()
        self._check(self._lib.dem_get_dt(self._h, ctypes.byref(v)))
        return v.value

    def set_cell_velgrad(self, L):
        L = _f64(L, (3, 3))
        self._check(self._lib.dem_set_cell_velgrad(self._h, _ptr(L)))

    def set_triax(self, goal, stress_mask, max_rate, grow_damping=0.25, glob_update=5):
        g = _f64(goal)
        m = _f64(max_rate)
        self._check(self._lib.dem_set_triax(self._h, _ptr(g), int(stress_mask), _ptr(m),
                                            float(grow_damping), int(glob_update)))

    # --- stepping
    def step(self, n=1):
        self._check(self._lib.dem_step(self._h, int(n)))

    # --- queries
    def state(self, force=True):
        it = ctypes.c_longlong()
        self._check(self._lib.dem_get_clock(self._h, ctypes.byref(it), None))
        n = self.n
        out = {k: np.empty((n, 3)) for k in ("pos", "vel", "angvel")}
        out["ori"] = np.empty((n, 4))
        if force:
            out["force"] = np.empty((n, 3))
            out["torque"] = np.empty((n, 3))
        self._check(self._lib.dem_get_state(self._h, _ptr(out["pos"]), _ptr(out["vel"]),
                                            _ptr(out["angvel"]), _ptr(out["ori"]),
                                            _ptr(out.get("force")), _ptr(out.get("torque"))))
        return out

    def get_state_into(self, pos=None, vel=None, angvel=None, ori=None, force=None, torque=None):
        """Copy state into caller-provided float64 host arrays (no allocation here)."""
        self._check(self._lib.dem_get_state(self._h, *(_ptr(a) for a in
                                                       (pos, vel, angvel, ori, force, torque))))

    def set_state(self, pos=None, vel=None, angvel=None, ori=None):
        keep = [_f64(pos, (-1, 3)), _f64(vel, (-1, 3)), _f64(angvel, (-1, 3)), _f64(ori, (-1, 4))]
        n = self.n
        for a, k in zip(keep, (3, 3, 3, 4)):
            if a is not None and a.shape != (n, k):
                raise ValueError("state array has the wrong shape")
        self._check(self._lib.dem_set_state(self._h, *(_ptr(a) for a in keep)))

    @property
    def n(self):
        v = ctypes.c_longlong()
        self._check(self._lib.dem_num_bodies(self._h, ctypes.byref(v)))
        return v.value

    # --- sub-scenes (independent scenes advanced by the same launches)
    def add_subscene(self, periodic=False, cell=None, box_lo=(0, 0, 0), box_hi=(1, 1, 1),
                     wall_mask=0, wall_material=0, gravity=(0, 0, 0), damping=0.2, dt=0.0,
                     verlet_dist=-0.5):
        d = SubsceneDesc()
        self._lib.dem_subscene_desc_init(ctypes.byref(d))
        d.periodic = int(bool(periodic))
        H = np.eye(3) if cell is None else np.asarray(cell, dtype=np.float64).reshape(3, 3)
        for q in range(9):
            d.cell_h[q] = float(H.flat[q])
        for k in range(3):
            d.box_lo[k] = float(box_lo[k])
            d.box_hi[k] = float(box_hi[k])
            d.gravity[k] = float(gravity[k])
        d.wall_mask = int(wall_mask)
        d.wall_material = int(wall_material)
        d.damping = float(damping)
        d.dt = float(dt)
        d.verlet_dist = float(verlet_dist)
        sub = ctypes.c_int()
        self._check(self._lib.dem_add_subscene(self._h, ctypes.byref(d), ctypes.byref(sub)))
        return sub.value

    def add_spheres_to(self, sub, pos, radius, mat_id=None, vel=None, angvel=None, fixed=None):
        pos = _f64(pos, (-1, 3))
        radius = _f64(radius)
        mat = None if mat_id is None else np.ascontiguousarray(mat_id, dtype=np.int32)
        vel = _f64(vel, (-1, 3))
        angvel = _f64(angvel, (-1, 3))
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        first = ctypes.c_longlong()
        self._check(self._lib.dem_add_spheres_to(self._h, int(sub), radius.size, _ptr(pos),
                                                 _ptr(radius), _ptr(mat), _ptr(vel), _ptr(angvel),
                                                 _ptr(fx), ctypes.byref(first)))
        return first.value

    def add_workload(self, w, material_base, dt=None):
        """Add workload w as a new sub-scene whose materials take the ids
        material_base + k; returns the sub-scene index."""
        for k, m in enumerate(w.materials):
            self.set_material(material_base + k, m.density, m.young, m.poisson, m.friction)
        sub = self.add_subscene(periodic=w.periodic, cell=w.cell, box_lo=w.box_lo,
                                box_hi=w.box_hi, wall_mask=w.wall_mask,
                                wall_material=material_base, gravity=w.gravity,
                                damping=w.damping, dt=0.0 if dt is None else dt)
        self.add_spheres_to(sub, w.pos, w.radius, np.asarray(w.mat_id) + material_base, w.vel,
                            w.angvel)
        if w.periodic and np.any(w.velgrad):
            self.set_subscene_velgrad(sub, w.velgrad)
        return sub

    def remove_subscene(self, sub):
        self._check(self._lib.dem_remove_subscene(self._h, int(sub)))

    def subscene(self, sub):
        first, n, it = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        t, dt = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.dem_get_subscene(self._h, int(sub), ctypes.byref(first),
                                               ctypes.byref(n), ctypes.byref(it), ctypes.byref(t),
                                               ctypes.byref(dt)))
        return {"first_id": first.value, "n": n.value, "iter": it.value, "time": t.value,
                "dt": dt.value}

    def subscene_stats(self, sub):
        st = Stats()
        self._check(self._lib.dem_get_subscene_stats(self._h, int(sub), ctypes.byref(st)))
        out = {name: getattr(st, name) for name, _ in Stats._fields_ if name != "stress"}
        out["stress"] = np.array(list(st.stress)).reshape(3, 3)
        return out

    def set_subscene_velgrad(self, sub, L):
        L = _f64(L, (3, 3))
        self._check(self._lib.dem_set_subscene_velgrad(self._h, int(sub), _ptr(L)))

    def set_peri3d(self, goal, stress_mask, n_steps, mod=0.1, max_strain_rate=1e3,
                   young_est=1e20, poisson_est=0.25, max_strain=1e6, paths=None, trsf0=None):
        """Peri3dController (dem_set_peri3d).  goal: xx, yy, zz, yz, zx, xy; paths:
        None or 6 sequences of (t, v) couples (empty: linear); trsf0: Cell.trsf now."""
        npath = np.zeros(6, dtype=np.int32)
        path = np.zeros((6, 16, 2))
        if paths is not None:
            for i, pth in enumerate(paths):
                pth = np.asarray(pth, dtype=np.float64).reshape(-1, 2)
                npath[i] = len(pth)
                path[i, :len(pth)] = pth
        g = _f64(goal, (6,))
        T0 = None if trsf0 is None else _f64(trsf0, (3, 3))
        self._check(self._lib.dem_set_peri3d(
            self._h, _ptr(g), int(stress_mask), int(n_steps), float(mod), float(max_strain_rate),
            float(young_est), float(poisson_est), float(max_strain),
            npath.ctypes.data_as(_P), _ptr(path), None if T0 is None else _ptr(T0)))

    def peri3d(self):
        st, sn, rt = np.empty(6), np.empty(6), np.empty(6)
        done = ctypes.c_int()
        self._check(self._lib.dem_get_peri3d(self._h, _ptr(st), _ptr(sn), _ptr(rt),
                                             ctypes.byref(done)))
        return {"stress": st, "strain": sn, "rate": rt, "done": bool(done.value)}

    def set_density_scaling(self, enable=True, target_dt=1.0, sub=0):
        """Density scaling to the step target_dt (dem_set_density_scaling); needs
        set_timestepper on the same sub-scene."""
        self._check(self._lib.dem_set_density_scaling(self._h, int(sub), int(bool(enable)),
                                                      float(target_dt)))

    def density_scaling(self):
        """Inertia factor f of every sphere, by id."""
        f = np.empty(self.n)
        self._check(self._lib.dem_get_density_scaling(self._h, _ptr(f)))
        return f

    def flip_cell(self, flip=None, sub=0):
        """utils.flipCell (dem_flip_cell): H' = H (I + flip), bodies and interactions
        unchanged; flip None: the automatic reduction.  Returns the applied matrix."""
        out = np.zeros((3, 3), dtype=np.int32)
        K = None if flip is None else np.ascontiguousarray(flip, dtype=np.int32).reshape(3, 3)
        self._check(self._lib.dem_flip_cell(self._h, int(sub),
                                            None if K is None else K.ctypes.data_as(_P),
                                            out.ctypes.data_as(_P)))
        return out

    def set_law(self, law, sub=0):
        """Contact law (dem_set_law): DEM_LAW_LINEAR or DEM_LAW_HERTZ_MINDLIN."""
        self._check(self._lib.dem_set_law(self._h, int(sub), int(law)))

    def set_timestepper(self, safety=0.8, interval=1, default_dt=-1.0, max_dt=0.0, sub=0):
        """GlobalStiffnessTimeStepper (dem_set_timestepper)."""
        self._check(self._lib.dem_set_timestepper(self._h, int(sub), float(safety), int(interval),
                                                  float(default_dt), float(max_dt)))

    def micro(self, sub=-1):
        """Fabric tensor and the normal / shear parts of the contact stress (dem_get_micro)."""
        F, SN, ST = np.empty((3, 3)), np.empty((3, 3)), np.empty((3, 3))
        nc = ctypes.c_longlong()
        self._check(self._lib.dem_get_micro(self._h, int(sub), _ptr(F), _ptr(SN), _ptr(ST),
                                            ctypes.byref(nc)))
        return {"fabric": F, "normal_stress": SN, "shear_stress": ST, "n_contacts": nc.value}

    def body_stress(self):
        """Per-sphere stress tensors (dem_get_body_stress), shape (n, 3, 3) in id order."""
        out = np.empty((self.n, 9))
        self._check(self._lib.dem_get_body_stress(self._h, _ptr(out)))
        return out.reshape(-1, 3, 3)

    def state_range(self, first_id, n):
        out = {k: np.empty((n, 3)) for k in ("pos", "vel", "angvel")}
        out["ori"] = np.empty((n, 4))
        self._check(self._lib.dem_get_state_range(self._h, int(first_id), int(n),
                                                  _ptr(out["pos"]), _ptr(out["vel"]),
                                                  _ptr(out["angvel"]), _ptr(out["ori"])))
        return out

    def subscene_state(self, sub):
        info = self.subscene(sub)
        return self.state_range(info["first_id"], info["n"])

    def cell(self):
        H, L, Lp, Hp = (np.empty((3, 3)) for _ in range(4))
        self._check(self._lib.dem_get_cell(self._h, _ptr(H), _ptr(L), _ptr(Lp), _ptr(Hp)))
        return {"H": H, "velgrad": L, "prev_velgrad": Lp, "prev_H": Hp}

    def set_cell(self, H=None, velgrad=None, prev_velgrad=None, prev_H=None):
        keep = [_f64(a, (3, 3)) for a in (H, velgrad, prev_velgrad, prev_H)]
        self._check(self._lib.dem_set_cell(self._h, *(_ptr(a) for a in keep)))

    def clock(self):
        it = ctypes.c_longlong()
        t = ctypes.c_double()
        self._check(self._lib.dem_get_clock(self._h, ctypes.byref(it), ctypes.byref(t)))
        return it.value, t.value

    def set_clock(self, it, t):
        self._check(self._lib.dem_set_clock(self._h, int(it), float(t)))

    def count_contacts(self):
        c = ctypes.c_longlong()
        self._check(self._lib.dem_count_contacts(self._h, ctypes.byref(c)))
        return c.value

    def contacts(self):
        m = self.count_contacts()
        out = {"id1": np.empty(m, np.int32), "id2": np.empty(m, np.int32),
               "c": np.empty((m, 3), np.int32), "fn": np.empty((m, 3)), "fs": np.empty((m, 3)),
               "normal": np.empty((m, 3)), "cpoint": np.empty((m, 3)), "phys": np.empty((m, 3)),
               "pen": np.empty(m)}
        cnt = ctypes.c_longlong()
        self._check(self._lib.dem_get_contacts(
            self._h, m, ctypes.byref(cnt), *(_ptr(out[k]) for k in
                                             ("id1", "id2", "c", "fn", "fs", "normal", "cpoint",
                                              "phys", "pen"))))
        return out

    def set_contacts(self, id1, id2, c, fs, nprev, phys):
        id1 = np.ascontiguousarray(id1, np.int32)
        id2 = np.ascontiguousarray(id2, np.int32)
        c = None if c is None else np.ascontiguousarray(c, np.int32).reshape(-1, 3)
        fs, nprev, phys = _f64(fs, (-1, 3)), _f64(nprev, (-1, 3)), _f64(phys, (-1, 3))
        if not (fs.shape[0] == nprev.shape[0] == phys.shape[0] == id1.size == id2.size):
            raise ValueError("contact arrays disagree in length")
        self._check(self._lib.dem_set_contacts(self._h, id1.size, _ptr(id1), _ptr(id2), _ptr(c),
                                               _ptr(fs), _ptr(nprev), _ptr(phys)))

    def stats(self):
        st = Stats()
        self._check(self._lib.dem_get_stats(self._h, ctypes.byref(st)))
        out = {name: getattr(st, name) for name, _ in Stats._fields_ if name != "stress"}
        out["stress"] = np.array(list(st.stress)).reshape(3, 3)
        return out


def _timing_methods():
    def set_timing(self, enable=True):
        self._check(self._lib.dem_set_timing(self._h, int(bool(enable))))

    def timing(self):
        t = Timing()
        self._check(self._lib.dem_get_timing(self._h, ctypes.byref(t)))
        return {name: getattr(t, name) for name, _ in Timing._fields_}

    def set_tuning(self, **shape):
        """Launch shapes (dem_tuning fields); unspecified fields keep their value."""
        t = Tuning()
        self._check(self._lib.dem_get_tuning(self._h, ctypes.byref(t)))
        for k, v in shape.items():
            setattr(t, k, int(v))
        self._check(self._lib.dem_set_tuning(self._h, ctypes.byref(t)))

    def tuning(self):
        t = Tuning()
        self._check(self._lib.dem_get_tuning(self._h, ctypes.byref(t)))
        return {name: getattr(t, name) for name, _ in Tuning._fields_}

    def autotune(self, steps_per_trial=20):
        """dem_autotune: time the launch shapes on this scene's own steps (they are
        real steps of the simulation); applies and returns the best shape."""
        t = Tuning()
        self._check(self._lib.dem_autotune(self._h, int(steps_per_trial), ctypes.byref(t)))
        return {name: getattr(t, name) for name, _ in Tuning._fields_}
    Scene.set_timing = set_timing
    Scene.timing = timing
    Scene.set_tuning = set_tuning
    Scene.tuning = tuning
    Scene.autotune = autotune


_timing_methods()


def _stats_dict(st):
    out = {name: getattr(st, name) for name, _ in Stats._fields_ if name != "stress"}
    out["stress"] = np.array(list(st.stress)).reshape(3, 3)
    return out


class Server:
    """dem_server_*: the continuous-batching request server of the library (its
    worker thread and scheduling run in the C++ library; this class marshals)."""

    WAITING, RESIDENT, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, precision=DEM_MIXED, budget_bytes=0, tick_steps=200, rows_per_body=8.0,
                 stream=None, device=-1):
        self._lib = load_library()
        d = ServerDesc()
        self._lib.dem_server_desc_init(ctypes.byref(d))
        d.precision = int(precision)
        d.budget_bytes = int(budget_bytes)
        d.tick_steps = int(tick_steps)
        d.rows_per_body = float(rows_per_body)
        d.cuda_stream = stream
        d.device = int(device)
        h = ctypes.c_void_p()
        rc = self._lib.dem_server_create(ctypes.byref(d), ctypes.byref(h))
        if rc != DEM_OK:
            raise DemError(rc, self._lib.dem_server_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != DEM_OK:
            raise DemError(rc, self._lib.dem_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dem_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, w, steps, velgrad=None, keep_state=False, dt=0.0):
        """Queue workload w (a workloads.Workload-like object) for `steps` steps;
        dt 0: 0.5 x p-wave step of its spheres.  Returns the ticket."""
        r = Request()
        self._lib.dem_request_init(ctypes.byref(r))
        sd = r.scene
        sd.periodic = int(bool(w.periodic))
        H = np.eye(3) if w.cell is None else np.asarray(w.cell, dtype=np.float64).reshape(3, 3)
        for q in range(9):
            sd.cell_h[q] = float(H.flat[q])
        for k in range(3):
            sd.box_lo[k] = float(w.box_lo[k])
            sd.box_hi[k] = float(w.box_hi[k])
            sd.gravity[k] = float(w.gravity[k])
        sd.wall_mask = int(w.wall_mask)
        sd.wall_material = 0
        sd.damping = float(w.damping)
        sd.dt = float(dt)
        mats = np.ascontiguousarray([[m.density, m.young, m.poisson, m.friction]
                                     for m in w.materials], dtype=np.float64)
        if velgrad is None and w.periodic and np.any(w.velgrad):
            velgrad = w.velgrad
        mat_id = None if w.mat_id is None else np.ascontiguousarray(w.mat_id, dtype=np.int32)
        keep = [mats, _f64(w.pos, (-1, 3)), _f64(w.radius), mat_id, _f64(w.vel, (-1, 3)),
                _f64(w.angvel, (-1, 3)), _f64(velgrad, (3, 3))]
        r.n_materials = len(w.materials)
        r.materials, r.pos, r.radius, r.mat_id, r.vel, r.angvel, r.velgrad = (
            _ptr(a) for a in keep)
        r.n = keep[2].size
        r.nsteps = int(steps)
        r.keep_state = int(bool(keep_state))
        t = ctypes.c_longlong()
        self._check(self._lib.dem_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        v = ctypes.c_int()
        self._check(self._lib.dem_server_poll(self._h, int(ticket), ctypes.byref(v)))
        return v.value

    def wait(self, ticket, timeout=3600.0):
        self._check(self._lib.dem_server_wait(self._h, int(ticket), float(timeout)))

    def result(self, ticket, state=False):
        info = RequestResult()
        n = None
        arrs = [None] * 4
        if state:
            self._check(self._lib.dem_server_result(self._h, int(ticket), ctypes.byref(info),
                                                    None, None, None, None))
            n = info.n
            arrs = [np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 4))]
        self._check(self._lib.dem_server_result(self._h, int(ticket), ctypes.byref(info),
                                                *(_ptr(a) for a in arrs)))
        out = {k: getattr(info, k) for k, _ in RequestResult._fields_ if k != "stats"}
        out["stats"] = _stats_dict(info.stats)
        if state:
            out["state"] = dict(zip(("pos", "vel", "angvel", "ori"), arrs))
        return out

    def release(self, ticket):
        self._check(self._lib.dem_server_release(self._h, int(ticket)))

    def stats(self):
        st = ServerSummary()
        self._check(self._lib.dem_server_stats(self._h, ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in ServerSummary._fields_}
        out["concurrency_hist"] = list(st.concurrency_hist)
        return out


def find_pairs(pos, radius, periodic=False, cell=None, margin=0.0, cap=None, stream=None,
               noalloc=False):
    """All pairs i < j with |x_j + H c - x_i| < r_i + r_j + margin (dem_find_pairs).

    pos (n, 3) and radius (n,) are float64 CUDA tensors; returns int32 CUDA tensors
    (i, j, c) in the library's fixed row order.  noalloc=True calls
    dem_find_pairs_noalloc, which uses the library's fixed scratch array instead of
    allocating (at most 65,536 spheres; the output tensors are still allocated here,
    by the caller of the C function)."""
    import torch
    lib = load_library()
    fn = lib.dem_find_pairs_noalloc if noalloc else lib.dem_find_pairs
    pos = pos.contiguous()
    radius = radius.contiguous()
    if pos.dtype != torch.float64 or radius.dtype != torch.float64 or not pos.is_cuda:
        raise ValueError("pos and radius must be float64 CUDA tensors")
    n = radius.numel()
    H = np.ascontiguousarray(np.eye(3) if cell is None else cell, dtype=np.float64).reshape(3, 3)
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    cap = max(16, 8 * n) if cap is None else int(cap)
    while True:
        I = torch.empty(cap, dtype=torch.int32, device=pos.device)
        J = torch.empty(cap, dtype=torch.int32, device=pos.device)
        C = torch.empty((cap, 3), dtype=torch.int32, device=pos.device)
        cnt = ctypes.c_longlong()
        rc = fn(pos.data_ptr(), radius.data_ptr(), n, int(bool(periodic)), H.ctypes.data,
                float(margin), cap, I.data_ptr(), J.data_ptr(), C.data_ptr(), ctypes.byref(cnt),
                st)
        if rc != DEM_OK:
            raise DemError(rc, lib.dem_last_error(None).decode())
        if cnt.value <= cap:
            m = cnt.value
            return I[:m], J[:m], C[:m]
        cap = cnt.value


def measure_fp64_peak(iters=6000, repeats=5, stream=None):
    """dem_measure_fp64_peak: the FP64 FMA throughput of this GPU in TFLOP/s."""
    lib = load_library()
    v = ctypes.c_double()
    st = _current_stream() if stream is None else stream
    rc = lib.dem_measure_fp64_peak(int(iters), int(repeats), st, ctypes.byref(v))
    if rc != DEM_OK:
        raise DemError(rc, lib.dem_last_error(None).decode())
    return v.value


def version() -> str:
    return load_library().dem_version().decode()
