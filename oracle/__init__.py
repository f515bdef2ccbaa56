"""Python binding of the plain FP64 CPU DEM oracle (``dem_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA path; only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and does not import the
product package.

Parity status of each oracle function (what pins it, in ``tests/test_oracle_*``):

* contact detection (cell list + exact test; a sort-and-sweep variant): pinned
  by brute force on small inputs, aperiodic, periodic and sheared.
* Ip2 stiffness and Law2 normal force: pinned by the closed-form binary impact
  (duration pi*sqrt(m*/kn), restitution 1) and the sphere resting on a wall
  (pen = m g / kn).
* shear transport and torques: pinned by rigid-body motion of a contact pair
  (objectivity: the shear force rotates with the pair, twist angle w*dt per step),
  the rolling transition v = 5/7 v0, and angular-momentum conservation.
* Coulomb cap: pinned by the bound |Fs| <= tan(phi) Fn on every contact.
* NewtonIntegrator, damping (eq. 2.9) and energy conventions: pinned by the
  falling-sphere energy doctest of the yade.plot reference (printed digits).
* p-wave time step: pinned by the SpherePWaveTimeStep doctest.
* periodic cell (cellDist, homoDeform, image velocity): pinned by the affine
  invariant (a pair riding the homogeneous field stays force-free) and by
  brute-force periodic detection.
* servo / stress: Love-Weber stress pinned by the static two-sphere closed form.
* orientation update q+ = dq q: pinned by scipy's rotation algebra (constant spin
  turns by k |w| dt; two spin phases compose in the world frame).
* unbalanced force, coordination, packing fraction: pinned by a hand-worked chain
  with a wall contact and a fixed sphere, and by sphere volumes over the box or
  current cell volume.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_HDR = os.path.join(_HERE, "dem_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_d = ctypes.c_double
_p = ctypes.c_void_p
_l = ctypes.c_long
_i = ctypes.c_int


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction (IEEE round-to-nearest,
    operation order as written)."""
    out = _LIB if not sanitize else os.path.join(_HERE, "liboracle_asan.so")
    stale = (not os.path.exists(out) or
             os.path.getmtime(out) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        flags = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                 "-Wall"]
        if sanitize:
            flags = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"] + \
                flags[2:]
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "orc_create": (_p, [_i, _p, _p, _p, _i, _p, _d, _d]),
        "orc_destroy": (None, [_p]),
        "orc_set_material": (_i, [_p, _i, _d, _d, _d, _d]),
        "orc_add_spheres": (_l, [_p, _l, _p, _p, _p, _p, _p, _p]),
        "orc_set_dt": (_i, [_p, _d]),
        "orc_set_velgrad": (_i, [_p, _p]),
        "orc_step": (_i, [_p, _l]),
        "orc_set_triax": (_i, [_p, _p, _i, _p, _d, _i]),
        "orc_set_timestepper": (_i, [_p, _d, _i, _d, _d]),
        "orc_set_law": (_i, [_p, _i]),
        "orc_set_density_scaling": (_i, [_p, _i, _d]),
        "orc_set_peri3d": (_i, [_p, _p, _i, _l, _d, _d, _d, _d, _d, _p, _p, _p]),
        "orc_get_peri3d": (_i, [_p, _p, _p, _p]),
        "orc_get_density_scaling": (None, [_p, _p]),
        "orc_num_bodies": (_l, [_p]),
        "orc_get_state": (None, [_p, _p, _p, _p, _p, _p, _p]),
        "orc_set_state": (_i, [_p, _p, _p, _p, _p]),
        "orc_get_cell": (None, [_p, _p, _p, _p, _p]),
        "orc_set_cell": (_i, [_p, _p, _p, _p, _p]),
        "orc_flip_cell": (_i, [_p, _p, _p]),
        "orc_get_clock": (None, [_p, _p, _p, _p]),
        "orc_set_clock": (_i, [_p, _l, _d]),
        "orc_num_contacts": (_l, [_p]),
        "orc_get_contacts": (_l, [_p, _l, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "orc_set_contacts": (_i, [_p, _l, _p, _p, _p, _p, _p, _p]),
        "orc_get_energy": (None, [_p, _p]),
        "orc_get_stats": (None, [_p, _p]),
        "orc_sphere_pwave_dt": (_d, [_d, _d, _d]),
        "orc_pwave_dt": (_d, [_p]),
        "orc_pairs_bruteforce": (_l, [_l, _p, _p, _i, _p, _d, _l, _p, _p, _p]),
        "orc_pairs_sweep": (_l, [_l, _p, _p, _i, _p, _d, _l, _p, _p, _p]),
        "orc_pairs_grid": (_l, [_l, _p, _p, _i, _p, _d, _l, _p, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def sphere_pwave_dt(radius: float, density: float, young: float) -> float:
    """utils.SpherePWaveTimeStep."""
    return _load().orc_sphere_pwave_dt(radius, density, young)


def pairs(pos, radius, periodic=False, H=None, margin=0.0, method="grid"):
    """All (i<j, c) with |x_j + H c - x_i| < r_i + r_j + margin, sorted by (i, j)."""
    lib = _load()
    pos = _f64(pos, (-1, 3))
    radius = _f64(radius)
    n = radius.size
    Hm = _f64(np.eye(3) if H is None else H, (3, 3))
    fn = {"sweep": lib.orc_pairs_sweep, "grid": lib.orc_pairs_grid,
          "brute": lib.orc_pairs_bruteforce}[method]
    cap = max(16, 8 * n)
    while True:
        I = np.empty(cap, np.int32)
        J = np.empty(cap, np.int32)
        C = np.empty((cap, 3), np.int32)
        m = fn(n, _ptr(pos), _ptr(radius), int(bool(periodic)), _ptr(Hm), float(margin), cap,
               _ptr(I), _ptr(J), _ptr(C))
        if m < 0:
            raise RuntimeError(f"oracle pair search failed ({m})")
        if m <= cap:
            return I[:m].copy(), J[:m].copy(), C[:m].copy()
        cap = m


class OracleScene:
    """One oracle scene (the CPU counterpart of a DEM scene)."""

    def __init__(self, periodic=False, cell=None, box_lo=(0, 0, 0), box_hi=(1, 1, 1),
                 wall_mask=0, gravity=(0, 0, 0), damping=0.2, dt=0.0):
        self._lib = _load()
        H = _f64(np.eye(3) if cell is None else cell, (3, 3))
        lo = _f64(box_lo)
        hi = _f64(box_hi)
        g = _f64(gravity)
        self._h = self._lib.orc_create(int(bool(periodic)), _ptr(H), _ptr(lo), _ptr(hi),
                                       int(wall_mask), _ptr(g), float(damping), float(dt))
        if not self._h:
            raise RuntimeError("orc_create failed")
        self.periodic = bool(periodic)
        self._box = (lo.copy(), hi.copy())
        self._radius = np.zeros(0)

    @classmethod
    def from_workload(cls, w, dt=None):
        s = cls(periodic=w.periodic, cell=w.cell, box_lo=w.box_lo, box_hi=w.box_hi,
                wall_mask=w.wall_mask, gravity=w.gravity, damping=w.damping, dt=1.0)
        for k, m in enumerate(w.materials):
            s.set_material(k, m.density, m.young, m.poisson, m.friction)
        s.add_spheres(w.pos, w.radius, w.mat_id, w.vel, w.angvel)
        s.set_dt(dt if dt is not None else w.dt_factor * s.pwave_dt())
        if w.periodic and np.any(w.velgrad):
            s.set_velgrad(w.velgrad)
        return s

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_material(self, mat, density, young, poisson, friction):
        if self._lib.orc_set_material(self._h, mat, density, young, poisson, friction) != 0:
            raise ValueError("bad material")

    def add_spheres(self, pos, radius, mat=None, vel=None, angvel=None, fixed=None):
        pos = _f64(pos, (-1, 3))
        radius = _f64(radius)
        mat = None if mat is None else np.ascontiguousarray(mat, np.int32)
        vel = _f64(vel, (-1, 3))
        angvel = _f64(angvel, (-1, 3))
        fx = None if fixed is None else np.ascontiguousarray(fixed, np.uint8)
        r = self._lib.orc_add_spheres(self._h, radius.size, _ptr(pos), _ptr(radius), _ptr(mat),
                                      _ptr(vel), _ptr(angvel), _ptr(fx))
        if r < 0:
            raise ValueError(f"add_spheres failed ({r})")
        self._radius = np.concatenate([self._radius, radius])
        return r

    def set_dt(self, dt):
        if self._lib.orc_set_dt(self._h, float(dt)) != 0:
            raise ValueError("bad dt")

    def pwave_dt(self):
        return self._lib.orc_pwave_dt(self._h)

    def set_velgrad(self, L):
        L = _f64(L, (3, 3))
        if self._lib.orc_set_velgrad(self._h, _ptr(L)) != 0:
            raise ValueError("set_velgrad needs a periodic scene")

    def set_triax(self, goal, stress_mask, max_rate, grow_damping=0.25, glob_update=5):
        g = _f64(goal)
        m = _f64(max_rate)
        if self._lib.orc_set_triax(self._h, _ptr(g), int(stress_mask), _ptr(m),
                                   float(grow_damping), int(glob_update)) != 0:
            raise ValueError("set_triax needs a periodic scene and valid parameters")

    def set_law(self, law):
        """0: Cundall-Strack (linear), 1: Hertz-Mindlin (reading R18 in dem_oracle.c)."""
        if self._lib.orc_set_law(self._h, int(law)) != 0:
            raise ValueError("unknown contact law")

    def set_timestepper(self, safety=0.8, interval=1, default_dt=-1.0, max_dt=0.0):
        """GlobalStiffnessTimeStepper (reading R17 in dem_oracle.c)."""
        if self._lib.orc_set_timestepper(self._h, float(safety), int(interval), float(default_dt),
                                         float(max_dt)) != 0:
            raise ValueError("bad time-stepper parameters")

    def set_peri3d(self, goal, stress_mask, n_steps, mod=0.1, max_strain_rate=1e3,
                   young_est=1e20, poisson_est=0.25, max_strain=1e6, paths=None, trsf0=None):
        """Peri3dController (reading R23 in dem_oracle.c).  goal: 6 values in the order
        xx, yy, zz, yz, zx, xy; paths: None or 6 sequences of (t, v) couples (empty:
        the default linear path); trsf0: Cell.trsf at the start (None: identity)."""
        npath = np.zeros(6, dtype=np.int32)
        path = np.zeros((6, 16, 2))
        if paths is not None:
            for i, pth in enumerate(paths):
                pth = np.asarray(pth, dtype=np.float64).reshape(-1, 2)
                npath[i] = len(pth)
                path[i, :len(pth)] = pth
        g = _f64(goal, (6,))
        rc = self._lib.orc_set_peri3d(self._h, _ptr(g), int(stress_mask), int(n_steps), float(mod),
                                      float(max_strain_rate), float(young_est), float(poisson_est),
                                      float(max_strain), npath.ctypes.data_as(ctypes.c_void_p),
                                      _ptr(path), _ptr(_f64(trsf0, (3, 3))))
        if rc != 0:
            raise ValueError("bad Peri3dController parameters (or an aperiodic scene)")

    def peri3d(self):
        st, sn, rt = np.empty(6), np.empty(6), np.empty(6)
        rc = self._lib.orc_get_peri3d(self._h, _ptr(st), _ptr(sn), _ptr(rt))
        if rc < 0:
            raise ValueError("no Peri3dController")
        return {"stress": st, "strain": sn, "rate": rt, "done": bool(rc)}

    def set_density_scaling(self, on=True, target_dt=1.0):
        """NewtonIntegrator.densityScaling with the stepper's targetDt (reading R22 in
        dem_oracle.c); needs set_timestepper first."""
        if self._lib.orc_set_density_scaling(self._h, int(bool(on)), float(target_dt)) != 0:
            raise ValueError("density scaling needs the time stepper and target_dt > 0")

    def density_scaling(self):
        """Per-body inertia factors f (1 where no scaling applies)."""
        f = np.empty(self.n)
        self._lib.orc_get_density_scaling(self._h, _ptr(f))
        return f

    def step(self, n=1):
        rc = self._lib.orc_step(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")

    @property
    def n(self):
        return self._lib.orc_num_bodies(self._h)

    def state(self):
        n = self.n
        out = {k: np.empty((n, 3)) for k in ("pos", "vel", "angvel", "force", "torque")}
        out["ori"] = np.empty((n, 4))
        self._lib.orc_get_state(self._h, _ptr(out["pos"]), _ptr(out["vel"]), _ptr(out["angvel"]),
                                _ptr(out["ori"]), _ptr(out["force"]), _ptr(out["torque"]))
        return out

    def set_state(self, pos=None, vel=None, angvel=None, ori=None):
        keep = [_f64(pos, (-1, 3)), _f64(vel, (-1, 3)), _f64(angvel, (-1, 3)), _f64(ori, (-1, 4))]
        for a, k in zip(keep, (3, 3, 3, 4)):
            if a is not None and a.shape != (self.n, k):
                raise ValueError("state array has the wrong shape")
        self._lib.orc_set_state(self._h, *(_ptr(a) for a in keep))

    def cell(self):
        H, L, Lp, Hp = (np.empty((3, 3)) for _ in range(4))
        self._lib.orc_get_cell(self._h, _ptr(H), _ptr(L), _ptr(Lp), _ptr(Hp))
        return {"H": H, "velgrad": L, "prev_velgrad": Lp, "prev_H": Hp}

    def set_cell(self, H=None, velgrad=None, prev_velgrad=None, prev_H=None):
        keep = [_f64(a, (3, 3)) for a in (H, velgrad, prev_velgrad, prev_H)]
        rc = self._lib.orc_set_cell(self._h, *(_ptr(a) for a in keep))
        if rc != 0:
            raise ValueError("set_cell needs a periodic scene")

    def flip_cell(self, flip=None):
        """utils.flipCell: H' = H (I + flip), interactions keep their images; flip None:
        the automatic reduction.  Returns the applied integer matrix."""
        out = np.zeros((3, 3), dtype=np.int32)
        K = None if flip is None else np.ascontiguousarray(flip, dtype=np.int32).reshape(3, 3)
        rc = self._lib.orc_flip_cell(self._h, None if K is None else K.ctypes.data_as(ctypes.c_void_p),
                                     out.ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise ValueError("flip_cell: aperiodic scene, det(I + flip) != 1, or a shift out of range")
        return out

    def clock(self):
        it = ctypes.c_long()
        t = ctypes.c_double()
        dt = ctypes.c_double()
        self._lib.orc_get_clock(self._h, ctypes.byref(it), ctypes.byref(t), ctypes.byref(dt))
        return it.value, t.value, dt.value

    def set_clock(self, it, t):
        self._lib.orc_set_clock(self._h, int(it), float(t))

    def contacts(self):
        m = self._lib.orc_num_contacts(self._h)
        out = {"id1": np.empty(m, np.int32), "id2": np.empty(m, np.int32),
               "c": np.empty((m, 3), np.int32), "fn": np.empty((m, 3)), "fs": np.empty((m, 3)),
               "normal": np.empty((m, 3)), "cpoint": np.empty((m, 3)), "phys": np.empty((m, 3)),
               "pen": np.empty(m)}
        self._lib.orc_get_contacts(self._h, m, *(_ptr(out[k]) for k in
                                                ("id1", "id2", "c", "fn", "fs", "normal",
                                                 "cpoint", "phys", "pen")))
        return out

    def set_contacts(self, id1, id2, c, fs, nprev, phys):
        id1 = np.ascontiguousarray(id1, np.int32)
        id2 = np.ascontiguousarray(id2, np.int32)
        c = np.ascontiguousarray(c, np.int32).reshape(-1, 3)
        fs, nprev, phys = _f64(fs, (-1, 3)), _f64(nprev, (-1, 3)), _f64(phys, (-1, 3))
        if not (c.shape[0] == fs.shape[0] == nprev.shape[0] == phys.shape[0] == id1.size == id2.size):
            raise ValueError("contact arrays disagree in length")
        rc = self._lib.orc_set_contacts(self._h, id1.size, _ptr(id1), _ptr(id2), _ptr(c),
                                        _ptr(fs), _ptr(nprev), _ptr(phys))
        if rc != 0:
            raise ValueError(f"set_contacts failed ({rc})")

    def energy(self):
        e = np.empty(7)
        self._lib.orc_get_energy(self._h, _ptr(e))
        keys = ("kinTrans", "kinRot", "gravWork", "nonviscDamp", "plastDissip",
                "elastPotential", "total")
        return dict(zip(keys, e.tolist()))

    def micro(self):
        """Micromechanics of the current contacts, from the utils reference of the text:
        fabricTensor F = (1/n_c) sum n n; normalShearStressTensors, read with compression
        negative and l the current centroid distance: normal part -(1/V) sum l N n n,
        shear part -(1/V) sum l n Fs; bodyStressTensors (1/V_b) sum x f per sphere, x the
        contact point relative to the centre, f the force on the sphere (walls included),
        x read in the configuration the contact forces were computed in (the contact
        geometry), not from the positions the integrator has since moved.  Written out
        from the contact list (numpy, FP64)."""
        c = self.contacts()
        pos = self.state()["pos"]
        r = self._radius
        if self.periodic:
            V = abs(np.linalg.det(self.cell()["H"]))
        else:
            lo, hi = self._box
            V = float(np.prod(hi - lo))
        ss = c["id1"] >= 0
        n = c["normal"][ss]
        fn, fs = c["fn"][ss], c["fs"][ss]
        i1, i2 = c["id1"][ss], c["id2"][ss]
        l = r[i1] + r[i2] - c["pen"][ss]
        N = np.einsum("ki,ki->k", fn, n)
        nc = n.shape[0]
        fabric = np.einsum("ki,kj->ij", n, n) / nc if nc else np.zeros((3, 3))
        normal = -np.einsum("k,ki,kj->ij", l * N, n, n) / V
        shear = -np.einsum("k,ki,kj->ij", l, n, fs) / V
        body = np.zeros((self.n, 3, 3))
        F = c["fn"] + c["fs"]                      # force on id2
        # contact point relative to each centre in the configuration the forces were
        # computed in: (r - pen/2) along the normal from body 1 (toward body 2), the
        # opposite way from body 2, and from the sphere toward a wall
        for k in range(len(c["id1"])):
            b2, nk, pk = c["id2"][k], c["normal"][k], c["pen"][k]
            if c["id1"][k] >= 0:
                b1 = c["id1"][k]
                body[b1] += np.outer((r[b1] - 0.5 * pk) * nk, -F[k])
                body[b2] += np.outer(-(r[b2] - 0.5 * pk) * nk, F[k])
            else:
                body[b2] += np.outer(-(r[b2] - 0.5 * pk) * nk, F[k])
        body /= (4.0 / 3.0 * np.pi * r ** 3)[:, None, None]
        return {"fabric": fabric, "normal_stress": normal, "shear_stress": shear,
                "body_stress": body, "n_contacts": nc}

    def stats(self):
        o = np.empty(14)
        self._lib.orc_get_stats(self._h, _ptr(o))
        return {"ke": o[0], "unbalanced": o[1], "Z": o[2], "phi": o[3], "n_contacts": int(o[4]),
                "stress": o[5:14].reshape(3, 3).copy()}
