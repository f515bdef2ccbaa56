"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances of the FP64 path, derived from its arithmetic:

* Contact pair set: exact, except pairs whose centre distance lies within
  BAND = 1e-9 r of the contact threshold (a rounding difference may decide
  those either way).
* Per-contact forces: within TOL = 1e-12 of the contact's sum of magnitudes
  |Fn| + |Fs| (cancellation-safe), plus the force that a few units in the last
  place of the branch length make through Fn = kn (r1 + r2 - l):
  kn * ULPS * eps * X, where X is the largest coordinate magnitude of the
  scene.  The two sides form the branch vector of a pair in possibly opposite
  orientations; across a periodic image that is x2 + h - x1 against
  x1 - h - x2, and the sum x2 + h is rounded at the scale of the coordinates,
  not of l.  For a contact whose penetration is a tiny fraction of its radii
  that rounding is a large relative change of Fn which no operation order
  removes.
* Per-body force, torque and velocity: within TOL of the body's sum of
  contact-force magnitudes (and r times it for torques, dt/m times it for the
  velocity change) plus the same ulp term summed over the body's contacts:
  a sum of terms that cancel is compared against the size of its terms.
* Positions within TOL of the coordinate scale; orientations within TOL.
"""
import numpy as np

BAND = 1e-9
TOL = 1e-12
ULPS = 4
EPS = 2.0 ** -52

_CTX = {}


def set_radii(radius, coord_scale=None):
    """Register the radii (by id) and the coordinate scale of the scene under comparison."""
    _CTX["r"] = np.asarray(radius, dtype=np.float64)
    _CTX["X"] = coord_scale


def set_coord_scale(x):
    _CTX["X"] = float(x)


def _coord_scale():
    X = _CTX.get("X")
    return 1.0 if X is None else X


def band_pairs(pos, radius, periodic, H, pairs_fn):
    """(i, j) pairs whose distance is within BAND * r of r_i + r_j at these positions."""
    I, J, C = pairs_fn(pos, radius, periodic=periodic, H=H, margin=BAND * float(radius.max()))
    out = set()
    for i, j, c in zip(I, J, C):
        d = pos[j] + (H @ c if periodic else 0) - pos[i]
        l = np.linalg.norm(d)
        if abs(l - (radius[i] + radius[j])) <= BAND * max(radius[i], radius[j]):
            out.add((int(i), int(j)))
    return out


def contact_keys(c):
    return [(int(a), int(b)) for a, b in zip(c["id1"], c["id2"])]


def compare_contact_sets(co, cg, band=frozenset()):
    ko = set(contact_keys(co)) - band
    kg = set(contact_keys(cg)) - band
    assert ko == kg, (f"contact sets differ: only oracle {sorted(ko - kg)[:10]}, "
                      f"only gpu {sorted(kg - ko)[:10]} ({len(ko)} vs {len(kg)})")
    return len(ko)


def compare_contacts(co, cg, band=frozenset(), tol=TOL, eps=EPS, coord=None):
    """Per-contact parity on the common set; returns (count, worst relative errors).
    eps and coord give the rounding unit and the coordinate scale of the branch
    vector (FP64: the scene's coordinates; mixed precision: FP32 offsets bounded by
    the contact distance)."""
    n = compare_contact_sets(co, cg, band)
    io = {k: t for t, k in enumerate(contact_keys(co))}
    ig = {k: t for t, k in enumerate(contact_keys(cg))}
    keys = [k for k in io if k in ig and k not in band]
    a = np.array([io[k] for k in keys], dtype=int)
    b = np.array([ig[k] for k in keys], dtype=int)
    worst = {}
    if len(keys) == 0:
        return n, worst
    scale = np.linalg.norm(co["fn"][a], axis=1) + np.linalg.norm(co["fs"][a], axis=1)
    X = _coord_scale() if coord is None else coord
    ulp_force = co["phys"][a, 0] * ULPS * eps * X
    widened = np.zeros(len(keys), dtype=bool)
    for f in ("fn", "fs"):
        d = np.max(np.abs(cg[f][b] - co[f][a]), axis=1)
        e = d / (tol * scale + ulp_force)
        worst[f] = float(e.max()) * tol
        widened |= d > tol * scale   # held only by the absolute rounding allowance
    # contacts whose force error is above the relative bar alone (the allowance for the
    # rounding of the penetration, a difference of two numbers of the reach's size)
    worst["widened_count"] = int(widened.sum())
    worst["widened_frac"] = float(widened.mean())
    worst["normal"] = float(np.max(np.abs(cg["normal"][b] - co["normal"][a]))) * (EPS / eps)
    rs = np.abs(co["phys"][a])
    worst["phys"] = float(np.max(np.abs(cg["phys"][b] - co["phys"][a]) / np.maximum(rs, 1e-300)))
    if eps != EPS:   # FP32 stiffnesses: a few FP32 roundings
        worst["phys"] *= tol / (8 * eps)
    worst["pen_abs"] = float(np.max(np.abs(cg["pen"][b] - co["pen"][a])))
    assert np.array_equal(cg["c"][b], co["c"][a]), "cell shifts differ"
    for f in ("fn", "fs", "normal", "phys"):
        assert worst[f] <= tol, (f, worst[f])
    return n, worst


def body_sums(co, n):
    """Per body: sum of |contact force| and sum of kn over its contacts (oracle contacts)."""
    F = np.linalg.norm(co["fn"] + co["fs"], axis=1)
    kn = co["phys"][:, 0]
    fsum = np.zeros(n)
    ksum = np.zeros(n)
    for ids in (co["id1"], co["id2"]):
        m = ids >= 0
        np.add.at(fsum, ids[m], F[m])
        np.add.at(ksum, ids[m], kn[m])
    return fsum, ksum


def compare_states(so, sg, length_scale, tol=TOL, co=None, masses=None, dt=0.0, gravity=0.0,
                   eps=EPS, coord=None):
    """State parity after one step.  With the oracle's contacts `co`, masses
    (m, I, r per body) and dt, velocities, spins, forces and torques are compared
    per body against the size of the terms that were summed; without them, against
    the largest magnitude of each field."""
    worst = {}
    worst["pos"] = float(np.max(np.abs(sg["pos"] - so["pos"]))) / length_scale
    worst["ori"] = float(np.max(np.abs(sg["ori"] - so["ori"])))
    if co is not None and masses is not None:
        m, I, r = masses
        n = len(m)
        fsum, ksum = body_sums(co, n)
        X = _coord_scale() if coord is None else coord
        fterm = tol * fsum + ULPS * eps * X * ksum
        fscale = fterm + tol * m * abs(gravity)
        dv = np.linalg.norm(sg["vel"] - so["vel"], axis=1)
        vs = tol * np.linalg.norm(so["vel"], axis=1) + dt * fscale / m
        worst["vel"] = float(np.max(dv / np.maximum(vs, 1e-300))) * tol
        dw = np.linalg.norm(sg["angvel"] - so["angvel"], axis=1)
        ws = tol * np.linalg.norm(so["angvel"], axis=1) + dt * r * fterm / I
        worst["angvel"] = float(np.max(dw / np.maximum(ws, 1e-300))) * tol
        if "force" in sg and "force" in so:
            df = np.linalg.norm(sg["force"] - so["force"], axis=1)
            worst["force"] = float(np.max(df / np.maximum(fterm, 1e-300))) * tol
            dtq = np.linalg.norm(sg["torque"] - so["torque"], axis=1)
            worst["torque"] = float(np.max(dtq / np.maximum(r * fterm, 1e-300))) * tol
    else:
        for f in ("vel", "angvel"):
            sc = max(float(np.max(np.abs(so[f]))), 1e-300)
            worst[f] = float(np.max(np.abs(sg[f] - so[f]))) / sc
    for f, v in worst.items():
        assert v <= tol, (f, v)
    return worst


def masses_of(w):
    """(m, I, r) per body of a workload, utils.sphere definitions."""
    rho = np.array([w.materials[k].density for k in w.mat_id])
    m = rho * 4.0 / 3.0 * np.pi * w.radius ** 3
    return m, 0.4 * m * w.radius ** 2, w.radius


def export_oracle(orc):
    """State, contact history, cell and clock of an oracle scene (to seed the GPU)."""
    return {"state": orc.state(), "contacts": orc.contacts(),
            "cell": orc.cell() if orc.periodic else None, "clock": orc.clock()}


def import_into_gpu(gpu, ex):
    st = ex["state"]
    gpu.set_state(pos=st["pos"], vel=st["vel"], angvel=st["angvel"], ori=st["ori"])
    c = ex["contacts"]
    gpu.set_contacts(c["id1"], c["id2"], c["c"], c["fs"], c["normal"], c["phys"])
    if ex["cell"] is not None:
        cl = ex["cell"]
        gpu.set_cell(H=cl["H"], velgrad=cl["velgrad"], prev_velgrad=cl["prev_velgrad"],
                     prev_H=cl["prev_H"])
    it, t, dt = ex["clock"]
    gpu.set_clock(it, t)
    gpu.set_dt(dt)
