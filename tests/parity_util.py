"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (FP64 path): the contact pair set is compared exactly, except
pairs whose centre distance lies within 1e-9 r of the contact threshold (a
rounding difference may legitimately decide those either way).  Per-contact
forces agree within 1e-12 relative to the contact's sum of magnitudes
|Fn| + |Fs| (cancellation-safe); one-step states within 1e-12 of the field's
scale (box size for positions, the largest speed for velocities).
"""
import numpy as np

BAND = 1e-9
TOL = 1e-12


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
                      f"only gpu {sorted(kg - ko)[:10]}")
    return len(ko)


def compare_contacts(co, cg, band=frozenset(), tol=TOL):
    """Per-contact parity on the common set; returns the worst relative errors."""
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
    scale = np.maximum(scale, 1e-300)
    for f in ("fn", "fs"):
        e = np.max(np.abs(cg[f][b] - co[f][a]), axis=1) / scale
        worst[f] = float(e.max())
    worst["normal"] = float(np.max(np.abs(cg["normal"][b] - co["normal"][a])))
    pen_scale = np.maximum(np.abs(co["pen"][a]), 1e-300)
    rs = np.abs(co["phys"][a])
    worst["phys"] = float(np.max(np.abs(cg["phys"][b] - co["phys"][a]) / np.maximum(rs, 1e-300)))
    # penetration: relative to the radius sum scale (it is a small difference of lengths)
    worst["pen_abs"] = float(np.max(np.abs(cg["pen"][b] - co["pen"][a])))
    assert np.array_equal(cg["c"][b], co["c"][a]), "cell shifts differ"
    for f in ("fn", "fs", "normal", "phys"):
        assert worst[f] <= tol, (f, worst[f])
    del pen_scale
    return n, worst


def compare_states(so, sg, length_scale, tol=TOL):
    worst = {}
    worst["pos"] = float(np.max(np.abs(sg["pos"] - so["pos"]))) / length_scale
    for f in ("vel", "angvel"):
        sc = max(float(np.max(np.abs(so[f]))), 1e-300)
        worst[f] = float(np.max(np.abs(sg[f] - so[f]))) / sc
    worst["ori"] = float(np.max(np.abs(sg["ori"] - so["ori"])))
    for f, v in worst.items():
        assert v <= tol, (f, v)
    return worst


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
