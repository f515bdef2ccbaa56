"""Sheared periodic cells (general H and grad v, section 2.1.6) on the GPU against
the oracle: one-step contact and state parity from a pre-sheared cell with a full
velocity gradient and unwrapped positions, FP64 and mixed precision, both contact
laws; one step from a history the oracle built under simple shear; a simple-shear
trajectory with frequent collider runs; a sheared sub-scene beside a walled box."""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, export_oracle,
                               import_into_gpu, masses_of, set_coord_scale, set_radii)

pytestmark = pytest.mark.gpu

GRAD = np.array([[-5.0, 30.0, 0.0], [0.0, -5.0, 10.0], [4.0, 0.0, -5.0]])


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def sheared_cloud(n, seed, shear=(0.12, -0.07, 0.1), unwrap=True, **kw):
    """A periodic cloud mapped into the cell H = D + off-diagonal shear (fractional
    coordinates kept), optionally moved by whole cell vectors several periods away."""
    w = workloads.periodic_cloud(n, seed, **kw)
    D = np.diag(w.cell).copy()
    H = np.diag(D)
    H[0, 1], H[0, 2], H[1, 2] = shear[0] * D[1], shear[1] * D[2], shear[2] * D[2]
    frac = w.pos / D
    if unwrap:
        frac = frac + ((workloads.uniform(3 * n, seed + 9).reshape(n, 3) * 5).astype(int) - 2)
    w.pos = frac @ H.T
    w.cell = H
    return w


def _band(before, w, H, oracle, band):
    import tests.parity_util as pu
    old = pu.BAND
    pu.BAND = band
    try:
        return band_pairs(before["pos"], w.radius, True, H, oracle.pairs)
    finally:
        pu.BAND = old


def _check_step(o, g, w, oracle, precision):
    tol = 1e-12 if precision == "fp64" else 1e-5
    eps = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    set_radii(w.radius)
    before = o.state()
    X = float(np.max(np.abs(before["pos"])))
    set_coord_scale(X)
    band = _band(before, w, o.cell()["H"], oracle, 1e-9 if precision == "fp64" else 1e-5)
    coord = None if precision == "fp64" else 2 * float(w.radius.max()) * 1.25
    o.step(1)
    g.step(1)
    co, cg = o.contacts(), g.contacts()
    n, _ = compare_contacts(co, cg, band, tol=tol, eps=eps, coord=coord)
    compare_states(o.state(), g.state(), X, tol=tol, co=co, masses=masses_of(w),
                   dt=o.clock()[2], eps=eps, coord=coord)
    Ho, Hg = o.cell()["H"], g.cell()["H"]
    assert np.allclose(Hg, Ho, rtol=0, atol=1e-15 * np.abs(Ho).max())
    return n, cg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("law", ["linear", "hertz"])
def test_one_step_sheared_cell_full_velgrad(mods, precision, law):
    oracle, pkg = mods
    w = sheared_cloud(1801, 61, phi=0.3, inflate=1.05, vel_scale=0.05, angvel_scale=30.0)
    o = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    if law == "hertz":
        o.set_law(1)
        g.set_law(pkg.DEM_LAW_HERTZ_MINDLIN)
    o.set_velgrad(GRAD)
    g.set_cell_velgrad(GRAD)
    n, cg = _check_step(o, g, w, oracle, precision)
    assert n > 400
    # contacts through images whose shift has a shear component
    assert np.any((cg["c"][:, 1] != 0) | (cg["c"][:, 2] != 0))


def test_one_step_from_a_history_under_simple_shear(mods):
    """The oracle shears a diagonal cell for 60 steps (the cell becomes sheared, the
    contacts carry shear forces); the GPU imports state, history and cell, and both
    take one more step."""
    oracle, pkg = mods
    w = workloads.periodic_cloud(1500, 62, phi=0.33, inflate=1.03, vel_scale=0.01,
                                 angvel_scale=5.0)
    set_radii(w.radius)
    o = oracle.OracleScene.from_workload(w)
    g = pkg.Scene.from_workload(w, dt=o.clock()[2])
    dt = o.clock()[2]
    L = np.zeros((3, 3))
    L[0, 1] = 0.05 / (60 * dt)
    o.set_velgrad(L)
    o.step(60)
    assert o.cell()["H"][0, 1] > 0.04 * w.cell[1, 1]
    ex = export_oracle(o)
    assert np.count_nonzero(np.linalg.norm(ex["contacts"]["fs"], axis=1)) > 20
    import_into_gpu(g, ex)
    n, _ = _check_step(o, g, w, oracle, "fp64")
    assert n > 40


def test_simple_shear_trajectory_with_collider_reruns(mods):
    """140 steps of simple shear on both sides with a small Verlet margin: every step's
    contact set matches outside the threshold band, forces agree to 1e-8 of their size
    (rounding differences grow along a chaotic trajectory: the one-step bar is 1e-12),
    and the cells agree."""
    oracle, pkg = mods
    w = sheared_cloud(1200, 63, shear=(0.05, 0.0, 0.0), unwrap=False, phi=0.3, inflate=1.06,
                      vel_scale=0.05, angvel_scale=20.0)
    set_radii(w.radius)
    o = oracle.OracleScene.from_workload(w)
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], verlet_dist=-0.02)
    dt = o.clock()[2]
    L = np.zeros((3, 3))
    L[0, 1] = 0.1 / (140 * dt)
    o.set_velgrad(L)
    g.set_cell_velgrad(L)
    X = float(np.max(np.abs(w.pos)))
    for k in range(140):
        before = o.state()
        band = _band(before, w, o.cell()["H"], oracle, 1e-9)
        o.step(1)
        g.step(1)
        set_coord_scale(float(np.max(np.abs(before["pos"]))))
        compare_contacts(o.contacts(), g.contacts(), band, tol=1e-8)
        if k % 35 == 34:
            compare_states(o.state(), g.state(), X, tol=1e-8)
    Ho, Hg = o.cell()["H"], g.cell()["H"]
    assert np.allclose(Hg, Ho, rtol=0, atol=1e-14 * np.abs(Ho).max())
    assert Hg[0, 1] > 0.14 * w.cell[1, 1]
    assert g.stats()["n_rebuilds"] >= 3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sheared_subscene_beside_a_walled_box(mods, precision):
    oracle, pkg = mods
    from tests.test_gpu_subscenes import _sub_contacts
    a = sheared_cloud(1300, 64, phi=0.3, inflate=1.05, vel_scale=0.05, angvel_scale=20.0)
    a.velgrad = GRAD
    b = workloads.box_cloud(1100, 65, phi=0.3, inflate=1.05, two_materials=True,
                            gravity=(0, 0, -9.81), vel_scale=0.05, angvel_scale=30.0)
    orcs = [oracle.OracleScene.from_workload(w) for w in (a, b)]
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    tol = 1e-12 if precision == "fp64" else 1e-5
    eps = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    g = pkg.Scene.from_workload(b, precision=prec, dt=orcs[1].clock()[2])
    sub = g.add_workload(a, material_base=8, dt=orcs[0].clock()[2])
    before = orcs[0].state()
    set_radii(a.radius)
    X = float(np.max(np.abs(before["pos"])))
    set_coord_scale(X)
    band = _band(before, a, orcs[0].cell()["H"], oracle, 1e-9 if precision == "fp64" else 1e-5)
    coord = None if precision == "fp64" else 2 * float(a.radius.max()) * 1.25
    g.step(1)
    for o in orcs:
        o.step(1)
    info = g.subscene(sub)
    co = orcs[0].contacts()
    cg = _sub_contacts(g.contacts(), info["first_id"], info["n"])
    k, _ = compare_contacts(co, cg, band, tol=tol, eps=eps, coord=coord)
    assert k > 300
    sg = g.subscene_state(sub)
    compare_states(orcs[0].state(), sg, X, tol=tol, co=co, masses=masses_of(a),
                   dt=orcs[0].clock()[2], eps=eps, coord=coord)


def _sheared_history(oracle, gamma=0.7, steps=150, n=1500, seed=66):
    """An oracle packing sheared to H_xy / H_yy = gamma while compacting (contacts with
    shear history), its velocity gradient still on."""
    w = workloads.periodic_cloud(n, seed, phi=0.34, inflate=1.06, vel_scale=0.02,
                                 angvel_scale=10.0)
    o = oracle.OracleScene.from_workload(w)
    dt = o.clock()[2]
    L = -5.0 * np.eye(3)
    L[0, 1] = gamma / (steps * dt)
    o.set_velgrad(L)
    o.step(steps)
    return o, w


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_flip_matches_the_oracle(mods, precision):
    """Both sides flip the same sheared cell (the automatic reduction), then step:
    the applied matrix, the new cell, the contacts with their new shifts and the
    states agree at the parity bar of one step, and again after 25 more steps."""
    oracle, pkg = mods
    o, w = _sheared_history(oracle)
    assert o.cell()["H"][0, 1] > 0.6 * o.cell()["H"][1, 1]
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    import_into_gpu(g, export_oracle(o))
    Ko, Kg = o.flip_cell(), g.flip_cell()
    assert np.array_equal(Ko, Kg) and Kg[0, 1] == -1
    assert np.array_equal(o.cell()["H"], g.cell()["H"])
    n, cg = _check_step(o, g, w, oracle, precision)
    assert n > 300
    assert np.any(cg["c"][:, 0] != 0)
    tol = 1e-9 if precision == "fp64" else 1e-4
    o.step(24)
    g.step(24)
    before = o.state()
    band = _band(before, w, o.cell()["H"], oracle, 1e-7 if precision == "fp64" else 1e-4)
    o.step(1)
    g.step(1)
    set_coord_scale(float(np.max(np.abs(before["pos"]))))
    compare_contacts(o.contacts(), g.contacts(), band, tol=tol,
                     eps=2.0 ** -52 if precision == "fp64" else 2.0 ** -23,
                     coord=None if precision == "fp64" else 2 * float(w.radius.max()) * 1.25)


def test_flip_does_not_change_the_run(mods):
    """Fig. 6 on the GPU: two copies of one state, one flipped with an explicit matrix
    (the cell vector a_1 minus a_0), step 40 times; the bodies follow the same
    trajectories and the contacts carry the same forces (shifts related by M^-1)."""
    oracle, pkg = mods
    o, w = _sheared_history(oracle)
    ex = export_oracle(o)
    a = pkg.Scene.from_workload(w, dt=o.clock()[2])
    b = pkg.Scene.from_workload(w, dt=o.clock()[2])
    import_into_gpu(a, ex)
    import_into_gpu(b, ex)
    a.step(1)
    b.step(1)
    K = np.zeros((3, 3), dtype=int)
    K[0, 1] = -1
    assert np.array_equal(a.flip_cell(K), K)
    a.step(40)
    b.step(40)
    ca, cb = a.contacts(), b.contacts()
    ka = {(i, j): t for t, (i, j) in enumerate(zip(ca["id1"], ca["id2"]))}
    kb = {(i, j): t for t, (i, j) in enumerate(zip(cb["id1"], cb["id2"]))}
    assert set(ka) == set(kb) and len(ka) > 300
    ia = np.array([ka[k] for k in kb])
    ib = np.array([kb[k] for k in kb])
    Minv = np.rint(np.linalg.inv(np.eye(3) + K)).astype(int)
    assert np.array_equal(ca["c"][ia], cb["c"][ib] @ Minv.T)
    scale = float(np.abs(cb["fn"]).max())
    assert np.abs(ca["fn"][ia] - cb["fn"][ib]).max() < 1e-8 * scale
    assert np.abs(ca["fs"][ia] - cb["fs"][ib]).max() < 1e-8 * scale
    sa, sb = a.state(), b.state()
    assert np.abs(sa["pos"] - sb["pos"]).max() < 1e-12 * np.abs(sb["pos"]).max()
    assert np.abs(sa["vel"] - sb["vel"]).max() < 1e-8 * np.abs(sb["vel"]).max()


def test_flip_errors(mods):
    oracle, pkg = mods
    w = workloads.periodic_cloud(300, 67, phi=0.3)
    g = pkg.Scene.from_workload(w)
    with pytest.raises(pkg.DemError) as e:
        g.flip_cell([[1, 0, 0], [0, 0, 0], [0, 0, 0]])   # det(I + K) = 2
    assert e.value.code == 1
    assert np.array_equal(g.flip_cell(), np.zeros((3, 3)))   # a right cell: nothing to do
    b = workloads.box_cloud(200, 68, phi=0.2)
    gb = pkg.Scene.from_workload(b)
    with pytest.raises(pkg.DemError):
        gb.flip_cell()
