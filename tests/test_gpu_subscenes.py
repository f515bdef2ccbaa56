"""Sub-scenes: independent scenes (own cell or walled box, wall material, gravity,
materials, time step) advanced together by the same launches.  Each sub-scene
must match its own oracle after a step (the parity bar of a single scene), keep
its own clock, follow the statistics of the same scene run alone, and survive the
removal of other sub-scenes and the arrival of new ones."""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, masses_of,
                               set_coord_scale, set_radii)  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def _workloads():
    a = workloads.periodic_cloud(1300, 51, phi=0.34, inflate=1.05, vel_scale=0.05,
                                 angvel_scale=20.0)
    a.velgrad = np.diag([-3.0, -2.0, -4.0])
    b = workloads.box_cloud(1100, 52, phi=0.3, inflate=1.05, two_materials=True,
                            gravity=(0, 0, -9.81), vel_scale=0.05, angvel_scale=30.0)
    c = workloads.periodic_cloud(900, 53, phi=0.33, inflate=1.04, friction=0.3, young=2e7,
                                 vel_scale=0.02)
    d = workloads.box_cloud(700, 54, phi=0.25, inflate=1.04, young=1e8, friction=0.6,
                            gravity=(0, -9.81, 0), vel_scale=0.03)
    return [a, b, c, d]


def _mix(pkg, ws, prec, dts=None):
    g = pkg.Scene.from_workload(ws[0], precision=prec,
                                dt=None if dts is None else dts[0])
    subs = [0]
    for k, w in enumerate(ws[1:]):
        subs.append(g.add_workload(w, material_base=8 * (k + 1),
                                   dt=None if dts is None else dts[k + 1]))
    return g, subs


def _sub_contacts(cg, first, n):
    """Contacts of one sub-scene with its ids made local (walls keep id1 < 0)."""
    in1 = (cg["id1"] >= first) & (cg["id1"] < first + n)
    in2 = (cg["id2"] >= first) & (cg["id2"] < first + n)
    m = in2 & ((cg["id1"] < 0) | in1)
    out = {k: v[m].copy() for k, v in cg.items()}
    out["id1"] = np.where(out["id1"] >= 0, out["id1"] - first, out["id1"])
    out["id2"] = out["id2"] - first
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_step_each_subscene_matches_its_oracle(mods, precision):
    oracle, pkg = mods
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    tol = 1e-12 if precision == "fp64" else 1e-5
    eps = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    ws = _workloads()
    orcs = [oracle.OracleScene.from_workload(w) for w in ws]
    dts = [o.clock()[2] for o in orcs]
    assert len(set(dts)) == len(dts)          # every sub-scene has its own step
    g, subs = _mix(pkg, ws, prec, dts)
    befores = [o.state() for o in orcs]
    g.step(1)
    cg = g.contacts()
    for w, o, sub, before in zip(ws, orcs, subs, befores):
        o.step(1)
        info = g.subscene(sub)
        assert info["iter"] == 1 and info["time"] == o.clock()[1] and info["dt"] == o.clock()[2]
        set_radii(w.radius)
        X = float(np.max(np.abs(before["pos"])))
        set_coord_scale(X)
        H = np.eye(3) if not w.periodic else np.asarray(w.cell)
        import tests.parity_util as pu
        old = pu.BAND
        pu.BAND = 1e-9 if precision == "fp64" else 1e-5   # FP32 decisions: wider band
        try:
            band = band_pairs(before["pos"], w.radius, w.periodic, H, oracle.pairs)
        finally:
            pu.BAND = old
        # mixed: FP32 rounding of coordinates bounded by the reach of a contact
        coord = None if precision == "fp64" else 2 * float(w.radius.max()) * 1.25
        co = o.contacts()
        n, _ = compare_contacts(co, _sub_contacts(cg, info["first_id"], info["n"]), band,
                                tol=tol, eps=eps, coord=coord)
        assert n > 100
        sg = g.subscene_state(sub)
        compare_states(o.state(), sg, X, tol=tol, co=co, masses=masses_of(w), dt=o.clock()[2],
                       gravity=float(np.linalg.norm(w.gravity)), eps=eps, coord=coord)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subscenes_follow_their_alone_runs(mods, precision):
    oracle, pkg = mods
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    ws = _workloads()
    g, subs = _mix(pkg, ws, prec)
    g.step(200)
    for w, sub in zip(ws, subs):
        alone = pkg.Scene.from_workload(w, precision=prec)
        alone.step(200)
        sa, sm = alone.stats(), g.subscene_stats(sub)
        info = g.subscene(sub)
        assert info["iter"] == 200 and info["time"] == alone.clock()[1]
        assert sm["n_bodies"] == w.n
        assert abs(sm["packing_fraction"] / sa["packing_fraction"] - 1) < 1e-12
        assert abs(sm["kinetic_energy"] / sa["kinetic_energy"] - 1) < 1e-3
        assert abs(sm["n_contacts"] - sa["n_contacts"]) <= max(2, 0.01 * sa["n_contacts"])
        assert abs(sm["n_wall_contacts"] - sa["n_wall_contacts"]) <= max(2, 0.01 * sa["n_wall_contacts"])


def test_removal_and_arrival(mods):
    oracle, pkg = mods
    ws = _workloads()
    g, subs = _mix(pkg, ws[:3], pkg.DEM_FP64)
    ref, rsubs = _mix(pkg, ws[:3], pkg.DEM_FP64)
    g.step(40)
    ref.step(40)
    n1 = ws[1].n
    first2 = g.subscene(subs[2])["first_id"]
    g.remove_subscene(subs[1])
    with pytest.raises(pkg.DemError):
        g.subscene(subs[1])
    g.step(1)
    assert g.n == ws[0].n + ws[2].n
    assert g.subscene(subs[2])["first_id"] == first2 - n1     # ids closed up
    # a new scene takes the free index and starts its own clock
    new = g.add_workload(ws[3], material_base=40)
    assert new == subs[1]
    o = oracle.OracleScene.from_workload(ws[3])
    g.step(1)
    o.step(1)
    info = g.subscene(new)
    assert info["iter"] == 1 and g.subscene(subs[2])["iter"] == 42
    assert info["first_id"] == ws[0].n + ws[2].n
    st = g.subscene_state(new)
    set_radii(ws[3].radius)
    X = float(np.max(np.abs(ws[3].pos)))
    set_coord_scale(X)
    compare_states(o.state(), st, X, co=o.contacts(), masses=masses_of(ws[3]), dt=o.clock()[2],
                   gravity=9.81)
    # the sub-scenes that stayed follow the run that never changed (the removal moved
    # their collider runs: rounding-level differences, amplified by the dynamics)
    g.step(19)
    ref.step(21)
    for a, b in ((subs[0], rsubs[0]), (subs[2], rsubs[2])):
        sg, sr = g.subscene_stats(a), ref.subscene_stats(b)
        assert sg["iter"] == sr["iter"] == 61
        assert abs(sg["kinetic_energy"] / sr["kinetic_energy"] - 1) < 1e-3
        assert abs(sg["n_contacts"] - sr["n_contacts"]) <= max(2, 0.01 * sr["n_contacts"])


def test_subscene_errors(mods):
    oracle, pkg = mods
    ws = _workloads()
    g, subs = _mix(pkg, ws[:2], pkg.DEM_FP64)
    with pytest.raises(pkg.DemError) as e:   # sub-scene 0 no longer holds the last ids
        g.add_spheres_to(subs[0], ws[0].pos[:1] + 0.5 * ws[0].cell[0, 0], ws[0].radius[:1])
    assert e.value.code == 10
    with pytest.raises(pkg.DemError) as e:
        g.remove_subscene(7)
    assert e.value.code == 1
    with pytest.raises(pkg.DemError) as e:
        g.add_subscene(wall_mask=0x3F, wall_material=999)
    assert e.value.code == 1
    with pytest.raises(pkg.DemError) as e:
        g.set_triax([-1e4] * 3, 7, [1.0] * 3, 0.2, 5)
    assert e.value.code in (9, 10)
