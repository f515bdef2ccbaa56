"""A sub-scene advanced in a batch is the same computation as the scene alone.

Rows are oriented by id and every per-body sum runs in increasing partner id, so in
FP64 the result of a step depends on the bodies and their contact histories only:
not on the slot order of the arrays, on when the collider runs (a batch runs it
whenever any sub-scene needs it), nor on the other sub-scenes.  So each sub-scene's
state must be bitwise equal to its alone run after 2000 steps, including across the
removal of another sub-scene and the arrival of a new one.  In mixed precision the
FP32 offsets are taken from the positions at the last collider run, which the batch
moves: there the bar is the statistics one (kinetic energy, coordination, packing
fraction within 1e-3).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

STEPS = 2000


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00611_gb300 as p
    return p


def _workloads():
    """Four uneven scenes: two gravity depositions in walled boxes (different sizes,
    materials, gravity directions) and two periodic clouds (one under compaction)."""
    a = workloads.box_cloud(2600, 61, phi=0.3, inflate=1.03, two_materials=True,
                            gravity=(0, 0, -9.81), vel_scale=0.05, angvel_scale=30.0)
    b = workloads.periodic_cloud(1500, 62, phi=0.34, inflate=1.05, vel_scale=0.05,
                                 angvel_scale=20.0)
    b.velgrad = np.diag([-3.0, -2.0, -4.0])
    c = workloads.box_cloud(700, 63, phi=0.25, inflate=1.04, young=1e8, friction=0.6,
                            gravity=(0, -9.81, 0), vel_scale=0.03)
    d = workloads.periodic_cloud(4100, 64, phi=0.33, inflate=1.04, friction=0.3, young=2e7,
                                 vel_scale=0.02)
    return [a, b, c, d]


def _batch(pkg, ws, prec):
    g = pkg.Scene(capacity_bodies=sum(w.n for w in ws) + 5000, precision=prec, dt=1.0)
    g.set_material(0, 1000.0, 1e6, 0.25, 0.5)
    subs = [g.add_workload(w, material_base=8 * (k + 1)) for k, w in enumerate(ws)]
    return g, subs


def _alone(pkg, w, prec, steps):
    s = pkg.Scene.from_workload(w, precision=prec)
    s.step(steps)
    st = s.state(force=True)
    stats = s.stats()
    s.close()
    return st, stats


def _assert_same_state(a, b, what):
    for k in ("pos", "vel", "angvel", "ori"):
        if not np.array_equal(a[k], b[k]):
            d = np.max(np.abs(a[k] - b[k]))
            raise AssertionError(f"{what}: {k} differs (max |diff| {d:.3e})")


def test_fp64_subscenes_equal_their_alone_runs_bitwise(pkg):
    ws = _workloads()
    g, subs = _batch(pkg, ws, pkg.DEM_FP64)
    g.step(10)
    # the inflated clouds start with a dense contact network (it relaxes later on)
    assert sum(g.subscene_stats(q)["n_contacts"] for q in subs) > 500
    g.step(STEPS - 10)
    rebuilds = []
    for k, (w, q) in enumerate(zip(ws, subs)):
        assert g.subscene(q)["iter"] == STEPS
        alone, stats = _alone(pkg, w, pkg.DEM_FP64, STEPS)
        _assert_same_state(g.subscene_state(q), alone, f"scene {k}")
        sm = g.subscene_stats(q)
        assert sm["n_contacts"] == stats["n_contacts"]
        assert sm["n_wall_contacts"] == stats["n_wall_contacts"]
        rebuilds.append(stats["n_rebuilds"])
    # the batch ran the collider whenever any scene asked: more often than each alone
    assert min(rebuilds) >= 2
    assert g.stats()["n_rebuilds"] > max(rebuilds)
    g.close()


def test_fp64_bitwise_across_a_removal_and_an_arrival(pkg):
    ws = _workloads()
    g, subs = _batch(pkg, ws[:3], pkg.DEM_FP64)
    g.step(700)
    g.remove_subscene(subs[1])
    g.step(600)
    new = g.add_workload(ws[3], material_base=64)
    g.step(700)
    for w, q in ((ws[0], subs[0]), (ws[2], subs[2])):
        assert g.subscene(q)["iter"] == STEPS
        alone, _ = _alone(pkg, w, pkg.DEM_FP64, STEPS)
        _assert_same_state(g.subscene_state(q), alone, "remaining scene")
    assert g.subscene(new)["iter"] == 700
    alone, _ = _alone(pkg, ws[3], pkg.DEM_FP64, 700)
    _assert_same_state(g.subscene_state(new), alone, "arrived scene")
    g.close()


def test_mixed_subscenes_follow_their_alone_runs(pkg):
    """Mixed precision, 200 steps: kinetic energy within 1e-3 of the mixed run alone,
    packing fraction to rounding, coordination within 1e-3 relative or one contact
    (2/N, the resolution of Z = 2C/N)."""
    ws = _workloads()
    g, subs = _batch(pkg, ws, pkg.DEM_MIXED)
    g.step(200)
    for k, (w, q) in enumerate(zip(ws, subs)):
        _, sa = _alone(pkg, w, pkg.DEM_MIXED, 200)
        sm = g.subscene_stats(q)
        assert abs(sm["packing_fraction"] / sa["packing_fraction"] - 1) < 1e-12
        assert abs(sm["kinetic_energy"] / sa["kinetic_energy"] - 1) < 1e-3, k
        assert abs(sm["coordination"] - sa["coordination"]) <= (1 + 1e-9) * max(
            1e-3 * sa["coordination"], 2.0 / w.n), k
    g.close()
