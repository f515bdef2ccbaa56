"""GlobalStiffnessTimeStepper on the GPU (dem_set_timestepper) against the oracle:
the step it picks after every update, on dense periodic and walled packings, in FP64
and mixed precision, alone and per sub-scene."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def _clouds():
    a = workloads.periodic_cloud(1800, 71, phi=0.34, inflate=1.06, vel_scale=0.05,
                                 angvel_scale=20.0)
    a.velgrad = np.diag([-5.0, -5.0, -5.0])
    b = workloads.box_cloud(1500, 72, phi=0.3, inflate=1.05, gravity=(0, 0, -9.81),
                            two_materials=True, vel_scale=0.03)
    return a, b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which,interval", [(0, 1), (1, 1), (1, 3)])
def test_step_sequence_matches_oracle(mods, precision, which, interval):
    oracle, pkg = mods
    w = _clouds()[which]
    o = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    for s in (o, g):
        s.set_timestepper(safety=0.7, interval=interval)
    tol = 1e-12 if precision == "fp64" else 1e-5
    changed = 0
    dt0 = o.clock()[2]
    seq = []
    for it in range(7):
        o.step(1)
        g.step(1)
        do, dg = o.clock()[2], g.dt()
        seq.append((it, do, dg))
        assert abs(dg / do - 1) < tol, seq
        changed += do != dt0
        assert g.clock()[1] == pytest.approx(o.clock()[1], rel=tol)
    assert changed >= 1


def test_per_subscene_steppers(mods):
    oracle, pkg = mods
    a, b = _clouds()
    oa, ob = oracle.OracleScene.from_workload(a), oracle.OracleScene.from_workload(b)
    g = pkg.Scene.from_workload(a, dt=oa.clock()[2])
    sb = g.add_workload(b, material_base=8, dt=ob.clock()[2])
    oa.set_timestepper(safety=0.6, interval=2)
    g.set_timestepper(safety=0.6, interval=2, sub=0)       # sub-scene b keeps its fixed dt
    for _ in range(5):
        oa.step(1)
        ob.step(1)
        g.step(1)
        assert abs(g.subscene(0)["dt"] / oa.clock()[2] - 1) < 1e-12
        assert g.subscene(sb)["dt"] == ob.clock()[2]
