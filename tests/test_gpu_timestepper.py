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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_density_scaling_matches_oracle(mods, precision):
    """Density scaling (reading R22 of dem_oracle.c) on a walled packing under gravity: the step is the
    target, the per-body inertia factors match the oracle's, and so do the states after
    one step and after 20 more."""
    oracle, pkg = mods
    from tests.parity_util import compare_states, masses_of, set_coord_scale, set_radii
    w = _clouds()[1]
    o = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    target = 30 * o.clock()[2]
    for s in (o, g):
        s.set_timestepper(safety=0.7, interval=1)
        s.set_density_scaling(True, target)
    tol = 1e-12 if precision == "fp64" else 1e-5
    set_radii(w.radius)
    X = float(np.max(np.abs(w.pos)))
    set_coord_scale(X)
    o.step(1)
    g.step(1)
    assert o.clock()[2] == target and g.dt() == target
    fo, fg = o.density_scaling(), g.density_scaling()
    scaled = fo != 1.0
    assert scaled.sum() > 500 and np.all(fo[scaled] > 1)
    assert np.array_equal(fg == 1.0, ~scaled)
    assert np.abs(fg / fo - 1).max() < (1e-12 if precision == "fp64" else 1e-5)
    compare_states(o.state(), g.state(), X, tol=tol, co=o.contacts(), masses=masses_of(w),
                   dt=target, gravity=9.81,
                   eps=2.0 ** -52 if precision == "fp64" else 2.0 ** -23,
                   coord=None if precision == "fp64" else 2 * float(w.radius.max()) * 1.25)
    # 20 more steps: every body agrees but a handful, which a decision that rounding
    # can flip (the damping sign of eq. 2.9, a contact at its threshold) sends apart
    o.step(20)
    g.step(20)
    d = np.linalg.norm(g.state()["pos"] - o.state()["pos"], axis=1)
    close = d < (1e-9 if precision == "fp64" else 1e-5) * X
    assert close.mean() > 0.99, (close.mean(), d.max())
    ko, kg = o.stats()["ke"], g.stats()["kinetic_energy"]
    assert abs(kg / ko - 1) < (1e-3 if precision == "fp64" else 1e-2)


def test_density_scaling_switch_and_errors(mods):
    oracle, pkg = mods
    w = _clouds()[1]
    g = pkg.Scene.from_workload(w)
    with pytest.raises(pkg.DemError) as e:
        g.set_density_scaling(True, 1e-4)          # no time stepper yet
    assert e.value.code == 9
    g.set_timestepper(safety=0.7, interval=1)
    with pytest.raises(pkg.DemError):
        g.set_density_scaling(True, -1.0)
    g.set_density_scaling(True, 1e-4)
    g.step(3)
    assert g.dt() == 1e-4 and np.any(g.density_scaling() != 1.0)
    g.set_density_scaling(False)
    assert np.all(g.density_scaling() == 1.0)
    g.step(1)
    assert g.dt() != 1e-4
