"""Peri3dController on the GPU (dem_set_peri3d) against the oracle: strain-controlled
paths step by step (strain, stress, cell), the first steps of a stress-controlled run,
a rotated start, and a full stress-controlled run reaching its goals in FP64 and mixed
precision."""
import numpy as np
import pytest

import workloads
from tests.test_oracle_peri3d import _tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def _pair(mods, precision="fp64", n=800, seed=91):
    oracle, pkg = mods
    w = workloads.periodic_cloud(n, seed, phi=0.36, inflate=1.05, friction=0.5, vel_scale=0.01)
    o = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    return o, g, w


def test_strain_paths_step_by_step(mods):
    """All components strain-controlled (a path with three couples on xy): strain and
    cell agree with the oracle every step; the stress of the contacts agrees at the
    one-step parity bar."""
    o, g, w = _pair(mods)
    goal = [-0.004, 0.002, -0.003, 0.0, 0.001, 0.006]
    paths = [[], [], [], [], [], [[1, 2], [2, -1], [3, 1]]]
    for s in (o, g):
        s.set_peri3d(goal, 0, 60, paths=paths)
    for k in range(60):
        o.step(1)
        g.step(1)
        ro, rg = o.peri3d(), g.peri3d()
        assert np.allclose(rg["strain"], ro["strain"], rtol=0, atol=1e-13), k
        scale = max(1.0, float(np.abs(ro["stress"]).max()))
        assert np.abs(rg["stress"] - ro["stress"]).max() < 1e-9 * scale, (k, rg["stress"], ro["stress"])
    assert rg["done"] and ro["done"]
    assert np.allclose(g.cell()["H"], o.cell()["H"], rtol=0, atol=1e-15)
    assert np.allclose(rg["strain"], goal, atol=1e-12)


def test_first_steps_of_a_stress_controlled_run(mods):
    """Normal stresses controlled, xy strain prescribed: the first update's elastic
    estimate and the next predictor updates give the same rates and cell as the
    oracle over the first 25 steps."""
    o, g, w = _pair(mods)
    goal = [-1e4, -1e4, -1e4, 0.0, 0.0, 0.01]
    for s in (o, g):
        s.set_peri3d(goal, 0b000111, 3000, young_est=1e9, max_strain_rate=5.0)
    for k in range(25):
        o.step(1)
        g.step(1)
        ro, rg = o.peri3d(), g.peri3d()
        assert np.allclose(rg["rate"], ro["rate"], rtol=1e-9, atol=1e-12), (k, rg["rate"], ro["rate"])
        assert np.allclose(rg["stress"], ro["stress"], rtol=1e-8, atol=1e-6), (k, rg["stress"], ro["stress"])
    assert np.allclose(g.cell()["H"], o.cell()["H"], rtol=1e-12, atol=0)


def test_rotated_start(mods):
    oracle, pkg = mods
    goal = np.array([0.01, -0.004, 0.0, 0.0, 0.003, 0.012])
    c, sn = np.cos(np.pi / 6), np.sin(np.pi / 6)
    R = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1.0]])
    w = workloads.periodic_cloud(300, 92, phi=0.2)
    g = pkg.Scene.from_workload(w)
    H0 = g.cell()["H"]
    g.set_peri3d(goal, 0, 200, trsf0=R)
    g.step(200)
    r = g.peri3d()
    assert r["done"] and np.allclose(r["strain"], goal, atol=1e-12)
    assert np.allclose(g.cell()["H"], (np.eye(3) + _tensor(goal)) @ H0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stress_goals_are_met(mods, precision):
    oracle, pkg = mods
    w = workloads.periodic_cloud(600, 81, phi=0.36, inflate=1.04, friction=0.5)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, precision=prec)
    g.set_peri3d([-2e4, -2e4, -2e4, 0.0, 0.0, 0.02], 0b000111, 2500, young_est=5e6)
    g.step(2500)
    r = g.peri3d()
    assert r["done"]
    assert np.all(np.abs(r["stress"][:3] / -2e4 - 1) < 0.03), r["stress"]
    assert r["strain"][5] == pytest.approx(0.02, rel=1e-9)


def test_controller_errors(mods):
    oracle, pkg = mods
    box = pkg.Scene.from_workload(workloads.box_cloud(100, 93, phi=0.2))
    with pytest.raises(pkg.DemError):
        box.set_peri3d([0] * 6, 0, 10)
    w = workloads.periodic_cloud(200, 94, phi=0.2)
    g = pkg.Scene.from_workload(w)
    with pytest.raises(pkg.DemError):
        g.peri3d()
    with pytest.raises(pkg.DemError):
        g.set_peri3d([0] * 6, 0, 0)
    g.set_peri3d([0.001, 0, 0, 0, 0, 0], 0, 10)
    with pytest.raises(pkg.DemError) as e:
        g.add_workload(workloads.periodic_cloud(50, 95, phi=0.2), material_base=8)
    assert e.value.code != 0
