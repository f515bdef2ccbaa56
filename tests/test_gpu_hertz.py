"""Hertz-Mindlin law (dem_set_law) on the GPU against the oracle: one-step contact
and state parity on walled and periodic packings, FP64 and mixed precision."""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, masses_of,
                               set_coord_scale, set_radii)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["box", "periodic"])
def test_hertz_one_step(mods, kind, precision):
    oracle, pkg = mods
    if kind == "box":
        w = workloads.box_cloud(1600, 81, phi=0.3, inflate=1.05, two_materials=True,
                                gravity=(0, 0, -9.81), vel_scale=0.05, angvel_scale=30.0)
    else:
        w = workloads.periodic_cloud(1700, 82, phi=0.34, inflate=1.06, vel_scale=0.05,
                                     angvel_scale=30.0)
        w.velgrad = np.diag([-4.0, -4.0, -4.0])
    o = oracle.OracleScene.from_workload(w)
    o.set_law(1)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    g.set_law(pkg.DEM_LAW_HERTZ_MINDLIN)
    tol = 1e-12 if precision == "fp64" else 1e-5
    eps = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    set_radii(w.radius)
    before = o.state()
    X = float(np.max(np.abs(before["pos"])))
    set_coord_scale(X)
    H = np.asarray(w.cell) if w.periodic else np.eye(3)
    import tests.parity_util as pu
    old = pu.BAND
    pu.BAND = 1e-9 if precision == "fp64" else 1e-5
    try:
        band = band_pairs(before["pos"], w.radius, w.periodic, H, oracle.pairs)
    finally:
        pu.BAND = old
    coord = None if precision == "fp64" else 2 * float(w.radius.max()) * 1.25
    o.step(1)
    g.step(1)
    co, cg = o.contacts(), g.contacts()
    n, _ = compare_contacts(co, cg, band, tol=tol, eps=eps, coord=coord)
    assert n > 500
    compare_states(o.state(), g.state(), X, tol=tol, co=co, masses=masses_of(w),
                   dt=o.clock()[2], gravity=float(np.linalg.norm(w.gravity)), eps=eps,
                   coord=coord)
    with pytest.raises(pkg.DemError) as e:        # chosen before the first step only
        g.set_law(pkg.DEM_LAW_LINEAR)
    assert e.value.code == 9


def test_hertz_statistics_over_many_steps(mods):
    oracle, pkg = mods
    w = workloads.periodic_cloud(1500, 83, phi=0.34, inflate=1.04, vel_scale=0.02)
    w.velgrad = np.diag([-10.0, -10.0, -10.0])
    o = oracle.OracleScene.from_workload(w)
    o.set_law(1)
    g = pkg.Scene.from_workload(w, dt=o.clock()[2])
    g.set_law(pkg.DEM_LAW_HERTZ_MINDLIN)
    o.step(150)
    g.step(150)
    so, sg = o.stats(), g.stats()
    assert abs(sg["kinetic_energy"] / so["ke"] - 1) < 1e-3
    assert abs(sg["n_contacts"] - so["n_contacts"]) <= max(2, 0.01 * so["n_contacts"])
    assert np.allclose(sg["stress"], so["stress"], rtol=1e-3, atol=1e-3 * np.abs(so["stress"]).max())
