"""Micromechanics on the GPU (dem_get_micro, dem_get_body_stress) against the oracle on
the same state: fabric, normal and shear stress parts, per-sphere stress tensors."""
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


@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_micro_matches_oracle(mods, kind, precision):
    oracle, pkg = mods
    if kind == "periodic":
        w = workloads.periodic_cloud(2100, 61, phi=0.34, inflate=1.06, vel_scale=0.05,
                                     angvel_scale=30.0)
    else:
        w = workloads.box_cloud(1900, 62, phi=0.3, inflate=1.05, two_materials=True,
                                gravity=(0, 0, -9.81), vel_scale=0.05, angvel_scale=30.0)
    o = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    g = pkg.Scene.from_workload(w, dt=o.clock()[2], precision=prec)
    o.step(2)
    g.step(2)
    mo, mg = o.micro(), g.micro()
    tol = 1e-11 if precision == "fp64" else 2e-4
    # contact sets agree away from the threshold band; compare the tensors as sums
    assert abs(mg["n_contacts"] - mo["n_contacts"]) <= (0 if precision == "fp64" else 3)
    for k in ("fabric", "normal_stress", "shear_stress"):
        scale = np.max(np.abs(mo["normal_stress"] if k != "fabric" else mo["fabric"]))
        assert np.max(np.abs(mg[k] - mo[k])) <= tol * scale, k
    sb_o, sb_g = mo["body_stress"], g.body_stress()
    scale = np.max(np.abs(sb_o), axis=(1, 2))
    err = np.max(np.abs(sb_g - sb_o), axis=(1, 2))
    assert np.sum(scale > 1e-6 * scale.max()) > 500
    # per sphere against its own load; mixed: a contact at the FP32 threshold may be
    # present on one side only, bounded by a small fraction of the largest load
    den = scale if precision == "fp64" else np.maximum(scale, 1e-3 * scale.max())
    den = np.maximum(den, 1e-300)
    assert np.max(err / den) <= (1e-10 if precision == "fp64" else 2e-3)
    # the whole-scene and sub-scene-0 views are the same reduction
    m0 = g.micro(0)
    assert np.array_equal(m0["fabric"], mg["fabric"])
    assert np.array_equal(m0["normal_stress"], mg["normal_stress"])
