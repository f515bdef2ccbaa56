"""The gravity-deposition workload exactly as specified (1000 spheres, radii
U[9, 11] mm, 0.3 x 0.3 x 0.6 m box with six walls, E = 5e7 Pa, friction 30 deg,
damping 0.2, dt = 0.5 p-wave step, 2000 steps), run in full on both sides."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deposition_full_run(precision):
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    w = workloads.deposition()
    orc = oracle.OracleScene.from_workload(w)
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    gpu = pkg.Scene.from_workload(w, precision=prec)
    assert gpu.dt() == orc.clock()[2]          # both take 0.5 * PWaveTimeStep
    tol = 1e-12 if precision == "fp64" else 1e-5
    for _ in range(4):
        orc.step(500)
        gpu.step(500)
        so, sg = orc.stats(), gpu.stats()
        assert abs(sg["kinetic_energy"] / so["ke"] - 1) < max(tol * 10, 1e-9 if tol < 1e-6 else 1e-4)
        nw = int(np.sum(orc.contacts()["id1"] < 0))
        if precision == "fp64":   # same decisions in the same precision: equal counts
            assert sg["n_contacts"] == so["n_contacts"] and sg["n_wall_contacts"] == nw
        else:   # FP32 contact tests: a sphere at the threshold may decide otherwise
            assert abs(sg["n_contacts"] - so["n_contacts"]) <= max(1, 0.01 * so["n_contacts"])
            assert abs(sg["n_wall_contacts"] - nw) <= max(1, 0.01 * nw)
    po, pg = orc.state()["pos"], gpu.state()["pos"]
    # FP64: rounding-level agreement (box scale 0.6 m); mixed: FP32 contact forces over
    # 2000 steps, bounded by 1e-4 of a radius (1 um)
    assert np.max(np.abs(pg - po)) < (0.6e-12 if precision == "fp64" else 1e-6)
    # the clock: 2000 additions of dt in the same order on both sides
    it, t = gpu.clock()
    assert it == 2000 and t == orc.clock()[1]
