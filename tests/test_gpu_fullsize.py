"""Parity at the full size of the benchmarked workload: one million polydisperse
spheres (log-normal radii, median 1 mm, sigma 0.25, clipped to [0.5, 2] mm) in a
periodic cell, radii inflated 5% after placement so that every sphere has
contacts, under isotropic compaction.  The oracle steps the same seeded scene;
the CUDA path runs in the launch configuration the bench times."""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, masses_of, set_coord_scale,
                               set_radii)

pytestmark = pytest.mark.gpu


def test_million_spheres_one_step_and_statistics():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    w = workloads.compaction(n=1_000_000, seed=1)
    w.radius = w.radius * 1.05
    set_radii(w.radius)
    orc = oracle.OracleScene.from_workload(w)
    dt = orc.clock()[2]
    L = np.diag([-26.8, -26.8, -26.8])
    orc.set_velgrad(L)
    gpu = pkg.Scene.from_workload(w, dt=dt)
    gpu.set_cell_velgrad(L)
    X = float(np.max(np.abs(w.pos)))
    set_coord_scale(X)
    band = band_pairs(w.pos, w.radius, True, w.cell, oracle.pairs)
    orc.step(1)
    gpu.step(1)
    co, cg = orc.contacts(), gpu.contacts()
    n, worst = compare_contacts(co, cg, band)
    assert n > 300_000
    compare_states(orc.state(), gpu.state(), X, co=co, masses=masses_of(w), dt=dt)
    for _ in range(4):
        orc.step(5)
        gpu.step(5)
    so, sg = orc.stats(), gpu.stats()
    assert abs(sg["kinetic_energy"] / so["ke"] - 1) < 1e-3
    assert abs(sg["coordination"] / so["Z"] - 1) < 1e-3
    assert abs(sg["packing_fraction"] / so["phi"] - 1) < 1e-3
