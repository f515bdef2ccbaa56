"""Mixed-precision path (DEM_MIXED) against the FP64 oracle.

Expected agreement, from the arithmetic: the FP32 branch vector is formed from
offsets bounded by the contact distance, so lengths carry ~1e-7 relative
rounding; contact sets agree outside a 1e-5 r band around the threshold;
per-contact forces within 1e-5 of |Fn| + |Fs| plus kn * 4 * 2^-23 * (r1 + r2 +
margin); one-step states within 1e-5 of their scales; statistics over many
steps within 1e-3.
"""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, masses_of,
                               set_coord_scale, set_radii)

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23
TOL32 = 1e-5


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def _pair(w, mods, **kw):
    oracle, pkg = mods
    set_radii(w.radius)
    orc = oracle.OracleScene.from_workload(w)
    gpu = pkg.Scene.from_workload(w, dt=orc.clock()[2], precision=pkg.DEM_MIXED, **kw)
    return orc, gpu


def _band32(before, w, H, oracle):
    import tests.parity_util as pu
    old = pu.BAND
    pu.BAND = 1e-5
    try:
        return band_pairs(before["pos"], w.radius, w.periodic, H, oracle.pairs)
    finally:
        pu.BAND = old


@pytest.mark.parametrize("kind", ["box", "periodic"])
def test_mixed_one_step(mods, kind):
    oracle, pkg = mods
    if kind == "box":
        w = workloads.box_cloud(1537, 3, phi=0.3, inflate=1.05, two_materials=True,
                                vel_scale=0.05, angvel_scale=30.0)
    else:
        w = workloads.periodic_cloud(1801, 4, phi=0.33, inflate=1.06, vel_scale=0.05,
                                     angvel_scale=30.0)
    orc, gpu = _pair(w, mods)
    if kind == "periodic":
        L = np.diag([-20.0, -20.0, -20.0])
        orc.set_velgrad(L)
        gpu.set_cell_velgrad(L)
    before = orc.state()
    H = orc.cell()["H"] if w.periodic else np.eye(3)
    band = _band32(before, w, H, oracle)
    orc.step(1)
    gpu.step(1)
    co, cg = orc.contacts(), gpu.contacts()
    reach = 2 * float(w.radius.max()) * 1.25
    n, worst = compare_contacts(co, cg, band, tol=TOL32, eps=EPS32, coord=reach)
    assert n > 500
    X = float(np.max(np.abs(before["pos"])))
    set_coord_scale(X)
    compare_states(orc.state(), gpu.state(), X, tol=TOL32, co=co, masses=masses_of(w),
                   dt=orc.clock()[2], gravity=float(np.linalg.norm(w.gravity)), eps=EPS32,
                   coord=reach)


def test_mixed_compaction_statistics(mods):
    """Periodic compaction from 0.33 to ~0.6 solid fraction over 500 steps with several
    collider runs: kinetic energy and coordination number within 1e-3 of the FP64
    oracle as means over the last 100 steps (every 10th step, once the packing carries
    thousands of contacts: one contact more or less must be below the tolerance for a
    count statistic to be comparable), packing fraction at every sampled step."""
    oracle, pkg = mods
    w = workloads.periodic_cloud(4000, 6, phi=0.33, inflate=1.02, vel_scale=0.02)
    orc, gpu = _pair(w, mods, verlet_dist=-0.1)
    dt = orc.clock()[2]
    g = workloads.compaction_rate(0.33, 0.6, 500, dt)
    L = np.diag([g, g, g])
    orc.set_velgrad(L)
    gpu.set_cell_velgrad(L)
    orc.step(400)
    gpu.step(400)
    ke, z = [], []
    for _ in range(11):
        so, sg = orc.stats(), gpu.stats()
        assert so["n_contacts"] > 3000
        assert abs(sg["packing_fraction"] / so["phi"] - 1) < 1e-6
        ke.append((sg["kinetic_energy"], so["ke"]))
        z.append((sg["coordination"], so["Z"]))
        orc.step(10)
        gpu.step(10)
    ke, z = np.array(ke), np.array(z)
    assert abs(ke[:, 0].mean() / ke[:, 1].mean() - 1) < 1e-3
    assert abs(z[:, 0].mean() / z[:, 1].mean() - 1) < 1e-3
    assert gpu.stats()["n_rebuilds"] >= 2


def test_mixed_deposition_statistics(mods):
    oracle, pkg = mods
    w = workloads.box_cloud(1000, 22, phi=0.3, inflate=1.02, friction=np.deg2rad(30),
                            vel_scale=0.05)
    orc, gpu = _pair(w, mods)
    for _ in range(3):
        orc.step(100)
        gpu.step(100)
        so, sg = orc.stats(), gpu.stats()
        assert abs(sg["kinetic_energy"] / so["ke"] - 1) < 1e-3
        assert abs(sg["coordination"] / so["Z"] - 1) < 1e-3


def test_mixed_history_import_and_determinism(mods):
    """A checkpointed FP64 history resumes in the mixed path; two mixed runs are
    bitwise identical."""
    oracle, pkg = mods
    w = workloads.periodic_cloud(2000, 8, phi=0.33, inflate=1.03, vel_scale=0.02)
    orc = oracle.OracleScene.from_workload(w)
    orc.step(20)
    c = orc.contacts()
    st = orc.state()
    outs = []
    for _ in range(2):
        gpu = pkg.Scene.from_workload(w, dt=orc.clock()[2], precision=pkg.DEM_MIXED)
        gpu.set_state(pos=st["pos"], vel=st["vel"], angvel=st["angvel"], ori=st["ori"])
        gpu.set_contacts(c["id1"], c["id2"], c["c"], c["fs"], c["normal"], c["phys"])
        gpu.step(60)
        outs.append(gpu.state())
        gpu.close()
    for k in ("pos", "vel", "angvel", "ori", "force"):
        assert np.array_equal(outs[0][k], outs[1][k]), k
