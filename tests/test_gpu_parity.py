"""CUDA path vs the FP64 oracle through the C ABI, on seeded inputs.

Sizes span several thread blocks and leave ragged tails (bodies and contact
rows are not multiples of the block size); inputs cover walls, periodic cells
(with unwrapped positions several periods away), two materials, fixed bodies,
random velocities and spins, imported contact histories and a deforming cell.
"""
import numpy as np
import pytest

import workloads
from tests.parity_util import (band_pairs, compare_contacts, compare_states, export_oracle,
                               import_into_gpu, masses_of, set_coord_scale, set_radii)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return oracle, pkg


def _pair(w, mods, dt=None, **kw):
    oracle, pkg = mods
    set_radii(w.radius)
    orc = oracle.OracleScene.from_workload(w)
    if dt is not None:
        orc.set_dt(dt)
    gpu = pkg.Scene.from_workload(w, dt=orc.clock()[2], **kw)
    return orc, gpu


def _one_step_check(orc, gpu, w, oracle):
    before = orc.state()
    X = float(np.max(np.abs(before["pos"])))
    set_coord_scale(X)
    H = orc.cell()["H"] if w.periodic else np.eye(3)
    band = band_pairs(before["pos"], w.radius, w.periodic, H, oracle.pairs)
    orc.step(1)
    gpu.step(1)
    co, cg = orc.contacts(), gpu.contacts()
    n, worst = compare_contacts(co, cg, band)
    so, sg = orc.state(), gpu.state()
    ws = compare_states(so, sg, X, co=co, masses=masses_of(w), dt=orc.clock()[2],
                        gravity=float(np.linalg.norm(w.gravity)))
    return n, worst, ws


@pytest.mark.parametrize("seed", [0, 1])
def test_one_step_walled_box_two_materials(mods, seed):
    oracle, pkg = mods
    w = workloads.box_cloud(1537, seed, phi=0.3, inflate=1.05, two_materials=True,
                            vel_scale=0.05, angvel_scale=30.0)
    orc, gpu = _pair(w, mods)
    n, worst, ws = _one_step_check(orc, gpu, w, oracle)
    assert n > 500
    c = gpu.contacts()
    assert np.sum(c["id1"] < 0) > 10, "walls must be in contact in this case"


@pytest.mark.parametrize("seed", [2, 3])
def test_one_step_periodic_unwrapped(mods, seed):
    oracle, pkg = mods
    w = workloads.periodic_cloud(1801, seed, phi=0.33, inflate=1.06, vel_scale=0.05,
                                 angvel_scale=30.0)
    L = w.cell[0, 0]
    shift = (workloads.uniform(w.pos.size, seed + 5).reshape(w.pos.shape) * 5).astype(int) - 2
    w.pos = w.pos + shift * L
    orc, gpu = _pair(w, mods)
    n, worst, ws = _one_step_check(orc, gpu, w, oracle)
    assert n > 500
    c = gpu.contacts()
    assert np.any(np.any(c["c"] != 0, axis=1))


def test_one_step_from_imported_history(mods):
    """The oracle builds a contact history over 40 steps; the GPU imports that state and
    history (checkpoint/resume) and both take one more step."""
    oracle, pkg = mods
    w = workloads.periodic_cloud(1500, 7, phi=0.33, inflate=1.02, vel_scale=0.01,
                                 angvel_scale=5.0)
    orc, gpu = _pair(w, mods)
    orc.set_velgrad(np.diag([-50.0, -30.0, 20.0]))
    orc.step(40)
    ex = export_oracle(orc)
    assert np.count_nonzero(np.linalg.norm(ex["contacts"]["fs"], axis=1)) > 20
    import_into_gpu(gpu, ex)
    n, worst, ws = _one_step_check(orc, gpu, w, oracle)
    assert n > 40


def test_fixed_bodies_and_gravity(mods):
    oracle, pkg = mods
    w = workloads.box_cloud(700, 9, phi=0.3, inflate=1.04, vel_scale=0.05, angvel_scale=10.0)
    fixed = (workloads.uniform(w.n, 99) < 0.2).astype(np.uint8)
    set_radii(w.radius)
    orc = oracle.OracleScene(periodic=False, box_lo=w.box_lo, box_hi=w.box_hi,
                             wall_mask=w.wall_mask, gravity=w.gravity, damping=w.damping)
    gpu = pkg.Scene(periodic=False, box_lo=w.box_lo, box_hi=w.box_hi, wall_mask=w.wall_mask,
                    gravity=w.gravity, damping=w.damping)
    for s in (orc, gpu):
        m = w.materials[0]
        s.set_material(0, m.density, m.young, m.poisson, m.friction)
        s.add_spheres(w.pos, w.radius, w.mat_id, w.vel, w.angvel, fixed=fixed)
    dt = 0.5 * orc.pwave_dt()
    orc.set_dt(dt)
    gpu.set_dt(dt)
    _one_step_check(orc, gpu, w, oracle)
    st = gpu.state()
    assert np.array_equal(st["vel"][fixed == 1], w.vel[fixed == 1])


def test_trajectory_and_collider_reruns(mods):
    """Step both sides 120 times from the same state: every step's contact set matches
    (outside the threshold band) and forces agree, across several collider runs.

    The run is chaotic: a difference of one rounding grows by orders of magnitude over
    120 steps.  Beside the two runs the oracle runs a third time from the same state
    with every coordinate moved by one ulp; each step's bar is the larger of 1e-9 and
    the largest deviation of that nudged run from the oracle so far (the method's own
    chaos floor): the GPU may not depart from the oracle more than the oracle departs
    from itself.  (Over these 120 steps that floor grows from 1e-12 to about 1e-8.)"""
    oracle, pkg = mods
    w = workloads.periodic_cloud(1200, 4, phi=0.33, inflate=1.04, vel_scale=0.5,
                                 angvel_scale=100.0)
    orc, gpu = _pair(w, mods, verlet_dist=-0.02)   # small margin: frequent collider runs
    nudged = oracle.OracleScene.from_workload(w)
    nudged.set_state(pos=np.nextafter(nudged.state()["pos"], np.inf))
    L = w.cell[0, 0]
    floor_c = floor_s = 0.0
    worst_c = worst_s = 0.0
    for k in range(120):
        before = orc.state()
        band = band_pairs(before["pos"], w.radius, True, orc.cell()["H"], oracle.pairs)
        orc.step(1)
        gpu.step(1)
        nudged.step(1)
        set_coord_scale(float(np.max(np.abs(before["pos"]))))
        co, cg = orc.contacts(), gpu.contacts()
        _, fl = compare_contacts(co, nudged.contacts(), band, tol=1.0)
        floor_c = max(floor_c, fl["fn"], fl["fs"])
        _, wc = compare_contacts(co, cg, band, tol=max(1e-9, floor_c))
        worst_c = max(worst_c, wc["fn"], wc["fs"])
        if k % 20 == 19:
            so = orc.state()
            fls = compare_states(so, nudged.state(), L, tol=1.0)
            floor_s = max(floor_s, *fls.values())
            ws = compare_states(so, gpu.state(), L, tol=max(1e-9, floor_s))
            worst_s = max(worst_s, *ws.values())
    print(f"\nforces: GPU {worst_c:.2e}, chaos floor {floor_c:.2e}; "
          f"states: GPU {worst_s:.2e}, chaos floor {floor_s:.2e}")
    assert gpu.stats()["n_rebuilds"] >= 3


def test_deposition_statistics_over_many_steps(mods):
    """Config-0-like deposition (walls, gravity, damping, friction 30 deg) at reduced size:
    kinetic energy, coordination number and packing fraction within 1e-3 relative over
    300 steps (the trajectories are chaotic, the statistics are not)."""
    oracle, pkg = mods
    w = workloads.box_cloud(1000, 21, phi=0.3, inflate=1.02, friction=np.deg2rad(30),
                            vel_scale=0.05)
    orc, gpu = _pair(w, mods)
    for _ in range(3):
        orc.step(100)
        gpu.step(100)
        so, sg = orc.stats(), gpu.stats()
        assert abs(sg["kinetic_energy"] / so["ke"] - 1) < 1e-3
        assert abs(sg["coordination"] / so["Z"] - 1) < 1e-3
        assert abs(sg["packing_fraction"] / so["phi"] - 1) < 1e-12


def test_stats_match_oracle_definitions(mods):
    oracle, pkg = mods
    w = workloads.periodic_cloud(900, 8, phi=0.33, inflate=1.05, vel_scale=0.05)
    orc, gpu = _pair(w, mods)
    orc.step(1)
    gpu.step(1)
    so, sg = orc.stats(), gpu.stats()
    assert sg["n_contacts"] == so["n_contacts"]
    for a, b in (("kinetic_energy", "ke"), ("unbalanced_force", "unbalanced"),
                 ("coordination", "Z"), ("packing_fraction", "phi")):
        assert abs(sg[a] / so[b] - 1) < 1e-11, (a, sg[a], so[b])
    assert np.allclose(sg["stress"], so["stress"], rtol=0, atol=1e-11 * np.abs(so["stress"]).max())


def test_bitwise_determinism(mods):
    """Two runs of the same scene give bitwise identical states (fixed-order gather, no
    force atomics): the reproducibility the text's summation-order example asks for."""
    oracle, pkg = mods
    w = workloads.periodic_cloud(3000, 5, phi=0.33, inflate=1.05, vel_scale=0.3,
                                 angvel_scale=50.0)
    outs = []
    for _ in range(2):
        gpu = pkg.Scene.from_workload(w, dt=2e-7)
        gpu.set_cell_velgrad(np.diag([-20.0, -20.0, -20.0]))
        gpu.step(150)
        st = gpu.state()
        outs.append(st)
        gpu.close()
    for k in ("pos", "vel", "angvel", "ori", "force", "torque"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_error_paths(mods):
    oracle, pkg = mods
    s = pkg.Scene(periodic=False, box_lo=(0, 0, 0), box_hi=(1, 1, 1))
    with pytest.raises(pkg.DemError) as e:
        s.add_spheres([[0.5, 0.5, 0.5]], [0.01])          # material 0 not set
    assert e.value.code == 1
    s.set_material(0, 2600, 5e7, 0.25, 0.5)
    with pytest.raises(pkg.DemError) as e:
        s.add_spheres([[np.nan, 0.5, 0.5]], [0.01])
    assert e.value.code == 5
    with pytest.raises(pkg.DemError) as e:
        s.set_material(5000, 2600, 5e7, 0.25, 0.5)
    assert e.value.code == 1
    s.add_spheres([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], [0.011, 0.011])
    with pytest.raises(pkg.DemError) as e:
        s.set_contacts([0], [5], None, [[0, 0, 0]], [[1, 0, 0]], [[1, 1, 0.5]])
    assert e.value.code == 2
    s.step(3)
    assert s.clock()[0] == 3
    # a sphere larger than a third of the periodic cell
    p = pkg.Scene(periodic=True, cell=np.eye(3) * 0.01)
    p.set_material(0, 2600, 5e7, 0.25, 0.5)
    p.add_spheres([[0.005, 0.005, 0.005]], [0.004])
    with pytest.raises(pkg.DemError) as e:
        p.step(1)
    assert e.value.code == 6
