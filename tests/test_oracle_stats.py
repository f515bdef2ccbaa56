"""Oracle pins for the orientation update and the scene statistics.

* Orientation (section 2.1.5, "Orientation (spherical)"): the rotation increment is
  the rotation by the vector omega+ dt, composed on the left of the current
  orientation (q+ = dq q).  Checked against scipy's rotation algebra (rotation
  vectors and matrices, not the oracle's quaternion product): a constant spin about
  a fixed axis turns the body by k |omega| dt after k steps, and two spin phases
  about different axes compose in the world frame (later rotation on the left).
  A swapped product (body-frame composition) or a half-angle slip is far outside
  the tolerance.
* Unbalanced force (utils.unbalancedForce, the mean/mean reading): mean over the dynamic bodies
  of the magnitude of the summed contact force (gravity excluded), over the mean
  magnitude of the interaction forces, on a hand-worked chain of spheres with a wall
  contact and a fixed sphere; the "max/max" sentence of section 1 and a variant that
  counts the weight give other numbers.
* Packing fraction (utils.porosity: phi = V_s / V): the volume of the
  spheres, overlaps ignored, over the box volume with walls, or the current cell
  volume |det H| of a periodic cell (sheared, and after a compaction, where the cell
  follows H_k = (1 + g dt)^k H_0 exactly up to rounding).
* Coordination (utils.avgNumInteractions): 2 C_ss / N, wall contacts
  excluded.
"""
import numpy as np
import pytest

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

PI = np.pi


def _rot_of(q_wxyz):
    q = np.asarray(q_wxyz, float)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])      # scipy: scalar last


def _free_scene(oracle_mod, n=1, damping=0.2):
    s = oracle_mod.OracleScene(damping=damping)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    pos = np.array([[0.1 * k, 0.05, -0.02] for k in range(n)])
    s.add_spheres(pos, np.full(n, 1e-3))
    return s


def test_constant_spin_turns_by_k_omega_dt(oracle_mod):
    """A free sphere spinning at constant omega about a fixed, oblique axis from a
    non-trivial start orientation: after k steps R(q_k) = Rot(k |omega| dt, axis) R(q_0)."""
    s = _free_scene(oracle_mod)
    axis = np.array([0.3, -0.5, 0.81])
    axis /= np.linalg.norm(axis)
    wmag, dt, k = 37.0, 1e-4, 250
    r0 = Rotation.from_rotvec([0.4, 1.1, -0.7])
    x0, y0, z0, w0 = r0.as_quat()
    s.set_state(angvel=[wmag * axis], ori=[[w0, x0, y0, z0]])
    s.set_dt(dt)
    s.step(k)
    st = s.state()
    np.testing.assert_allclose(st["angvel"][0], wmag * axis, rtol=0, atol=1e-12 * wmag)
    got = _rot_of(st["ori"][0]).as_matrix()
    want = (Rotation.from_rotvec(k * wmag * dt * axis) * r0).as_matrix()
    assert np.max(np.abs(got - want)) < 1e-12
    # the quaternion stays a unit quaternion
    assert abs(np.linalg.norm(st["ori"][0]) - 1.0) < 1e-13
    # a half-angle slip (rotation by 2 k |omega| dt) would be caught
    slip = (Rotation.from_rotvec(2 * k * wmag * dt * axis) * r0).as_matrix()
    assert np.max(np.abs(slip - want)) > 1e-2


def test_two_spin_phases_compose_in_the_world_frame(oracle_mod):
    """Spin about x for k1 steps, then about y for k2 steps: the orientation is
    Rot_y(theta2) Rot_x(theta1) R0 (the increment on the left, omega in world axes).
    The body-frame composition R0 Rot_x Rot_y (a swapped product) is rejected."""
    s = _free_scene(oracle_mod, damping=0.0)
    dt, k1, k2, w1, w2 = 2e-4, 300, 200, 11.0, -7.0
    r0 = Rotation.from_rotvec([-0.9, 0.2, 0.5])
    x0, y0, z0, w0 = r0.as_quat()
    s.set_dt(dt)
    s.set_state(angvel=[[w1, 0, 0]], ori=[[w0, x0, y0, z0]])
    s.step(k1)
    st = s.state()
    s.set_state(angvel=[[0, w2, 0]])
    s.step(k2)
    got = _rot_of(s.state()["ori"][0]).as_matrix()
    rx = Rotation.from_rotvec([k1 * w1 * dt, 0, 0])
    ry = Rotation.from_rotvec([0, k2 * w2 * dt, 0])
    want = (ry * rx * r0).as_matrix()
    assert np.max(np.abs(got - want)) < 1e-12
    swapped = (r0 * rx * ry).as_matrix()
    assert np.max(np.abs(swapped - want)) > 1e-2
    order = (rx * ry * r0).as_matrix()
    assert np.max(np.abs(order - want)) > 1e-2
    assert st["ori"].shape == (1, 4)


def _chain_scene(oracle_mod, g):
    """Spheres 0-1-2-3 along x (3 fixed), sphere 0 resting on the floor wall.
    Overlaps a, b, c between neighbours, w with the floor; zero velocities."""
    r, E = 0.01, 5e7
    pa, pb, pc, pw = 4e-6, 1e-6, 2.4e-6, 6e-7
    x = [0.05, 0.05 + 2 * r - pa, 0.05 + 4 * r - pa - pb, 0.05 + 6 * r - pa - pb - pc]
    z0 = r - pw
    pos = np.array([[x[0], 0.05, z0], [x[1], 0.05, z0 + 0.02 * r], [x[2], 0.05, z0 + 0.02 * r],
                    [x[3], 0.05, z0 + 0.02 * r]])
    # the three upper spheres are lifted a little: their x overlaps follow from the
    # exact distances computed below
    s = oracle_mod.OracleScene(box_lo=(0, 0, 0), box_hi=(0.2, 0.1, 0.1), wall_mask=1 << 4,
                               gravity=(0, 0, -g), damping=0.2)
    s.set_material(0, 2600.0, E, 0.25, 0.5)
    s.add_spheres(pos, np.full(4, r), fixed=[0, 0, 0, 1])
    s.set_dt(1e-6)
    return s, pos, r, E


def test_unbalanced_force_hand_worked_chain(oracle_mod):
    g = 100.0                         # a weight comparable to the contact forces
    s, pos, r, E = _chain_scene(oracle_mod, g)
    s.step(1)
    kn = E * r                        # equal radii and materials; the wall: refR = r
    # contact forces at the step's start positions (zero velocities: no shear force)
    F = np.zeros((4, 3))
    mags = []
    for i, j in ((0, 1), (1, 2), (2, 3)):
        d = pos[j] - pos[i]
        l = np.linalg.norm(d)
        fn = kn * (2 * r - l)
        F[j] += fn * d / l
        F[i] -= fn * d / l
        mags.append(fn)
    fw = kn * (r - pos[0, 2])         # floor wall: pen = r - z
    F[0, 2] += fw
    mags.append(fw)
    body = np.linalg.norm(F[:3], axis=1)          # dynamic bodies only (3 is fixed)
    want = body.mean() / np.mean(mags)
    st = s.stats()
    assert st["n_contacts"] == 3                  # sphere-sphere contacts
    assert abs(st["unbalanced"] - want) <= 1e-12 * want
    # Z = 2 C_ss / N with the wall contact left out
    assert st["Z"] == 2 * 3 / 4
    # planted variants of the definition are far off
    maxmax = body.max() / max(mags)
    m = 2600.0 * 4 / 3 * PI * r ** 3
    Fw = F[:3] + np.array([0, 0, -m * g])
    with_weight = np.linalg.norm(Fw, axis=1).mean() / np.mean(mags)
    all_bodies = np.linalg.norm(F, axis=1).mean() / np.mean(mags)
    for bad in (maxmax, with_weight, all_bodies):
        assert abs(bad - want) > 1e-3 * want
    # the force the oracle reports per body is the contact sum (no weight)
    np.testing.assert_allclose(s.state()["force"], F, rtol=0, atol=1e-12 * max(mags))


def test_packing_fraction_walled_box(oracle_mod):
    """Two overlapping spheres and a loose one in a 0.2 x 0.1 x 0.3 box: phi = sum of the
    full sphere volumes / box volume (overlap ignored), whichever walls are present."""
    radii = np.array([0.01, 0.012, 0.007])
    pos = np.array([[0.05, 0.05, 0.05], [0.05 + 0.015, 0.05, 0.05], [0.15, 0.05, 0.2]])
    for mask in (0b111111, 1 << 4):
        s = oracle_mod.OracleScene(box_lo=(0, 0, 0), box_hi=(0.2, 0.1, 0.3), wall_mask=mask,
                                   gravity=(0, 0, -9.81))
        s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
        s.add_spheres(pos, radii)
        s.set_dt(1e-6)
        s.step(1)
        want = np.sum(4.0 / 3.0 * PI * radii ** 3) / (0.2 * 0.1 * 0.3)
        assert abs(s.stats()["phi"] - want) <= 1e-14 * want


def test_packing_fraction_sheared_and_compacted_cell(oracle_mod):
    """Periodic cell: phi uses the current |det H|.  A sheared cell first, then an
    isotropic compaction with grad v = g I, where H_k = (1 + g dt)^k H_0 exactly."""
    H0 = np.array([[0.1, 0.03, 0.0], [0.0, 0.12, -0.02], [0.0, 0.0, 0.09]])
    radii = np.array([0.004, 0.005, 0.006, 0.0045])
    pos = np.array([[0.01, 0.02, 0.03], [0.05, 0.06, 0.02], [0.08, 0.03, 0.07],
                    [0.03, 0.09, 0.05]])
    s = oracle_mod.OracleScene(periodic=True, cell=H0, damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    s.add_spheres(pos, radii)
    dt, gr, k = 1e-5, -3.0, 40
    s.set_dt(dt)
    vs = np.sum(4.0 / 3.0 * PI * radii ** 3)
    s.step(1)
    assert abs(s.stats()["phi"] - vs / abs(np.linalg.det(H0))) <= 1e-13 * vs / abs(np.linalg.det(H0))
    s.set_velgrad(gr * np.eye(3))
    s.step(k)              # the gradient set between steps drives the next step
    Hk = (1 + gr * dt) ** k * H0
    want = vs / abs(np.linalg.det(Hk))
    assert np.allclose(s.cell()["H"], Hk, rtol=1e-13, atol=0)
    assert abs(s.stats()["phi"] - want) <= 1e-12 * want
    # the reference volume (H_0) would be off by the compaction
    assert abs(vs / abs(np.linalg.det(H0)) - want) > 1e-3 * want
