"""Oracle pinned on sheared periodic cells (non-diagonal H and grad v).

The periodic cell of section 2.1.6 is a general parallelepiped H whose columns are the
cell vectors; a sheared cell is the case the diagonal-only shortcuts would get
wrong.  Each pin fails under a plausible slip: an image shift that uses only the
diagonal of H (the chain's closing contact is missed or lands at the wrong
distance), a homoDeform term that keeps only the diagonal of grad v (the lone
body leaves the affine field), or a cell update that is not (I + dt L) H.
"""
import numpy as np
import pytest


def _ip2_kn(E1, r1, E2, r2):
    k1, k2 = E1 * 2 * r1, E2 * 2 * r2
    return k1 * k2 / (k1 + k2)


def test_simple_shear_cell_update_is_exact(oracle_mod):
    """grad v = gamma_dot e_x (x) e_y is nilpotent, so (I + dt L)^n = I + n dt L exactly:
    H_xy grows by n dt gamma_dot L_y and nothing else moves."""
    Lx, Ly, Lz, gd, dt = 0.05, 0.04, 0.06, 2.0, 1e-4
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([Lx, Ly, Lz]), damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    s.add_spheres([[0.01, 0.02, 0.03]], [1e-3])
    s.set_dt(dt)
    L = np.zeros((3, 3))
    L[0, 1] = gd
    s.set_velgrad(L)
    s.step(300)
    H = s.cell()["H"]
    expect = np.diag([Lx, Ly, Lz])
    expect[0, 1] = 300 * dt * gd * Ly
    assert np.allclose(H, expect, rtol=1e-12, atol=1e-18)


def test_affine_body_follows_a_sheared_field(oracle_mod):
    """homoDeform = 2 with a full grad v (shear plus stretch): a lone body tracks the cell
    map x_k = H_k H_0^-1 x_0 from a cell that is already sheared."""
    H0 = np.array([[0.05, 0.012, -0.004], [0.0, 0.045, 0.009], [0.0, 0.0, 0.06]])
    s = oracle_mod.OracleScene(periodic=True, cell=H0, damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    x0 = np.array([0.031, 0.007, 0.044])
    s.add_spheres([x0], [1e-3])
    s.set_dt(1e-4)
    L = np.array([[-1.0, 3.0, 0.5], [0.7, 0.4, -2.0], [1.1, 0.0, -0.8]])
    s.set_velgrad(L)
    s.step(400)
    x = s.state()["pos"][0]
    H = s.cell()["H"]
    assert np.allclose(x, H @ np.linalg.solve(H0, x0), rtol=1e-11, atol=0)
    # the body is not trivially at rest: it moved along with the cell
    assert np.linalg.norm(x - x0) > 1e-3


def test_love_weber_stress_of_a_chain_along_a_sheared_cell_vector(oracle_mod):
    """Four equal spheres on the cell vector a_2 = H e_y of a sheared cell, each
    overlapping its neighbours by delta; the fourth contact closes through the image
    c = (0, 1, 0), shifted by the whole column a_2 (its x part is the shear).  Each
    contact carries F = kn delta along n = a_2 / |a_2| at arm l = |a_2| / 4, so
    sigma = -(kn delta |a_2| / det H) n (x) n (compression negative)."""
    r, delta, E = 1e-3, 2e-6, 5e7
    l = 2 * r - delta
    a2 = 4 * l
    th = 0.35                                    # tilt of a_2 from the y axis, in the x-y plane
    H = np.array([[6 * r, a2 * np.sin(th), 0.0],
                  [0.0, a2 * np.cos(th), 0.0],
                  [0.0, 0.0, 5.5 * r]])
    n = H[:, 1] / np.linalg.norm(H[:, 1])
    s = oracle_mod.OracleScene(periodic=True, cell=H, damping=0.0)
    s.set_material(0, 2600.0, E, 0.25, 0.5)
    base = np.array([2.5 * r, 0.3 * r, 2.7 * r])
    pos = [base + k * l * n for k in range(4)]
    s.add_spheres(pos, [r] * 4, fixed=[1] * 4)
    s.set_dt(1e-7)
    s.step(1)
    st = s.stats()
    assert st["n_contacts"] == 4
    c = s.contacts()
    assert sorted(map(tuple, np.abs(c["c"]))).count((0, 1, 0)) == 1
    F = _ip2_kn(E, r, E, r) * delta
    expect = -(F * np.linalg.norm(H[:, 1]) / np.linalg.det(H)) * np.outer(n, n)
    assert np.allclose(st["stress"], expect, rtol=1e-9, atol=1e-12 * abs(expect).max())
    assert st["Z"] == 2.0


def _sheared_packing(oracle_mod, n=600, seed=71, gamma=0.0, steps=0):
    """A periodic packing with a contact network and shear history, sheared by simple
    shear until H_xy / H_yy = gamma while it is slowly compacted (the oracle's own
    stepping; the compaction makes the image velocity grad(v)_prev H_prev c depend on
    every column of H_prev, so a flip must carry H_prev too)."""
    import workloads
    w = workloads.periodic_cloud(n, seed, phi=0.34, inflate=1.06, vel_scale=0.02,
                                 angvel_scale=10.0)
    s = oracle_mod.OracleScene.from_workload(w)
    if steps:
        dt = s.clock()[2]
        L = -5.0 * np.eye(3)
        L[0, 1] = gamma / (steps * dt)
        s.set_velgrad(L)
        s.step(steps)
    return s, w


def test_automatic_flip_of_a_simple_shear_cell(oracle_mod):
    """Simple shear H_xy = 0.8 L_x: the reduction subtracts the first cell vector once,
    H'_xy = -0.2 L_x; the new cell spans the same lattice (H^-1 H' integer, det 1) and
    a second call finds nothing to reduce."""
    Lx, Ly, Lz = 0.03, 0.025, 0.028
    H = np.diag([Lx, Ly, Lz])
    H[0, 1] = 0.8 * Lx
    s = oracle_mod.OracleScene(periodic=True, cell=H, damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    s.add_spheres([[0.01, 0.01, 0.01]], [1e-3])
    K = s.flip_cell()
    assert K.tolist() == [[0, -1, 0], [0, 0, 0], [0, 0, 0]]
    Hn = s.cell()["H"]
    assert np.isclose(Hn[0, 1], -0.2 * Lx, rtol=1e-12)
    T = np.linalg.solve(H, Hn)
    assert np.allclose(T, np.rint(T), atol=1e-12) and round(np.linalg.det(T)) == 1
    assert s.flip_cell().tolist() == [[0] * 3] * 3
    with pytest.raises(ValueError):
        s.flip_cell([[1, 0, 0], [0, 0, 0], [0, 0, 0]])     # det(I + K) = 2


def test_flip_keeps_every_interaction(oracle_mod):
    """Fig. 6: flipping the cell does not change the simulation.  Two copies of a
    sheared packing step on together, one flipped half way: the same contacts carry
    the same forces (their shifts related by M^-1) and the bodies follow the same
    trajectory, to rounding."""
    a, w = _sheared_packing(oracle_mod, gamma=0.7, steps=150)
    b, _ = _sheared_packing(oracle_mod, gamma=0.7, steps=150)
    assert a.cell()["H"][0, 1] > 0.65 * a.cell()["H"][1, 1]
    a.step(20)
    b.step(20)
    K = a.flip_cell()
    assert K[0, 1] == -1
    Minv = np.linalg.inv(np.eye(3) + K)
    a.step(30)
    b.step(30)
    ca, cb = a.contacts(), b.contacts()
    assert len(ca["id1"]) == len(cb["id1"]) > 120
    assert np.array_equal(ca["id1"], cb["id1"]) and np.array_equal(ca["id2"], cb["id2"])
    assert np.array_equal(ca["c"], np.rint(cb["c"] @ Minv.T).astype(int))
    assert np.any(ca["c"] != cb["c"])
    fs = np.linalg.norm(cb["fs"], axis=1)
    assert np.count_nonzero(fs) > 60
    scale = np.abs(cb["fn"]).max()
    assert np.abs(ca["fn"] - cb["fn"]).max() < 1e-8 * scale
    assert np.abs(ca["fs"] - cb["fs"]).max() < 1e-8 * scale
    sa, sb = a.state(), b.state()
    assert np.abs(sa["pos"] - sb["pos"]).max() < 1e-12 * np.abs(sb["pos"]).max()
    assert np.abs(sa["vel"] - sb["vel"]).max() < 1e-8 * np.abs(sb["vel"]).max()
