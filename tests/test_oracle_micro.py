"""Oracle micromechanics (fabricTensor, normalShearStressTensors, bodyStressTensors of
the utils reference) pinned to closed forms and to identities with the separately
computed Love-Weber stress.  A dropped sign, a transposed product or a wrong arm
(centre-to-centre instead of centre-to-contact) fails one of them."""
import numpy as np

import workloads

PI = np.pi


def _ip2_kn(E1, r1, E2, r2):
    k1, k2 = E1 * 2 * r1, E2 * 2 * r2
    return k1 * k2 / (k1 + k2)


def test_force_chain_closed_forms(oracle_mod):
    """Periodic chain of four spheres along x overlapping by delta: every contact has
    n = e_x and N = kn delta, so F = e_x e_x, normal stress -l N / (Ly Lz a) ... per
    contact summed over four contacts in a cell of length 4a, shear part zero, and each
    sphere is squeezed from both sides: sigma_b,xx = -2 (r - delta/2) N / V_b."""
    r, delta = 1e-3, 2e-6
    a = 2 * r - delta
    Lx, Ly, Lz = 4 * a, 5 * r, 5.5 * r
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([Lx, Ly, Lz]), damping=0.0)
    E = 5e7
    s.set_material(0, 2600.0, E, 0.25, 0.5)
    s.add_spheres([[k * a + 0.1 * r, 2 * r, 2.5 * r] for k in range(4)], [r] * 4, fixed=[1] * 4)
    s.set_dt(1e-7)
    s.step(1)
    m = s.micro()
    N = _ip2_kn(E, r, E, r) * delta
    assert m["n_contacts"] == 4
    assert np.allclose(m["fabric"], np.diag([1.0, 0, 0]), atol=1e-15)
    V = Lx * Ly * Lz
    assert np.isclose(m["normal_stress"][0, 0], -4 * a * N / V, rtol=1e-9)
    assert np.all(np.abs(m["normal_stress"] - np.diag([m["normal_stress"][0, 0], 0, 0])) < 1e-20)
    assert np.all(np.abs(m["shear_stress"]) < 1e-12 * abs(m["normal_stress"][0, 0]))
    Vb = 4.0 / 3.0 * PI * r ** 3
    for b in range(4):
        sb = m["body_stress"][b]
        assert np.isclose(sb[0, 0], -2 * (r - delta / 2) * N / Vb, rtol=1e-9)
        off = sb.copy()
        off[0, 0] = 0
        assert np.all(np.abs(off) < 1e-12 * abs(sb[0, 0]))


def test_sphere_on_floor_body_stress(oracle_mod):
    """A sphere resting on the floor wall carries m g at the contact point
    x = -(r - pen/2) e_z below its centre: sigma_zz = -(r - pen/2) m g / V_b."""
    r, E, rho, g = 0.01, 5e7, 2600.0, 9.81
    s = oracle_mod.OracleScene(box_lo=(0, 0, 0), box_hi=(0.1, 0.1, 0.1), wall_mask=1 << 4,
                               gravity=(0, 0, -g), damping=0.2)
    s.set_material(0, rho, E, 0.25, 0.5)
    s.add_spheres([[0.05, 0.05, r]], [r])
    m_ = rho * 4.0 / 3.0 * PI * r ** 3
    s.set_dt(2 * PI * np.sqrt(m_ / (E * r)) / 60)
    s.step(6000)
    pen = s.contacts()["pen"][0]
    sb = s.micro()["body_stress"][0]
    Vb = 4.0 / 3.0 * PI * r ** 3
    assert np.isclose(sb[2, 2], -(r - pen / 2) * m_ * g / Vb, rtol=1e-6)
    assert abs(sb[0, 0]) < 1e-9 * abs(sb[2, 2]) and abs(sb[1, 1]) < 1e-9 * abs(sb[2, 2])


def test_identities_on_a_dense_packing(oracle_mod):
    """On a sheared, rotating dense packing: the fabric tensor is symmetric with unit
    trace; normal + transpose(shear) is the Love-Weber stress of the stats (computed in
    C from the same contacts); the volume-weighted body stresses sum to V times the
    transpose of that stress; an isotropic packing has a nearly isotropic fabric."""
    w = workloads.periodic_cloud(1500, 11, phi=0.34, inflate=1.06, vel_scale=0.05,
                                 angvel_scale=30.0)
    s = oracle_mod.OracleScene.from_workload(w)
    s.step(3)
    m = s.micro()
    F = m["fabric"]
    assert m["n_contacts"] > 800
    assert np.allclose(F, F.T, atol=1e-15) and abs(np.trace(F) - 1) < 1e-14
    assert np.all(np.abs(F - np.eye(3) / 3) < 0.06)
    sig = s.stats()["stress"]
    scale = np.max(np.abs(sig))
    assert np.all(np.abs(m["normal_stress"] + m["shear_stress"].T - sig) < 1e-10 * scale)
    assert np.any(np.abs(m["shear_stress"]) > 1e-4 * scale)      # friction carries load
    V = abs(np.linalg.det(s.cell()["H"]))
    Vb = 4.0 / 3.0 * PI * w.radius ** 3
    tot = np.einsum("b,bij->ij", Vb, m["body_stress"])
    assert np.all(np.abs(tot - V * sig.T) < 1e-9 * V * scale)
