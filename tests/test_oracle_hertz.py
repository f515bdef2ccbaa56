"""Oracle Hertz-Mindlin law (Ip2_FrictMat_FrictMat_MindlinPhys and
Law2_ScGeom_MindlinPhys_Mindlin; reading R18 of dem_oracle.c) pinned to Hertz theory: the static
force of an overlap, the duration of a head-on impact (from the energy integral,
evaluated here by quadrature), restitution 1 without damping, the text's shear
constant for equal materials, and energy conservation over a collision cascade."""
import numpy as np
import pytest

import workloads

PI = np.pi


def _mass(rho, r):
    return rho * 4.0 / 3.0 * PI * r ** 3


def _estar(E1, nu1, E2, nu2):
    return 1.0 / ((1 - nu1 ** 2) / E1 + (1 - nu2 ** 2) / E2)


def test_static_overlap_force(oracle_mod):
    r1, r2, E1, E2, nu1, nu2, d = 1e-3, 1.5e-3, 5e7, 2e8, 0.25, 0.3, 3e-6
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_law(1)
    s.set_material(0, 2600.0, E1, nu1, 0.5)
    s.set_material(1, 1500.0, E2, nu2, 0.5)
    s.add_spheres([[0, 0, 0], [r1 + r2 - d, 0, 0]], [r1, r2], [0, 1], fixed=[1, 1])
    s.set_dt(1e-8)
    s.step(1)
    c = s.contacts()
    Rs = r1 * r2 / (r1 + r2)
    F = 4.0 / 3.0 * _estar(E1, nu1, E2, nu2) * np.sqrt(Rs) * d ** 1.5
    assert np.isclose(c["fn"][0, 0], F, rtol=1e-9)
    assert np.isclose(c["pen"][0], d, rtol=1e-9)


def test_equal_material_shear_constant_is_the_texts(oracle_mod):
    """For equal materials the text writes kso = 2 sqrt(4R) G / (2 - nu), R the
    effective radius r/2 of two equal spheres."""
    r, E, nu = 1e-3, 5e7, 0.3
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_law(1)
    s.set_material(0, 2600.0, E, nu, 0.5)
    s.add_spheres([[0, 0, 0], [2 * r - 1e-6, 0, 0]], [r, r], fixed=[1, 1])
    s.set_dt(1e-8)
    s.step(1)
    G = E / (2 * (1 + nu))
    R = r / 2
    kso = 2 * np.sqrt(4 * R) * G / (2 - nu)
    kno = 4.0 / 3.0 * (E / (2 * (1 - nu ** 2))) * np.sqrt(R)
    phys = s.contacts()["phys"][0]
    assert np.isclose(phys[1], kso, rtol=1e-12) and np.isclose(phys[0], kno, rtol=1e-12)


def test_impact_duration_and_restitution(oracle_mod):
    """m* x'' = -K x^3/2: the maximum overlap follows from 1/2 m* v^2 = 2/5 K x^5/2 and
    the contact lasts 2 (x_max / v) * int_0^1 (1 - u^5/2)^-1/2 du; restitution 1."""
    quad = pytest.importorskip("scipy.integrate").quad
    r1, r2, E, nu, rho, v = 1e-3, 1.2e-3, 5e7, 0.25, 2600.0, 0.1
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_law(1)
    s.set_material(0, rho, E, nu, 0.0)
    e = np.array([0.6, 0.0, 0.8])
    x1 = np.zeros(3)
    m1, m2 = _mass(rho, r1), _mass(rho, r2)
    ms = m1 * m2 / (m1 + m2)
    K = 4.0 / 3.0 * _estar(E, nu, E, nu) * np.sqrt(r1 * r2 / (r1 + r2))
    xmax = (5 * ms * v ** 2 / (4 * K)) ** 0.4
    integral = quad(lambda u: (1 - u ** 2.5) ** -0.5, 0, 1)[0]
    T = 2 * xmax / v * integral
    gap = 0.02 * v * T
    s.add_spheres([x1, x1 + (r1 + r2 + gap) * e], [r1, r2], vel=[m2 / (m1 + m2) * v * e,
                                                                 -m1 / (m1 + m2) * v * e])
    dt = T / 2000
    s.set_dt(dt)
    n_in = 0
    seen = False
    for _ in range(6000):
        s.step(1)
        if len(s.contacts()["id1"]):
            seen = True
            n_in += 1
        elif seen:
            break
    assert abs(n_in * dt - T) <= 3 * dt
    st = s.state()
    vrel = np.dot(st["vel"][1] - st["vel"][0], e)
    assert np.isclose(vrel, v, rtol=2e-3)


def _cascade_spread(oracle_mod, dt_factor):
    w = workloads.periodic_cloud(300, 5, phi=0.3, inflate=1.0, friction=0.0, vel_scale=0.3,
                                 damping=0.0)
    s = oracle_mod.OracleScene.from_workload(w)
    s.set_law(1)
    s.set_dt(s.clock()[2] * dt_factor)
    s.step(1)
    E0, spread, nc = None, [], 0
    for _ in range(int(400 / dt_factor)):
        s.step(1)
        en = s.energy()
        tot = en["kinTrans"] + en["kinRot"] + en["elastPotential"]
        E0 = tot if E0 is None else E0
        spread.append(tot / E0 - 1)
        nc = max(nc, len(s.contacts()["id1"]))
    return float(np.max(np.abs(spread))), nc


def test_energy_conserved_in_a_frictionless_cascade(oracle_mod):
    """Kinetic + Hertz elastic energy (2/5 Fn pen per contact) of a frictionless,
    undamped periodic cloud stays constant up to the leapfrog's O(dt) oscillation:
    small, and halved when dt is halved (a wrong elastic-energy factor or force law
    would leave an offset that does not shrink)."""
    a, nc = _cascade_spread(oracle_mod, 1.0)
    b, _ = _cascade_spread(oracle_mod, 0.5)
    assert nc >= 10
    assert a < 2e-3 and b < 0.7 * a
