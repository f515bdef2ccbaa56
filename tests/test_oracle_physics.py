"""Oracle pinned to closed forms and invariants of the mechanics it integrates.

Each test would fail under a plausible slip in the oracle: a wrong stiffness
length (impact duration off by sqrt(2)), a wrong sign of the shear increment or
torque arm (rolling never reaches 5/7 v0; angular momentum drifts), a missing
half in the twist term (shear force turns twice as fast), a missing image
velocity or homoDeform term (periodic pair gains shear force; affine body lags).
"""
import numpy as np
import pytest

import workloads

PI = np.pi


def _ip2_kn(E1, r1, E2, r2):
    # series springs with l_i = 2 r_i (Ip2_FrictMat_FrictMat_FrictPhys, section 2.1.2)
    k1, k2 = E1 * 2 * r1, E2 * 2 * r2
    return k1 * k2 / (k1 + k2)


def _mass(rho, r):
    return rho * 4.0 / 3.0 * PI * r ** 3


@pytest.mark.parametrize("direction", [(1, 0, 0), (0.3, -0.5, 0.8)])
def test_binary_impact_duration_and_restitution(oracle_mod, direction):
    """Head-on impact, no damping, no friction: a linear spring of stiffness kn between
    masses m1, m2 gives contact duration pi*sqrt(m*/kn) and restitution 1."""
    r1, r2, E1, E2, rho1, rho2 = 1e-3, 1.4e-3, 5e7, 2e8, 2600.0, 1500.0
    e = np.asarray(direction, float)
    e /= np.linalg.norm(e)
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_material(0, rho1, E1, 0.25, 0.0)
    s.set_material(1, rho2, E2, 0.25, 0.0)
    m1, m2 = _mass(rho1, r1), _mass(rho2, r2)
    mstar = m1 * m2 / (m1 + m2)
    kn = _ip2_kn(E1, r1, E2, r2)
    T = PI * np.sqrt(mstar / kn)
    u = 0.05
    gap = u * T                      # closed in about T/2
    x1 = np.array([0.01, 0.02, 0.03])
    x2 = x1 + (r1 + r2 + gap) * e
    s.add_spheres([x1, x2], [r1, r2], [0, 1], vel=[u * e, -u * e])
    dt = T / 400
    s.set_dt(dt)
    in_contact = 0
    seen = False
    for _ in range(4000):
        s.step(1)
        c = s.contacts()
        if len(c["id1"]):
            seen = True
            in_contact += 1
            assert np.isclose(c["phys"][0, 0], kn, rtol=1e-14)
        elif seen:
            break
    assert abs(in_contact * dt - T) <= 2 * dt
    st = s.state()
    vrel_after = np.dot(st["vel"][1] - st["vel"][0], e)
    assert vrel_after > 0
    assert abs(vrel_after / (2 * u) - 1.0) < 1e-3


def test_resting_sphere_on_wall(oracle_mod):
    """A sphere on the floor wall under gravity settles at pen = m g / kn with kn = E r
    (wall equivalent radius = sphere radius) and carries exactly m g."""
    r, E, rho, g = 0.01, 5e7, 2600.0, 9.81
    s = oracle_mod.OracleScene(box_lo=(0, 0, 0), box_hi=(0.1, 0.1, 0.1), wall_mask=1 << 4,
                               gravity=(0, 0, -g), damping=0.2)
    s.set_material(0, rho, E, 0.25, 0.5)
    s.add_spheres([[0.05, 0.05, r]], [r])
    m = _mass(rho, r)
    kn = E * r
    T = 2 * PI * np.sqrt(m / kn)
    s.set_dt(T / 60)
    s.step(6000)
    c = s.contacts()
    assert list(c["id1"]) == [-5] and list(c["id2"]) == [0]
    pen_eq = m * g / kn
    assert abs(c["pen"][0] / pen_eq - 1) < 1e-6
    assert abs(c["fn"][0, 2] / (m * g) - 1) < 1e-6
    assert np.isclose(c["phys"][0, 0], kn, rtol=1e-14)


def test_sliding_sphere_reaches_rolling_at_five_sevenths(oracle_mod):
    """Sphere launched sliding (v0, no spin) on a frictional floor: Coulomb friction
    decelerates it and spins it up until rolling without slip at v = 5/7 v0,
    w_y = v / r (textbook solid-sphere result)."""
    r, E, rho, g, phi = 0.01, 5e7, 2600.0, 9.81, np.arctan(0.5)
    s = oracle_mod.OracleScene(box_lo=(-10, -1, 0), box_hi=(10, 1, 1), wall_mask=1 << 4,
                               gravity=(0, 0, -g), damping=0.0)
    s.set_material(0, rho, E, 0.25, phi)
    m = _mass(rho, r)
    kn = E * r
    v0 = 0.5
    s.add_spheres([[0.0, 0.0, r - m * g / kn]], [r], vel=[[v0, 0, 0]])
    T = 2 * PI * np.sqrt(m / kn)
    dt = T / 40
    s.set_dt(dt)
    t_slide = (2.0 / 7.0) * v0 / (0.5 * g)
    nsteps = int(1.5 * t_slide / dt)
    s.step(nsteps)
    vs, ws = [], []
    for _ in range(400):
        s.step(1)
        st = s.state()
        vs.append(st["vel"][0, 0])
        ws.append(st["angvel"][0, 1])
    vmean, wmean = np.mean(vs), np.mean(ws)
    assert abs(vmean / (5.0 / 7.0 * v0) - 1) < 5e-3
    assert abs(wmean * r / vmean - 1) < 5e-3


def _contact_pair_scene(oracle_mod, fixed=True):
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_material(0, 2600.0, 5e7, 0.25, 1.5)
    r1, r2 = 1e-3, 1.2e-3
    n0 = np.array([0.0, 0.0, 1.0])
    x1 = np.array([0.1, 0.2, 0.3])
    x2 = x1 + (r1 + r2 - 1e-4) * n0
    s.add_spheres([x1, x2], [r1, r2], fixed=[1, 1] if fixed else None)
    return s, x1, x2, r1, r2, n0


def test_twist_rotates_shear_force_with_the_pair(oracle_mod):
    """Both spheres spinning at W about the contact normal (kinematics imposed): the shear
    force must turn about n at the same rate W (twist term dt/2 n.(w1+w2)), exactly
    atan(W dt) per step for the first-order update, without any normal component."""
    s, x1, x2, r1, r2, n0 = _contact_pair_scene(oracle_mod)
    W = 40.0
    s.set_state(angvel=[W * n0, W * n0])
    dt = 1e-5
    s.set_dt(dt)
    s.step(1)
    c = s.contacts()
    fs0 = np.array([2e-3, 0.0, 0.0])
    s.set_contacts(c["id1"], c["id2"], c["c"], [fs0], c["normal"], c["phys"])
    k = 200
    s.step(k)
    fs = s.contacts()["fs"][0]
    ang = np.arctan2(fs[1], fs[0])
    assert abs(ang - k * np.arctan(W * dt)) < 1e-12
    assert abs(ang - W * k * dt) < 1e-5 * W * k * dt
    assert abs(fs[2]) < 1e-15
    assert np.isclose(np.linalg.norm(fs), np.linalg.norm(fs0) * (1 + (W * dt) ** 2) ** (k / 2),
                      rtol=1e-12)


def test_rigid_rotation_of_the_pair_rotates_shear_force(oracle_mod):
    """Pair driven along an exact rigid rotation (angular velocity W perpendicular to n):
    the ratchet-free relative velocity vanishes and the shear force must follow the
    rotation R(W t) fs0 and stay in the contact plane, up to O((W dt)^2) per step."""
    s, x1, x2, r1, r2, n0 = _contact_pair_scene(oracle_mod)
    Wv = np.array([30.0, 0.0, 0.0])
    ctr = 0.5 * (x1 + x2)
    dt = 2e-5
    s.set_dt(dt)

    def rot(t):
        a = Wv[0] * t
        return np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])

    def drive(t):
        R = rot(t)
        p = [ctr + R @ (x1 - ctr), ctr + R @ (x2 - ctr)]
        v = [np.cross(Wv, p[0] - ctr), np.cross(Wv, p[1] - ctr)]
        s.set_state(pos=p, vel=v, angvel=[Wv, Wv])

    drive(0.0)
    s.step(1)
    c = s.contacts()
    fs0 = np.array([0.0, 1.5e-3, 0.0])      # in the plane of n0 = z, along y
    s.set_contacts(c["id1"], c["id2"], c["c"], [fs0], c["normal"], c["phys"])
    k = 300
    for step in range(1, k + 1):
        drive(step * dt)
        s.step(1)
    c = s.contacts()
    fs, n = c["fs"][0], c["normal"][0]
    target = rot(k * dt) @ fs0
    th = Wv[0] * dt
    assert np.linalg.norm(fs - target) < 5 * k * th ** 2 * np.linalg.norm(fs0)
    assert abs(np.dot(fs, n)) < 5 * k * th ** 2 * np.linalg.norm(fs0)
    # a sign slip in the frame term would turn fs the other way: error O(k th)
    wrong = rot(-k * dt) @ fs0
    assert np.linalg.norm(fs - wrong) > 0.5 * k * th * np.linalg.norm(fs0)


def _cluster(oracle_mod, friction, seed=3, n=300):
    w = workloads.box_cloud(n, seed, phi=0.3, inflate=1.04, wall_mask=0, gravity=(0, 0, 0),
                            friction=friction, vel_scale=0.05, angvel_scale=20.0, damping=0.0)
    s = oracle_mod.OracleScene.from_workload(w)
    s.set_dt(0.1 * s.pwave_dt())
    return s, w


def _momenta(s, w):
    st = s.state()
    m = w.materials[0].density * 4.0 / 3.0 * PI * w.radius ** 3
    I = 0.4 * m * w.radius ** 2
    P = (m[:, None] * st["vel"]).sum(0)
    L = (np.cross(st["pos"], m[:, None] * st["vel"]) + I[:, None] * st["angvel"]).sum(0)
    pscale = (m[:, None] * np.abs(st["vel"])).sum()
    lscale = (np.abs(np.cross(st["pos"], m[:, None] * st["vel"])).sum() +
              (I[:, None] * np.abs(st["angvel"])).sum())
    return P, L, pscale, lscale


def test_momentum_conservation(oracle_mod):
    """No walls, no gravity, no damping: action = reaction gives exact linear momentum; the
    contact-point torque arms (C - x_i) give exact angular momentum (leapfrog form)."""
    s, w = _cluster(oracle_mod, friction=0.5)
    P0, L0, ps, ls = _momenta(s, w)
    s.step(1)
    assert s.stats()["n_contacts"] > 50
    s.step(299)
    P1, L1, _, _ = _momenta(s, w)
    assert np.all(np.abs(P1 - P0) < 1e-13 * ps)
    assert np.all(np.abs(L1 - L0) < 1e-12 * ls)


def test_energy_conservation_frictionless(oracle_mod):
    """No damping, no friction: kinetic + normal-spring energy is conserved up to the
    leapfrog's bounded oscillation (kinetic energy sits half a step away from the spring
    energy, an O(w dt) term: halving dt halves it) and does not drift."""
    devs, drifts = [], []
    for f in (1.0, 0.5):
        s, w = _cluster(oracle_mod, friction=0.0, seed=4, n=200)
        s.set_dt(f * 0.1 * s.pwave_dt())
        s.step(1)                     # the first contact pass measures the initial overlaps
        e0 = s.energy()
        E0 = e0["kinTrans"] + e0["kinRot"] + e0["elastPotential"]
        series = []
        for _ in range(int(800 / f)):
            s.step(1)
            e = s.energy()
            series.append(e["kinTrans"] + e["kinRot"] + e["elastPotential"])
        series = np.asarray(series)
        devs.append(np.max(np.abs(series - E0)) / E0)
        drifts.append(abs(series[-int(100 / f):].mean() - series[:int(100 / f)].mean()) / E0)
    assert devs[0] < 0.05
    assert 0.35 < devs[1] / devs[0] < 0.7
    assert max(drifts) < 0.5 * devs[0]


def test_energy_balance_with_friction(oracle_mod):
    """With friction the tracked total (kinetic + elastic + plastic dissipation) stays
    constant: slip dissipates exactly what the elastic and kinetic parts lose."""
    s, w = _cluster(oracle_mod, friction=0.3, seed=5, n=200)
    s.set_dt(0.05 * s.pwave_dt())
    s.step(1)
    E0 = s.energy()["total"]
    for _ in range(600):
        s.step(1)
    e = s.energy()
    assert e["plastDissip"] > 1e-3 * E0
    assert abs(e["total"] - E0) / E0 < 5e-3


def test_coulomb_bound_every_contact_every_step(oracle_mod):
    s, w = _cluster(oracle_mod, friction=0.2, seed=6, n=250)
    capped = 0
    for _ in range(150):
        s.step(1)
        c = s.contacts()
        fn = np.linalg.norm(c["fn"], axis=1)
        fs = np.linalg.norm(c["fs"], axis=1)
        assert np.all(fs <= c["phys"][:, 2] * fn * (1 + 1e-15) + 1e-300)
        capped += int(np.sum(fs >= c["phys"][:, 2] * fn * (1 - 1e-12)))
    assert capped > 0


def test_affine_body_stays_on_the_homogeneous_field(oracle_mod):
    """homoDeform = 2: a lone body in a cell deformed at constant grad(v) follows the cell
    map exactly: x_k = H_k H_0^-1 x_0 (to rounding)."""
    L = 0.05
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([L, L, 1.2 * L]), damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    x0 = np.array([0.031, 0.007, 0.044])
    s.add_spheres([x0], [1e-3])
    s.set_dt(1e-4)
    D = np.diag([-3.0, 1.5, -0.5])
    s.set_velgrad(D)
    H0 = s.cell()["H"]
    s.step(500)
    x = s.state()["pos"][0]
    H = s.cell()["H"]
    assert np.allclose(x, H @ np.linalg.solve(H0, x0), rtol=1e-12, atol=0)
    assert np.allclose(np.diag(H), np.diag(H0) * (1 + np.diag(D) * 1e-4) ** 500, rtol=1e-12)


def test_pair_across_boundary_under_isotropic_compaction_has_no_shear(oracle_mod):
    """Two spheres touching through the periodic image while the cell shrinks isotropically:
    their relative motion is along n, so no shear force may appear (needs the image
    velocity grad(v)_prev H_prev c and the homoDeform velocity terms).  No damping: the
    per-component damping of eq. 2.9 is not rotation invariant and would tilt the force."""
    L = 0.02
    s = oracle_mod.OracleScene(periodic=True, cell=np.eye(3) * L, damping=0.0)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    r = 1e-3
    dy, dz = 0.3 * r, 0.1 * r
    dx = np.sqrt((2.005 * r) ** 2 - dy ** 2 - dz ** 2)      # gap 0.005 r through the image
    s.add_spheres([[0.9 * r, 0.013, 0.007], [L + 0.9 * r - dx, 0.013 + dy, 0.007 + dz]], [r, r])
    s.set_dt(1e-6)
    s.set_velgrad(-20.0 * np.eye(3))
    seen = 0
    for _ in range(600):
        s.step(1)
        c = s.contacts()
        if len(c["id1"]):
            seen += 1
            assert tuple(c["c"][0]) == (-1, 0, 0)
            fn = np.linalg.norm(c["fn"][0])
            assert np.linalg.norm(c["fs"][0]) <= 1e-12 * fn + 1e-300
    assert seen > 10


def test_love_weber_stress_of_a_force_chain(oracle_mod):
    """Periodic chain of four equal spheres along x, each overlapping its neighbours by
    delta: the chain carries F = kn delta through the cross-section Ly*Lz, so
    sigma_xx = -F/(Ly Lz) (compression negative) and the other entries vanish."""
    r, delta = 1e-3, 2e-6
    a = 2 * r - delta
    Lx, Ly, Lz = 4 * a, 5 * r, 5.5 * r
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([Lx, Ly, Lz]), damping=0.0)
    E = 5e7
    s.set_material(0, 2600.0, E, 0.25, 0.5)
    pos = [[k * a + 0.1 * r, 2 * r, 2.5 * r] for k in range(4)]
    s.add_spheres(pos, [r] * 4, fixed=[1] * 4)
    s.set_dt(1e-7)
    s.step(1)
    st = s.stats()
    assert st["n_contacts"] == 4
    F = _ip2_kn(E, r, E, r) * delta
    sig = st["stress"]
    assert np.isclose(sig[0, 0], -F / (Ly * Lz), rtol=1e-9)
    off = sig.copy()
    off[0, 0] = 0
    assert np.all(np.abs(off) < 1e-12 * abs(sig[0, 0]))
    assert st["Z"] == 2.0


def test_stress_servo_reaches_its_goal(oracle_mod):
    """PeriTriaxController reading: lateral axes under stress control settle at the goal
    stress while the third axis is driven at its prescribed strain rate (and therefore
    loads up): the behaviour the controller's goal/stressMask attributes describe."""
    w = workloads.periodic_cloud(400, 31, phi=0.34, inflate=1.06, friction=0.5)
    s = oracle_mod.OracleScene.from_workload(w)
    goal = -5e4
    s.set_triax([goal, goal, -2.0], 0b011, [50.0, 50.0, 50.0], 0.25, 5)
    s.step(2500)
    sig = np.diag(s.stats()["stress"])
    L = np.diag(s.cell()["velgrad"])
    assert abs(sig[0] / goal - 1) < 0.02 and abs(sig[1] / goal - 1) < 0.02
    assert L[2] == -2.0
    s.step(1000)
    sig2 = np.diag(s.stats()["stress"])
    assert abs(sig2[0] / goal - 1) < 0.02 and abs(sig2[1] / goal - 1) < 0.02
    assert sig2[2] < sig[2] < 0          # the strain-controlled axis keeps compressing
