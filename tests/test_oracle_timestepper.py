"""Oracle GlobalStiffnessTimeStepper (section 2.1.5, eq. 2.12-2.14) pinned to closed
forms: a dimer (the text's two masses in opposite motion, dt_cr = sqrt(2 m / kn)), a
sphere caged by six fixed neighbours where the rotational stiffness sets the step,
the no-contact default, the cap and the update interval; density scaling (reading
R22 of dem_oracle.c) pinned by the same chain's stability limit at a step far above the natural one,
by the invariance of a trajectory counted in steps under a change of the target step,
and by the static penetration m g / kn (the weight is not scaled)."""
import numpy as np

PI = np.pi


def _mass(rho, r):
    return rho * 4.0 / 3.0 * PI * r ** 3


def test_dimer_step_is_safety_times_sqrt_2m_over_kn(oracle_mod):
    r, E, rho = 1e-3, 5e7, 2600.0
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_material(0, rho, E, 0.25, 0.5)
    s.add_spheres([[0, 0, 0], [2 * r - 1e-6, 0, 0]], [r, r])
    s.set_dt(1e-9)
    s.set_timestepper(safety=0.8, interval=1)
    s.step(1)
    kn = E * r                                   # series springs E 2r / 2
    m = _mass(rho, r)
    # translational: sqrt(2m/kn) along n, sqrt(2m/ks) across; rotational sqrt(2I/(ks d^2))
    # is larger (I = 0.4 m r^2, ks = kn/4): the normal mode sets it
    assert np.isclose(s.clock()[2], 0.8 * np.sqrt(2 * m / kn), rtol=1e-12)


def test_caged_sphere_rotational_stiffness_sets_the_step(oracle_mod):
    """Poisson ratio 1 makes ks = kn: the centre sphere's translational stiffness is
    2 kn + 4 ks = 6 kn per axis, its rotational stiffness 4 ks d^2 per axis, so
    sqrt(2 I / (4 kn d^2)) < sqrt(2 m / (6 kn)) and the rotation sets the step."""
    r, E, rho, delta = 1e-3, 5e7, 2600.0, 2e-6
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_material(0, rho, E, 1.0, 0.5)
    a = 2 * r - delta
    c = np.array([0.1, 0.1, 0.1])
    nb = [c + a * e for e in np.vstack([np.eye(3), -np.eye(3)])]
    s.add_spheres([c] + nb, [r] * 7, fixed=[0] + [1] * 6)
    s.set_dt(1e-9)
    s.set_timestepper(safety=0.5, interval=1)
    s.step(1)
    kn = E * r
    m = _mass(rho, r)
    I = 0.4 * m * r * r
    d = r - delta / 2
    rot = np.sqrt(2) * np.sqrt(I / (4 * kn * d * d))
    trans = np.sqrt(2) * np.sqrt(m / (6 * kn))
    assert rot < trans
    assert np.isclose(s.clock()[2], 0.5 * rot, rtol=1e-12)


def test_default_cap_and_interval(oracle_mod):
    r, E, rho = 1e-3, 5e7, 2600.0
    s = oracle_mod.OracleScene(damping=0.0)
    s.set_material(0, rho, E, 0.25, 0.5)
    s.add_spheres([[0, 0, 0], [0.01, 0, 0]], [r, r])      # apart: no contact
    s.set_dt(1e-9)
    s.set_timestepper(safety=0.8, interval=1)
    s.step(1)
    assert np.isclose(s.clock()[2], 0.8 * r / np.sqrt(E / rho), rtol=1e-14)
    s.set_timestepper(safety=0.8, interval=1, default_dt=3e-8)
    s.step(1)
    assert s.clock()[2] == 3e-8
    s.set_timestepper(safety=0.8, interval=1, max_dt=1e-8)
    s.step(1)
    assert s.clock()[2] == 1e-8
    # interval 4: the step changes only when the step count is a multiple of 4
    t = oracle_mod.OracleScene(damping=0.0)
    t.set_material(0, rho, E, 0.25, 0.5)
    t.add_spheres([[0, 0, 0], [2 * r - 1e-6, 0, 0]], [r, r])
    t.set_dt(1e-9)
    t.step(1)                                              # iter 1 before the stepper
    t.set_timestepper(safety=0.8, interval=4)
    t.step(2)
    assert t.clock()[2] == 1e-9                            # iters 1, 2: not due
    t.step(1)
    assert t.clock()[2] == 1e-9                            # iter 3: not due
    t.step(1)
    assert t.clock()[2] != 1e-9                            # iter 4: due


def _chain_growth(oracle_mod, safety):
    """Periodic chain of four overlapping spheres (springs kn between equal masses),
    started in its highest mode: the largest speed reached over 400 steps, relative
    to the initial one."""
    r, E, rho, delta, v0 = 1e-3, 5e7, 2600.0, 2e-5, 1e-4
    a = 2 * r - delta
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([4 * a, 5 * r, 5 * r]), damping=0.0)
    s.set_material(0, rho, E, 0.25, 0.0)
    s.add_spheres([[k * a + 0.1 * r, 2 * r, 2 * r] for k in range(4)], [r] * 4,
                  vel=[[v0 * (-1) ** k, 0, 0] for k in range(4)])
    s.set_dt(1e-9)
    s.set_timestepper(safety=safety, interval=1)
    vmax = 0.0
    for _ in range(400):
        s.step(1)
        vmax = max(vmax, float(np.abs(s.state()["vel"]).max()))
    return vmax / v0


def test_stepper_sits_at_the_chain_stability_limit(oracle_mod):
    """The highest mode of a chain of springs kn between masses m has omega =
    2 sqrt(kn/m), i.e. critical step sqrt(m/kn); each sphere has K = 2 kn, so eq. 2.12
    gives exactly that step.  Below it (safety 0.95) the leapfrog stays bounded,
    above it (1.05) the mode grows without bound."""
    assert _chain_growth(oracle_mod, 0.95) < 10
    assert _chain_growth(oracle_mod, 1.05) > 1e3


def _chain_growth_scaled(oracle_mod, safety, target):
    """The chain of _chain_growth under density scaling with step `target`."""
    r, E, rho, delta, v0 = 1e-3, 5e7, 2600.0, 2e-5, 1e-4
    a = 2 * r - delta
    s = oracle_mod.OracleScene(periodic=True, cell=np.diag([4 * a, 5 * r, 5 * r]), damping=0.0)
    s.set_material(0, rho, E, 0.25, 0.0)
    s.add_spheres([[k * a + 0.1 * r, 2 * r, 2 * r] for k in range(4)], [r] * 4,
                  vel=[[v0 * (-1) ** k, 0, 0] for k in range(4)])
    s.set_dt(1e-9)
    s.set_timestepper(safety=safety, interval=1)
    s.set_density_scaling(True, target)
    vmax = 0.0
    for _ in range(400):
        s.step(1)
        vmax = max(vmax, float(np.abs(s.state()["vel"]).max()))
    assert s.clock()[2] == target
    return vmax / v0


def test_density_scaling_moves_the_stability_limit_to_the_target_step(oracle_mod):
    """With every body's inertia scaled so that safety * sqrt(f) * t_b = targetDt, the
    chain's highest mode is stable at safety 0.95 and unstable at 1.05 whatever the
    target step (here 1000 times the natural critical step)."""
    r, E, rho = 1e-3, 5e7, 2600.0
    tcr = np.sqrt(_mass(rho, r) / (E * r))
    assert _chain_growth_scaled(oracle_mod, 0.95, 1000 * tcr) < 10
    assert _chain_growth_scaled(oracle_mod, 1.05, 1000 * tcr) > 1e3


def _resting(oracle_mod, target, steps):
    r, E, rho = 1e-3, 5e7, 2600.0
    s = oracle_mod.OracleScene(periodic=False, box_lo=(0, 0, 0), box_hi=(0.01, 0.01, 0.01),
                               wall_mask=0b010000, gravity=(0, 0, -9.81), damping=0.3)
    s.set_material(0, rho, E, 0.25, 0.5)
    s.add_spheres([[0.005, 0.005, r - 1e-7]], [r])    # touching the floor from the start
    s.set_dt(1e-9)
    s.set_timestepper(safety=0.5, interval=1)
    s.set_density_scaling(True, target)
    s.step(steps)
    return s


def test_density_scaling_trajectory_counted_in_steps_does_not_depend_on_the_target(oracle_mod):
    """x_{k+1} = x_k + dt v, v += dt F / (f m) with f proportional to target^2 and dt =
    target: the positions after each step are the same for any target step (to
    rounding), gravity included because the weight is m g and dt^2 g / f is fixed."""
    a = _resting(oracle_mod, 1e-3, 300).state()["pos"]
    b = _resting(oracle_mod, 7e-2, 300).state()["pos"]
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    assert abs(a[0, 2] - (1e-3 - 1e-7)) > 1e-9          # it moved


def test_density_scaling_keeps_the_static_penetration(oracle_mod):
    """A sphere resting on the floor settles at pen = m g / kn (kn = E r for the wall),
    the true weight: density scaling changes the dynamics, not the equilibrium."""
    r, E, rho = 1e-3, 5e7, 2600.0
    s = _resting(oracle_mod, 3e-2, 4000)
    pen = r - s.state()["pos"][0, 2]
    assert np.isclose(pen, _mass(rho, r) * 9.81 / (E * r), rtol=1e-6)
    f = s.density_scaling()[0]
    assert f > 1e6                                   # the inertia really was scaled
