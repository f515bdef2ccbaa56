"""Oracle Peri3dController (class reference; reading R23 in dem_oracle.c) pinned by:
the worked example of the xxPath attribute (tests/golden/peri3d_path.json), exact
strain paths under strain control (the cell ends at (I + E) H0 with E the goal
tensor), the same cell when the controller starts from a rotated transformation
(the global increment is carried into the cell frame and back), and a packing whose
three normal stresses reach their goals while a shear strain is prescribed."""
import json
import os

import numpy as np
import pytest

import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden", "peri3d_path.json")


def _lone(oracle_mod, H=None):
    H = np.diag([0.04, 0.05, 0.045]) if H is None else H
    s = oracle_mod.OracleScene(periodic=True, cell=H, damping=0.2)
    s.set_material(0, 2600.0, 5e7, 0.25, 0.5)
    s.add_spheres([[0.01, 0.02, 0.015]], [1e-3])
    s.set_dt(1e-4)
    return s


def _tensor(e6):
    xx, yy, zz, yz, zx, xy = e6
    return np.array([[xx, xy / 2, zx / 2], [xy / 2, yy, yz / 2], [zx / 2, yz / 2, zz]])


def test_xx_path_worked_example(oracle_mod):
    """The text's example with the value read as a strain (goal 300 scaled to 3e-3):
    strain-controlled xx follows the piecewise-linear path exactly, step by step."""
    g = json.load(open(GOLD))
    scale = 1e-5
    s = _lone(oracle_mod)
    goal = [g["goal_xx"] * scale, 0, 0, 0, 0, 0]
    s.set_peri3d(goal, 0, g["n_steps"], paths=[g["path"], [], [], [], [], []])
    done = 0
    for step, value in g["values_at_steps"]:
        s.step(step - done)
        done = step
        assert s.peri3d()["strain"][0] == pytest.approx(value * scale, rel=1e-9, abs=1e-15)
    assert s.peri3d()["done"]


def test_strain_control_reaches_the_goal_tensor(oracle_mod):
    """All six components strain-controlled on a linear path: after n steps the strain
    vector equals the goal, half way it is half the goal, and the cell is (I + E) H0."""
    s = _lone(oracle_mod)
    H0 = s.cell()["H"]
    goal = np.array([-0.01, 0.005, 0.002, 0.004, -0.003, 0.02])
    s.set_peri3d(goal, 0, 400)
    s.step(200)
    assert np.allclose(s.peri3d()["strain"], goal * 0.5, rtol=1e-9, atol=1e-15)
    s.step(200)
    r = s.peri3d()
    assert r["done"] and np.allclose(r["strain"], goal, rtol=1e-9, atol=1e-15)
    assert np.allclose(s.cell()["H"], (np.eye(3) + _tensor(goal)) @ H0, rtol=0, atol=1e-14)


def test_rotated_start_gives_the_same_global_deformation(oracle_mod):
    """Starting from Cell.trsf = R (a 30 degree rotation about z) the polar decomposition
    returns U = R, the prescribed global increments are rotated into the cell frame and
    back, and the cell deforms exactly as from trsf = I: H = (I + E) H0."""
    goal = np.array([0.01, -0.004, 0.0, 0.0, 0.003, 0.012])
    c, sn = np.cos(np.pi / 6), np.sin(np.pi / 6)
    R = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1.0]])
    out = []
    for trsf0 in (None, R):
        s = _lone(oracle_mod)
        H0 = s.cell()["H"]
        s.set_peri3d(goal, 0, 300, trsf0=trsf0)
        s.step(300)
        assert np.allclose(s.peri3d()["strain"], goal, rtol=1e-9, atol=1e-14)
        out.append(s.cell()["H"])
    assert np.allclose(out[0], (np.eye(3) + _tensor(goal)) @ H0, atol=1e-14)
    assert np.allclose(out[1], out[0], rtol=0, atol=1e-14)


def test_stress_goals_are_met_under_a_prescribed_shear(oracle_mod):
    """xx, yy, zz stress-controlled at -2e4 Pa from a loose packing while the shear
    strain xy follows its path: at the end the normal stresses are within 3% of the
    goal and the shear strain is exactly prescribed."""
    w = workloads.periodic_cloud(600, 81, phi=0.36, inflate=1.04, friction=0.5)
    s = oracle_mod.OracleScene.from_workload(w)
    goal = [-2e4, -2e4, -2e4, 0.0, 0.0, 0.02]
    s.set_peri3d(goal, 0b000111, 2500, young_est=5e6)
    s.step(2500)
    r = s.peri3d()
    assert r["done"]
    assert np.all(np.abs(r["stress"][:3] / -2e4 - 1) < 0.03), r["stress"]
    assert r["strain"][5] == pytest.approx(0.02, rel=1e-9)
    assert abs(r["strain"][3]) < 1e-12 and abs(r["strain"][4]) < 1e-12


def test_bad_parameters(oracle_mod):
    s = _lone(oracle_mod)
    with pytest.raises(ValueError):
        s.set_peri3d([0] * 6, 0, 0)
    with pytest.raises(ValueError):
        s.set_peri3d([0] * 6, 0, 10, paths=[[[2, 1], [1, 2]], [], [], [], [], []])
    box = oracle_mod.OracleScene(periodic=False, box_lo=(0, 0, 0), box_hi=(1, 1, 1))
    with pytest.raises(ValueError):
        box.set_peri3d([0] * 6, 0, 10)
