"""Oracle contact detection pinned against brute force and hand-worked cases."""
import numpy as np
import pytest

import workloads


def _set(I, J, C):
    return {(int(i), int(j), tuple(int(x) for x in c)) for i, j, c in zip(I, J, C)}


def test_hand_worked_periodic_pair(oracle_mod):
    # cell of edge 1: spheres at x=0.05 and x=0.95 (r=0.1) touch through the image c=(-1,0,0)
    pos = np.array([[0.05, 0.5, 0.5], [0.95, 0.5, 0.5], [0.5, 0.5, 0.5]])
    rad = np.array([0.1, 0.1, 0.1])
    for method in ("sweep", "grid", "brute"):
        I, J, C = oracle_mod.pairs(pos, rad, periodic=True, H=np.eye(3), method=method)
        assert _set(I, J, C) == {(0, 1, (-1, 0, 0))}
        I, J, C = oracle_mod.pairs(pos, rad, periodic=False, method=method)
        assert len(I) == 0
    # unwrapped positions two periods away find the same pair with the shifted image
    pos2 = pos.copy()
    pos2[1, 0] += 2.0
    I, J, C = oracle_mod.pairs(pos2, rad, periodic=True, H=np.eye(3))
    assert _set(I, J, C) == {(0, 1, (-3, 0, 0))}


def test_threshold_is_strict(oracle_mod):
    # exactly touching spheres are not in contact (real iff l < r1 + r2)
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    rad = np.array([0.25, 0.25])
    I, J, C = oracle_mod.pairs(pos, rad)
    assert len(I) == 0
    rad2 = np.array([0.25, 0.25 + 4e-16])   # r1 + r2 one ulp above 0.5
    I, J, C = oracle_mod.pairs(pos, rad2)
    assert len(I) == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("margin", [0.0, 2e-4])
def test_sweep_equals_bruteforce_aperiodic(oracle_mod, seed, margin):
    w = workloads.box_cloud(1500, seed, phi=0.3, inflate=1.05, wall_mask=0)
    a = oracle_mod.pairs(w.pos, w.radius, margin=margin, method="sweep")
    b = oracle_mod.pairs(w.pos, w.radius, margin=margin, method="brute")
    g = oracle_mod.pairs(w.pos, w.radius, margin=margin, method="grid")
    assert _set(*a) == _set(*b) == _set(*g)
    assert len(a[0]) > 500


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("margin", [0.0, 2e-4])
def test_sweep_equals_bruteforce_periodic(oracle_mod, seed, margin):
    w = workloads.periodic_cloud(1200, seed, phi=0.33, inflate=1.06)
    pos = w.pos.copy()
    # unwrap some bodies by whole periods: the search must not depend on wrapping
    L = w.cell[0, 0]
    shift = (workloads.uniform(pos.size, seed + 99).reshape(pos.shape) * 5).astype(int) - 2
    pos += shift * L
    a = oracle_mod.pairs(pos, w.radius, periodic=True, H=w.cell, margin=margin, method="sweep")
    b = oracle_mod.pairs(pos, w.radius, periodic=True, H=w.cell, margin=margin, method="brute")
    g = oracle_mod.pairs(pos, w.radius, periodic=True, H=w.cell, margin=margin, method="grid")
    sa = _set(*a)
    assert sa == _set(*b) == _set(*g)
    assert len(sa) > 500
    assert any(c != (0, 0, 0) for _, _, c in sa)


def test_sweep_equals_bruteforce_sheared_cell(oracle_mod):
    w = workloads.periodic_cloud(800, 5, phi=0.3, inflate=1.05)
    H = w.cell.copy()
    H[0, 1] = 0.3 * H[1, 1]       # sheared cell: second base vector leans along x
    a = oracle_mod.pairs(w.pos, w.radius, periodic=True, H=H, method="sweep")
    b = oracle_mod.pairs(w.pos, w.radius, periodic=True, H=H, method="brute")
    g = oracle_mod.pairs(w.pos, w.radius, periodic=True, H=H, method="grid")
    assert _set(*a) == _set(*b) == _set(*g)


def test_planted_missing_image_is_caught(oracle_mod):
    """Guard for the check above: an aperiodic search on a periodic cloud misses the pairs
    that touch through the boundary, so the brute-force comparison would fail."""
    w = workloads.periodic_cloud(600, 3, phi=0.33, inflate=1.06)
    a = _set(*oracle_mod.pairs(w.pos, w.radius, periodic=True, H=w.cell))
    b = {(i, j, (0, 0, 0)) for i, j, _ in _set(*oracle_mod.pairs(w.pos, w.radius))}
    assert a != b


def test_grid_on_a_tiny_periodic_cell_with_few_cells(oracle_mod):
    """Cells fewer than three per axis (neighbour cells repeat through the wrap)."""
    w = workloads.periodic_cloud(40, 9, phi=0.3, inflate=1.05)
    a = oracle_mod.pairs(w.pos, w.radius, periodic=True, H=w.cell, method="grid")
    b = oracle_mod.pairs(w.pos, w.radius, periodic=True, H=w.cell, method="brute")
    assert _set(*a) == _set(*b)
