"""dem_find_pairs (collision detection on a bare configuration) against the
oracle's brute-force search: the pair sets, with their cell shifts, must be
identical -- both sides evaluate the same exact test in the same operation order."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_00611_gb300 as pkg
    return torch, oracle, pkg


def _gpu_set(torch, pkg, pos, rad, **kw):
    P = torch.tensor(pos, dtype=torch.float64, device="cuda")
    R = torch.tensor(rad, dtype=torch.float64, device="cuda")
    I, J, C = pkg.find_pairs(P, R, **kw)
    I, J, C = I.cpu().numpy(), J.cpu().numpy(), C.cpu().numpy()
    assert np.all(I < J)
    return {(int(i), int(j), tuple(int(x) for x in c)) for i, j, c in zip(I, J, C)}, (I, J, C)


def _orc_set(oracle, pos, rad, periodic=False, H=None, margin=0.0):
    I, J, C = oracle.pairs(pos, rad, periodic=periodic, H=H, margin=margin, method="brute")
    return {(int(i), int(j), tuple(int(x) for x in c)) for i, j, c in zip(I, J, C)}


@pytest.mark.parametrize("margin", [0.0, 3e-4])
@pytest.mark.parametrize("seed", [0, 1])
def test_pairs_aperiodic(env, seed, margin):
    torch, oracle, pkg = env
    w = workloads.box_cloud(2500, seed, phi=0.3, inflate=1.05, wall_mask=0)
    g, _ = _gpu_set(torch, pkg, w.pos, w.radius, margin=margin)
    o = _orc_set(oracle, w.pos, w.radius, margin=margin)
    assert g == o and len(o) > 1000


@pytest.mark.parametrize("margin", [0.0, 3e-4])
def test_pairs_periodic_unwrapped(env, margin):
    torch, oracle, pkg = env
    w = workloads.periodic_cloud(2200, 3, phi=0.33, inflate=1.05)
    L = w.cell[0, 0]
    pos = w.pos + ((workloads.uniform(w.pos.size, 7).reshape(w.pos.shape) * 7).astype(int) - 3) * L
    g, _ = _gpu_set(torch, pkg, pos, w.radius, periodic=True, cell=w.cell, margin=margin)
    o = _orc_set(oracle, pos, w.radius, periodic=True, H=w.cell, margin=margin)
    assert g == o and len(o) > 1000
    assert any(c != (0, 0, 0) for _, _, c in g)


def test_pairs_capacity_and_determinism(env):
    torch, oracle, pkg = env
    w = workloads.periodic_cloud(1500, 4, phi=0.33, inflate=1.05)
    full, (I, J, C) = _gpu_set(torch, pkg, w.pos, w.radius, periodic=True, cell=w.cell)
    again, (I2, J2, C2) = _gpu_set(torch, pkg, w.pos, w.radius, periodic=True, cell=w.cell)
    assert np.array_equal(I, I2) and np.array_equal(J, J2) and np.array_equal(C, C2)
    P = torch.tensor(w.pos, dtype=torch.float64, device="cuda")
    R = torch.tensor(w.radius, dtype=torch.float64, device="cuda")
    Ic, Jc, Cc = pkg.find_pairs(P, R, periodic=True, cell=w.cell, cap=len(I))
    assert len(Ic) == len(I)


def test_pairs_errors(env):
    torch, oracle, pkg = env
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    rad = torch.full((4,), 0.1, dtype=torch.float64, device="cuda")
    rad[2] = float("nan")
    with pytest.raises(pkg.DemError) as e:
        pkg.find_pairs(pos, rad)
    assert e.value.code == 5
    rad[2] = 0.1
    H = np.eye(3)
    H[0, 1] = 0.2
    with pytest.raises(pkg.DemError) as e:
        pkg.find_pairs(pos, rad, periodic=True, cell=H)
    assert e.value.code == 1
    with pytest.raises(pkg.DemError) as e:
        pkg.find_pairs(pos, rad, periodic=True, cell=np.eye(3) * 0.5)
    assert e.value.code == 6
