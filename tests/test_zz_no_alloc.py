"""dem_find_pairs_noalloc: the pair query for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Its output must equal
dem_find_pairs's on the same input, on two calls in a row -- the second call also
shows that the shared scratch left by the first call does not leak into the
result.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00611_gb300 as pkg
    return torch, pkg


def _inputs(torch, w, shift_periods=False):
    pos = w.pos
    if shift_periods:
        L = w.cell[0, 0]
        pos = pos + ((workloads.uniform(pos.size, 3).reshape(pos.shape) * 5).astype(int) - 2) * L
    return (torch.tensor(pos, dtype=torch.float64, device="cuda"),
            torch.tensor(w.radius, dtype=torch.float64, device="cuda"))


def _same(a, b):
    # integer outputs: exact equality, rows in the same fixed order
    return all(np.array_equal(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(a, b))


def test_noalloc_matches_allocating_query_on_two_calls(env):
    torch, pkg = env
    w1 = workloads.periodic_cloud(6000, 21, phi=0.33, inflate=1.05)
    w2 = workloads.box_cloud(4000, 22, phi=0.3, inflate=1.04, wall_mask=0)
    P1, R1 = _inputs(torch, w1, shift_periods=True)
    P2, R2 = _inputs(torch, w2)
    ref1 = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4)
    ref2 = pkg.find_pairs(P2, R2, margin=0.0)
    got1 = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4, noalloc=True)
    got2 = pkg.find_pairs(P2, R2, margin=0.0, noalloc=True)
    assert len(ref1[0]) > 3000 and len(ref2[0]) > 1000
    assert _same(got1, ref1)
    assert _same(got2, ref2)
    again = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4, noalloc=True)
    assert _same(again, ref1)


def test_noalloc_rejects_more_spheres_than_its_scratch_holds(env):
    torch, pkg = env
    n = (1 << 16) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    rad = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DemError) as e:
        pkg.find_pairs(pos, rad, noalloc=True)
    assert e.value.code == 4
    assert "65536" in str(e.value)
