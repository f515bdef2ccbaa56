"""Launch shapes (dem_set_tuning / dem_autotune) change no result: every row and
every body is computed by one thread with the same arithmetic whatever the block
size, persistent grid, body order or whether a batch of steps is replayed from a
captured CUDA graph, so trajectories must be bit-identical."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(contact_block=256, contact_blocks_per_sm=8, integrate_block=256, degree_order=1,
         step_graphs=1),
    dict(contact_block=128, contact_blocks_per_sm=3, integrate_block=512, degree_order=0,
         step_graphs=0),
    dict(contact_block=256, contact_blocks_per_sm=1, integrate_block=128, degree_order=1,
         step_graphs=1),
]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00611_gb300 as pkg
    return pkg


def _workloads():
    return [workloads.periodic_cloud(3000, 41, phi=0.34, inflate=1.05, vel_scale=0.05,
                                     angvel_scale=20.0),
            workloads.box_cloud(2500, 42, phi=0.3, inflate=1.04, gravity=(0, 0, -9.81),
                                vel_scale=0.05)]


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("pos", "vel", "angvel", "ori"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_shapes_give_identical_trajectories(pkg, precision):
    prec = pkg.DEM_MIXED if precision == "mixed" else pkg.DEM_FP64
    for w in _workloads():
        states = []
        for shape in SHAPES:
            g = pkg.Scene.from_workload(w, precision=prec)
            g.set_tuning(**shape)
            assert g.tuning() == shape
            g.step(150)
            states.append(g.state())
            assert g.stats()["n_rebuilds"] >= 1
        assert _same(states[0], states[1]) and _same(states[0], states[2])


def test_autotune_picks_a_valid_shape_on_the_same_trajectory(pkg):
    w = _workloads()[0]
    a = pkg.Scene.from_workload(w)
    chosen = a.autotune(steps_per_trial=3)
    assert chosen["contact_block"] in (128, 256) and chosen["integrate_block"] in (128, 256, 512)
    assert 1 <= chosen["contact_blocks_per_sm"] <= 64 and chosen["degree_order"] in (0, 1)
    assert a.tuning() == chosen
    n = a.clock()[0]
    assert n == 17 * 4   # 6 contact shapes twice, 5 integrator shapes, 1 + 3 steps each
    b = pkg.Scene.from_workload(w)
    b.step(n)
    assert _same(a.state(), b.state())


def test_tuning_rejects_out_of_range(pkg):
    w = _workloads()[1]
    g = pkg.Scene.from_workload(w)
    for bad in (dict(contact_block=64), dict(contact_blocks_per_sm=0), dict(integrate_block=1024),
                dict(degree_order=2), dict(step_graphs=3), dict(step_graphs=-2)):
        with pytest.raises(pkg.DemError) as e:
            g.set_tuning(**bad)
        assert e.value.code == 1
