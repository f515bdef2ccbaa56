"""Oracle pinned to the values the Yade text prints (tests/golden/yade_doctests.json)."""
import numpy as np


def _prefix_match(value: float, printed: str) -> bool:
    s = repr(float(value))
    if printed.startswith("-") != s.startswith("-"):
        return False
    return s.startswith(printed) or f"{value:.{len(printed) + 4}f}".startswith(printed)


def test_falling_sphere_energy_doctest(oracle_mod, golden):
    """yade.plot energy doctest: damping (eq. 2.9) on gravity, first leapfrog step and the
    energy-tracker sign conventions, to the printed digits."""
    g = golden["energy_falling_sphere"]
    m = g["material"]
    s = oracle_mod.OracleScene(gravity=g["gravity"], damping=g["damping"])
    s.set_material(0, m["density"], m["young"], m["poisson"], m["friction"])
    s.add_spheres([[0.0, 0.0, 0.0]], [g["radius"]])
    s.set_dt(s.pwave_dt())
    s.step(1)
    e = s.energy()
    got = {"gravWork": e["gravWork"], "kinRot": e["kinRot"], "kinTrans": e["kinTrans"],
           "nonviscDamp": e["nonviscDamp"],
           "total energy": e["kinTrans"] + e["kinRot"] + e["gravWork"] + e["nonviscDamp"]}
    for k, printed in g["printed"].items():
        assert _prefix_match(got[k], printed), (k, got[k], printed)


def test_damping_is_what_reduces_the_work(oracle_mod, golden):
    """Planted-mistake guard: without damping the same step gives kinTrans = -gravWork/2
    (leapfrog from rest) and no damping work, so the doctest values above are not met by
    accident."""
    g = golden["energy_falling_sphere"]
    m = g["material"]
    s = oracle_mod.OracleScene(gravity=g["gravity"], damping=0.0)
    s.set_material(0, m["density"], m["young"], m["poisson"], m["friction"])
    s.add_spheres([[0.0, 0.0, 0.0]], [g["radius"]])
    s.set_dt(s.pwave_dt())
    s.step(1)
    e = s.energy()
    assert e["nonviscDamp"] == 0.0
    assert np.isclose(e["kinTrans"], -0.5 * e["gravWork"], rtol=1e-14)
    assert not _prefix_match(e["kinTrans"], g["printed"]["kinTrans"])


def test_sphere_pwave_timestep_doctest(oracle_mod, golden):
    g = golden["sphere_pwave_timestep"]
    dt = oracle_mod.sphere_pwave_dt(g["radius"], g["density"], g["young"])
    assert repr(dt) == g["printed"]


def test_step_advances_time_by_dt(oracle_mod, golden):
    g = golden["step_advances_time"]
    s = oracle_mod.OracleScene()
    s.set_material(0, 1000, 1e7, 0.3, 0.5)
    s.add_spheres([[0.0, 0.0, 0.0]], [1.0])
    s.set_dt(g["dt"])
    s.step(1)
    it, t, dt = s.clock()
    assert it == 1 and repr(t) == g["printed_time_after_one_step"]


def test_summation_order_changes_the_last_bit(golden):
    """The text's example that FP64 addition order matters (section 2.1.7): the reason the
    CUDA path sums per-body forces in one fixed order and must be bitwise reproducible."""
    g = golden["summation_order"]
    assert repr((1 / 10.) + (1 / 13.) + (1 / 17.)) == g["forward"]
    assert repr((1 / 17.) + (1 / 13.) + (1 / 10.)) == g["reversed"]
