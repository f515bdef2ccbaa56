"""The request server of the C ABI (dem_server_*) on the GPU.

Twelve requests -- gravity depositions and periodic compactions of 1,000 to 6,000
spheres with their own materials and step budgets -- arrive in three bursts while
earlier ones are resident, so their work overlaps on the device.  In FP64 every
result must be bitwise the state of the same scene run alone; in mixed precision
the energy and packing statistics must agree with the mixed run alone (kinetic
energy within 1e-3 relative, packing fraction to rounding, coordination within 1e-3
relative or one contact, the resolution of Z = 2C/N).  Errors stay with their
request."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00611_gb300 as pkg
    from paper_2301_00611_gb300 import serve
    return pkg, serve


def _requests():
    reqs = workloads.serving_requests(12, 7, 200.0, nmin=1000, nmax=6000, smin=200, smax=600)
    return [(rq, workloads.request_workload(rq)) for rq in reqs]


def _velgrad(rq, w, dt):
    if not w.periodic:
        return None
    return workloads.compaction_rate(0.30, 0.40, rq["steps"], dt) * np.eye(3)


def _serve(pkg, serve, built, precision):
    """Submit in three bursts, each once the server has something resident."""
    out = {}
    with pkg.Server(precision=precision, budget_bytes=2 << 30, tick_steps=50) as srv:
        tickets = {}
        for burst in (built[:4], built[4:8], built[8:]):
            for rq, w in burst:
                dt = serve.pwave_dt(w)
                tickets[rq["id"]] = (srv.submit(w, rq["steps"], velgrad=_velgrad(rq, w, dt),
                                                keep_state=True, dt=dt), dt)
            t0 = time.time()
            while time.time() - t0 < 30 and not any(
                    srv.poll(t) == pkg.Server.RESIDENT for t, _ in tickets.values()):
                time.sleep(0.001)
        for rid, (t, dt) in tickets.items():
            srv.wait(t, 600)
            out[rid] = (srv.result(t, state=True), dt)
            srv.release(t)
        summary = srv.stats()
    return out, summary


def _overlapped(results):
    """Some request was admitted while another one, admitted before it, was resident."""
    spans = sorted((r["t_admit"], r["t_done"]) for r, _ in results.values())
    return any(spans[k][0] < spans[j][1] for j in range(len(spans))
               for k in range(j + 1, len(spans)))


def test_fp64_results_equal_alone_runs_bitwise(env):
    pkg, serve = env
    built = _requests()
    results, summary = _serve(pkg, serve, built, pkg.DEM_FP64)
    assert summary["completed"] == 12 and summary["failed"] == 0
    assert summary["max_resident"] >= 3
    # every tick lands in one histogram bin; some ran three or more requests at once
    assert sum(summary["concurrency_hist"]) == summary["ticks"]
    assert sum(summary["concurrency_hist"][2:]) > 0
    assert _overlapped(results)
    assert summary["latency_p99"] >= summary["latency_p50"] > 0
    kinds = set()
    for rq, w in built:
        res, dt = results[rq["id"]]
        assert res["iter"] == rq["steps"] and res["n"] == w.n
        st, alone = serve.run_alone(w, rq["steps"], pkg.DEM_FP64,
                                    velgrad=_velgrad(rq, w, dt), dt=dt, state=True)
        for k in ("pos", "vel", "angvel", "ori"):
            assert np.array_equal(res["state"][k], alone[k]), (rq["id"], k)
        assert res["stats"]["n_contacts"] == st["n_contacts"]
        kinds.add(w.periodic)
    assert kinds == {True, False}


def test_mixed_results_follow_alone_runs(env):
    pkg, serve = env
    built = _requests()
    results, summary = _serve(pkg, serve, built, pkg.DEM_MIXED)
    assert summary["completed"] == 12
    assert _overlapped(results)
    for rq, w in built:
        res, dt = results[rq["id"]]
        sa = serve.run_alone(w, rq["steps"], pkg.DEM_MIXED, velgrad=_velgrad(rq, w, dt), dt=dt)
        sm = res["stats"]
        assert abs(sm["kinetic_energy"] / sa["kinetic_energy"] - 1) <= 1e-3, rq["id"]
        assert abs(sm["packing_fraction"] / sa["packing_fraction"] - 1) <= 1e-12
        assert abs(sm["coordination"] - sa["coordination"]) <= (1 + 1e-9) * max(
            1e-3 * sa["coordination"], 2.0 / w.n), rq["id"]


def test_errors_stay_with_their_request(env):
    pkg, serve = env
    built = _requests()
    with pkg.Server(precision=pkg.DEM_FP64, budget_bytes=64 << 20, tick_steps=50) as srv:
        # too large for the budget on its own
        big = workloads.compaction(n=200_000, seed=3, steps=100)
        with pytest.raises(pkg.DemError) as e:
            srv.submit(big, 100)
        assert e.value.code == 4
        # a periodic cell narrower than three grid slabs fails at admission, alone
        rq, w = next((rq, w) for rq, w in built if w.periodic)
        bad = workloads.compaction(n=1000, seed=5, steps=100)
        bad.cell = bad.cell * 0.05
        bad.pos = bad.pos * 0.05
        ok_t = srv.submit(w, 60)
        bad_t = srv.submit(bad, 60)
        with pytest.raises(pkg.DemError) as e:
            srv.wait(bad_t, 60)
        assert e.value.code == 6
        srv.wait(ok_t, 60)
        assert srv.poll(ok_t) == pkg.Server.DONE and srv.poll(bad_t) == pkg.Server.FAILED
        with pytest.raises(pkg.DemError):
            srv.poll(123456)
        with pytest.raises(pkg.DemError):        # no state without keep_state
            srv.result(ok_t, state=True)
        st = srv.stats()
        assert st["completed"] == 1 and st["failed"] == 1
