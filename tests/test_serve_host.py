"""Host logic of the continuous-batching server (no GPU): admission in arrival order
within the body budget, ticks that never overshoot a budget, retirement with the
freed room and material ids reused, and results for every request."""
import numpy as np

from paper_2301_00611_gb300.serve import Server, percentile


class FakeScene:
    """Records the calls the server makes; every sub-scene advances with each step."""

    def __init__(self):
        self.subs = {}
        self.free = []
        self.mats = {}
        self.steps = []
        self.next = 1

    def set_material(self, k, *a):
        self.mats[k] = a

    def add_workload(self, w, material_base, dt=None):
        for k, m in enumerate(w.materials):
            self.set_material(material_base + k, m)
        sub = self.free.pop(0) if self.free else self.next
        if sub == self.next:
            self.next += 1
        self.subs[sub] = {"n": w.n, "iter": 0, "mats": (material_base, len(w.materials))}
        return sub

    def subscene(self, sub):
        return {"dt": 1e-5, "iter": self.subs[sub]["iter"]}

    def set_subscene_velgrad(self, sub, L):
        self.subs[sub]["L"] = L

    def step(self, k):
        self.steps.append(k)
        for v in self.subs.values():
            v["iter"] += k

    def subscene_stats(self, sub):
        return {"iter": self.subs[sub]["iter"], "n_bodies": self.subs[sub]["n"]}

    def subscene_state(self, sub):
        return {"pos": np.zeros((self.subs[sub]["n"], 3))}

    def remove_subscene(self, sub):
        del self.subs[sub]
        self.free.append(sub)

    def close(self):
        pass


class W:
    def __init__(self, n, nmat=1):
        self.n = n
        self.materials = [object()] * nmat
        self.periodic = False


def test_admission_ticks_and_retirement():
    fake = FakeScene()
    srv = Server(capacity_bodies=1000, tick_steps=50, scene=fake)
    srv.submit(0, W(600), 120, arrival=0.0)
    srv.submit(1, W(500), 70, arrival=0.1)     # does not fit beside request 0
    srv.submit(2, W(300), 30, arrival=0.2)     # fits, but waits behind request 1 (FIFO)
    steps = []
    while not srv.idle:
        steps.append(srv.tick())
    # request 0 alone: 50, 50, 20 steps; then 1 and 2 together: 30, then 1 alone: 40
    assert steps == [50, 50, 20, 30, 40]
    assert fake.steps == steps
    by_id = {r.rid: r for r in srv.results}
    assert sorted(by_id) == [0, 1, 2]
    assert by_id[0].stats["iter"] == 120 and by_id[1].stats["iter"] == 70
    assert by_id[2].stats["iter"] == 30
    assert srv.resident_bodies == 0 and not fake.subs
    assert srv.scene_steps == 120 + 70 + 30
    assert srv.body_steps == 600 * 120 + 500 * 70 + 300 * 30
    # sub-scene indices and material ids come back for reuse
    assert fake.free and srv._free_mats == [(1, 3999)]


def test_budget_never_exceeded_and_latency():
    fake = FakeScene()
    srv = Server(capacity_bodies=1000, tick_steps=100, scene=fake)
    rng = np.random.default_rng(0)
    for k in range(30):
        srv.submit(k, W(int(rng.integers(50, 600)), int(rng.integers(1, 3))),
                   int(rng.integers(10, 300)), arrival=0.0)
    peak = 0
    while not srv.idle:
        srv.tick()
        peak = max(peak, srv.resident_bodies)
        assert srv.resident_bodies <= 1000
    assert len(srv.results) == 30 and peak > 500
    lat = [r.latency for r in srv.results]
    assert min(lat) >= 0 and percentile(lat, 50) <= percentile(lat, 99)
