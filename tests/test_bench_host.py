"""Host logic of the benchmark line: a stored DRAM-traffic figure is reported only for
the kernel sources it was measured with."""
import bench


def test_traffic_is_reported_only_for_the_measured_sources(monkeypatch):
    digest = bench.kernel_digest("contact", "fp64")
    entry = {"bytes": 1.5e8, "rows": 10, "real": 5, "step": 4990, "digest": digest}
    monkeypatch.setattr(bench, "TRAFFIC", {("fp64", "contact"): entry})
    tb, note = bench._traffic("fp64", "contact", lambda r, c: 100 * r + 10 * c)
    assert tb == 1.5e8 and "1050" in note
    monkeypatch.setattr(bench, "TRAFFIC", {("fp64", "contact"): {**entry, "digest": "0" * 16}})
    assert bench._traffic("fp64", "contact", lambda r, c: 0) == (None, None)
    assert bench._traffic("mixed", "integrate", lambda r, c: 0) == (None, None)


def test_digests_cover_each_kernel_source():
    d = {(n, p): bench.kernel_digest(n, p) for n in ("contact", "integrate") for p in ("fp64", "mixed")}
    assert d[("contact", "fp64")] != d[("contact", "mixed")]
    assert d[("integrate", "fp64")] == d[("integrate", "mixed")]   # one source file
    assert all(len(v) == 16 for v in d.values())
