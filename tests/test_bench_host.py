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


def test_other_workloads_carry_no_stored_traffic():
    """The stored DRAM figures belong to the 1M compaction: a roofline of another
    workload (the triaxial mode) reports traffic as null, with the algorithmic rate."""
    tm = {"integrate_ms": 2.0, "integrate_launches": 4, "contact_ms": 1.0}
    res = {"tm": tm, "mean_real": 2.0e6, "avg_ms": 0.25, "rows_avg": 4.0e6}
    line, out = bench._kernel_rooflines(res, "mixed", 1_000_000, 6800.0, "measured",
                                        traffic=False)
    assert all(o["traffic"] is None and "traffic_note" not in o for o in out.values())
    by = bench.ROW_BYTES_ALL_MIXED * 4.0e6 + bench.ROW_BYTES_REAL_MIXED * 2.0e6
    assert abs(out["contact"]["achieved"] - by / 0.25e-3 / 1e9) < 1e-6
    assert line["kernel"].startswith("integrate")   # the larger share of the step
