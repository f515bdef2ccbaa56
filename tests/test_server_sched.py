"""The request server's scheduling core (csrc/server_sched.h) on the host, with a
fake device backend compiled into a small C++ harness (no GPU): admission in
arrival order within the device-memory budget, ticks that never overshoot a step
budget, requests that join while a tick runs, the footprint estimate from the
measured rows per body, admission and device failures, deadlines, release, and the
latency percentiles against numpy's."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_00611_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = tmp_path_factory.mktemp("sched") / "harness"
    subprocess.run(["g++", "-std=c++17", "-O1", "-pthread", "-Wall", "-I", CSRC,
                    os.path.join(ROOT, "tests", "server_sched_harness.cpp"), "-o", str(exe)],
                   check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    return res.stdout.splitlines()


@pytest.mark.parametrize("name", ["budget_and_order", "join_while_running",
                                  "footprint_and_capacity", "failures", "wait_release_state",
                                  "stop_drops_pending"])
def test_scenario(harness, name):
    assert f"{name} ok" in harness


def test_percentiles_match_numpy(harness):
    line = [ln for ln in harness if ln.startswith("percentiles ")][0]
    got = [float(x) for x in line.split()[1:]]
    v = [3.0, 1.0, 4.0, 1.5, 9.0, 2.6, 5.0]
    want = [np.percentile(v, 50), np.percentile(v, 99), np.percentile(v, 12.5)]
    assert np.allclose(got, want, rtol=1e-15, atol=0)
