"""Host logic of the benchmark's measurement keys, on CPU (no GPU, no timing).

The roofline entry names the kernel group with the most time per solve and divides its
algorithmic bytes per launch by the launch time and the peak; the recorded DRAM traffic is
reported only while the source of the kernels it was captured from is unchanged; the CPU
baseline extrapolates one timed oracle step to the oracle's own full solve.
"""
import hashlib
import json
import os

import pytest

import bench


def _kernels():
    # two groups as profile_kernels() returns them: sorted by time per solve, largest first
    ks = [{"kernel": "coarse_cycle", "avg_launch_us": 40.0, "launches_per_solve": 600,
           "ms_per_solve": 24.0, "bytes_pass": 1.0e6, "bytes_once": 5.0e4,
           "achieved_gbs_pass": 25.0, "achieved_gbs_once": 1.25, "sampled_launches": 300},
          {"kernel": "mid_level_tiles", "avg_launch_us": 10.0, "launches_per_solve": 3600,
           "ms_per_solve": 36.0, "bytes_pass": 1.0e7, "bytes_once": 1.5e6,
           "achieved_gbs_pass": 1000.0, "achieved_gbs_once": 150.0, "sampled_launches": 1800}]
    ks.sort(key=lambda x: -x["ms_per_solve"])
    return ks


def test_roofline_entry_names_the_largest_group_and_divides_by_the_peak():
    r = bench.roofline_entry(_kernels(), 6786.6, "measured")
    assert r["kernel"] == bench.KERNEL_NAMES["mid_level_tiles"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_kind"] == "measured"
    assert r["achieved"] == 1000.0
    assert r["frac"] == pytest.approx(1000.0 / 6786.6)
    assert r["per_launch_once"]["frac"] == pytest.approx(150.0 / 6786.6)
    assert r["share_of_kernel_time"] == pytest.approx(36.0 / 60.0)
    # achieved = algorithmic bytes per launch / launch time
    assert r["algorithmic_bytes_per_launch"] / (r["avg_launch_us"] * 1e-6) / 1e9 == \
        pytest.approx(r["achieved"])
    assert bench.roofline_entry([], 6786.6, "measured") is None


def test_recorded_traffic_is_current_and_goes_null_when_the_source_changes(monkeypatch):
    t = bench.NCU_TRAFFIC["mid_level_tiles"]
    path, start, end = t["source"]
    with open(os.path.join(bench.ROOT, path)) as f:
        src = f.read()
    i, j = src.find(start), src.find(end)
    assert 0 <= i < j
    current = hashlib.sha256(src[i:j].encode()).hexdigest() == t["sha256"]
    assert bench.traffic_if_current("mid_level_tiles") == (t["bytes"] if current else None)
    stale = dict(t, sha256="0" * 64)
    monkeypatch.setitem(bench.NCU_TRAFFIC, "mid_level_tiles", stale)
    assert bench.traffic_if_current("mid_level_tiles") is None
    assert bench.traffic_if_current("no_such_group") is None


def test_measured_peak_comes_from_the_driver_file_when_present():
    hbm, kind = bench.measured_peaks()
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            assert hbm == json.load(f).get("hbm_gbs", 6800.0)
        assert kind == "measured"
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_oracle_extrapolation_counts_assembly_once_and_every_step_and_iteration():
    s = {"build_s": 2.0, "step_s": 11.0, "krylov_s": 8.0, "iters": 16}
    # assembly 2 s once; 3 s of set-up per IPM step; 0.5 s per FGMRES iteration
    assert bench.oracle_solve_seconds(s, (9, 150)) == pytest.approx(2.0 + 9 * 3.0 + 150 * 0.5)
    counts = bench.oracle_reference_counts(1)
    assert counts is not None
    k, K = counts
    assert k >= 1 and K >= k


def test_percentiles_and_throughput():
    assert bench.pct([1.0, 2.0, 3.0, 4.0, 5.0], 50) == 3.0
    assert bench.pct([1.0, 2.0], 99) == pytest.approx(1.99)
    assert bench.throughput(2, 9, 1500.0) == pytest.approx(12.0)
