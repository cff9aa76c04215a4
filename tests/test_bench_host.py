"""Host logic of bench.py that needs no GPU: clock-sample summary, whole-job
rate on one rank, and the ncu traffic figure gated on the kernel source."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, then the four flags
    return f"0, {sm}, {mx}, 950.25, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2055, 2070),
                "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"]
    s = cs.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0            # median of 1980, 2055, 2070
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_every_slowdown():
    cs = bench.ClockSampler(0)
    cs.lines = [_line(1500, 2070, hw="Active"), _line(1500, 2070, hwt="Active"),
                _line(1500, 2070, swt="Active")]
    assert cs.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                       "sw_thermal_slowdown"]


def test_clock_summary_unsampled():
    s = bench.ClockSampler(0).summary()
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_job_rate_one_rank():
    t, rate = bench.job_rate(1, 362, 0.05, "cpu")
    assert t == 0.05 and rate == pytest.approx(7240.0)


def test_captured_traffic_gated_on_source(monkeypatch):
    key = ("sphere_r2_L5", "mixed", 362, "far_stage2")
    assert key in bench.NCU_TRAFFIC
    # a source whose code hashes to the recorded value reports the captured figure
    text = ""
    for path in bench.NCU_TRAFFIC_SOURCE[0]:
        with open(os.path.join(ROOT, path)) as f:
            text += f.read()
    now = bench.code_hash(text)
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCE", (bench.NCU_TRAFFIC_SOURCE[0], now))
    assert bench.captured_traffic(*key) == bench.NCU_TRAFFIC[key]
    # not captured: other kernel, precision or RHS count
    assert bench.captured_traffic("sphere_r2_L5", "mixed", 362, "near") is None
    assert bench.captured_traffic("sphere_r2_L5", "fp64", 362, "far_stage2") is None
    assert bench.captured_traffic("sphere_r2_L5", "mixed", 100, "far_stage2") is None
    # a changed kernel source turns the figure off
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCE", (bench.NCU_TRAFFIC_SOURCE[0], "0" * 64))
    assert bench.captured_traffic(*key) is None


def test_workload_description_of_the_benchmark():
    # both arms (native and the oracle's) name the workload with this string
    from hm_workloads import get_workload
    assert bench.workload_desc(get_workload("sphere_r2_L5"), 30720, 362) == (
        "sphere_r2_L5: PEC sphere r=2 lambda, icosphere L5, N=30720, leaves<=128, ACA 1e-4, "
        "362 monostatic RHS (theta 0..180 step 1, theta/phi pol)")


def test_openblas_thread_control_and_single_thread_entry():
    import numpy as np
    a = np.ones((64, 64))
    a @ a                                          # BLAS loaded and initialised
    ob = bench.openblas_threads()
    if ob is not None:                             # NumPy built on OpenBLAS
        set_t, get_t = ob
        n = int(get_t())
        set_t(1)
        try:
            assert int(get_t()) == 1
        finally:
            set_t(n)
        assert int(get_t()) == n
    e = bench.one_thread_entry({"one_thread": {"n": 4, "ts": [2.0, 1.0]}})
    assert e["value"] == 4.0 and e["cores"] == 1
    assert bench.one_thread_entry({"one_thread": None})["value"] is None


def test_code_hash_ignores_comments_only():
    src = "int f(int a) {  // add one\n  return a + 1; /* done */ }\n"
    assert bench.code_hash(src) == bench.code_hash("int f(int a) { return a + 1; }")
    assert bench.code_hash(src) != bench.code_hash("int f(int a) { return a + 2; }")
