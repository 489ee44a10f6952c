"""Host-side pieces of the benchmark that decide what its line reports,
checked without a GPU: the clock and throttle-reason summary of the sampled
nvidia-smi rows, the FP32 peak arithmetic, and when the recorded DRAM traffic
of the pair kernel may be quoted."""
import os

import pytest

import bench


def _summary(rows):
    s = bench.ClockSampler(0)
    s.proc = object()            # rows written below stand in for nvidia-smi's
    with open(s.path, "w") as f:
        f.write("".join(r + "\n" for r in rows))
    try:
        return s.summary()
    finally:
        os.remove(s.path)


def test_clock_summary_median_max_and_reasons():
    na = "Not Active"
    rows = [f"1965, 2070, 812.31, {na}, {na}, {na}, Active",
            f"2070, 2070, 905.00, {na}, {na}, {na}, {na}",
            "[N/A], 2070, 880.0, Not Active, Not Active, Not Active, Not Active",
            "garbled",
            f"2010, 2070, 850.00, {na}, {na}, {na}, {na}"]
    c = _summary(rows)
    assert c["sm_mhz"] == 2010 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]


@pytest.mark.parametrize("col,name", [(3, "hw_slowdown"), (4, "hw_thermal_slowdown"),
                                      (5, "sw_thermal_slowdown")])
def test_clock_summary_reports_rejecting_reasons(col, name):
    flags = ["Not Active"] * 4
    flags[col - 3] = "Active"
    c = _summary(["1500, 2070, 990.0, " + ", ".join(flags)])
    assert c["reasons"] == [name] and c["sm_mhz"] == 1500


def test_clock_summary_without_samples():
    assert _summary([])["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_fp32_peak():
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz = 80.5 TFLOP/s."""
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9


def test_traffic_quoted_only_for_the_captured_shape():
    t = bench.PAIR_TRAFFIC
    shape = {"bodies_per_thread": t["bodies_per_thread"], "blocks_per_sm": t["blocks_per_sm"]}
    got = bench.pair_traffic(t["n"], t["precision"], shape)
    if bench.pair_source_digest() == t["source_sha256"]:
        assert got == t["bytes_per_launch"]
    else:
        assert got is None
    assert bench.pair_traffic(t["n"] // 2, t["precision"], shape) is None
    assert bench.pair_traffic(t["n"], "fp32", shape) is None
    assert bench.pair_traffic(t["n"], t["precision"], {**shape, "blocks_per_sm": 6}) is None
    assert bench.pair_traffic(t["n"], t["precision"], {**shape, "bodies_per_thread": 4}) is None


def test_error_statistics_of_the_accuracy_sweep():
    """Global relative RMS plus per-body median and 99th percentile of the
    relative error; a body with a zero reference is left out of the latter."""
    import numpy as np
    import bench_workloads as bw
    ref = np.ones((101, 3))
    e = np.linspace(0.0, 1e-6, 100)
    a = ref.copy()
    a[:100] *= (1 + e)[:, None]
    ref[100] = 0.0
    a[100] = 1e-3
    s = bw._err_stats(a, ref)
    assert abs(s["per_body_median"] - np.median(e)) < 1e-15
    assert abs(s["per_body_p99"] - np.percentile(e, 99)) < 1e-15
    want = np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())
    assert abs(s["rel_rms"] - want) <= 1e-15 * want
