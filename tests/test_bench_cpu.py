"""Host-side arithmetic of bench.py (no GPU): the clock summary that goes into every
JSON line, the algorithmic byte and flop counts behind the roofline, the peaks."""
import math

import pytest

import bench

ROW = "0, {sm}, 2070, 900.5, {act}, {hw}, Not Active, Not Active, {pc}"


def test_clock_summary():
    text = "\n".join([
        ROW.format(sm=2070, act="0x0", hw="Not Active", pc="Not Active"),
        ROW.format(sm=1980, act="0x4", hw="Not Active", pc="Active"),
        ROW.format(sm=2055, act="0x0", hw="Not Active", pc="Not Active"),
        "garbage line",
        "0, [N/A], 2070, 1, 0, a, b, c, d",
    ])
    c = bench.summarise_clocks(text)
    assert c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3


def test_clock_summary_reasons_and_empty():
    text = ROW.format(sm=1500, act="0x8", hw="Active", pc="Not Active")
    c = bench.summarise_clocks(text)
    assert c["reasons"] == ["hw_slowdown"] and c["sm_mhz"] == 1500.0
    e = bench.summarise_clocks("")
    assert e["sm_mhz"] is None and e["samples"] == 0 and e["reasons"] == []


@pytest.mark.parametrize("n", [2, 3, 64, 6400])
def test_panel_bytes_closed_form(n):
    # lower triangle of the trailing matrix once per column: 8 B x (n-i-1)^2 / 2, i < n-1
    assert bench.panel_bytes(n) == pytest.approx(4.0 * (n - 1) * n * (2 * n - 1) / 6.0, rel=1e-12)


def test_workload_flops_of_the_bench_molecule():
    f = bench.workload_flops(200, 40, 600)
    n = 40 * 160
    assert f["tridiag_panel"] + f["tridiag_syr2k"] == pytest.approx(4.0 / 3.0 * n ** 3 + 128.0 * n * n)
    assert f["ri_mo_transform"] == 4.0 * 600 * 200 ** 3
    assert f["backtransform"] == 4.0 * 600 * n * n
    assert 0.9e12 < sum(f.values()) < 0.92e12     # 0.908 TFLOP per iteration


def test_peaks():
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856, rel=1e-6)
    p = bench.measured_peaks()
    assert p["kind"] in ("measured", "fallback") and p["hbm_gbs"] > 1000 and p["bf16_tflops"] > 500
    assert math.isclose(bench.PANEL_TRAFFIC_RATIO, 4.569 / 6.629)
