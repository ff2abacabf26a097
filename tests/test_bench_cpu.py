"""Host-side arithmetic of bench.py (no GPU): the clock summary that goes into every
JSON line, the algorithmic byte and flop counts behind the roofline, the peaks."""
import json
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
    # residues over the pairs m <= p only (w^s_pm = w^s_mp), counted pair by pair
    pairs = sum(1 for p in range(200) for m in range(p + 1))
    assert f["sigma"] == pytest.approx(2.0 * pairs * 600 * n + 2.0 * 200 ** 3 * n)
    assert 0.75e12 < sum(f.values()) < 0.76e12     # 0.755 TFLOP per iteration


def test_stage_rooflines_fractions():
    ms = {"tridiag_panel": 365.0, "tridiag_syr2k": 155.0, "sigma": 247.0, "bisect": 33.0, "twisted": 17.0,
          "backtransform": 108.0, "gemm_f64": 43.0, "misc": 1.0}
    r = bench.stage_rooflines(200, 40, 600, ms)
    assert set(r) == set(ms) - {"misc"}
    n = 40 * 160
    panel = 2.0 / 3.0 * n ** 3 + 128.0 * n * n + 2.0 / 3.0 * 200 ** 3
    assert r["tridiag_panel"]["achieved"] == pytest.approx(panel / 0.365 / 1e12, rel=1e-3)
    assert r["tridiag_panel"]["frac"] == pytest.approx(panel / 0.365 / 1e12 / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert all(0 < v["frac"] < 1.5 for v in r.values())
    # with the 7-digit engine the trailing updates are tensor-bound, 28 digit products each
    r7 = bench.stage_rooflines(200, 40, 600, {"tridiag_syr2k": 31.0}, "bf16x10", bench.FLAG_EIG_TC_BIT)
    assert r7["tridiag_syr2k"]["bound"] == "tensor"
    useful = 2.0 / 3.0 * (n ** 3 + 200 ** 3)
    assert r7["tridiag_syr2k"]["fp64_equivalent_tflops"] == pytest.approx(useful / 0.031 / 1e12, rel=1e-3)
    rf = bench.stage_rooflines(200, 40, 600, {"sigma": 8.1, "gemm_tc": 9.4}, "bf16x10", bench.FLAG_TC_AB_BIT)
    assert rf["sigma"]["bound"] == "hbm" and rf["gemm_tc"]["bound"] == "tensor"
    # with EIG_TC the panel's integer mat-vec reads 8-byte tile images: HBM-bound, bytes
    # n^3/6 elements x 8 per column sweep + the image built once per 64-column panel
    ri = bench.stage_rooflines(200, 40, 600, {"tridiag_panel": 252.6}, "bf16x10", bench.FLAG_EIG_TC_BIT)
    p = ri["tridiag_panel"]
    assert p["bound"] == "hbm" and p["unit"] == "GB/s"
    assert p["achieved"] == pytest.approx((8.0 * n ** 3 / 6.0 + 16.0 * n ** 3 / 384.0) / 0.2526 / 1e9, rel=1e-3)
    assert p["frac"] == pytest.approx(p["achieved"] / bench.measured_peaks()["hbm_gbs"], rel=1e-3)
    assert p["fp64_equivalent_tflops"] == pytest.approx(panel / 0.2526 / 1e12, rel=1e-2)


def test_headline_is_short_and_complete():
    stage = {"frac": 0.4}
    line = {"value": 0.9, "roofline": {"frac": 0.39}, "roofline_stages": {"tridiag_panel": stage},
            "mixed": {"ms_per_step": 700.0, "speedup_vs_fp64": 1.39, "qp_error_vs_fp64_meV": 0.18},
            "config_C": {"fp64": {"s_per_pass": 34.8, "vs_oracle": {"qp_max_abs_meV": 1e-4}, "meets_bar": True},
                         "mixed": {"s_per_pass": 26.0, "speedup_vs_fp64": 1.34,
                                   "vs_oracle": {"qp_max_abs_meV": 0.03}, "meets_bar": True}},
            "config_E": {"s_per_pass": 171.0, "roofline_stages": {"tridiag_panel": stage},
                         "checks": {"omega_min_ge_min_D": True, "finite": True, "sum_omega2_vs_trace_M_rel": 1e-9}},
            "batch_D": {"error": "RuntimeError: x"}}
    h = bench.headline(line)
    assert h["C_mixed_x"] == 1.34 and h["C_fp64_ok"] and h["E_checks_ok"] and h["D_error"].startswith("Runtime")
    assert len(json.dumps(h)) < 1400


def test_oracle_arm_step_counts():
    assert bench.oracle_step_counts(bench.WORKLOADS["B"], 20, 5) == (20, 5)
    assert bench.oracle_step_counts(bench.WORKLOADS["B"], 50, 5) == (24, 1)
    assert bench.oracle_step_counts(bench.WORKLOADS["E"], 20, 5) == (1, 1)


def test_peaks():
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856, rel=1e-6)
    p = bench.measured_peaks()
    assert p["kind"] in ("measured", "fallback") and p["hbm_gbs"] > 1000 and p["bf16_tflops"] > 500
    assert math.isclose(bench.PANEL_TRAFFIC_RATIO, 4.564 / 6.629)   # profiles/k_panel_n6400.md
