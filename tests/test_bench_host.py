"""bench.py's roofline arithmetic and profile lookup (host logic, no GPU)."""
import math
import os

import bench

PK = dict(hbm=6780.0, bf16=1939.8, bf16_sus=1726.0, sm_max=2070.0, source="measured",
          ffma_tflops=70.0, gather_gbs=38000.0)


def test_histogram_roofline_counts_l1_bytes_per_working_launch():
    # 3 launches over 2 steps of which 2 work; 1e10 bytes per pass in 1 ms of each working launch
    r = bench.roofline_for("hist_segmented", 2.0, 2, 10**9, PK, "c2", hist_units=1e10)
    assert r["unit"] == "GB/s" and r["bound"] == "alu"
    assert math.isclose(r["achieved"], 1e10 / 1e-3 / 1e9)
    assert math.isclose(r["peak"], PK["gather_gbs"]) and math.isclose(r["frac"], r["achieved"] / PK["gather_gbs"])


def test_tensor_roofline_uses_24_flops_and_both_peaks():
    units = 16384 * 1024 * 1024
    r = bench.roofline_for("moments_bf16x3_tc", 0.25, 1, units, PK, "c2")
    assert r["unit"] == "TFLOP/s" and r["bound"] == "tensor"
    assert math.isclose(r["achieved"], 24.0 * units / 0.25e-3 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / PK["bf16"])
    assert math.isclose(r["frac_sustained"], r["achieved"] / PK["bf16_sus"])
    tf = bench.roofline_for("moments_tf32x3_tc", 0.25, 1, units, PK, "c2")
    assert math.isclose(tf["peak"], PK["bf16"] * 1.1 / 2.25)
    t1 = bench.roofline_for("moments_tf32_tc", 0.25, 1, units, PK, "c2")
    assert math.isclose(t1["achieved"], 8.0 * units / 0.25e-3 / 1e12)


def test_fp32_roofline_uses_the_measured_fma_ceiling():
    units = 16384 * 1024 * 1024
    r = bench.roofline_for("moments_fp32_simt", 2.0, 1, units, PK, "c2")
    assert r["bound"] == "alu" and math.isclose(r["peak"], PK["ffma_tflops"])
    assert math.isclose(r["achieved"], 8.0 * units / 2e-3 / 1e12)


def test_traffic_comes_from_the_kernel_profile_summary():
    t = bench.traffic_for("hist_segmented", "c2")
    line = [l for l in open(os.path.join(bench.ROOT, "profiles", "hist_segmented_c2.md"))
            if l.startswith("traffic_bytes_per_launch:")][0]
    assert t == float(line.split(":")[1])
    assert bench.traffic_for("hist_segmented", "no_such_workload") is None
