"""The benchmark's roofline bookkeeping on CPU: the dominant relaxation kernel is the one with the largest
share of the step, its bound is the resource whose minimum time is longer, achieved / peak is the
fraction, and DRAM traffic is reported only for phases the traffic file lists."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
pytest.importorskip("torch")

import bench  # noqa: E402

WL = {"nx": 4096, "nt": 16384, "order": 3, "m": 8, "max_coarsest": 8}


def stats(fine64_ms, coarse_ms, fine32_ms):
    return {"phase_ms": {"fine64_res": fine64_ms, "coarse": coarse_ms, "fine32_res": fine32_ms, "departure": 5.0},
            "phase_launches": {"fine64_res": 17, "coarse": 153, "fine32_res": 17, "departure": 1}}


def test_level_steps_follow_the_coarsening_rule():
    assert bench.level_steps(WL) == [16384, 2048, 256, 32, 4]


def test_dominant_kernel_is_the_largest_share_and_traffic_only_where_listed():
    traffic = {"fine64_res": 2.5e9}
    dom, others = bench.roofline(stats(10.2, 9.9, 2.4), WL, 6686.1, "measured", 17, traffic)
    assert dom["phase"] == "fine64_res" and [o["phase"] for o in others] == ["coarse", "fine32_res"]
    assert dom["traffic"] == 2.5e9 and all(o["traffic"] is None for o in others)
    dom2, _ = bench.roofline(stats(10.2, 10.4, 2.4), WL, 6686.1, "measured", 17, traffic)
    assert dom2["phase"] == "coarse"


def test_bound_and_fraction():
    dom, others = bench.roofline(stats(10.2, 9.9, 2.4), WL, 6686.1, "measured", 17, None)
    # level-0 FP64 residual: 2(p+1) flop against 2 + 8(p+1) bytes per point-step; at 2 FP64 FMA a clock
    # per SM the flops take longer than the bytes at HBM speed, so the pass is ALU bound
    assert dom["bound"] == "alu" and dom["unit"] == "TFLOP/s"
    pts = WL["nx"] * WL["nt"]
    assert dom["algorithmic_flops"] == pts * 2 * (WL["order"] + 1)
    avg_s = 10.2e-3 / 17
    assert dom["achieved"] == pytest.approx(dom["algorithmic_flops"] / avg_s / 1e12)
    assert dom["frac"] == pytest.approx(dom["achieved"] / bench.FP64_PEAK_TFLOPS)
    f32 = [o for o in others if o["phase"] == "fine32_res"][0]
    # level-0 FP32 error pass: eps (4 B) and shift (2 B) per point-step plus two slice rows per interval
    assert f32["bound"] == "hbm" and f32["unit"] == "GB/s"
    assert f32["algorithmic_bytes"] == pts * 6 + 2 * (WL["nt"] // WL["m"]) * WL["nx"] * 4
    assert f32["frac"] == pytest.approx(f32["algorithmic_bytes"] / (2.4e-3 / 17) / 1e9 / 6686.1)


def test_phases_without_launches_are_left_out():
    s = stats(10.2, 9.9, 2.4)
    s["phase_launches"]["fine32_res"] = 0
    _, others = bench.roofline(s, WL, 6686.1, "measured", 17, None)
    assert [o["phase"] for o in others] == ["coarse"]
