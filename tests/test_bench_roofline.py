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


def test_batched_bookkeeping_sums_the_problems_over_their_cycles():
    import workloads as W

    probs = W.batched_problems(4)
    iters = [3, 5, 2, 4]
    w = bench.batch_phase_work("fine32_res", probs, iters)
    want = sum(it * (q.nx * q.nt * 6 + (q.nt // q.m) * q.nx * 8) for q, it in zip(probs, iters))
    assert w["bytes"] == want and w["fp"] == 32
    lv = bench.batch_levels(probs[0])
    # coarsen by m while the level has more than one step and m divides it (1024 / 8: 128, 16, 2)
    assert lv[0] == probs[0].nt and (lv[-1] <= 1 or lv[-1] % probs[0].m) and all(a == b * probs[0].m for a, b in zip(lv, lv[1:]))
    ph_ms = {"fine64_res": 40.0, "fine32_res": 10.0, "coarse": 30.0, "coarsest": 5.0, "departure": 20.0}
    ph_n = {"fine64_res": 5, "fine32_res": 25, "coarse": 100, "coarsest": 5, "departure": 4}
    dom, others = bench.batch_roofline(ph_ms, ph_n, probs, iters, 6686.1, "measured", None)
    assert dom["phase"] == "fine64_res" and [o["phase"] for o in others] == ["coarse", "fine32_res", "coarsest"]
    assert dom["avg_launch_ms"] == pytest.approx(8.0)
    f32 = [o for o in others if o["phase"] == "fine32_res"][0]
    assert f32["achieved"] == pytest.approx(want / 10e-3 / 1e9)
    assert f32["algorithmic_bytes_per_launch"] == pytest.approx(want / 25)
