#!/usr/bin/env python
"""Benchmark: space-time DOF/s of MGRIT solves to a 1e-10 relative residual on one GB300.

Default workload (batched): 256 independent 1D problems u_t + alpha u_x = 0 on periodic [-1, 1),
alpha = 1 + a sin(2 pi k x) cos(2 pi t), drawn with SplitMix64 (seed 20260004): nx in 256 .. 4096 and
nt in 1024 .. 16384 (powers of two), order p = r in {1, 3, 5}, a in [0.1, 0.7], k in {1, 2, 3}, m in
{4, 8}; dt = 0.85 h, u0 = sin^4(pi x), random U[0,1] initial iterate; FP32 bulk with FP64 residual;
all problems' cycles in one launch per phase (mgrit_setup_batched / mgrit_solve_batched).

One step = mgrit_setup_batched (departure points, backtracking, sigma, coefficients) + the batched solve
to 1e-10 + mgrit_destroy_batched, with every u0 and initial iterate already resident in HBM.
value = sum of nx * nt over the problems / time per step, summed over ranks (replicas).

Also reported: the same-GPU sequential SL stepping comparator (every problem in one launch, with the
setup it needs), the roofline of the dominant kernel, the CPU oracle on a bounded sample of the workload,
an end-to-end figure through the host-buffer entry point, SM clocks sampled during the timed region and
the number of kernels launched.  --workload advection1d | advection2d | adjoint2d | twolevel measure the
single-problem rows (advection1d: the 4096 x 16384 variable-speed problem, p = 3, m = 8).

`--impl reference` times the CPU oracle (the method restated in numpy from the paper) on a bounded
sample of the same workload and prints the same JSON line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "space-time DOF/s to 1e-10 rel. residual vs sequential SL stepping, same GB300"
WORKLOAD = {
    "workload": "advection1d_alpha_1+0.5sin2pix_cos2pit_nx4096_nt16384_p3_m8_max8coarsest",
    "nx": 4096,
    "nt": 16384,
    "order": 3,
    "m": 8,
    "wave": "sin_kx_cos_t",
    "a": 0.5,
    "k": 1.0,
    "max_coarsest": 8,
    "cfl": 0.85,
    "u0": "3 gaussian bumps, seed 20260001",
    "rtol": 1e-10,
}
CPU_SAMPLE_NT = 512  # bounded oracle sample: the first 512 time steps of the same problem
REF_SAMPLE_NT = 256

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak derived from unit counts: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 issue peak for the FP32-pair passes: 152 SMs x 128 FP32 lanes x 2.07 GHz, one operation a lane a clock
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
# FP32 operations per point-step of the FP32-pair SL step (df32.cuh df_interp) by order p
DF_OPS = {1: 31, 3: 92, 5: 153}


def peaks():
    hbm, src = 6800.0, "fallback"
    if os.path.exists(MEASURED):
        with open(MEASURED) as f:
            d = json.load(f)
        hbm, src = float(d.get("hbm_gbs", hbm)), "measured"
    return hbm, src


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the replicas' step time is the slowest rank's)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(dof_per_rank: int, world: int, ms: float) -> float:
    """DOF/s of all ranks together: every rank solves its own replica of the workload."""
    return world * dof_per_rank / (ms / 1e3)


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.path.join("/tmp", f"clocks_{os.getpid()}.csv"), "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.out.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# roofline of the dominant kernel
# ------------------------------------------------------------------------------------------------

def level_steps(wl: dict) -> list[int]:
    """Steps per level under the coarsening rule of the library (m on every level, stop at <= max_coarsest)."""
    out = [wl["nt"]]
    while out[-1] > wl["max_coarsest"] and out[-1] % wl["m"] == 0:
        out.append(out[-1] // wl["m"])
    return out


def phase_work(phase: str, wl: dict, launches: int, iterations: int) -> dict | None:
    """Algorithmic bytes and flops per launch of a phase (averaged over the launches of one solve)."""
    nx, nt, p, m = wl["nx"], wl["nt"], wl["order"], wl["m"]
    J = nt // m
    pts = nx * nt
    if phase in ("fine64_res", "fine64_post") and wl.get("precision") in ("fp32bulk", "fp32bulk_coarse64"):
        # FP32-pair passes: per point-step eps hi, eps lo (4 B each) and shift (2 B); per interval the start slice
        # and C value in (8 B each), the residual out in FP64 and FP32; POST writes every F-point (8 B)
        byts = pts * 10 + J * nx * (8 + 8 + 8 + 4)
        if phase == "fine64_post":
            byts = pts * 10 + pts * 8 + J * nx * 16
        return {"bytes": byts, "flops": pts * DF_OPS[p], "fp": "df"}
    if phase in ("fine64_res", "fine64_fc", "fine64_post"):
        # per point-step: 2 B shift + (p+1) FP64 weights; per interval: start slice, C value in, C value out
        byts = pts * (2 + 8 * (p + 1)) + 3 * J * nx * 8
        if phase == "fine64_post":
            byts = pts * (2 + 8 * (p + 1)) + pts * 8 + J * nx * 16  # writes every slice of the solution
        flops = pts * 2 * (p + 1)
        return {"bytes": byts, "flops": flops, "fp": 64}
    if phase == "fine32_res":
        byts = pts * (2 + 4) + 2 * J * nx * 4
        flops = pts * (2 * (p + 1) + 3 * (p + 1))
        return {"bytes": byts, "flops": flops, "fp": 32}
    if phase == "coarse" and wl.get("coarse_levels_fp64"):
        # FP64 coarse levels: per point-step the shift (2 B), p+1 FP64 weights, the stored factorisation
        # of M (solver reals per row, FP64) and the right-hand side row (8 B); each stored factor value
        # enters one FMA, plus the gather's p+1 FMAs
        nts = level_steps(wl)
        B, P = (p + 1) // 2, nx // 8
        T = P.bit_length() - 1
        q = 8 - B
        reals = (q * (2 * B + 1) + 2 * q * B + 2 * B * B) * P + T * 2 * B * B * P + B * B * P
        per_pt_b = 2 + 8 * (p + 1) + 8 * reals / nx + 8
        per_pt_f = 2 * (p + 1) + 2 * reals / nx
        byts = flops = 0.0
        for l in range(1, len(nts) - 1):
            ntl, Jl = nts[l], nts[l] // m
            steps = 2 * ntl * nx + (ntl - Jl) * nx  # FC, RES (m steps an interval), POST (m - 1)
            byts += steps * per_pt_b + 7 * Jl * nx * 8 + (ntl - Jl) * nx * 8
            flops += steps * per_pt_f
        return {"bytes": byts * iterations / max(launches, 1), "flops": flops * iterations / max(launches, 1),
                "fp": 64}
    if phase == "coarse":
        # relaxation levels 1 .. L-2, passes FC, RES, POST per cycle; per coarse point-step the staged
        # tables (eps 4 B, shift 2 B, sigma 4 B) and the right-hand side row (4 B), POST also stores
        # every F-point (4 B); per interval the start slice and one C-point row in / out (4 B each)
        nts = level_steps(wl)
        per_cycle = 0
        for l in range(1, len(nts) - 1):
            ntl, Jl = nts[l], nts[l] // m
            per_cycle += ntl * nx * 14 + 2 * Jl * nx * 4          # FC
            per_cycle += ntl * nx * 14 + 3 * Jl * nx * 4          # RES
            per_cycle += (ntl - Jl) * nx * 18 + 2 * Jl * nx * 4   # POST
        return {"bytes": per_cycle * iterations / max(launches, 1), "flops": 0, "fp": 32}
    return None


def roofline_of(phase: str, stats: dict, wl: dict, hbm_peak: float, hbm_src: str, iterations: int,
                traffic: dict | None) -> dict | None:
    ms, nl = stats["phase_ms"], stats["phase_launches"]
    if nl.get(phase, 0) == 0:
        return None
    w = phase_work(phase, wl, nl[phase], iterations)
    if w is None:
        return None
    avg_s = ms[phase] / nl[phase] / 1e3
    t_hbm = w["bytes"] / (hbm_peak * 1e9)
    alu_peak = {64: FP64_PEAK_TFLOPS, "df": FP32_PEAK_TOPS}.get(w["fp"])
    t_alu = w["flops"] / (alu_peak * 1e12) if alu_peak else 0.0
    kern = {"coarse": "k_relax_1d<p, %s, coarse> (coarse levels)" % ("double" if wl.get("coarse_levels_fp64") else "float"), "fine32_res": "k_relax_1d<p, float> (level 0)",
            "fine64_res": ("k_relax_df_1d<p> (level 0 residual, FP32 pairs)" if w["fp"] == "df"
                           else "k_relax_1d<p, double> (level 0 residual)")}.get(phase, f"k_relax_1d ({phase})")
    out = {"kernel": kern, "phase": phase, "phase_share": ms[phase] / max(sum(ms.values()), 1e-30),
           "avg_launch_ms": avg_s * 1e3}
    if t_alu > t_hbm and w["fp"] == "df":
        out.update({"bound": "alu", "achieved": w["flops"] / avg_s / 1e12, "peak": FP32_PEAK_TOPS,
                    "unit": "Tops/s (FP32)", "peak_source": "derived: 152 SM x 128 FP32 lanes x 2.07 GHz; work = FP32 "
                                                            "operations of the FP32-pair step (df_interp)"})
    elif t_alu > t_hbm:
        out.update({"bound": "alu", "achieved": w["flops"] / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"})
    else:
        out.update({"bound": "hbm", "achieved": w["bytes"] / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "peak_source": f"{hbm_src} hbm_gbs"})
    out["frac"] = out["achieved"] / out["peak"]
    out["algorithmic_bytes"] = w["bytes"]
    out["algorithmic_flops"] = w["flops"]
    out["traffic"] = (traffic or {}).get(phase)
    return out


def roofline(stats: dict, wl: dict, hbm_peak: float, hbm_src: str, iterations: int,
             traffic: dict | None) -> tuple[dict, list]:
    """The dominant kernel (largest phase share among the relaxation kernels) and the others."""
    ms = stats["phase_ms"]
    cands = [k for k in ("coarse", "fine64_res", "fine32_res") if stats["phase_launches"].get(k, 0)]
    cands.sort(key=lambda k: -ms[k])
    lines = [roofline_of(k, stats, wl, hbm_peak, hbm_src, iterations, traffic) for k in cands]
    lines = [x for x in lines if x]
    if not lines:
        return {"bound": None}, []
    return lines[0], lines[1:]


# ------------------------------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ------------------------------------------------------------------------------------------------

def oracle_sample(nt_sample: int) -> tuple[float, int]:
    """Oracle MGRIT solve of the workload truncated to its first nt_sample steps; returns (seconds, iterations)."""
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    wl = WORKLOAD
    t0 = time.perf_counter()
    H = omg.build_hierarchy(osl.Grid(wl["nx"], nt_sample, cfl=wl["cfl"]), osl.WaveSpeed(wl["wave"], a=wl["a"], k=wl["k"]),
                            wl["order"], wl["m"], max_coarsest=wl["max_coarsest"])
    R = omg.mgrit_solve(H, W.u0_bumps_1d(wl["nx"], W.SEED_C2_BUMPS, 3), W.initial_iterate(nt_sample, wl["nx"]),
                        rtol=wl["rtol"])
    return time.perf_counter() - t0, R.iterations


def cores_used() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", "1"))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args) -> None:
    rank, _, world = rank_info()
    if rank != 0:
        return
    wl = WORKLOAD
    dof = wl["nx"] * REF_SAMPLE_NT
    for _ in range(args.warmup):
        oracle_sample(REF_SAMPLE_NT)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        _, its = oracle_sample(REF_SAMPLE_NT)
    el = time.perf_counter() - t0
    value = dof * args.steps / el
    sample = f"oracle MGRIT solve to 1e-10 of the first {REF_SAMPLE_NT} of {wl['nt']} time steps (nx={wl['nx']})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**wl, "sample_nt": REF_SAMPLE_NT}, "iterations": its,
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# the GPU arm
# ------------------------------------------------------------------------------------------------

def run_ours(args) -> None:
    import torch

    import paper_2203_13382_gb300 as mg

    rank, local_rank, world = rank_info()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = dict(WORKLOAD)
    if args.nt:  # another time axis (profiling captures, the long-axis case); not the benchmark workload
        wl["nt"] = args.nt
        wl["workload"] = wl["workload"].replace(f"nt{WORKLOAD['nt']}", f"nt{args.nt}")
    if args.nx:  # another slice length (the long-axis case nx 512, nt 131072); not the benchmark workload
        wl["nx"] = args.nx
        wl["workload"] = wl["workload"].replace(f"nx{WORKLOAD['nx']}", f"nx{args.nx}")
    nx, nt = wl["nx"], wl["nt"]
    dof = nx * nt
    prec = 0 if args.precision == "fp64" else 1
    cf64 = 1 if args.precision == "fp32bulk_coarse64" else 0
    wl["precision"] = args.precision
    wl["coarse_levels_fp64"] = 1 if (prec == 0 or cf64) else 0
    u0_h = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
    U_h = W.initial_iterate(nt, nx)
    u0 = torch.from_numpy(u0_h).cuda()
    U0 = torch.from_numpy(U_h).cuda()
    u_out = torch.empty(nt + 1, nx, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step(profile: int):
        h = mg.mgrit_setup(nx, nt, wl["order"], wl["m"], wave=wl["wave"], a=wl["a"], k=wl["k"], cfl=wl["cfl"],
                           max_coarsest=wl["max_coarsest"], precision=prec, coarse_fp64=cf64, rtol=wl["rtol"],
                           profile=profile)
        _, st = h.solve(u0, U0, u_out)
        h.destroy()
        return st

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        one_step(0)
    barrier()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id)
    sampler.start()
    # timed region 1 (the value): K solves with no instrumentation inside
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(one_step(0))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    # timed region 2 (kernel durations): K more solves with CUDA events around every kernel launch on the
    # launching stream; events serialise the stream, so these solves run slightly longer (reported)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    pstats = [one_step(1) for _ in range(args.steps)] if not args.no_phase_events else []
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_events = f0.elapsed_time(f1) / args.steps if pstats else None
    if not pstats:  # phase table from one solve outside the timed regions
        pstats = [one_step(1)]
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_value(dof, world, ms)

    # phase sums over the instrumented timed steps
    agg_ms = {k: sum(s["phase_ms"][k] for s in pstats) for k in pstats[0]["phase_ms"]}
    agg_nl = {k: sum(s["phase_launches"][k] for s in pstats) for k in pstats[0]["phase_launches"]}
    launches = int(sum(s["kernel_launches"] for s in stats))
    iters = [s["iterations"] for s in stats]
    hbm, hbm_src = peaks()
    traffic = None
    if os.path.exists(os.path.join(ROOT, "profiles", "traffic.json")):
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f).get(args.precision)
    roof, roof_others = roofline({"phase_ms": agg_ms, "phase_launches": agg_nl}, wl, hbm, hbm_src,
                                 sum(s["iterations"] for s in pstats), traffic)

    seq_ms, seq_best, seq_full_ms, fixed_point, e2e = {}, None, None, None, None
    if not args.no_comparator:
        # comparator: sequential SL stepping on the same GPU (one thread-block cluster per slice), FP64 and FP32,
        # each timed like the MGRIT step: a fine_only setup (departure points and the fine level's tables) +
        # the nt steps + destroy, CUDA events; the faster one is the reported comparator
        seq_ms, seq_steps = {}, {}
        for name, pr in (("fp64", 0), ("fp32", 1)):
            def seq_step():
                hs = mg.mgrit_setup(nx, nt, wl["order"], wl["m"], wave=wl["wave"], a=wl["a"], k=wl["k"], cfl=wl["cfl"],
                                    precision=pr, fine_only=1)
                out = hs.sequential(u0, store_all=False)
                hs.destroy()
                return out
            for _ in range(2):
                seq_step()
            torch.cuda.synchronize()
            nseq = max(3, args.steps)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(nseq):
                last = seq_step()
            s1.record(stream)
            torch.cuda.synchronize()
            seq_ms[name] = s0.elapsed_time(s1) / nseq
            hs = mg.mgrit_setup(nx, nt, wl["order"], wl["m"], wave=wl["wave"], a=wl["a"], k=wl["k"], cfl=wl["cfl"],
                                precision=pr, fine_only=1)
            hs.sequential(u0, store_all=False)
            torch.cuda.synchronize()
            s0.record(stream)
            for _ in range(nseq):
                hs.sequential(u0, store_all=False)
            s1.record(stream)
            torch.cuda.synchronize()
            seq_steps[name] = s0.elapsed_time(s1) / nseq
            hs.destroy()
            if pr == 0:
                seq_last = last.clone()
        seq_best = min(seq_ms, key=seq_ms.get)
        seq_full_ms = seq_ms[seq_best]
        fixed_point = float((seq_last - u_out[-1]).norm() / seq_last.norm())

        # end to end through the host-buffer entry point (inputs from pinned host memory, solution back)
        u0_pin = torch.from_numpy(u0_h).pin_memory()
        U_pin = torch.from_numpy(U_h).pin_memory()
        out_pin = torch.empty(nt + 1, nx, dtype=torch.float64).pin_memory()
        ne2e = max(2, args.steps // 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            he = mg.mgrit_setup(nx, nt, wl["order"], wl["m"], wave=wl["wave"], a=wl["a"], k=wl["k"], cfl=wl["cfl"],
                                max_coarsest=wl["max_coarsest"], precision=prec, coarse_fp64=cf64, rtol=wl["rtol"])
            he.solve_host(u0_pin.numpy(), U_pin.numpy(), out_pin.numpy())
            he.destroy()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / ne2e
        J = nt // wl["m"]
        e2e = {"value": world * dof / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": nx * 8 + J * nx * 8,
               "d2h_bytes_per_step": (nt + 1) * nx * 8,
               "path": "mgrit_setup + mgrit_solve_host (pinned host buffers) + mgrit_destroy, wall clock"}


    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        secs, cpu_its = oracle_sample(CPU_SAMPLE_NT)
        cpu = {"value": nx * CPU_SAMPLE_NT / secs, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle",
               "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
               "sample": f"oracle MGRIT solve to 1e-10 of the first {CPU_SAMPLE_NT} of {nt} time steps "
                         f"(nx={nx}; {cpu_its} iterations, {secs:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
            "config": {**wl, "precision": args.precision, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2: per-step gather tables alone exceed 2 GB"},
            "iterations": iters[0], "iterations_all_steps": sorted(set(iters)),
            "device_bytes": int(stats[0]["device_bytes"]),
            "setup_ms_per_step": float(np.median([st["setup_ms"] for st in stats])),
            "solve_only_ms_per_step": float(np.median([st["solve_ms"] for st in stats])),
            "solve_only_value": dof / (float(np.median([st["solve_ms"] for st in stats])) / 1e3),
            "comparator": None if args.no_comparator else {"sequential_dof_per_s": dof / (seq_full_ms / 1e3),
                           "sequential_ms": seq_full_ms, "sequential_precision": seq_best,
                           "sequential_ms_by_precision": seq_ms, "sequential_steps_only_ms": seq_steps,
                           "sequential_includes": "mgrit_setup(fine_only: FP64 departure points + fine-level tables) "
                                                  "+ nt SL steps (one thread-block cluster per slice) + destroy, "
                                                  "CUDA events",
                           "mgrit_over_sequential": (dof / (ms / 1e3)) / (dof / (seq_full_ms / 1e3)),
                           "fixed_point_rel_diff_final_slice": fixed_point},
            "roofline": roof, "roofline_others": roof_others, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "phases_ms_per_step": {k: v / len(pstats) for k, v in agg_ms.items() if agg_nl[k]},
            "phase_launches_per_step": {k: v // len(pstats) for k, v in agg_nl.items() if v},
            "timing": {"value": "K solves without instrumentation (CUDA events around the K solves)",
                       "kernels": "K further solves with CUDA events around every launch on its stream",
                       "ms_per_step_with_kernel_events": ms_events},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()



# ------------------------------------------------------------------------------------------------
# further workloads (--workload): the 2D solve, the batched problems and the 2D adjoint gradient
# ------------------------------------------------------------------------------------------------

WORKLOAD_2D = {"workload": "advection2d_alpha_1+0.5sin2piy_cos2pit_1+0.5cos2pix_sin2pit_512x512_nt2048_p5_m4",
               "nx": 512, "nt": 2048, "order": 5, "m": 4, "wave": "sin_cos2", "a": 0.5, "cfl": 0.85,
               "u0": "5 gaussian bumps, seed 20260002", "rtol": 1e-10, "precision": "fp32bulk",
               "coarse_solve": "GMRES from zero, rtol 1e-2 or 10 iterations"}
WORKLOAD_ADJ = {"workload": "adjoint2d_alpha_sin_cos2_a0.5_256x256_nt1024_p3_m4",
                "nx": 256, "nt": 1024, "order": 3, "m": 4, "wave": "sin_cos2", "a": 0.5, "cfl": 0.85,
                "u0": "5 gaussian bumps, seed 20260005",
                "u_target": "sequential solution at a = 0.4 from 5 bumps, seed 20260006", "rtol": 1e-10,
                "precision": "fp64"}
WORKLOAD_BATCH = {"workload": "batched1d_256_problems_seed20260004", "problems": 256, "precision": "fp32bulk",
                  "rtol": 1e-10, "u0": "sin^4(pi x)",
                  "draws": "nx in 256..4096, nt in 1024..16384 (powers of two), p in {1,3,5}, a in [0.1,0.7], "
                           "k in {1,2,3}, m in {4,8}"}


def _timed(fn, steps: int, warmup: int):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs = [fn() for _ in range(steps)]
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, outs


def _line(args, metric: str, value: float, unit: str, ms: float, cfg: dict, **extra) -> None:
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if cfg.get("precision") == "fp32bulk" else "f64", "data": "synthetic", "config": cfg}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_2d(args) -> None:
    import torch

    import paper_2203_13382_gb300 as mg

    wl = dict(WORKLOAD_2D)
    if args.nx or args.nt:  # smaller grids (profiling captures only)
        wl["nx"], wl["nt"] = args.nx or wl["nx"], args.nt or wl["nt"]
        wl["workload"] += f"_override_{wl['nx']}x{wl['nx']}_nt{wl['nt']}"
    nx, nt, p, m = wl["nx"], wl["nt"], wl["order"], wl["m"]
    npts = nx * nx
    u0 = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C3_BUMPS, 5).ravel().copy()).cuda()
    U0 = torch.zeros(nt + 1, npts, dtype=torch.float64, device="cuda")
    rows = np.arange(m, nt + 1, m)  # the solve reads the initial iterate at the C-points only
    U0[rows] = torch.from_numpy(W.initial_iterate(nt, npts, rows=rows)).cuda()
    out = torch.empty(nt + 1, npts, dtype=torch.float64, device="cuda")

    def step(profile=0):
        h = mg.mgrit_setup(nx, nt, p, m, wave=wl["wave"], a=wl["a"], a2=wl["a"], dim=2, precision=1, profile=profile)
        _, st = h.solve(u0, U0, out)
        h.destroy()
        return st

    sampler = ClockSampler("0")
    sampler.start()
    ms, stats = _timed(step, args.steps, args.warmup)
    clocks = sampler.stop()
    prof = step(1)
    h = mg.mgrit_setup(nx, nt, p, m, wave=wl["wave"], a=wl["a"], a2=wl["a"], dim=2, precision=1, profile=1)
    seq_ms, _ = _timed(lambda: h.sequential(u0, store_all=False), 3, 1)
    last = h.sequential(u0, store_all=False)
    fixed32 = float((last - out[-1]).norm() / last.norm())
    h.destroy()
    # the fixed point in FP64: sequential stepping of an FP64 handle (the MGRIT solve converges to the
    # FP64 discrete solution; the FP32 stepper differs from it by its own rounding)
    h = mg.mgrit_setup(nx, nt, p, m, wave=wl["wave"], a=wl["a"], a2=wl["a"], dim=2, precision=0)
    last64 = h.sequential(u0, store_all=False)
    fixed = float((last64 - out[-1]).norm() / last64.norm())
    h.destroy()
    dof = npts * nt
    ph = prof["phase_ms"]
    seq_full = seq_ms + ph["departure"] + ph["tables"] * nt / sum(nt // m ** l for l in range(prof["levels"]))
    _line(args, METRIC, dof / (ms / 1e3), "DOF/s", ms, wl, iterations=stats[0]["iterations"],
          comparator={"sequential_ms": seq_full, "sequential_steps_only_ms": seq_ms,
                      "sequential_dof_per_s": dof / (seq_full / 1e3),
                      "mgrit_over_sequential": seq_full / ms, "fixed_point_rel_diff_final_slice": fixed,
                      "fp32_sequential_rel_diff_final_slice": fixed32},
          phases_ms_per_step={k: v for k, v in ph.items() if v}, clocks=clocks,
          gpu_launches=int(stats[0]["kernel_launches"]), device_bytes=int(stats[0]["device_bytes"]))


# ---- the batched workload (the default benchmark line) -----------------------------------------------

BATCH_CPU_SAMPLE = (8, 256)   # cpu_baseline: the first 8 problems, each on its first 256 time steps
BATCH_REF_SAMPLE = (2, 256)   # --impl reference: one step = the first 2 problems on their first 256 steps


def batch_levels(q, max_coarsest: int = 1) -> list[int]:
    """Steps per level of one batched problem under the library's rule (factor m until <= max_coarsest)."""
    out = [q.nt]
    while out[-1] > max_coarsest and out[-1] % q.m == 0:
        out.append(out[-1] // q.m)
    return out


def batch_phase_work(phase: str, probs, iters: list[int]) -> dict | None:
    """Algorithmic bytes and flops of one phase over a whole batched solve (problem q takes part in
    iters[q] cycles; the per-pass figures are those of phase_work for one problem)."""
    byts = flops = 0.0
    fp = 32
    for q, it in zip(probs, iters):
        nx, p, m = q.nx, q.order, q.m
        nts = batch_levels(q)
        J = q.nt // m
        pts = nx * q.nt
        if phase == "fine64_res":
            # FP32 pairs: per point-step eps hi, eps lo (4 B each) and shift (2 B); per interval the start slice and
            # C value in (8 B each), the residual out in FP64 and FP32; work: FP32 operations of the pair step
            byts += it * (pts * 10 + J * nx * (8 + 8 + 8 + 4))
            flops += it * pts * DF_OPS[p]
            fp = "df"
        elif phase == "fine32_res":
            byts += it * (pts * 6 + J * nx * (4 + 4))
            flops += it * pts * 2 * (p + 1)
        elif phase == "coarse":
            per_cycle = 0
            for l in range(1, len(nts) - 1):
                ntl, Jl = nts[l], nts[l] // m
                per_cycle += ntl * nx * 14 + 2 * Jl * nx * 4          # FC
                per_cycle += ntl * nx * 14 + 3 * Jl * nx * 4          # RES
                per_cycle += (ntl - Jl) * nx * 18 + 2 * Jl * nx * 4   # POST
            byts += it * per_cycle
        elif phase == "coarsest":
            byts += it * nts[-1] * nx * 14
        else:
            return None
    return {"bytes": byts, "flops": flops, "fp": fp}


BATCH_KERNELS = {"fine64_res": "k_relax_batched_df (level-0 residual in FP32 pairs, every problem)",
                 "fine32_res": "k_relax_batched<float, false, NT> (level-0 FP32 error pass, per CTA size)",
                 "coarse": "k_relax_batched<float, true, NT> (coarse levels FC/RES/POST)",
                 "coarsest": "k_sequential_batched<float, true> (coarsest levels)"}


def batch_roofline(phase_ms: dict, phase_n: dict, probs, iters, hbm_peak: float, hbm_src: str,
                   traffic: dict | None) -> tuple[dict, list]:
    """Roofline of every relaxation phase of the batched solve; the first is the one with the largest share."""
    total = max(sum(phase_ms.values()), 1e-30)
    lines = []
    for ph in ("fine64_res", "fine32_res", "coarse", "coarsest"):
        n = phase_n.get(ph, 0)
        if not n:
            continue
        w = batch_phase_work(ph, probs, iters)
        t = phase_ms[ph] / 1e3  # seconds over the solve
        t_hbm = w["bytes"] / (hbm_peak * 1e9)
        t_alu = w["flops"] / (FP32_PEAK_TOPS * 1e12) if w["fp"] == "df" else 0.0
        out = {"kernel": BATCH_KERNELS[ph], "phase": ph, "phase_share": phase_ms[ph] / total, "launches": n,
               "avg_launch_ms": phase_ms[ph] / n}
        if t_alu > t_hbm:
            out.update({"bound": "alu", "achieved": w["flops"] / t / 1e12, "peak": FP32_PEAK_TOPS,
                        "unit": "Tops/s (FP32)", "peak_source": "derived: 152 SM x 128 FP32 lanes x 2.07 GHz; work = "
                                                                "FP32 operations of the FP32-pair step (df_interp)"})
        else:
            out.update({"bound": "hbm", "achieved": w["bytes"] / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "peak_source": f"{hbm_src} hbm_gbs"})
        out["frac"] = out["achieved"] / out["peak"]
        out["algorithmic_bytes_per_launch"] = w["bytes"] / n
        out["algorithmic_flops_per_launch"] = w["flops"] / n
        out["traffic"] = (traffic or {}).get(ph)
        lines.append(out)
    lines.sort(key=lambda x: -x["phase_share"])
    if not lines:
        return {"bound": None}, []
    return lines[0], lines[1:]


def batch_inputs(probs):
    """u0 = sin^4(pi x) and the random initial iterate (read at the C-points only) of every problem."""
    u0s = [W.u0_sin4(q.nx) for q in probs]
    rows = [np.arange(0, q.nt + 1, q.m) for q in probs]
    inits_c = [W.initial_iterate(q.nt, q.nx, rows=r) for q, r in zip(probs, rows)]  # row 0 is zero (ignored)
    return u0s, rows, inits_c


def oracle_batch_sample(nprob: int, nt_s: int) -> tuple[float, int, list[int]]:
    """Oracle MGRIT solves of the first nprob batched problems, each on its first nt_s steps (same nx, p, m,
    alpha, u0, initial iterate); returns (seconds, DOF, iterations)."""
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    probs = W.batched_problems(WORKLOAD_BATCH["problems"])[:nprob]
    t0 = time.perf_counter()
    its = []
    for q in probs:
        H = omg.build_hierarchy(osl.Grid(q.nx, nt_s), osl.WaveSpeed("sin_kx_cos_t", a=q.a, k=float(q.k)), q.order, q.m)
        its.append(omg.mgrit_solve(H, W.u0_sin4(q.nx), W.initial_iterate(nt_s, q.nx), rtol=WORKLOAD_BATCH["rtol"]).iterations)
    return time.perf_counter() - t0, sum(q.nx * nt_s for q in probs), its


def run_reference_batched(args) -> None:
    rank, _, _ = rank_info()
    if rank != 0:
        return
    nprob, nt_s = BATCH_REF_SAMPLE
    for _ in range(args.warmup):
        oracle_batch_sample(nprob, nt_s)
    el, dof, its = 0.0, 0, []
    for _ in range(args.steps):
        t, dof, its = oracle_batch_sample(nprob, nt_s)
        el += t
    value = dof * args.steps / el
    sample = (f"oracle MGRIT solves to 1e-10 of the first {nprob} of {WORKLOAD_BATCH['problems']} batched problems, "
              f"each on its first {nt_s} time steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**WORKLOAD_BATCH, "sample_problems": nprob, "sample_nt": nt_s}, "iterations": its,
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_mem_available() -> int | None:
    """MemAvailable of /proc/meminfo in bytes (None if unknown)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def run_batched(args) -> None:
    import torch

    import paper_2203_13382_gb300 as mg

    rank, local_rank, world = rank_info()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = dict(WORKLOAD_BATCH)
    probs = W.batched_problems(wl["problems"])
    if args.problems and args.problems < wl["problems"]:  # the first problems of the draw (profiling captures only)
        probs = probs[:args.problems]
        wl["workload"] += f"_first{args.problems}"
        wl["problems_used"] = args.problems
    specs = [dict(nx=q.nx, nt=q.nt, order=q.order, m=q.m, a=q.a, k=float(q.k)) for q in probs]
    u0_h, rows, inits_c = batch_inputs(probs)
    u0s = [torch.from_numpy(u).cuda() for u in u0_h]
    inits, outs = [], []
    for q, r, ic in zip(probs, rows, inits_c):
        U = torch.zeros(q.nt + 1, q.nx, dtype=torch.float64, device="cuda")
        U[torch.from_numpy(r).cuda()] = torch.from_numpy(ic).cuda()
        inits.append(U)
        outs.append(torch.empty(q.nt + 1, q.nx, dtype=torch.float64, device="cuda"))
    dof = sum(q.nx * q.nt for q in probs)
    stream = torch.cuda.current_stream()

    def one_step(profile: int):
        b = mg.mgrit_setup_batched(specs, rtol=wl["rtol"], profile=profile)
        _, st = b.solve(u0s, inits, outs)
        b.destroy()
        return st

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):  # the first setup also runs the tuner (its choices are cached per batch)
        one_step(0)
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(_gpu_id(torch, local_rank))
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [one_step(0) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    # kernel durations: a few more steps with CUDA events around every launch on its stream
    nprof = max(1, min(3, args.steps))
    pstats = [one_step(1) for _ in range(nprof)]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    value = whole_job_value(dof, world, ms)
    iters = [st["iterations"] for st in stats[0]]
    conv = all(st["converged"] for st in stats[0])
    launches = int(sum(st[0]["kernel_launches"] for st in stats))
    # phase table per step: setup phases summed over the problems, cycle phases from the batch totals
    setup_ph = ("departure", "backtrack", "tables", "factor")
    ph_ms = {k: 0.0 for k in pstats[0][0]["phase_ms"]}
    ph_n = {k: 0 for k in ph_ms}
    for st in pstats:
        for k in ph_ms:
            if k in setup_ph:
                ph_ms[k] += sum(x["phase_ms"][k] for x in st) / nprof
                ph_n[k] += sum(x["phase_launches"][k] for x in st) // nprof
            else:
                ph_ms[k] += st[0]["phase_ms"][k] / nprof
                ph_n[k] += st[0]["phase_launches"][k] // nprof
    hbm, hbm_src = peaks()
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f).get("batched")
    roof, roof_others = batch_roofline(ph_ms, ph_n, probs, [x["iterations"] for x in pstats[0]], hbm, hbm_src,
                                       traffic)

    comparator, e2e = None, None
    if not args.no_comparator:
        # comparator: sequential SL stepping of every problem on the same GPU, all problems in one launch (one CTA
        # each, FP32), with the setup it needs (fine departure points and fine-level tables: a fine_only batch),
        # timed like the MGRIT step: setup + stepping + destroy, CUDA events
        def seq_step():
            bs = mg.mgrit_setup_batched(specs, fine_only=1)
            out = bs.sequential(u0s)
            bs.destroy()
            return out

        for _ in range(2):
            seq_step()
        torch.cuda.synchronize()
        nseq = max(3, min(args.steps, 10))
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(nseq):
            last = seq_step()
        s1.record(stream)
        torch.cuda.synchronize()
        seq_ms = s0.elapsed_time(s1) / nseq
        bs = mg.mgrit_setup_batched(specs, fine_only=1)
        bs.sequential(u0s)
        torch.cuda.synchronize()
        s0.record(stream)
        for _ in range(nseq):
            last = bs.sequential(u0s)
        s1.record(stream)
        torch.cuda.synchronize()
        seq_steps_ms = s0.elapsed_time(s1) / nseq
        bs.destroy()
        # against the solution's scale (some final slices decay far below |u0|)
        fixed = max(float((l - o[-1]).norm() / max(float(l.norm()), float(u.norm()))) for l, o, u in zip(last, outs, u0s))
        comparator = {"sequential_dof_per_s": dof / (seq_ms / 1e3), "sequential_ms": seq_ms,
                      "sequential_steps_only_ms": seq_steps_ms, "sequential_setup_ms": seq_ms - seq_steps_ms,
                      "sequential_precision": "fp32",
                      "sequential_includes": "mgrit_setup_batched(fine_only: FP64 departure points + fine tables of "
                                             "every problem) + sl_step_sequential_batched (all problems in one launch, "
                                             "one CTA each, FP32) + destroy, CUDA events",
                      "mgrit_over_sequential": seq_ms / ms,
                      "fp32_sequential_vs_mgrit_final_slice_max_diff_rel_to_scale": fixed}
        # end to end through the host-buffer entry point: inputs from pinned host memory, every solution back
        need = sum((q.nt + 1) * q.nx * 8 for q in probs)
        avail = host_mem_available()
        try:
            if avail is not None and avail < 2 * need:
                raise RuntimeError("not enough host memory to pin the solutions")
            u0_pin = [torch.from_numpy(u).pin_memory() for u in u0_h]
            ic_pin = [torch.from_numpy(ic).pin_memory() for ic in inits_c]
            out_pin = [torch.empty(q.nt + 1, q.nx, dtype=torch.float64, pin_memory=True) for q in probs]
            pinned = True
        except RuntimeError:
            u0_pin = [torch.from_numpy(u) for u in u0_h]
            ic_pin = [torch.from_numpy(ic) for ic in inits_c]
            out_pin = [torch.empty(q.nt + 1, q.nx, dtype=torch.float64) for q in probs]
            pinned = False
        ne2e = 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            be = mg.mgrit_setup_batched(specs, rtol=wl["rtol"])
            be.solve_host([u.numpy() for u in u0_pin], [x.numpy() for x in ic_pin], [x.numpy() for x in out_pin])
            be.destroy()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / ne2e
        e2e = {"value": world * dof / e2e_s, "unit": "DOF/s",
               "h2d_bytes_per_step": int(sum((q.nx + (q.nt // q.m) * q.nx) * 8 for q in probs)),
               "d2h_bytes_per_step": int(sum((q.nt + 1) * q.nx * 8 for q in probs)), "pinned": pinned,
               "path": "mgrit_setup_batched + mgrit_solve_batched_host (host u0, C-point iterate in; every full "
                       "solution out) + mgrit_destroy_batched, wall clock"}
        del u0_pin, ic_pin, out_pin

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        nprob, nt_s = BATCH_CPU_SAMPLE
        secs, sdof, sits = oracle_batch_sample(nprob, nt_s)
        cpu = {"value": sdof / secs, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle", "cpu_model": cpu_model(),
               "host_cores": os.cpu_count(),
               "sample": f"oracle MGRIT solves to 1e-10 of the first {nprob} of {len(probs)} problems, each on its "
                         f"first {nt_s} time steps (iterations {sits}, {secs:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {**wl, "dof": dof, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (per-step gather tables of the batch exceed 10 GB)"},
            "iterations_min_max": [min(iters), max(iters)], "converged": conv,
            "device_bytes": int(sum(x["device_bytes"] for x in stats[0])),
            "setup_ms_per_step": float(np.median([max(x["setup_ms"] for x in st) for st in stats])),
            "comparator": comparator, "roofline": roof, "roofline_others": roof_others, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "phases_ms_per_step": {k: v for k, v in ph_ms.items() if ph_n[k]},
            "phase_launches_per_step": {k: v for k, v in ph_n.items() if v},
            "timing": {"value": "K steps (batched setup + solve + destroy) without instrumentation, CUDA events",
                       "kernels": f"{nprof} further steps with CUDA events around every launch on its stream; setup "
                                  "phases summed over the problems (their setups overlap on 8 streams)"},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _gpu_id(torch, local_rank: int) -> str:
    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    return gpu_id


def run_adjoint2d(args) -> None:
    import torch

    import paper_2203_13382_gb300 as mg

    wl = WORKLOAD_ADJ
    nx, nt, p, m = wl["nx"], wl["nt"], wl["order"], wl["m"]
    npts = nx * nx
    u0 = torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_BUMPS, 5).ravel().copy()).cuda()
    ht = mg.mgrit_setup(nx, nt, p, m, wave="sin_cos2", a=0.4, dim=2)
    ut = ht.sequential(torch.from_numpy(W.u0_bumps_2d(nx, W.SEED_C5_TARGET, 5).ravel().copy()).cuda(),
                       store_all=False).clone()
    ht.destroy()
    U0 = torch.zeros(nt + 1, npts, dtype=torch.float64, device="cuda")
    rows = np.arange(m, nt + 1, m)
    U0[rows] = torch.from_numpy(W.initial_iterate(nt, npts, rows=rows)).cuda()
    out = torch.empty(nt + 1, npts, dtype=torch.float64, device="cuda")
    times = {}

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        h = mg.mgrit_setup(nx, nt, p, m, wave=wl["wave"], a=wl["a"], dim=2, precision=0)
        _, st = h.solve(u0, U0, out)
        e[1].record()
        g_u0, g_a, ast = h.adjoint(ut, out[::m].contiguous())
        e[2].record()
        h.destroy()
        torch.cuda.synchronize()
        times.setdefault("fwd", []).append(e[0].elapsed_time(e[1]))
        times.setdefault("adj", []).append(e[1].elapsed_time(e[2]))
        return st, ast, float(g_a)

    sampler = ClockSampler("0")
    sampler.start()
    ms, res = _timed(step, args.steps, args.warmup)
    clocks = sampler.stop()
    st, ast, g_a = res[0]
    dof = npts * nt
    k = args.steps
    _line(args, "space-time DOF/s of the gradient (MGRIT forward + adjoint MGRIT) to 1e-10", dof / (ms / 1e3),
          "DOF/s", ms, wl, forward_ms=float(np.mean(times["fwd"][-k:])), adjoint_ms=float(np.mean(times["adj"][-k:])),
          iterations_forward=st["iterations"], iterations_adjoint=ast["iterations"], dJ_da=g_a, clocks=clocks)


def run_twolevel(args) -> None:
    """The two-level constant-speed case (nx = nt = 256, alpha = 1, p = 1, m = 4, FP64): GPU MGRIT and
    sequential stepping, and the oracle's MGRIT and sequential stepping on one core (the whole case)."""
    import torch

    import paper_2203_13382_gb300 as mg
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    nx, nt = 256, 256
    u0 = torch.from_numpy(W.u0_sin4(nx)).cuda()
    U0 = torch.from_numpy(W.initial_iterate(nt, nx)).cuda()

    def step():
        h = mg.mgrit_setup(nx, nt, 1, 4, wave="const", a=1.0, levels=2)
        _, st = h.solve(u0, U0)
        h.destroy()
        return st

    ms, stats = _timed(step, max(args.steps, 10), args.warmup)
    h = mg.mgrit_setup(nx, nt, 1, 4, wave="const", a=1.0, levels=2)
    seq_ms, _ = _timed(lambda: h.sequential(u0, store_all=False), 10, 2)
    h.destroy()
    t0 = time.perf_counter()
    H = omg.build_hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("const", a=1.0), 1, 4, levels=2)
    R = omg.mgrit_solve(H, W.u0_sin4(nx), W.initial_iterate(nt, nx))
    t_or = time.perf_counter() - t0
    t0 = time.perf_counter()
    omg.sequential_solve(omg.Hierarchy(osl.Grid(nx, nt), osl.WaveSpeed("const", a=1.0), 1, []), W.u0_sin4(nx))
    t_seq = time.perf_counter() - t0
    dof = nx * nt
    _line(args, METRIC, dof / (ms / 1e3), "DOF/s", ms,
          {"workload": "advection1d_const_alpha1_nx256_nt256_p1_m4_two_levels", "precision": "fp64"},
          iterations=stats[0]["iterations"], iterations_oracle=R.iterations,
          comparator={"sequential_ms": seq_ms, "sequential_dof_per_s": dof / (seq_ms / 1e3)},
          cpu_baseline={"value": dof / t_or, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle",
                        "sample": "the whole case (oracle MGRIT, setup included)"},
          cpu_sequential={"value": dof / t_seq, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle"})


def run_cpu(args) -> None:
    """The oracle's sequential stepping and MGRIT on bounded samples of the 1D workload (one core)."""
    from oracle import mgrit as omg
    from oracle import semi_lagrangian as osl

    wl = WORKLOAD
    nx = wl["nx"]
    out = {}
    for name, nts in (("sequential", 2048), ("mgrit", CPU_SAMPLE_NT)):
        g = osl.Grid(nx, nts, cfl=wl["cfl"])
        ws = osl.WaveSpeed(wl["wave"], a=wl["a"], k=wl["k"])
        u0 = W.u0_bumps_1d(nx, W.SEED_C2_BUMPS, 3)
        t0 = time.perf_counter()
        if name == "sequential":
            omg.sequential_solve(omg.Hierarchy(g, ws, wl["order"], []), u0)
            its = None
        else:
            H = omg.build_hierarchy(g, ws, wl["order"], wl["m"], max_coarsest=wl["max_coarsest"])
            its = omg.mgrit_solve(H, u0, W.initial_iterate(nts, nx), rtol=wl["rtol"]).iterations
        el = time.perf_counter() - t0
        out[name] = {"value": nx * nts / el, "unit": "DOF/s", "cores": cores_used(), "kind": "oracle",
                     "sample": f"first {nts} of {wl['nt']} steps, nx = {nx}, departure points included",
                     "seconds": el, "iterations": its}
    print(json.dumps({"impl": "oracle", "workload": wl["workload"], **out}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32bulk", "fp64", "fp32bulk_coarse64"], default="fp32bulk",
                    help="fp32bulk_coarse64: FP32 error relaxation on level 0, FP64 coarse cycle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true", help="skip the sequential comparator and e2e runs")
    ap.add_argument("--nt", type=int, default=0, help="override nt (small profiling cases only)")
    ap.add_argument("--nx", type=int, default=0,
                    help="override nx (1D: another slice length, e.g. the long-axis case; 2D: small profiling cases)")
    ap.add_argument("--workload", choices=["batched", "advection1d", "advection2d", "adjoint2d", "twolevel", "cpu"],
                    default="batched", help="batched (256 problems) is the benchmark; the others measure further rows")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched: use only the first N problems of the 256 (small profiling cases only)")
    ap.add_argument("--no-phase-events", action="store_true",
                    help="skip the second, instrumented timed region (phase table from one solve)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        if args.workload == "batched":
            run_reference_batched(args)
        else:
            run_reference(args)
    elif args.workload == "advection2d":
        run_2d(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint2d":
        run_adjoint2d(args)
    elif args.workload == "twolevel":
        run_twolevel(args)
    elif args.workload == "cpu":
        run_cpu(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
