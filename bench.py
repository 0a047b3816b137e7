"""Benchmark: Jacobian columns per second of the standing-wave shooting map.

One step = one full shoot_jacobian (all RK4 stages of all columns, setup and
outputs included) on the seeded N = 2048 workload (512 Fourier unknowns + T,
1024 RK4 steps, h = 1, c_1 = 0.4, c_k = 0.4^k u_k).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form mixed|fp64]
                  [--impl ours|reference] [--workload NAME] [--no-fp64-form]

--form mixed (default) is the tensor-core form (FP32-accurate inverse, FP64-
accurate Ozaki products, iterative refinement to a 1e-13 residual).  Its line
also carries the metric's comparison: `fp64_form`, one timed Jacobian of the
plain FP64 form on the same workload (~1.5 minutes), and `error_vs_oracle`,
both forms' errors against the oracle's stored samples of the workload.
--form fp64 times the plain FP64 form alone.  `value` is timed with the
library's phase events off; one more Jacobian with them on gives the
per-kernel `rooflines` (and, in the mixed form, the measured refinement
residual in `stats`).

--impl reference times the CPU FP64 oracle (the only baseline: the paper's
code is not available) on a bounded sample of the same workload, scaled to
the full Jacobian (marked "extrapolated").  Under torchrun every rank runs an
independent replica (its own seed; the path has no exchange step), the
slowest rank's time is reported and value counts the columns of all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1210_5672_gb300 import workloads as W  # noqa: E402

METRIC = "Jacobian columns/s at N=2048, mixed vs plain FP64 at 1e-12 rel err; % roofline"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# FP64 pipe of GB300: 2 FP64 FMA per clock per SM (1/64 of FP32), 152 SMs,
# 2070 MHz maximum -> 2 * 2 * 152 * 2.07e9 = 1.259 TFLOP/s.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_rate(local_step_s, ws, columns):
    """Whole-job rate of ws independent replicas: each rank ran `columns` columns
    per step in local_step_s seconds; the slowest rank's step time sets the job's."""
    t = allmax(local_step_s, ws)
    return t, ws * columns / t


def allmax(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def flush_l2(buf):
    buf.add_(1.0)   # 512 MB read + write: evicts the 129 MB L2


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel, from one ncu capture of the current kernel on the N = 2048 workload
# (summaries under profiles/); a kernel changed since its capture has none (null).
TRAFFIC_BYTES = {("mixed", "N2048_n512_steps1024_h1", "k_ozaki"): 85.35e6,
                 # mean of the update's two launches, profiles/k_tc_gemm_N2048.md: two CTAs
                 # per SM (54.6 and 89.9 MB) and one (54.1 and 101.2 MB)
                 ("mixed", "N2048_n512_steps1024_h1", "k_tc_gemm<128,3,3,32,2>"): 72.27e6,
                 ("mixed", "N2048_n512_steps1024_h1", "k_tc_gemm<128,3,3,32>"): 77.65e6,
                 # 59.05 + 1.78 MB, profiles/k_col_rhs_N2048.md (per-pass twiddle rows)
                 ("mixed", "N2048_n512_steps1024_h1", "k_col_rhs"): 60.84e6}

# slice pairs (p, q) with p + q <= 6 of the 7 x 7 integer digits: 28 bf16 GEMMs
OZAKI_PAIRS = 28
# slice pairs with p + q <= 2 of the 3 x 3 bf16 slices of the inverse update's products
NS_PAIRS = 6
# FP32 pipe of GB300: 128 FP32 lanes per SM, 152 SMs, FMA = 2 flop, 2070 MHz
FP32_PEAK_TFLOPS = 128 * 2 * 152 * 2.07e9 / 1e12
# k_col_rhs, double-float Stockham radix-8 FFTs: about 120 FP32 flop per point and
# radix-8 pass, log8(N) passes, 5.5 transforms of N points per column
DF_FLOP_PER_POINT_PASS = 120
COLRHS_FFTS = 5.5
# k_assemble_sym: about 80 FP64 flop per unordered pair (i, j) for both A and G
ASM_FLOP_PER_PAIR = 80


def _entry(kernel, bound, flops, dur, peak, unit, src, w, form, **extra):
    achieved = flops / dur / 1e12
    e = {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
         "frac": achieved / peak, "traffic": TRAFFIC_BYTES.get((form, w.name, kernel)),
         "launch_ms": dur * 1e3, "peak_source": src}
    e.update(extra)
    return e


def tc_gemm_name(sched):
    """The inverse update's kernel under a schedule: its column tile, and a
    fifth template argument 2 when two CTAs share an SM."""
    return f"k_tc_gemm<{sched['inv_bn']},3,3,32{',2' if sched.get('inv_ctas', 1) == 2 else ''}>"


def rooflines(form, timing, w, pk, sched=None):
    """Per-kernel rooflines of the profiled Jacobian, from the phase events that
    bracket single kernels on the stream each runs on: gkernel (the column
    G-apply product), inverse (the two products of the inverse update),
    assembly (k_assemble_sym), colrhs (k_col_rhs).  Returns (dominant, list):
    the dominant kernel is the one with the largest share of the stage."""
    N, nc = w.N, w.n + 1
    out = []

    def dur(phase, per_phase=1):
        ms, cnt = timing.get(phase, (0.0, 0))
        return (ms / cnt / per_phase / 1e3, cnt) if cnt else (None, 0)

    g_fp64 = 2.0 * N * N * nc                 # the FP64 product G Gamma the G-apply delivers
    fp64_src = "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"
    if form == "fp64":
        d, _ = dur("gkernel")
        if d:
            out.append(_entry("k_dgemm", "alu", g_fp64, d, FP64_PEAK_TFLOPS, "TFLOP/s", fp64_src, w, form,
                              role="column G-apply", work=f"2 N^2 (n+1) FP64 flop, N={N}, n+1={nc}",
                              share_ms_per_stage=d * 1e3))
    else:
        peak = pk.get("bf16_tflops_sustained") or 1700.0
        src = "of measured (bf16_tflops_sustained)" if pk.get("bf16_tflops_sustained") else "of fallback (sustained)"
        d, _ = dur("gkernel")
        if d:
            out.append(_entry("k_ozaki", "tensor", OZAKI_PAIRS * g_fp64, d, peak, "TFLOP/s", src, w, form,
                              role="column G-apply (7+7 digits)",
                              work=f"{OZAKI_PAIRS} bf16 digit-pair GEMMs of {N} x {nc} x {N}",
                              method_fp64_tflops=g_fp64 / d / 1e12, share_ms_per_stage=d * 1e3))
        d, n_upd = dur("inverse", 2)
        if d:
            ns = NS_PAIRS * 2.0 * N ** 3
            # the phase events time the updates of the even stages (which always move the
            # inverse); odd-stage updates run through the device-side decision untimed
            stages = timing.get("assembly", (0.0, 0))[1] or n_upd
            out.append(_entry(tc_gemm_name(sched or {"inv_bn": 128}), "tensor", ns, d, peak, "TFLOP/s", src, w, form,
                              role="inverse update X <- X (2I - A X), one of its two products",
                              work=f"{NS_PAIRS} bf16 slice-pair GEMMs of {N}^3",
                              method_fp32_tflops=2.0 * N ** 3 / d / 1e12, updates_per_stage=n_upd / stages,
                              share_ms_per_stage=2 * d * 1e3 * n_upd / stages))
    d, _ = dur("assembly")
    if d:
        out.append(_entry("k_assemble_sym", "alu", ASM_FLOP_PER_PAIR * N * N / 2.0, d, FP64_PEAK_TFLOPS, "TFLOP/s",
                          fp64_src, w, form, role="A = 1/2 I + K and G",
                          work=f"~{ASM_FLOP_PER_PAIR} FP64 flop per unordered pair, N^2/2 pairs",
                          share_ms_per_stage=d * 1e3))
    d, _ = dur("colrhs")
    if d:
        if form == "fp64":
            work = COLRHS_FFTS * 5.0 * N * math.log2(N) * nc
            out.append(_entry("k_col_rhs", "alu", work, d, FP64_PEAK_TFLOPS, "TFLOP/s", fp64_src, w, form,
                              role="variational RHS + RK update", work=f"{COLRHS_FFTS} FP64 FFTs (5 N log2 N) per column",
                              share_ms_per_stage=d * 1e3))
        else:
            work = DF_FLOP_PER_POINT_PASS * N * (math.log2(N) / 3.0) * COLRHS_FFTS * nc
            out.append(_entry("k_col_rhs", "alu", work, d, FP32_PEAK_TFLOPS, "TFLOP/s",
                              "derived: 128 FP32 lanes x 2 flop/clk/SM x 152 SMs x 2070 MHz", w, form,
                              role="variational RHS + RK update (double-float FFTs)",
                              work=f"{COLRHS_FFTS} double-float FFTs per column, ~{DF_FLOP_PER_POINT_PASS} FP32 "
                                   f"flop per point and radix-8 pass", share_ms_per_stage=d * 1e3))
    if not out:
        return None, []
    dom = max(out, key=lambda e: e["share_ms_per_stage"])
    return dom, out


def error_vs_oracle(w, r, J, f):
    """Errors of one Jacobian against the oracle's stored samples of the same
    workload (tests/golden/full_n2048_samples.json, written from the oracle
    alone): |df|/|f|, ||dr||/||r|| and per sampled column ||dJ_k|| /
    max(||J_k||, 1e-4 max_j ||J_j||) over every 16th row.  Each is also given
    as a ratio to the oracle's own one-ulp spread (how far the oracle moves
    when c_1 moves by one ulp), the parity test's tolerance unit."""
    path = os.path.join(ROOT, "tests", "golden", "full_n2048_samples.json")
    if w.name != W.LARGE.name or not os.path.exists(path):
        return None
    with open(path) as fh:
        g = json.load(fh)
    rows = np.asarray(g["rows"])
    big = max(v["norm"] for v in g["columns"].values())
    ej = {}
    for k, v in g["columns"].items():
        ref = np.asarray(v["values"])
        den = max(np.linalg.norm(ref), 1e-4 * big * math.sqrt(len(rows) / g["N"]))
        ej[k] = float(np.linalg.norm(J[0 if k == "T" else int(k), rows] - ref) / den)
    worst = max(ej, key=ej.get)
    out = {"f_rel": abs(f - g["f"]) / abs(g["f"]),
           "r_rel": float(np.linalg.norm(r[rows] - np.asarray(g["r"])) / np.linalg.norm(g["r"])),
           "J_max_col_rel": ej[worst], "J_worst_col": worst, "J_median_col_rel": float(np.median(list(ej.values()))),
           "columns_compared": len(ej), "rows_compared": len(rows),
           "reference": "oracle samples (tests/golden/full_n2048_samples.json)"}
    sp = g.get("spread")
    if sp:
        out["J_max_ratio_to_oracle_ulp_spread"] = max(ej[k] / sp["columns"][k] for k in ej)
        out["oracle_ulp_spread_f"] = sp["f"]
    return out


def _jacobian_rate(ww, ctx, ct, outs, stream, flush, k, warm):
    """Warm-up calls, then k device-timed calls (L2 flushed between them, outside
    the events): (seconds per call, kernel launches of the timed calls)."""
    r, J, f = outs
    import torch
    for _ in range(warm):
        ww.shoot_jacobian(ctx, ct, r, J, f)
    torch.cuda.synchronize()
    times, launches = [], 0
    for _ in range(k):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ww.shoot_jacobian(ctx, ct, r, J, f)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        launches += ctx.stats()["launches"]   # the library counts the kernel nodes it replays
    return times, launches


def run_fp64_form(ww, w, c, dev, flush):
    """The plain FP64 form on the same workload, for the metric's comparison: one
    timed Jacobian (device-resident inputs, L2 flushed before it).  Its warm-up
    is one call of a one-step context of the same sizes (loads the kernels and
    sizes the allocator); the timed call includes the capture of its own step
    graph, a few milliseconds against minutes."""
    import torch
    cw = c.copy()
    cw[0] = c[0] / w.steps
    with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=1, precision=ww.WW_FP64) as warm:
        r, J, f = warm.empty_outputs()
        ww.shoot_jacobian(warm, torch.tensor(cw, dtype=torch.float64, device=dev), r, J, f)
    torch.cuda.synchronize()
    ctx = ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=ww.WW_FP64)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream)
    outs = ctx.empty_outputs()
    ct = torch.tensor(c, dtype=torch.float64, device=dev)
    times, launches = _jacobian_rate(ww, ctx, ct, outs, stream, flush, 1, 0)
    res = (outs[0].cpu().numpy(), outs[1].cpu().numpy(), float(outs[2].item()))
    ctx.close()
    return times[0], launches, res


def run_ours(args):
    import torch
    import paper_1210_5672_gb300 as ww

    rank, ws, local = dist_init()
    w = W.ALL[args.workload]
    form = args.form
    c, seed_used = W.coefficients(w, seed=w.seed + rank)
    if args.rk_steps:
        # profiling: fewer RK4 steps at the full run's dt (T scaled), not a bench number
        c[0] *= args.rk_steps / w.steps
        w = W.shrink(w, steps=args.rk_steps, name=f"{w.name}[profile: {args.rk_steps} RK steps at full dt]")
    prec = ww.WW_MIXED if form == "mixed" else ww.WW_FP64
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=prec)
    ct = torch.tensor(c, dtype=torch.float64, device=dev)
    outs = ctx.empty_outputs()
    r, J, f = outs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream)
    # ---- timed region: K Jacobians, phase events off, L2 flushed between them
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times, gpu_launches = _jacobian_rate(ww, ctx, ct, outs, stream, flush, args.steps, args.warmup)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.summary()
    t_step, value = replica_rate(sum(times) / len(times), ws, w.n + 1)
    res = (r.cpu().numpy(), J.cpu().numpy(), float(f.item()))
    # ---- end to end through the host-buffer entry point (pinned host memory)
    ch = torch.tensor(c, dtype=torch.float64).pin_memory().numpy()
    rh = torch.empty(w.N, dtype=torch.float64).pin_memory().numpy()
    Jh = torch.empty((w.n + 1, w.N), dtype=torch.float64).pin_memory().numpy()
    fh = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
    e2e_t = []
    for _ in range(max(1, min(args.steps, 2))):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ww.shoot_jacobian_host(ctx, ch, rh, Jh, fh)
        e2e_t.append(time.perf_counter() - t0)
    _, e2e_value = replica_rate(sum(e2e_t) / len(e2e_t), ws, w.n + 1)
    # ---- profiled Jacobian: phase events on (per-kernel durations on the streams
    # the kernels run on) and, in the mixed form, the refinement residual
    # measured after the last correction of every 256th solve
    sched = ctx.schedule()
    ctx.set_timing(True)
    if form == "mixed":
        ctx.set_verify(256)
    _jacobian_rate(ww, ctx, ct, outs, stream, flush, 1, 0)
    timing = ctx.timing()
    stats = ctx.stats()
    ctx.set_timing(False)
    ctx.close()
    dom, roofs = rooflines(form, timing, w, peaks(), sched)
    errors = {form: error_vs_oracle(w, *res)} if ws == 1 else {}
    fp64 = None
    if form == "mixed" and ws == 1 and not args.no_fp64_form and not args.rk_steps:
        t64, l64, res64 = run_fp64_form(ww, w, c, dev, flush)
        fp64 = {"value": (w.n + 1) / t64, "unit": "Jacobian columns/s", "ms_per_step": t64 * 1e3,
                "steps": 1, "gpu_launches": l64,
                "timing": "one device-timed Jacobian (CUDA events), L2 flushed before it",
                "mixed_over_fp64": value / ((w.n + 1) / t64)}
        errors["fp64"] = error_vs_oracle(w, *res64)
        norms = np.linalg.norm(res64[1], axis=1)
        col = np.linalg.norm(res[1] - res64[1], axis=1) / np.maximum(norms, 1e-4 * norms.max())
        errors["mixed_vs_fp64"] = {"J_max_col_rel": float(col.max()), "J_worst_col": int(col.argmax()),
                                   "J_median_col_rel": float(np.median(col)),
                                   "f_rel": abs(res[2] - res64[2]) / abs(res64[2]),
                                   "columns_compared": int(len(col)), "rows_compared": int(w.N)}
    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if form == "fp64" else "f64+f32/bf16-tensor",
        "data": "synthetic (seeded PCG64 standing-wave coefficients)",
        "config": {"workload": w.name, "N": w.N, "n": w.n, "columns": w.n + 1, "rk4_steps": w.steps,
                   "h": w.h, "g": w.g, "tau": w.tau, "form": form, "seed": seed_used,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": {"value": e2e_value, "unit": "Jacobian columns/s",
                "h2d_bytes_per_step": 8 * (w.n + 1), "d2h_bytes_per_step": 8 * (w.N + w.N * (w.n + 1) + 1)},
        "roofline": dom,
        "rooflines": roofs,
        "roofline_timing": "phase events around each kernel in one more Jacobian of the same workload "
                           "(value itself is timed with phase events off)",
        "phases_ms_per_step": {p: v[0] for p, v in timing.items()},
        "stats": stats,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if fp64 is not None:
        out["fp64_form"] = fp64
    if errors:
        out["error_vs_oracle"] = errors
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(w, c)
    return out


GRAD_METRIC = "gradients/s of f(c) by the discrete adjoint at N=1024 (256 modes + T, 2048 RK4 steps)"


def run_gradient(args):
    """--mode gradient: one step = one objective_and_grad (forward shot, then
    the transposed RK4 sweep) on a gradient workload (default: N = 1024, 256
    modes + T, 2048 steps, deep water, tau = 0.1; the shallow one reaches the
    bottom before T/4 and runs with --rk-steps 512), with the base trajectory checkpointed
    every --checkpoint steps (default 45 ~ sqrt(2048); 0 keeps every stage's
    record resident).  The other memory mode and the forward Jacobian route
    (shoot_jacobian, then J^T r) on the same problem are timed once beside it,
    with their device memory and agreement."""
    import torch
    import paper_1210_5672_gb300 as ww

    rank, ws, local = dist_init()
    w = W.ALL[args.workload]
    c, seed_used = W.coefficients(w, seed=w.seed + rank)
    if args.rk_steps:
        # profiling: fewer RK4 steps at the full run's dt (T scaled), not a bench number
        c[0] *= args.rk_steps / w.steps
        w = W.shrink(w, steps=args.rk_steps, name=f"{w.name}[profile: {args.rk_steps} RK steps at full dt]")
    prec = ww.WW_MIXED if args.form == "mixed" else ww.WW_FP64
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=prec)
    ct = torch.tensor(c, dtype=torch.float64, device=dev)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(w.n + 1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream)
    ckpt = min(args.checkpoint, w.steps)
    ctx.set_checkpoint(ckpt)
    for _ in range(args.warmup):
        ww.objective_and_grad(ctx, ct, f, grad)
    torch.cuda.synchronize()
    times, gpu_launches = [], 0
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ww.objective_and_grad(ctx, ct, f, grad)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            gpu_launches += ctx.stats()["launches"]
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.summary()
    t_step, value = replica_rate(sum(times) / len(times), ws, 1)
    stats = ctx.stats()
    # end to end: c from pinned host memory in, f and grad back to pinned host memory
    ch = torch.tensor(c, dtype=torch.float64).pin_memory()
    fh = torch.empty(1, dtype=torch.float64).pin_memory()
    gh = torch.empty(w.n + 1, dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(max(1, min(args.steps, 2))):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ct.copy_(ch, non_blocking=True)
            ww.objective_and_grad(ctx, ct, f, grad)
            fh.copy_(f, non_blocking=True)
            gh.copy_(grad, non_blocking=True)
        stream.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    _, e2e_value = replica_rate(sum(e2e_t) / len(e2e_t), ws, 1)
    # the other memory mode, once (after one untimed call that sizes its workspace)
    g_main = grad.cpu().numpy()
    other = 0 if ckpt else max(1, round(math.sqrt(w.steps)))
    ctx.set_checkpoint(other)
    ww.objective_and_grad(ctx, ct, f, grad)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ww.objective_and_grad(ctx, ct, f, grad)
    e1.record(stream)
    e1.synchronize()
    st_other = ctx.stats()
    g_other = grad.cpu().numpy()
    other_mode = {"checkpoint_every": other, "seconds": e0.elapsed_time(e1) / 1e3,
                  "adjoint_bytes": st_other["adjoint_bytes"], "device_bytes": st_other["device_bytes"],
                  "rel_diff_grad": float(np.linalg.norm(g_other - g_main) / np.linalg.norm(g_main))}
    ctx.set_checkpoint(ckpt)
    # the forward route for comparison: n + 1 variational columns, then J^T r
    r, J, fj = ctx.empty_outputs()
    ww.shoot_jacobian(ctx, ct, r, J, fj)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ww.shoot_jacobian(ctx, ct, r, J, fj)
    e1.record(stream)
    e1.synchronize()
    t_jac = e0.elapsed_time(e1) / 1e3
    jtr = (J @ r).cpu().numpy()
    g_adj = g_main
    agree = float(np.linalg.norm(g_adj - jtr) / np.linalg.norm(jtr))
    ctx.close()
    if rank != 0:
        return None
    out = {
        "metric": GRAD_METRIC, "value": value, "unit": "gradients/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f64+f32/bf16-tensor",
        "data": "synthetic (seeded PCG64 standing-wave coefficients)",
        "config": {"workload": w.name, "N": w.N, "n": w.n, "rk4_steps": w.steps, "h": w.h, "g": w.g,
                   "tau": w.tau, "form": args.form, "seed": seed_used, "mode": "gradient",
                   "checkpoint_every": ckpt,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": {"value": e2e_value, "unit": "gradients/s", "h2d_bytes_per_step": 8 * (w.n + 1),
                "d2h_bytes_per_step": 8 * (w.n + 2)},
        "roofline": None,
        "forward_route": {"shoot_jacobian_s": t_jac, "adjoint_s": t_step,
                          "speedup": t_jac / t_step, "rel_diff_grad_vs_JTr": agree},
        "memory": {"checkpoint_every": ckpt, "adjoint_bytes": stats["adjoint_bytes"],
                   "device_bytes": stats["device_bytes"]},
        "other_memory_mode": other_mode,
        "stats": stats,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline_gradient(w, c)
    return out


BATCH_METRIC = "Jacobian columns/s over a batch of 32 uneven shots (N 256..4096, 8..64 columns each)"


def run_batch(args):
    """--mode batch: one step = shoot_jacobian_batch (ONE graph launch) over the
    32 seeded shots of the uneven batch, each shot's step count capped at
    --batch-step-cap at its own dt, after the autotuner picked each shot's
    schedule.  Beside it, timed once each: the per-shot loop of the same tuned
    contexts (bitwise the batch's results) and the plain FP64 per-shot loop,
    whose Jacobians the batch is compared with column by column."""
    import torch
    import paper_1210_5672_gb300 as ww

    rank, ws, local = dist_init()
    shots = W.uneven_shots(n_shots=32, seed=rank, step_cap=args.batch_step_cap or None)
    prec = ww.WW_MIXED if args.form == "mixed" else ww.WW_FP64
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctxs = [ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=prec) for w, _ in shots]
    cs = [torch.tensor(c, dtype=torch.float64, device=dev) for _, c in shots]
    outs = [ctx.empty_outputs() for ctx in ctxs]
    cols = sum(w.n + 1 for w, _ in shots)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    # the autotuner: each shot's schedule from timed probes (or the cache file)
    cache = args.tune_cache or os.path.join(tempfile.mkdtemp(prefix="ww_tune_"), "schedules.txt")
    t0 = time.perf_counter()
    tuned = []
    for (w, _), ctx, c in zip(shots, ctxs, cs):
        ms = ctx.autotune(c, probe_steps=3, cache_path=cache)
        tuned.append({"shot": w.name, "schedule": ctx.schedule(), "probe_ms_per_step": ms})
    t_tune = time.perf_counter() - t0

    def batch():
        ww.shoot_jacobian_batch(ctxs, cs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])

    for _ in range(args.warmup):
        batch()
    torch.cuda.synchronize()
    times = []
    barrier(ws)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch()                      # returns when every shot is done (device synchronised)
            times.append(time.perf_counter() - t0)
    barrier(ws)
    clocks = clk.summary()
    t_step, value = replica_rate(sum(times) / len(times), ws, cols)
    launches = sum(ctx.stats()["launches"] for ctx in ctxs) * args.steps
    got = [(o[0].cpu(), o[1].cpu(), o[2].cpu()) for o in outs]
    # the per-shot loop on the same (tuned) contexts
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx, c, o in zip(ctxs, cs, outs):
        ww.shoot_jacobian(ctx, c, o[0], o[1], o[2])
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    same = all(torch.equal(a[0], o[0].cpu()) and torch.equal(a[1], o[1].cpu()) and torch.equal(a[2], o[2].cpu())
               for a, o in zip(got, outs))
    for ctx in ctxs:
        ctx.close()
    # the plain FP64 per-shot loop (one context per shot, first call captures its graph)
    fp64 = None
    if prec == ww.WW_MIXED and not args.no_fp64_form:
        worst, t64 = 0.0, 0.0
        for (w, _), c, a in zip(shots, cs, got):
            with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=ww.WW_FP64) as ctx:
                r, J, f = ctx.empty_outputs()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ww.shoot_jacobian(ctx, c, r, J, f)
                torch.cuda.synchronize()
                t64 += time.perf_counter() - t0
                Jd = J.cpu().numpy()
            norms = np.linalg.norm(Jd, axis=1)
            col = np.linalg.norm(a[1].numpy() - Jd, axis=1) / np.maximum(norms, 1e-4 * norms.max())
            worst = max(worst, float(col.max()))
        fp64 = {"seconds": t64, "columns_per_s": cols / t64, "batch_speedup": t64 / t_step,
                "J_max_col_rel_batch_vs_fp64": worst,
                "timing": "host wall clock, one shoot_jacobian per shot in turn (synchronised)"}
    if rank != 0:
        return None
    out = {
        "metric": BATCH_METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f64+f32/bf16-tensor",
        "data": "synthetic (seeded uneven-batch recipe)",
        "config": {"workload": ("uneven batch of 32 shots, steps capped at "
                                f"{args.batch_step_cap} (each shot's own dt)") if args.batch_step_cap else
                               "uneven batch of 32 shots at their full step counts",
                   "shots": [w.name + f"_steps{w.steps}" for w, _ in shots], "columns": cols, "form": args.form,
                   "mode": "batch", "timing": "host wall clock around the batch call (one graph launch; it "
                                              "synchronises)",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": None,
        "roofline": None,
        "autotune": {"seconds": t_tune, "cache": "per (N, n+1, form) text file", "choices": tuned},
        "per_shot_loop": {"seconds": t_loop, "columns_per_s": cols / t_loop, "batch_speedup": t_loop / t_step,
                          "bitwise_equal_to_batch": same},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if fp64 is not None:
        out["fp64_per_shot_loop"] = fp64
    return out


SEG_METRIC = "Jacobian columns/s of the segmented DOP853 shot on adaptive meshes (4 segments, M 512..2048)"


def run_segments(args):
    """--mode segments: one step = shoot_jacobian_segments of the segmented
    workload (four time segments with rho = 1, 0.4, 0.1, 0.1 refined near
    x = 0, M = 512, 1024, 2048, 2048, DOP853 steps 21, 48, 64, 53, 170 modes +
    T), in the chosen form; the same shot in the other form is timed once
    beside it, and the two compared column by column.  The line also carries
    the timed form's own one-ulp sensitivity and the gradient of the same
    shot by the discrete adjoint (time, agreement with J^T r)."""
    import torch
    import paper_1210_5672_gb300 as ww

    rank, ws, local = dist_init()
    wl = W.SEGMENTED
    segs = wl.meta["segments"]
    c, seed_used = W.coefficients(W.Workload("seg", N=segs[0][0], n=wl.n, steps=1, h=wl.h, amp=wl.amp,
                                             seed=wl.seed + rank))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ct = torch.tensor(c, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)

    def build(prec):
        ctxs = []
        for (M, steps, theta, rho, centre) in segs:
            ctx = ww.Context(M, wl.n, g=wl.g, tau=wl.tau, h=wl.h, steps=steps, precision=prec)
            ww.set_segment(ctx, steps, theta, rho, centre, wl.meta["tableau"])
            ctxs.append(ctx)
        stream = torch.cuda.Stream(dev)
        ctxs[0].set_stream(stream)
        M = segs[-1][0]
        out = (torch.empty(M, dtype=torch.float64, device=dev), torch.empty(wl.n + 1, M, dtype=torch.float64, device=dev),
               torch.empty(1, dtype=torch.float64, device=dev))
        return ctxs, stream, out

    def timed(ctxs, stream, out, k, warm):
        for _ in range(warm):
            ww.shoot_jacobian_segments(ctxs, ct, *out)
        torch.cuda.synchronize()
        ts, launches = [], 0
        for _ in range(k):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ww.shoot_jacobian_segments(ctxs, ct, *out)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
            launches += ctxs[0].stats()["launches"]
        return ts, launches

    prec = ww.WW_MIXED if args.form == "mixed" else ww.WW_FP64
    ctxs, stream, out = build(prec)
    barrier(ws)
    with ClockSampler(local) as clk:
        times, gpu_launches = timed(ctxs, stream, out, args.steps, args.warmup)
    barrier(ws)
    clocks = clk.summary()
    t_step, value = replica_rate(sum(times) / len(times), ws, wl.n + 1)
    J1 = out[1].cpu().numpy()
    jtr = J1 @ out[0].cpu().numpy()

    # the gradient of the same segmented shot by its discrete adjoint, in the timed form
    fg = torch.empty(1, dtype=torch.float64, device=dev)
    gg = torch.empty(wl.n + 1, dtype=torch.float64, device=dev)
    ww.objective_and_grad_segments(ctxs, ct, fg, gg)
    torch.cuda.synchronize()
    gts = []
    for _ in range(2):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ww.objective_and_grad_segments(ctxs, ct, fg, gg)
        e1.record(stream)
        e1.synchronize()
        gts.append(e0.elapsed_time(e1) / 1e3)
    gvec = gg.cpu().numpy()
    gradient = {"seconds": sum(gts) / len(gts), "gradients_per_s": len(gts) / sum(gts),
                "rel_diff_vs_JT_r": float(np.linalg.norm(gvec - jtr) / np.linalg.norm(jtr)),
                "adjoint_bytes": int(sum(x.stats()["adjoint_bytes"] for x in ctxs)),
                "device_bytes": int(sum(x.stats()["device_bytes"] for x in ctxs)),
                "what": "objective_and_grad_segments (discrete adjoint) in the timed form; J^T r from its Jacobian"}

    def col_rel(A, B):
        norms = np.linalg.norm(B, axis=1)
        return np.linalg.norm(A - B, axis=1) / np.maximum(norms, 1e-4 * norms.max())

    # the timed form's own rounding sensitivity: the same shot with c_1 one ulp up
    cp = c.copy()
    cp[1] = np.nextafter(c[1], np.inf)
    ww.shoot_jacobian_segments(ctxs, torch.tensor(cp, dtype=torch.float64, device=dev), *out)
    torch.cuda.synchronize()
    spread = col_rel(out[1].cpu().numpy(), J1)
    for x in ctxs:
        x.close()
    other = None
    if ws == 1:
        oprec = ww.WW_FP64 if prec == ww.WW_MIXED else ww.WW_MIXED
        octx, ostream, oout = build(oprec)
        ot, _ = timed(octx, ostream, oout, 1, 1)
        J2 = oout[1].cpu().numpy()
        for x in octx:
            x.close()
        col = col_rel(J1, J2)
        other = {"form": "fp64" if oprec == ww.WW_FP64 else "mixed", "seconds": ot[0],
                 "columns_per_s": (wl.n + 1) / ot[0], "J_max_col_rel_between_forms": float(col.max()),
                 "worst_column": int(col.argmax())}
    sens = {"J_max_col_rel": float(spread.max()), "J_median_col_rel": float(np.median(spread)),
            "worst_column": int(spread.argmax()),
            "what": "the timed form's J moved by one ulp of c_1 (its own rounding sensitivity)"}
    if rank != 0:
        return None
    stages = sum(st for (_, st, _, _, _) in segs) * 12
    return {
        "metric": SEG_METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f64+f32/bf16-tensor",
        "data": "synthetic (seeded PCG64 standing-wave coefficients, the segmented workload)",
        "config": {"workload": wl.name, "segments": [list(x) for x in segs], "tableau": wl.meta["tableau"],
                   "columns": wl.n + 1, "dtn_stages": stages, "h": wl.h, "form": args.form, "seed": seed_used,
                   "mode": "segments", "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": None,
        "roofline": None,
        "other_form": other,
        "one_ulp_sensitivity": sens,
        "gradient": gradient,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }


def cpu_baseline_gradient(w, c):
    """The oracle's discrete adjoint on one RK4 step of the workload (the full
    run's dt), scaled to the full step count."""
    import oracle as O
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=1)
    cs = c.copy()
    cs[0] = c[0] / w.steps
    t0 = time.perf_counter()
    O.objective_and_grad(prob, cs)
    t1 = time.perf_counter() - t0
    return {"value": 1.0 / (t1 * w.steps), "unit": "gradients/s", "cores": O.threads(), "kind": "oracle",
            "sample": f"1 RK4 step (forward + adjoint) of the {w.name} workload, {t1:.2f} s, "
                      f"scaled x{w.steps} steps",
            "extrapolated": True, "measured_rk4_steps": 1, "full_rk4_steps": w.steps}


def cpu_baseline(w, c, target_s=20.0):
    """The oracle (untuned) on this host's cores, on a bounded sample of the same
    workload: all columns, as many RK4 steps as fit in ~target_s; scaled to
    columns/s of the full 1024-step Jacobian."""
    import oracle as O
    threads = O.threads()
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=1)
    cs = c.copy()
    cs[0] = c[0] / w.steps    # one step of the full run's dt
    t0 = time.perf_counter()
    O.shoot_jacobian(prob, cs)
    t1 = time.perf_counter() - t0
    k = max(1, min(int(target_s / max(t1, 1e-3)), 8))
    if k > 1:
        prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=k)
        cs[0] = c[0] * k / w.steps
        t0 = time.perf_counter()
        O.shoot_jacobian(prob, cs)
        t1 = (time.perf_counter() - t0) / k
    per_jac = t1 * w.steps
    return {"value": (w.n + 1) / per_jac, "unit": "Jacobian columns/s", "cores": threads, "kind": "oracle",
            "sample": f"{k} RK4 step(s) of the {w.name} workload (all {w.n + 1} columns), "
                      f"{t1:.2f} s per step, scaled x{w.steps} steps",
            "extrapolated": True, "measured_rk4_steps": k, "full_rk4_steps": w.steps}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    w = W.ALL[args.workload]
    c, _ = W.coefficients(w)
    import oracle as O
    O.build()
    times = []
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=1)
    cs = c.copy()
    cs[0] = c[0] / w.steps
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.shoot_jacobian(prob, cs)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_jac = statistics.mean(times) * w.steps
    value = (w.n + 1) / per_jac
    cpu = {"value": value, "unit": "Jacobian columns/s", "cores": O.threads(), "kind": "oracle",
           "sample": f"1 RK4 step of {w.name} per timed step (all {w.n + 1} columns), scaled x{w.steps}",
           "extrapolated": True, "measured_rk4_steps": 1, "full_rk4_steps": w.steps}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_jac * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "extrapolated": True,
            "timing": f"each timed step runs 1 of the {w.steps} RK4 steps (all {w.n + 1} columns); "
                      f"ms_per_step and value are scaled to the full {w.steps}-step Jacobian",
            "config": {"workload": w.name, "N": w.N, "n": w.n, "columns": w.n + 1, "rk4_steps": w.steps,
                       "h": w.h, "g": w.g, "tau": w.tau, "form": "cpu-oracle", "seed": 0,
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "Jacobian columns/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default=None, choices=sorted(W.ALL),
                    help=f"default {W.LARGE.name} (jacobian mode), {W.DEEP_TENSION.name} (gradient mode)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="jacobian mode, mixed form: leave out the timed plain-FP64 Jacobian of the comparison")
    ap.add_argument("--batch-step-cap", type=int, default=32,
                    help="batch mode: RK4 steps per shot at most (T scaled, each shot's dt kept); 0: no cap")
    ap.add_argument("--tune-cache", default=None,
                    help="batch mode: the autotuner's cache file (default: a fresh temporary file)")
    ap.add_argument("--mode", default="jacobian", choices=["jacobian", "gradient", "batch", "segments"],
                    help="gradient: objective_and_grad by the discrete adjoint (default workload "
                         "N1024_n256_steps2048_deep_tau0.1); batch: the uneven batch; segments: the "
                         "segmented DOP853 workload")
    ap.add_argument("--checkpoint", type=int, default=45,
                    help="gradient mode: checkpoint the base state every K steps (0: every stage's record resident)")
    ap.add_argument("--rk-steps", type=int, default=0,
                    help="profiling only: override the workload's RK4 step count (not a bench number)")
    args = ap.parse_args()
    if args.workload is None:
        args.workload = W.DEEP_TENSION.name if args.mode == "gradient" else W.LARGE.name
    if args.impl == "reference":
        out = run_reference(args)
    else:
        from paper_1210_5672_gb300 import build as B
        B.build()
        out = {"gradient": run_gradient, "batch": run_batch, "segments": run_segments}.get(args.mode, run_ours)(args)
    if out is not None:
        # numpy scalars and arrays (should any reach the line) print as plain numbers / lists
        print(json.dumps(out, default=lambda v: v.tolist() if hasattr(v, "tolist") else str(v)), flush=True)


if __name__ == "__main__":
    main()
