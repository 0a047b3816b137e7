"""Benchmark: Jacobian columns per second of the standing-wave shooting map.

One step = one full shoot_jacobian (all RK4 stages of all columns, setup and
outputs included) on the seeded N = 2048 workload (512 Fourier unknowns + T,
1024 RK4 steps, h = 1, c_1 = 0.4, c_k = 0.4^k u_k).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form mixed|fp64]
                  [--impl ours|reference] [--workload NAME]

--form mixed (default) is the tensor-core form (FP32-accurate inverse, FP64-
accurate Ozaki products, iterative refinement to a 1e-13 residual); --form
fp64 is the plain FP64 form it is compared with (~2 minutes per Jacobian at
N = 2048: run it with --warmup 3 --steps 1).

--impl reference times the CPU FP64 oracle (the only baseline: the paper's
code is not available) on a bounded sample of the same workload.  Under
torchrun every rank runs an independent replica (its own seed; the path has
no exchange step), the slowest rank's time is reported and value counts the
columns of all ranks.
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


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the timed product
# kernel, from the ncu captures summarised under profiles/ (None: not captured
# since the kernel last changed).
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# roofline kernel, from one ncu capture of the current k_ozaki's column G-apply
# launch on the N = 2048 workload; other workloads and forms have no capture of
# their current kernel: null.
TRAFFIC_BYTES = {("mixed", "N2048_n512_steps1024_h1"): 85.35e6}

# slice pairs (p, q) with p + q <= 6 of the 7 x 7 integer digits: 28 bf16 GEMMs
OZAKI_PAIRS = 28


def roofline_for(form, timing, w, pk):
    """Roofline of the dominant kernel, from the GKERNEL phase: the events around
    the one product kernel of each stage's column G-apply (k_ozaki in the mixed
    form, k_dgemm in the FP64 form; the same kernels carry the solves and the
    FP64 factorisation), so duration = GKERNEL ms / launches."""
    N, nc = w.N, w.n + 1
    ms, cnt = timing["gkernel"]
    if cnt == 0:
        return None
    dur = ms / cnt / 1e3
    fp64_flops = 2.0 * N * N * nc          # the FP64 product G Gamma it delivers
    if form == "fp64":
        achieved = fp64_flops / dur / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES.get(("fp64", w.name)), "kernel": "k_dgemm",
                "launch_ms": dur * 1e3,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"}
    peak = pk.get("bf16_tflops_sustained") or 1700.0
    src = "of measured (bf16_tflops_sustained)" if pk.get("bf16_tflops_sustained") else "of fallback (sustained)"
    achieved = OZAKI_PAIRS * fp64_flops / dur / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC_BYTES.get(("mixed", w.name)), "kernel": "k_ozaki",
            "launch_ms": dur * 1e3, "fp64_equivalent_tflops": fp64_flops / dur / 1e12,
            "work": f"{OZAKI_PAIRS} bf16 digit-pair GEMMs of {N} x {nc} x {N}",
            "peak_source": src}


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
    r, J, f = ctx.empty_outputs()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream)
    ctx.set_timing(True)     # the same step program (with its event nodes) in warm-up and timed steps
    for _ in range(args.warmup):
        ww.shoot_jacobian(ctx, ct, r, J, f)
    torch.cuda.synchronize()
    # ---- timed region: K Jacobians, L2 flushed between them (outside the events)
    times, phase, gpu_launches = [], {p: [0.0, 0] for p in ww.PHASES}, 0
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ww.shoot_jacobian(ctx, ct, r, J, f)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            # our kernels in this call: the library counts the kernel nodes it replays
            gpu_launches += ctx.stats()["launches"]
            for p, (ms, cnt) in ctx.timing().items():
                phase[p][0] += ms
                phase[p][1] += cnt
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.summary()
    ctx.set_timing(False)
    t_step, value = replica_rate(sum(times) / len(times), ws, w.n + 1)
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
    timing = {p: tuple(v) for p, v in phase.items()}
    roof = roofline_for(form, timing, w, peaks())
    stats = ctx.stats()
    ctx.close()
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
        "roofline": roof,
        "phases_ms_per_step": {p: v[0] / args.steps for p, v in timing.items()},
        "stats": stats,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(w, c)
    return out


GRAD_METRIC = "gradients/s of f(c) by the discrete adjoint at N=1024 (256 modes + T, 2048 RK4 steps)"


def run_gradient(args):
    """--mode gradient: one step = one objective_and_grad (forward shot that
    records every stage, then the transposed RK4 sweep) on a gradient workload
    (default: N = 1024, 256 modes + T, 2048 steps, h = 0.05).  The forward
    Jacobian route (shoot_jacobian, then J^T r) on the same problem is timed
    once beside it."""
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
    g_adj = grad.cpu().numpy()
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
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": {"value": e2e_value, "unit": "gradients/s", "h2d_bytes_per_step": 8 * (w.n + 1),
                "d2h_bytes_per_step": 8 * (w.n + 2)},
        "roofline": None,
        "forward_route": {"shoot_jacobian_s": t_jac, "adjoint_s": t_step,
                          "speedup": t_jac / t_step, "rel_diff_grad_vs_JTr": agree},
        "stats": stats,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline_gradient(w, c)
    return out


BATCH_METRIC = "Jacobian columns/s over a batch of 32 uneven shots (N 256..4096, 8..64 columns each)"


def run_batch(args):
    """--mode batch: one step = shoot_jacobian_batch over the 32 seeded shots of
    the uneven batch (each shot's step count capped at --batch-step-cap at its
    own dt); the per-shot loop (shoot_jacobian on each context in turn) on the
    same shots is timed beside it, and the two must agree bitwise."""
    import torch
    import paper_1210_5672_gb300 as ww

    rank, ws, local = dist_init()
    shots = W.uneven_shots(n_shots=32, seed=rank, step_cap=args.batch_step_cap)
    prec = ww.WW_MIXED if args.form == "mixed" else ww.WW_FP64
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctxs = [ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=prec) for w, _ in shots]
    cs = [torch.tensor(c, dtype=torch.float64, device=dev) for _, c in shots]
    outs = [ctx.empty_outputs() for ctx in ctxs]
    cols = sum(w.n + 1 for w, _ in shots)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)

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
    got = [(o[0].cpu(), o[1].cpu(), o[2].cpu()) for o in outs]
    # the per-shot loop on the same contexts
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx, c, o in zip(ctxs, cs, outs):
        ww.shoot_jacobian(ctx, c, o[0], o[1], o[2])
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    same = all(torch.equal(a[0], o[0].cpu()) and torch.equal(a[1], o[1].cpu()) and torch.equal(a[2], o[2].cpu())
               for a, o in zip(got, outs))
    launches = sum(ctx.stats()["launches"] for ctx in ctxs) * args.steps
    for ctx in ctxs:
        ctx.close()
    if rank != 0:
        return None
    return {
        "metric": BATCH_METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f64+f32/bf16-tensor",
        "data": "synthetic (seeded uneven-batch recipe)",
        "config": {"workload": f"uneven batch of 32 shots, steps capped at {args.batch_step_cap} (each shot's own dt)",
                   "shots": [w.name + f"_steps{w.steps}" for w, _ in shots], "columns": cols, "form": args.form,
                   "mode": "batch", "timing": "host wall clock around the batch call (it synchronises)",
                   "l2": "flushed between timed steps (512 MB write)"},
        "e2e": None,
        "roofline": None,
        "per_shot_loop": {"seconds": t_loop, "columns_per_s": cols / t_loop, "batch_speedup": t_loop / t_step,
                          "bitwise_equal_to_batch": same},
        "gpu_launches": launches,
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
                      f"scaled x{w.steps} steps"}


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
                      f"{t1:.2f} s per step, scaled x{w.steps} steps"}


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
           "sample": f"1 RK4 step of {w.name} per timed step (all {w.n + 1} columns), scaled x{w.steps}"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Jacobian columns/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_jac * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "n": w.n, "form": "cpu-oracle"},
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
                    help=f"default {W.LARGE.name} (jacobian mode), {W.SHALLOW.name} (gradient mode)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-step-cap", type=int, default=64,
                    help="batch mode: RK4 steps per shot at most (T scaled, each shot's dt kept)")
    ap.add_argument("--mode", default="jacobian", choices=["jacobian", "gradient", "batch"],
                    help="gradient: objective_and_grad by the discrete adjoint (default workload "
                         "N1024_n256_steps2048_h0.05)")
    ap.add_argument("--rk-steps", type=int, default=0,
                    help="profiling only: override the workload's RK4 step count (not a bench number)")
    args = ap.parse_args()
    if args.workload is None:
        args.workload = W.SHALLOW.name if args.mode == "gradient" else W.LARGE.name
    if args.impl == "reference":
        out = run_reference(args)
    else:
        from paper_1210_5672_gb300 import build as B
        B.build()
        out = {"gradient": run_gradient, "batch": run_batch}.get(args.mode, run_ours)(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
