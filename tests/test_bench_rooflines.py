"""bench.py's per-kernel rooflines from phase timings (host arithmetic, no GPU):
achieved = algorithmic work / mean launch time, frac = achieved / peak, the
inverse update's launches split per timed stage, the kernel names of the
schedule's variants, and the dominant kernel chosen by its share of the stage."""
import importlib.util
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_names_follow_the_schedule(bench):
    assert bench.tc_gemm_name({"inv_bn": 128, "inv_ctas": 2}) == "k_tc_gemm<128,3,3,32,2>"
    assert bench.tc_gemm_name({"inv_bn": 256, "inv_ctas": 1}) == "k_tc_gemm<256,3,3,32>"
    assert bench.tc_gemm_name({"inv_bn": 64}) == "k_tc_gemm<64,3,3,32>"


def test_mixed_rooflines_from_phase_totals(bench):
    w = bench.W.LARGE                     # N = 2048, 513 columns
    stages = 4 * w.steps
    pk = {"bf16_tflops_sustained": 1700.0}
    # phase totals (ms, records): the G-apply kernel 0.1 ms a stage; the inverse
    # update timed on half the stages, two launches of 0.09 ms each; assembly
    # 0.25 ms and the column right-hand sides 0.2 ms every stage
    timing = {"gkernel": (0.1 * stages, stages), "inverse": (0.18 * stages / 2, stages // 2),
              "assembly": (0.25 * stages, stages), "colrhs": (0.2 * stages, stages)}
    dom, roofs = bench.rooflines("mixed", timing, w, pk, {"inv_bn": 128, "inv_ctas": 2})
    by = {r["kernel"]: r for r in roofs}
    N, nc = w.N, w.n + 1
    oz = by["k_ozaki"]
    assert math.isclose(oz["launch_ms"], 0.1)
    assert math.isclose(oz["achieved"], 28 * 2.0 * N * N * nc / 1e-4 / 1e12)
    assert math.isclose(oz["frac"], oz["achieved"] / 1700.0)
    tc = by["k_tc_gemm<128,3,3,32,2>"]
    assert math.isclose(tc["launch_ms"], 0.09)                      # per launch
    assert math.isclose(tc["achieved"], 6 * 2.0 * N ** 3 / 0.09e-3 / 1e12)
    assert math.isclose(tc["updates_per_stage"], 0.5)
    assert math.isclose(tc["share_ms_per_stage"], 0.09)             # two launches on half the stages
    asm = by["k_assemble_sym"]
    assert math.isclose(asm["achieved"], bench.ASM_FLOP_PER_PAIR * N * N / 2 / 0.25e-3 / 1e12)
    assert math.isclose(asm["peak"], bench.FP64_PEAK_TFLOPS)
    assert by["k_col_rhs"]["peak"] == bench.FP32_PEAK_TFLOPS
    assert dom["kernel"] == "k_assemble_sym"                         # the largest share of the stage
    for r in roofs:
        assert r["unit"] == "TFLOP/s" and r["bound"] in ("tensor", "alu")


def test_fp64_rooflines(bench):
    w = bench.W.LARGE
    stages = 4 * w.steps
    timing = {"gkernel": (4.0 * stages, stages), "assembly": (0.25 * stages, stages)}
    dom, roofs = bench.rooflines("fp64", timing, w, {}, None)
    by = {r["kernel"]: r for r in roofs}
    assert set(by) == {"k_dgemm", "k_assemble_sym"}
    assert math.isclose(by["k_dgemm"]["achieved"], 2.0 * w.N * w.N * (w.n + 1) / 4e-3 / 1e12)
    assert dom["kernel"] == "k_dgemm"
