"""The rounding floor of the FP64 oracle on a workload: the same C computed in
double and in long double (x87 extended on x86-64, binary128 on aarch64), on
the same discrete map, compared on the metrics the parity tests use.  Two
correct FP64 programs that differ only in rounding cannot be expected to agree
better than about twice this floor.

    python -m oracle.roundoff_floor N64_n12_steps64_h1 [--shot-only] [--threads T]

Prints one JSON line: the workload, the relative error of r and f, and the
largest per-column Jacobian error |dJ_k| / max(|J_k|, 1e-4 max_j |J_j|).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1210_5672_gb300 import workloads as W  # noqa: E402


def col_rel(J, J0):
    norms = np.linalg.norm(J0, axis=0)
    floor = 1e-4 * norms.max()
    return max(float(np.linalg.norm(J[:, k] - J0[:, k]) / max(norms[k], floor)) for k in range(J0.shape[1]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--shot-only", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args(argv)
    if not O.wide_available():
        print(json.dumps({"workload": a.workload, "unavailable": "long double is double on this platform"}))
        return
    if a.threads:
        O.set_threads(a.threads)
    w = W.ALL[a.workload]
    c, seed = W.coefficients(w)
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    wp, _ = O.wide_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    out = {"workload": w.name, "seed": seed, "long_double_eps": float(np.finfo(np.longdouble).eps),
           "threads": O.threads()}
    t = time.time()
    if a.shot_only:
        r, f = O.shoot(prob, c)
        rw, fw = O.wide_shoot(wp, c)
    else:
        r, J, f = O.shoot_jacobian(prob, c)
        rw, Jw, fw = O.wide_shoot_jacobian(wp, c)
        Jw = Jw.astype(np.float64)
        out["J_col_rel"] = col_rel(J, Jw)
        out["J_abs_max"] = float(np.max(np.abs(J - Jw)))
    rw64 = rw.astype(np.float64)
    out["r_rel"] = float(np.linalg.norm(r - rw64) / np.linalg.norm(rw64))
    out["f_rel"] = float(abs(f - fw) / fw)
    out["seconds"] = round(time.time() - t, 1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
