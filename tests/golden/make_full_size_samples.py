"""Write full_n2048_samples.json: the oracle's shooting map and sampled Jacobian
columns on the N = 2048 workload (512 modes + T, 1024 RK4 steps, h = 1,
c_1 = 0.4, c_k = 0.4^k u_k, seed 0), for the full-size parity test.

Only the oracle computes here.  A Jacobian column d r / d c_k depends on the
other coefficients only through the base trajectory, so the oracle runs a
problem whose basis is [sum_k c_k cos kx, cos k1 x, cos k2 x, ...] with
coefficients [1, 0, 0, ...]: the same initial surface and the same base
trajectory, and variational columns only for the sampled modes (plus T).
That keeps the run to ~38 columns; it is still the full 4096-stage trajectory
with one N = 2048 LU per stage (about 45 minutes on 8 cores).

With --spread the oracle runs once more with c_1 one ulp larger and records,
per output, how far its own result moves (the sensitivity floor of the
problem at this size: two correct FP64 evaluations that differ only in
rounding cannot be expected to agree better than a few times this).

With --wide the oracle's long double build runs the base shot (r and f, no
columns) on the same workload and records how far the double oracle's r and
f are from it: the double oracle's own rounding error at this size.  It is
slow: about 1.6 s per RK4 stage on 8 x86-64 cores in x87 extended precision
(LU and long double cotangents), 6 to 7 hours for the 4096 stages, and far
longer where long double is software binary128.

    python tests/golden/make_full_size_samples.py [--spread | --wide]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1210_5672_gb300 import workloads as W  # noqa: E402

# sampled Jacobian columns (mode numbers; column 0 is T): the first three
# modes, every 16th mode and the two below the last
MODES = sorted({1, 2, 3, 255, 511} | set(range(16, 513, 16)))
ROW_STRIDE = 16                        # sampled rows of r and J


def run(c):
    w = W.LARGE
    x = 2 * np.pi * np.arange(w.N) / w.N
    basis = np.zeros((2 * w.N, 1 + len(MODES)))
    basis[: w.N, 0] = np.cos(np.outer(x, np.arange(1, w.n + 1))) @ c[1:]
    for i, k in enumerate(MODES):
        basis[: w.N, 1 + i] = np.cos(k * x)
    cr = np.zeros(2 + len(MODES))
    cr[0] = c[0]
    cr[1] = 1.0
    prob, keep = O.make_problem(w.N, 1 + len(MODES), g=w.g, tau=w.tau, h=w.h, steps=w.steps, basis=basis)
    r, J, f = O.shoot_jacobian(prob, cr)
    cols = {"T": J[:, 0]}
    for i, k in enumerate(MODES):
        cols[str(k)] = J[:, 2 + i]
    return r, cols, f


def main():
    O.build()
    w = W.LARGE
    c, seed = W.coefficients(w)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_n2048_samples.json")
    rows = list(range(0, w.N, ROW_STRIDE))
    if "--wide" in sys.argv:
        with open(path) as fh:
            out = json.load(fh)
        wp, _ = O.wide_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
        t0 = time.time()
        rw, fw = O.wide_shoot(wp, c)
        rs = rw.astype(np.float64)[rows]
        out["wide"] = {
            "what": "the oracle's long double build, base shot: f, and the double oracle's distance to it",
            "long_double_eps": float(np.finfo(np.longdouble).eps),
            "f": float(fw),
            "f_rel_double_oracle": float(abs(out["f"] - fw) / abs(fw)),
            "r_rel_double_oracle": float(np.linalg.norm(np.asarray(out["r"]) - rs) / np.linalg.norm(rs)),
            "r": [float(v) for v in rs],
            "oracle_threads": O.threads(), "oracle_seconds": round(time.time() - t0, 1),
        }
    elif "--spread" in sys.argv:
        with open(path) as fh:
            out = json.load(fh)
        cp = c.copy()
        cp[1] = np.nextafter(c[1], np.inf)
        t0 = time.time()
        r, cols, f = run(cp)
        out["spread"] = {
            "what": "relative change of each sampled output when c_1 moves by one ulp (oracle, same sampling)",
            "f": abs(f - out["f"]) / abs(out["f"]),
            "r": float(np.linalg.norm(r[rows] - np.asarray(out["r"])) / np.linalg.norm(out["r"])),
            "columns": {k: float(np.linalg.norm(v[rows] - np.asarray(out["columns"][k]["values"]))
                                 / np.linalg.norm(out["columns"][k]["values"])) for k, v in cols.items()},
            "oracle_seconds": round(time.time() - t0, 1),
        }
    else:
        t0 = time.time()
        r, cols, f = run(c)
        elapsed = time.time() - t0
        out = {
            "what": "oracle shoot_jacobian on the N2048_n512_steps1024_h1 workload, sampled",
            "workload": w.name, "seed": seed, "N": w.N, "n": w.n, "steps": w.steps,
            "T": c[0], "f": f, "r_norm": float(np.linalg.norm(r)),
            "rows": rows, "r": [float(r[i]) for i in rows],
            "columns": {k: {"norm": float(np.linalg.norm(v)), "values": [float(v[i]) for i in rows]}
                        for k, v in cols.items()},
            "oracle_threads": O.threads(), "oracle_seconds": round(elapsed, 1),
        }
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
