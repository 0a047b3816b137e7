"""Write medium_n512_samples.json: the oracle's shooting Jacobian on the N = 512
workload (128 modes + T, 512 RK4 steps, h = 1, c_1 = 0.2, c_k = 0.2^k u_k,
seed 0), every 16th row of r and of every column, for the full-run parity test
of that size.

Only the oracle computes here.  The double oracle gives the reference values;
its long double build (x87 extended on x86-64, binary128 on aarch64) runs the
same Jacobian, and the per-column distance between the two is stored as the
double oracle's own rounding floor: two correct FP64 evaluations that round
differently cannot agree better than about twice it.  About 20 minutes on 8
x86-64 cores, almost all of it in long double.

    python tests/golden/make_medium_samples.py
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

ROW_STRIDE = 16


def main():
    O.build()
    w = W.MEDIUM
    c, seed = W.coefficients(w)
    rows = list(range(0, w.N, ROW_STRIDE))
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    t0 = time.time()
    r, J, f = O.shoot_jacobian(prob, c)
    t_double = time.time() - t0
    out = {
        "what": "oracle shoot_jacobian on the N512_n128_steps512_h1 workload, every 16th row",
        "workload": w.name, "seed": seed, "N": w.N, "n": w.n, "steps": w.steps, "T": c[0], "f": f,
        "rows": rows, "r": [float(r[i]) for i in rows],
        "column_norms": [float(v) for v in np.linalg.norm(J, axis=0)],
        "J": [[float(J[i, k]) for i in rows] for k in range(w.n + 1)],
        "oracle_threads": O.threads(), "oracle_seconds": round(t_double, 1),
    }
    if O.wide_available():
        wp, _ = O.wide_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
        t0 = time.time()
        rw, Jw, fw = O.wide_shoot_jacobian(wp, c)
        rw, Jw, fw = rw.astype(np.float64), Jw.astype(np.float64), float(fw)
        out["floor"] = {
            "what": "distance of the double oracle from its long double build (same discrete map)",
            "long_double_eps": float(np.finfo(np.longdouble).eps),
            "f": abs(f - fw) / abs(fw),
            "r": float(np.linalg.norm(r - rw) / np.linalg.norm(rw)),
            "columns_abs": [float(v) for v in np.linalg.norm(J - Jw, axis=0)],
            "seconds": round(time.time() - t0, 1),
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "medium_n512_samples.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
        fh.write("\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
