"""Parity of full-length shots, in the launch configuration bench.py times (one
context, the captured step graph replayed `steps` times), on outputs stored from
the oracle's run of the same problem.

* N = 512, 128 modes + T, all 512 RK4 steps (tests/golden/medium_n512_samples.json,
  tests/golden/make_medium_samples.py): f, and r and EVERY column of J at every
  16th point.  Each output is held to max(1e-11, 4 x its measured rounding
  floor): the distance of the double oracle from its own long double build,
  stored per column with the samples (two correct FP64 evaluations of the same
  discrete map that round differently agree to about twice that).
* N = 2048, 512 modes + T, all 1024 RK4 steps (tests/golden/full_n2048_samples.json,
  tests/golden/make_full_size_samples.py): f, r at every 16th point, and the T
  column, the first three modes and every 16th mode of J at the same points.
  A long double run of the oracle at this size takes hours, so each output is
  held to max(1e-11, 4 x its one-ulp spread): how far the oracle's own output
  moves when c_1 moves by one ulp, i.e. when only the rounding pattern changes.

Both forms (plain FP64 and mixed) run every case, and the mixed form is also
compared with the FP64 form on every entry of J at full size.  With the
measurement of ww_set_verify on, the mixed form's true refinement residual,
recomputed after the last correction of sampled solves, must be <= 1e-13.

Error measures: |df|/|f|; ||dr|| / ||r|| over the sampled points; per column
||dJ_k|| / max(||J_k||, 1e-4 max_j ||J_j||) over the sampled points (the
column floor of the other parity tests).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1210_5672_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN_FULL = os.path.join(HERE, "golden", "full_n2048_samples.json")
GOLDEN_MEDIUM = os.path.join(HERE, "golden", "medium_n512_samples.json")
TOL = 1e-11
RESID_TOL = 1e-13
VERIFY_EVERY = 64          # stages between measured residuals (64 of the 4096 at N = 2048)

_runs = {}


def _golden(path):
    if not os.path.exists(path):
        pytest.skip(f"{os.path.basename(path)} not generated")
    with open(path) as fh:
        return json.load(fh)


def _run(precision, w):
    """One shoot_jacobian of workload w (cached per form and workload)."""
    key = (precision, w.name)
    if key not in _runs:
        import torch
        from paper_1210_5672_gb300 import build as B
        B.build()
        import paper_1210_5672_gb300 as ww
        c, _ = W.coefficients(w)
        with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=precision) as ctx:
            if precision == ww.WW_MIXED:
                ctx.set_verify(VERIFY_EVERY)
            r, J, f = ctx.empty_outputs()
            ww.shoot_jacobian(ctx, torch.tensor(c, dtype=torch.float64, device="cuda"), r, J, f)
            st = ctx.stats()
            _runs[key] = (r.cpu().numpy(), J.cpu().numpy(), float(f.item()), st)
    return _runs[key]


def _col_err(ref_rows, got_rows, big_rows):
    den = max(np.linalg.norm(ref_rows), 1e-4 * big_rows)
    return float(np.linalg.norm(got_rows - ref_rows) / den)


def _check_resid(precision, st):
    import paper_1210_5672_gb300 as ww
    if precision == ww.WW_MIXED:
        assert st["verified_solves"] > 0
        assert 0 <= st["refine_resid_measured"] <= RESID_TOL, st


# ------------------------------------------------------------ N = 512, every column
def _check_medium(precision):
    g = _golden(GOLDEN_MEDIUM)
    if "floor" not in g:
        pytest.skip("medium_n512_samples.json has no long double floor")
    w = W.MEDIUM
    r, J, f, st = _run(precision, w)
    rows = np.asarray(g["rows"])
    Jg = np.asarray(g["J"])                       # (n + 1, rows)
    norms = np.asarray(g["column_norms"])         # full-column norms of the oracle's J
    floor_abs = np.asarray(g["floor"]["columns_abs"])
    floor_rel = floor_abs / np.maximum(norms, 1e-4 * norms.max())
    big = np.linalg.norm(Jg, axis=1).max()
    ej = np.array([_col_err(Jg[k], J[k, rows], big) for k in range(w.n + 1)])
    tol = np.maximum(TOL, 4.0 * floor_rel)
    ef = abs(f - g["f"]) / abs(g["f"])
    er = np.linalg.norm(r[rows] - np.asarray(g["r"])) / np.linalg.norm(g["r"])
    ratio = ej / np.maximum(floor_rel, 1e-300)
    print(f"\nN=512 full run precision={precision}: |df|/|f| {ef:.2e}  r {er:.2e}  J worst column "
          f"{ej.max():.2e} (column {int(ej.argmax())}, tolerance {tol[ej.argmax()]:.2e}), median {np.median(ej):.2e}; "
          f"error / floor: median {np.median(ratio):.2f}, worst {ratio.max():.2f} (column {int(ratio.argmax())}); "
          f"stats {st}")
    assert ef < max(TOL, 4 * g["floor"]["f"])
    assert er < max(TOL, 4 * g["floor"]["r"])
    bad = np.nonzero(ej >= tol)[0]
    assert bad.size == 0, [(int(k), float(ej[k]), float(tol[k])) for k in bad]
    _check_resid(precision, st)


def test_medium_full_run_fp64_every_column_within_rounding_floor():
    import paper_1210_5672_gb300 as ww
    _check_medium(ww.WW_FP64)


def test_medium_full_run_mixed_every_column_within_rounding_floor():
    import paper_1210_5672_gb300 as ww
    _check_medium(ww.WW_MIXED)


# ------------------------------------------------------------ N = 2048, sampled columns
def _errors_full(g, r, J, f):
    rows = np.asarray(g["rows"])
    ef = abs(f - g["f"]) / abs(g["f"])
    r0 = np.asarray(g["r"])
    er = np.linalg.norm(r[rows] - r0) / np.linalg.norm(r0)
    cols = g["columns"]
    big = max(v["norm"] for v in cols.values())
    ej = {}
    for k, v in cols.items():
        j = 0 if k == "T" else int(k)
        ref = np.asarray(v["values"])
        den = max(np.linalg.norm(ref), 1e-4 * big * math.sqrt(len(rows) / g["N"]))
        ej[k] = float(np.linalg.norm(J[j, rows] - ref) / den)
    return ef, er, ej


def _tol_full(g, key, col=None):
    sp = g.get("spread")
    if sp is None:
        pytest.skip("the oracle's one-ulp spread is not in the samples file (make_full_size_samples.py --spread)")
    s = sp["columns"][col] if col is not None else sp[key]
    return max(TOL, 4.0 * s)


def _check_full(precision):
    g = _golden(GOLDEN_FULL)
    r, J, f, st = _run(precision, W.LARGE)
    ef, er, ej = _errors_full(g, r, J, f)
    worst = max(ej, key=lambda k: ej[k] / _tol_full(g, None, k))
    print(f"\nfull N=2048 precision={precision}: |df|/|f| {ef:.2e}  r {er:.2e}  {len(ej)} sampled columns, "
          f"worst J[{worst}] {ej[worst]:.2e} (tolerance {_tol_full(g, None, worst):.2e}), "
          f"median {np.median(list(ej.values())):.2e}  stats {st}")
    assert ef < _tol_full(g, "f")
    assert er < _tol_full(g, "r")
    for k, e in ej.items():
        assert e < _tol_full(g, None, k), (k, e)
    _check_resid(precision, st)


def test_full_size_mixed_matches_oracle_samples():
    import paper_1210_5672_gb300 as ww
    _check_full(ww.WW_MIXED)


def test_full_size_fp64_matches_oracle_samples():
    import paper_1210_5672_gb300 as ww
    _check_full(ww.WW_FP64)


def test_full_size_mixed_matches_fp64_form():
    """Every entry of J: the mixed form against the plain FP64 GPU form."""
    import paper_1210_5672_gb300 as ww
    rm, Jm, fm, _ = _run(ww.WW_MIXED, W.LARGE)
    rd, Jd, fd, _ = _run(ww.WW_FP64, W.LARGE)
    norms = np.linalg.norm(Jd, axis=1)
    floor = 1e-4 * norms.max()
    col = np.linalg.norm(Jm - Jd, axis=1) / np.maximum(norms, floor)
    print(f"\nfull N=2048 mixed vs FP64: |df|/|f| {abs(fm - fd) / abs(fd):.2e}  "
          f"r {np.linalg.norm(rm - rd) / np.linalg.norm(rd):.2e}  J max column {col.max():.2e} "
          f"(column {int(col.argmax())}), median {np.median(col):.2e}")
    g = _golden(GOLDEN_FULL)
    worst = max(g["spread"]["columns"].values()) if "spread" in g else TOL
    assert col.max() < max(TOL, 4.0 * worst)
