"""The seeded input recipe (paper_1210_5672_gb300/workloads.py), no GPU:
initial periods against the values the paper prints, the geometry redraw rule,
and the uneven-batch recipe's ranges and step rule."""
import math

import numpy as np

from paper_1210_5672_gb300 import workloads as W


def test_linear_periods_match_the_paper():
    # Sec. 4: T = 2 pi / sqrt(tanh h) = 7.19976 at h = 1; 28.1110 at h = 0.05;
    # deep water with sigma/rho = 1: 2 pi / sqrt(2) = 4.443
    assert abs(W.linear_period(1.0, 0.0, 1.0) - 7.19976) < 1e-5
    assert abs(W.linear_period(1.0, 0.0, 0.05) - 28.1110) < 1e-4
    assert abs(W.linear_period(1.0, 1.0, math.inf) - 4.443) < 1e-3
    for w in (W.LARGE, W.SHALLOW, W.DEEP_TENSION):
        c, _ = W.coefficients(w)
        assert c[0] == W.linear_period(w.g, w.tau, w.h)


def test_redraw_keeps_the_surface_above_half_depth():
    for w in (W.SMALL, W.MEDIUM, W.LARGE, W.SHALLOW):
        c, seed = W.coefficients(w)
        x = W.grid(w.N)
        surf = w.h + np.cos(np.outer(x, np.arange(1, w.n + 1))) @ c[1:]
        assert surf.min() >= 0.5 * w.h
        assert seed >= w.seed
    # the draw is reproducible
    a, sa = W.coefficients(W.LARGE)
    b, sb = W.coefficients(W.LARGE)
    assert sa == sb and np.array_equal(a, b)


def test_uneven_batch_recipe():
    shots = W.uneven_shots()
    assert len(shots) == 32
    for w, c in shots:
        assert w.N in (256, 512, 1024, 2048, 4096)
        assert 8 <= w.n + 1 <= 64
        assert 0.1 <= w.h <= 2.0 and w.tau in (0.0, 0.05)
        assert 0.01 <= c[1] <= 0.5 and c[1] < 0.45 * w.h
        assert w.steps == W.stable_steps(w.N, w.g, w.tau, w.h, c[0]) >= w.N // 2
    capped = W.uneven_shots(step_cap=64)
    for (w, c), (wc, cc) in zip(shots, capped):
        assert wc.steps == min(w.steps, 64)
        # the cap keeps each shot's dt
        assert abs(cc[0] / (4 * wc.steps) - c[0] / (4 * w.steps)) <= 1e-15 * c[0]


def test_segmented_recipe():
    """The segmented workload (shaped like the paper's solution O, Table
    param:OA): theta sums to 1, the first segment is uniform on N points, the
    grids are powers of two, the spacing rule of Sec. 2.2 holds, and the
    steps add up.  The printed table itself breaks the rule between its second
    and third segments (6912 / 6144 = 1.125 < 6.2 / 5.3), which the rule check
    detects."""
    w = W.SEGMENTED
    segs = w.meta["segments"]
    assert abs(sum(s[2] for s in segs) - 1.0) < 1e-12
    assert segs[0][0] == w.N and segs[0][3] == 1.0
    assert all(s[0] & (s[0] - 1) == 0 for s in segs)
    assert sum(s[1] for s in segs) == w.steps
    assert W.spacing_rule_ok(segs)
    printed = ((4608, 192, 0.2, 1.0), (6144, 432, 0.3, 0.4), (6912, 576, 0.3, 0.1), (8192, 480, 0.2, 0.09))
    assert not W.spacing_rule_ok(printed)
    assert W.spacing_rule_ok(printed[:2]) and not W.spacing_rule_ok(printed[1:3]) and W.spacing_rule_ok(printed[2:])
    assert w.name not in W.ALL


def test_stored_oracle_samples_match_the_workload_recipe():
    """The golden files of the full-length parity tests were written by the
    oracle for exactly the workloads the recipe builds today (sizes, steps,
    the seed actually used, T): a stale file would hold a test to the wrong
    problem."""
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for name, w in (("medium_n512_samples.json", W.MEDIUM), ("full_n2048_samples.json", W.LARGE)):
        with open(os.path.join(here, name)) as fh:
            g = json.load(fh)
        c, seed = W.coefficients(w)
        assert (g["N"], g["n"], g["steps"], g["seed"], g["workload"]) == (w.N, w.n, w.steps, seed, w.name), name
        assert g["T"] == c[0], name
        assert g["rows"] == list(range(0, w.N, 16)), name
