"""The FP64 oracle's own rounding error, no GPU: the same C compiled with long
double (x87 extended on x86-64, binary128 on aarch64) computes the same
discrete map with at least 11 more bits, so the difference is the double
build's rounding error.  This is the floor under every GPU-vs-oracle
comparison: two correct FP64 programs that round differently cannot agree
better than about twice it.

* the long double build is what it claims: on a flat surface the DtN is
  k tanh(kh) on each mode to 1e-17, where the double build stops near 1e-14;
* on the N = 64, 12-mode, 64-step workload the floor is far below the 1e-11
  parity tolerance, on the parity tests' own metrics.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300 import workloads as W

pytestmark = pytest.mark.skipif(not O.wide_available(), reason="long double is double here")


def test_wide_build_is_wider():
    pi = np.longdouble("3.14159265358979323846264338327950288")
    N = 64
    x = 2 * pi * np.arange(N, dtype=np.longdouble) / N           # the wide build's own grid
    for k in (1, 3, 7):
        kk = np.longdouble(k)
        phi = np.cos(kk * x)
        G = O.wide_dtn(np.ones(N, dtype=np.longdouble), phi, 1.0)
        assert float(np.max(np.abs(G - kk * np.tanh(kk) * phi))) < 1e-16
        xd = 2 * np.pi * np.arange(N) / N
        Gd = O.dtn(np.ones(N), np.cos(k * xd), 1.0)
        assert np.max(np.abs(Gd - k * math.tanh(k) * np.cos(k * xd))) > 1e-16


def col_rel(J, J0):
    norms = np.linalg.norm(J0, axis=0)
    floor = 1e-4 * norms.max()
    return max(np.linalg.norm(J[:, k] - J0[:, k]) / max(norms[k], floor) for k in range(J0.shape[1]))


def test_rounding_floor_of_the_small_workload():
    w = W.SMALL
    c, _ = W.coefficients(w)
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    wp, _ = O.wide_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    r, J, f = O.shoot_jacobian(prob, c)
    rw, Jw, fw = O.wide_shoot_jacobian(wp, c)
    rw, Jw, fw = rw.astype(np.float64), Jw.astype(np.float64), float(fw)
    assert np.linalg.norm(r - rw) / np.linalg.norm(rw) < 1e-13
    assert abs(f - fw) / fw < 1e-13
    assert col_rel(J, Jw) < 2e-12
    # and the double build does round: the floor is not zero
    assert np.max(np.abs(J - Jw)) > 0.0
