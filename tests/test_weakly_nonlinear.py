"""Weakly nonlinear standing waves against the classical expansions the paper
compares with, no GPU.  The oracle's shooting map and Jacobian drive the
host Levenberg-Marquardt solver (App. D) to time-periodic solutions of the
k = 1 family at two small amplitudes; the frequency shift between them gives
the second-order coefficient, which is fixed by perturbation theory:

* Tadjbakhsh and Keller, Eq. (omega:correction) of Sec. 4.2: with
  omega_0^2 = tanh h and g = k = 1,
      omega = omega_0 + eps^2 omega_2 / 2 + O(eps^3),
      omega_2 = (9 omega_0^-7 - 12 omega_0^-3 - 3 omega_0 - 2 omega_0^5) / 32,
  eps agreeing with the linear eta amplitude A of Eq. (lin:soln) to first
  order (A = omega_0 B, B the linear phi amplitude); deep water gives
  omega_2 = -1/4, Rayleigh's omega = 1 - eps^2 / 8;
* Concus, Eq. (concus) of Sec. 4.6: deep water, g = 1, sigma/rho = 1 (so
  delta = 1/2), T = sqrt(2) pi (1 + 197/320 c_1^2) with c_1 = phi^_1(0).

These test the nonlinear terms of the oracle's right-hand side (finite-depth
image kernels, the quadratic terms of Eq. ww, the surface-tension curvature
term) at second order, which the linear pins do not reach.

T(c_1) is even in c_1 (c_1 -> -c_1 is the shift x -> x + pi), so the
expansion has no odd terms and the difference quotient between amplitudes a
and 2a carries a relative error O(a^2); the discrete scheme's own error in
the linear period cancels in the difference.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as O
from paper_1210_5672_gb300.levmar import LMOptions, levmar


def tk_omega2(h):
    """Eq. (omega:correction): omega_2 with omega_0^2 = tanh h (g = k = 1)."""
    w0 = 1.0 if math.isinf(h) else math.sqrt(math.tanh(h))
    return (9 * w0 ** -7 - 12 * w0 ** -3 - 3 * w0 - 2 * w0 ** 5) / 32


def standing_wave_period(c1, h, tau, N=32, n=12, steps=96):
    """Period of the k = 1 standing wave with phi^_1(0) = c_1 held fixed:
    Eq. (init:stand) (c_k on phi^_{+-k} for odd k, on eta^_{+-k} for even k,
    i.e. 2 c_k cos kx), the other c_k and T solved for by App. D's solver."""
    x = 2 * np.pi * np.arange(N) / N
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        basis[(N if k % 2 else 0):(2 * N if k % 2 else N), k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, g=1.0, tau=tau, h=h, steps=steps, basis=basis)
    w0 = math.sqrt((1.0 + tau) * (1.0 if math.isinf(h) else math.tanh(h)))
    c0 = np.zeros(n + 1)
    c0[0] = 2 * math.pi / w0
    c0[1] = c1
    free = np.array([0] + list(range(2, n + 1)))

    def full(z):
        c = c0.copy()
        c[free] = z
        return c

    out = levmar(lambda z: O.shoot(prob, full(z))[0],
                 lambda z: (lambda rJ: (rJ[0], rJ[1][:, free]))(O.shoot_jacobian(prob, full(z))),
                 c0[free], 0.01 * c0[0], LMOptions())
    assert out.f < 1e-28, (c1, h, tau, out.f, out.reason)
    del keep
    return full(out.c)[0], w0


def test_tadjbakhsh_keller_formula_changes_sign_where_printed():
    """Sec. 4.2 prints the depth where omega_2 changes sign: h = 1.0581
    (positive below, so the period first falls with amplitude at h = 1, as
    the unit-depth family of Fig. bif10 does)."""
    root = brentq(tk_omega2, 0.5, 2.0, xtol=1e-12)
    assert abs(root - 1.0581) < 5e-5
    assert tk_omega2(1.0) > 0 > tk_omega2(1.07)
    assert tk_omega2(math.inf) == -0.25


@pytest.mark.parametrize("h", [0.5, 2.0, math.inf])
def test_tadjbakhsh_keller_frequency_correction(h):
    a = 0.005                                     # phi^_1(0): B = 2 c_1 = 0.01 and 0.02
    T1, w0 = standing_wave_period(a, h, 0.0)
    T2, _ = standing_wave_period(2 * a, h, 0.0)
    e1, e2 = w0 * 2 * a, w0 * 4 * a             # eps = A = omega_0 B to first order
    omega2 = 2 * (2 * math.pi / T2 - 2 * math.pi / T1) / (e2 ** 2 - e1 ** 2)
    assert abs(omega2 / tk_omega2(h) - 1.0) < 2e-3, (h, omega2, tk_omega2(h))


def test_concus_gravity_capillary_period():
    """Deep water, g = 1, sigma/rho = 1: T_lin = 2 pi / sqrt 2 and the
    quadratic coefficient 197/320 in c_1 = phi^_1(0)."""
    T0 = math.sqrt(2.0) * math.pi
    T1, w0 = standing_wave_period(0.02, math.inf, 1.0)
    T2, _ = standing_wave_period(0.04, math.inf, 1.0)
    assert abs(2 * math.pi / w0 - T0) < 1e-14
    coef = (T2 - T1) / T0 / (0.04 ** 2 - 0.02 ** 2)
    assert abs(coef / (197 / 320) - 1.0) < 1e-3, coef
    assert T1 > T0 and T2 > T1                   # the period increases with amplitude
