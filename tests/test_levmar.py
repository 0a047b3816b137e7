"""Levenberg-Marquardt with delayed Jacobian updates (App. D), host logic, no GPU.

* the trust-region step from the thin SVD against the KKT conditions of the
  constrained quadratic model and against a library least-squares solve;
* convergence on textbook problems (Rosenbrock's residuals: zero residual; an
  exponential fit: nonzero residual, against scipy's least_squares);
* the standing-wave problem of Sec. 3 on the CPU oracle (paper basis: even k on
  eta, odd k on phi; c_1 fixed): the solver reaches the round-off regime, reuses
  its Jacobian (fewer Jacobians than accepted steps), and the period obeys the
  weakly nonlinear law T(eps) = T_lin + O(eps^2) with T_lin = 2 pi / sqrt(g tanh h)
  (Eq. lin:soln): halving eps divides T - T_lin by 4;
* numerical continuation along the unit-depth family (Sec. 4, Fig. bif10: the
  family bifurcates from T = 2 pi / sqrt(tanh 1) ~ 7.200 and its period first
  decreases with amplitude): one Jacobian per solution, a decreasing period, and
  the same solutions as direct solves.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300.levmar import LMOptions, continue_branch, levmar, trust_region_step


def _svd(J):
    U, s, Vt = np.linalg.svd(J, full_matrices=False)
    return U, s, Vt.T


def test_trust_region_step_kkt():
    rng = np.random.default_rng(0)
    J = rng.standard_normal((30, 8))
    r = rng.standard_normal(30)
    U, s, V = _svd(J)
    gn = np.linalg.lstsq(J, -r, rcond=None)[0]
    # inactive constraint: the Gauss-Newton step, lam = 0
    p, lam, df = trust_region_step(U, s, V, r, 2 * np.linalg.norm(gn))
    assert lam == 0.0 and np.allclose(p, gn, rtol=1e-12, atol=1e-14)
    # active constraint: |p| = Delta and (J^T J + lam I) p = -J^T r with lam > 0
    delta = 0.3 * np.linalg.norm(gn)
    p, lam, df = trust_region_step(U, s, V, r, delta)
    assert lam > 0 and abs(np.linalg.norm(p) - delta) <= 1e-11 * delta
    ref = np.linalg.solve(J.T @ J + lam * np.eye(8), -J.T @ r)
    assert np.allclose(p, ref, rtol=1e-10, atol=1e-14)
    # predicted change of the quadratic model
    g, B = J.T @ r, J.T @ J
    assert abs(df - (g @ p + 0.5 * p @ B @ p)) <= 1e-12 * abs(df)


def test_rosenbrock_zero_residual():
    def res(x):
        return np.array([10.0 * (x[1] - x[0] ** 2), 1.0 - x[0]])

    def resj(x):
        return res(x), np.array([[-20.0 * x[0], 10.0], [-1.0, 0.0]])

    out = levmar(res, resj, [-1.2, 1.0], 1.0)
    assert np.allclose(out.c, [1.0, 1.0], atol=1e-12)
    assert out.f < 1e-26


def test_exponential_fit_matches_library():
    scipy_opt = pytest.importorskip("scipy.optimize")
    t = np.linspace(0.0, 3.0, 40)
    rng = np.random.default_rng(2)
    y = 2.5 * np.exp(-1.3 * t) + 0.4 + 0.01 * rng.standard_normal(t.size)

    def res(x):
        return x[0] * np.exp(-x[1] * t) + x[2] - y

    def jac(x):
        e = np.exp(-x[1] * t)
        return np.stack([e, -x[0] * t * e, np.ones_like(t)], axis=1)

    out = levmar(res, lambda x: (res(x), jac(x)), [1.0, 1.0, 0.0], 1.0)
    ref = scipy_opt.least_squares(res, [1.0, 1.0, 0.0], jac=jac, xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert np.allclose(out.c, ref.x, rtol=1e-8, atol=1e-10)
    assert out.f > 1e-4                       # a genuine nonzero-residual minimum


def _problem(N=32, n=12, steps=96, h=1.0):
    x = 2 * np.pi * np.arange(N) / N
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):   # Eq. init:stand: even k on eta, odd k on phi, 2 cos(k x)
        if k % 2 == 0:
            basis[:N, k - 1] = 2 * np.cos(k * x)
        else:
            basis[N:, k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, h=h, steps=steps, basis=basis)
    free = np.array([0] + list(range(2, n + 1)))

    def solve(guess):
        def full(z):
            c = guess.copy()
            c[free] = z
            return c

        out = levmar(lambda z: O.shoot(prob, full(z))[0],
                     lambda z: (lambda rJ: (rJ[0], rJ[1][:, free]))(O.shoot_jacobian(prob, full(z))),
                     guess[free], 0.01 * guess[0], LMOptions())
        out.c = full(out.c)
        return out

    return solve, keep


def test_continuation_along_the_unit_depth_family():
    solve, keep = _problem()
    T_lin = 2 * math.pi / math.sqrt(math.tanh(1.0))
    assert abs(T_lin - 7.200) < 1e-3             # Fig. bif10's bifurcation point
    lin = lambda e: np.concatenate([[T_lin, e], np.zeros(11)])
    a, b = solve(lin(0.01)), solve(lin(0.015))
    values = [0.02, 0.025, 0.03, 0.035, 0.04]
    branch = continue_branch(solve, a.c, b.c, 1, values)
    Ts = [a.c[0], b.c[0]] + [r.c[0] for r in branch]
    assert all(r.f < 1e-24 for r in branch)
    assert sum(r.jacobians == 1 for r in branch) >= 4    # one Jacobian per solution, as a rule
    assert all(t1 > t2 for t1, t2 in zip(Ts, Ts[1:]))    # the period decreases with amplitude
    assert Ts[-1] < T_lin
    direct = solve(lin(values[-1]))
    assert np.max(np.abs(direct.c - branch[-1].c)) < 1e-9 * values[-1]


def _standing_wave(eps, N=32, n=12, steps=96, h=1.0):
    x = 2 * np.pi * np.arange(N) / N
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):   # Eq. init:stand: even k on eta, odd k on phi, 2 cos(k x)
        if k % 2 == 0:
            basis[:N, k - 1] = 2 * np.cos(k * x)
        else:
            basis[N:, k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, h=h, steps=steps, basis=basis)
    T_lin = 2 * math.pi / math.sqrt(math.tanh(h))
    c0 = np.zeros(n + 1)
    c0[0] = T_lin
    c0[1] = eps
    free = np.array([0] + list(range(2, n + 1)))

    def full(z):
        c = c0.copy()
        c[free] = z
        return c

    def res(z):
        return O.shoot(prob, full(z))[0]

    def resj(z):
        r, J, _ = O.shoot_jacobian(prob, full(z))
        return r, J[:, free]

    out = levmar(res, resj, c0[free], 0.1 * T_lin, LMOptions())
    return out, T_lin, keep


def test_standing_wave_period_is_second_order_in_amplitude():
    outs = []
    for eps in (0.02, 0.01):
        out, T_lin, _ = _standing_wave(eps)
        assert out.f < 1e-24, (eps, out.f, out.reason)
        assert out.jacobians < out.accepted    # the Jacobian was reused across steps
        outs.append(out.c[0] - T_lin)
    d1, d2 = outs
    # the unit-depth period first decreases with amplitude (Sec. 4, Fig. bif10)
    assert d1 < -1e-6 and d2 < 0
    assert abs(d1 / d2 - 4.0) < 0.1, (d1, d2)


def test_solver_on_a_segmented_dop853_shot():
    """The paper's own setting (Sec. 2.2): the shot over time segments, the second
    on twice the points with the mesh refined near x = pi, stepped by DOP853
    (16 steps in all), drives the solver to the same standing wave as uniform
    RK4, and its period is the RK4 periods' Richardson extrapolation to dt -> 0
    (RK4 error ~ dt^4, so T_exact = T_128 - (T_64 - T_128) / 15)."""
    N, n = 64, 12
    x = 2 * np.pi * np.arange(N) / N
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):   # Eq. init:stand: even k on eta, odd k on phi, 2 cos(k x)
        basis[(N if k % 2 else 0):(2 * N if k % 2 else N), k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, h=1.0, basis=basis)
    T_lin = 2 * math.pi / math.sqrt(math.tanh(1.0))
    c0 = np.zeros(n + 1)
    c0[0], c0[1] = T_lin, 0.02
    free = np.array([0] + list(range(2, n + 1)))

    def solve(segs, tab):
        def full(z):
            c = c0.copy()
            c[free] = z
            return c

        out = levmar(lambda z: O.shoot_segments(prob, segs, tab, full(z))[0],
                     lambda z: (lambda rJ: (rJ[0], rJ[1][:, free]))(O.shoot_jacobian_segments(prob, segs, tab,
                                                                                                full(z))),
                     c0[free], 0.01 * T_lin, LMOptions())
        assert out.f < 1e-28
        return full(out.c)

    seg = solve([(N, 8, 0.5, 1.0), (2 * N, 8, 0.5, 0.5, 1)], "dop853")
    r64 = solve([(N, 64, 1.0, 1.0)], "rk4")
    r128 = solve([(N, 128, 1.0, 1.0)], "rk4")
    T_exact = r128[0] - (r64[0] - r128[0]) / 15
    assert abs(r128[0] - T_exact) > 1e-9                 # RK4 at 128 steps is still visibly off
    assert abs(seg[0] - T_exact) < 1e-12
    assert np.max(np.abs(seg[2:] - r128[2:])) < 1e-11   # the same initial data
