"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test names the passage it follows.  Together they are chosen
so that a dropped term, a wrong sign, a transposed operand or a wrong RK
coefficient in the oracle fails at least one of them:

* FFT / multipliers   -- textbook DFT, closed forms of d/dx and H on cos/sin.
* flat DtN            -- Eq. (lin): G e^{ikx} = k tanh(kh) e^{ikx} (|k| deep);
                         pins the sign of the image kernels (reading R1).
* analytic-potential  -- G phi = phi_y - eta' phi_x for an exact harmonic
                         function on a NON-flat surface (Eq. DNO:def); pins
                         K1/G1, zeta'(alpha) vs zeta'(beta), diagonal limits.
* high precision      -- the same discrete operator in 40-digit arithmetic at
                         tiny N (independent cot, independent elimination).
* linear dispersion   -- Eq. (lin:soln): phi(T/4) = O(eps^2) at the linear
                         period, amplitude ratio sqrt(tanh h / g); with tension.
* energy              -- Sec. 4 energy monitor conserved; error falls like dt^4.
* time reversal, evenness -- Sec. 2.3.
* linearisation       -- App. B, Eqs. (l5a)/(l6a) against a central directional
                         difference of the discrete RHS.
* Jacobian            -- Eq. (Jik) columns against central differences of the
                         objective, T column included (reading R2).
* adjoint gradient    -- Sec. 3.2 / App. C by the discrete adjoint (reading R18):
                         equals J^T r of the forward variational columns (an
                         independent algorithm) to roundoff, and central
                         differences of f to the linearisation's accuracy;
                         the transposed DtN is the explicit matrix transpose,
                         and the discrete DtN is nearly self-adjoint (App. C,
                         Green's identity), more so as N grows.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300 import workloads as W


def x_grid(N):
    return 2 * np.pi * np.arange(N) / N


# ----------------------------------------------------------------- FFT, multipliers
def test_fft_matches_textbook_dft():
    rng = np.random.default_rng(1)
    for N in (2, 8, 64):
        z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        j = np.arange(N)
        dft = np.exp(-2j * np.pi * np.outer(j, j) / N) @ z
        assert np.max(np.abs(O.fft(z) - dft)) < 1e-12 * N
        assert np.max(np.abs(O.fft(O.fft(z), inverse=True) - z)) < 1e-14 * N


def test_multipliers_closed_forms():
    N = 64
    x = x_grid(N)
    for k in (1, 5, 31):
        assert np.max(np.abs(O.spectral(O.MUL_DERIV, np.sin(k * x)) - k * np.cos(k * x))) < 1e-12
        # H cos = sin, H sin = -cos (symbol -i sgn k)
        assert np.max(np.abs(O.spectral(O.MUL_HILBERT, np.cos(k * x)) - np.sin(k * x))) < 1e-13
        assert np.max(np.abs(O.spectral(O.MUL_HILBERT, np.sin(k * x)) + np.cos(k * x))) < 1e-13
        fac = math.exp(-36.0 * (k / (N / 2)) ** 36)
        assert np.max(np.abs(O.spectral(O.MUL_FILTER, np.cos(k * x)) - fac * np.cos(k * x))) < 5e-14
    # Nyquist: derivative and Hilbert annihilate it, filter multiplies by e^-36
    nyq = np.cos(N / 2 * x)
    assert np.max(np.abs(O.spectral(O.MUL_DERIV, nyq))) < 1e-13
    assert np.max(np.abs(O.spectral(O.MUL_HILBERT, nyq))) < 1e-13
    assert np.max(np.abs(O.spectral(O.MUL_FILTER, nyq) - math.exp(-36) * nyq)) < 1e-16
    # projection removes exactly the mean
    f = 3.0 + np.cos(x)
    assert np.max(np.abs(O.spectral(O.MUL_PROJECT, f) - np.cos(x))) < 1e-14


# ----------------------------------------------------------------- DtN
@pytest.mark.parametrize("h", [1.0, 0.3, 0.05, math.inf])
def test_flat_dtn_symbol(h):
    """Eq. (lin): on the flat surface G e^{ikx} = k tanh(kh) e^{ikx}."""
    # the image kernel of a shallow layer has width ~ h: resolve it with N >> 2 pi / h
    N, tol = (512, 1e-11) if h < 0.1 else (64, 2e-13)
    x = x_grid(N)
    eta = np.full(N, 0.0 if math.isinf(h) else h)
    for k in (1, 2, 5, 13):
        sym = k if math.isinf(h) else k * math.tanh(k * h)
        for f in (np.cos(k * x), np.sin(k * x)):
            assert np.max(np.abs(O.dtn(eta, f, h) - sym * f)) < tol * max(1.0, sym)


def test_flat_dtn_rejects_printed_plus_sign():
    """The symbol is tanh, not coth: |G cos x - coth(h) cos x| must be large."""
    N, h = 64, 1.0
    x = x_grid(N)
    out = O.dtn(np.full(N, h), np.cos(3 * x), h)
    assert abs(out[0] - 3 * math.tanh(3)) < 1e-12
    assert abs(out[0] - 3 / math.tanh(3)) > 1e-2


def _analytic_case(deep, N, k=2):
    x = x_grid(N)
    if deep:
        eta = 0.15 * np.cos(x) + 0.03 * np.cos(2 * x) - 0.02 * np.cos(3 * x)
        z = x + 1j * eta
        Phi, dPhi = np.exp(-1j * k * z), -1j * k * np.exp(-1j * k * z)  # decays as y -> -inf
        h = math.inf
    else:
        eta = 1.0 + 0.15 * np.cos(x) + 0.03 * np.cos(2 * x) - 0.02 * np.cos(3 * x)
        z = x + 1j * eta
        Phi, dPhi = np.cos(k * z), -k * np.sin(k * z)                   # Phi_y = 0 at y = 0
        h = 1.0
    phi = Phi.real
    u, v = dPhi.real, -dPhi.imag                                        # Phi' = u - i v
    eta_x = O.spectral(O.MUL_DERIV, eta)
    return eta, phi, v - eta_x * u, h


@pytest.mark.parametrize("deep", [False, True])
def test_analytic_potential_dtn_converges_spectrally(deep):
    """Eq. (DNO:def): G phi = sqrt(1+eta'^2) dphi/dn = phi_y - eta' phi_x for an
    exact harmonic function with the bottom condition; error falls spectrally."""
    errs = []
    for N in (16, 32, 64):
        eta, phi, exact, h = _analytic_case(deep, N)
        errs.append(np.max(np.abs(O.dtn(eta, phi, h) - exact)))
    assert errs[-1] < 1e-12
    assert errs[0] > 10 * errs[1] > 100 * errs[2] or errs[1] < 1e-12


def _mp_tools(mp, N):
    """40-digit trigonometric-interpolant operators on N points (explicit DFT)."""
    def coeffs(vals):
        return {k: sum(mp.mpf(vals[j]) * mp.expjpi(-2 * mp.mpf(k * j) / N) for j in range(N)) / N
                for k in range(-N // 2 + 1, N // 2 + 1)}

    def apply(vals, mult):
        ck = coeffs(vals)
        return [mp.re(sum(ck[k] * mult(k) * mp.expjpi(2 * mp.mpf(k * i) / N) for k in ck)) for i in range(N)]

    nyq = N // 2
    deriv = lambda v: apply(v, lambda k: 0 if abs(k) == nyq else 1j * k)             # Nyquist dropped
    hilbert = lambda v: apply(v, lambda k: 0 if (k == 0 or abs(k) == nyq) else -1j * mp.sign(k))
    filt = lambda v: apply(v, lambda k: mp.exp(-36 * (mp.mpf(abs(k)) / nyq) ** 36))
    proj = lambda v: apply(v, lambda k: 0 if k == 0 else 1)
    return deriv, hilbert, filt, proj


def _mp_dtn(mp, N, h, e, phi):
    """The discrete DtN of Eq. (K1K2) (images with the minus sign) in mpmath:
    its own cot, its own elimination and an explicit DFT."""
    deriv, hilbert, _, _ = _mp_tools(mp, N)
    # cos/sin rather than mpmath's complex cot, which loses its relative accuracy
    # near its zeros (cot(-pi/2 + 1e-41 i) comes out near 1e-8 i): points pi apart
    # with equal heights put the direct kernel exactly there.
    cot = lambda w: mp.cos(w) / mp.sin(w)
    ex = deriv(e)
    exx = deriv(ex)
    al = [2 * mp.pi * j / N for j in range(N)]
    z = [al[j] + 1j * e[j] for j in range(N)]
    dz = [1 + 1j * ex[j] for j in range(N)]
    ddz = [1j * exx[j] for j in range(N)]
    A = mp.matrix(N, N)
    G = mp.matrix(N, N)
    for i in range(N):
        for j in range(N):
            if i == j:
                k1 = -mp.im(ddz[i] / (2 * dz[i]))
                g1 = mp.re(ddz[i] / (2 * dz[i]))
            else:
                c = cot((z[i] - z[j]) / 2)
                k1 = mp.im(dz[j] / 2 * c)
                g1 = mp.re(dz[i] / 2 * c - cot((al[i] - al[j]) / 2) / 2)
            k2 = g2 = 0
            if not math.isinf(h):
                cb = cot((z[i] - mp.conj(z[j])) / 2)
                k2 = -mp.im(mp.conj(dz[j]) / 2 * cb)
                g2 = -mp.re(dz[i] / 2 * cb)
            A[i, j] = (k1 + k2) / N + (mp.mpf(1) / 2 if i == j else 0)
            G[i, j] = (g1 + g2) / N
    mu = mp.lu_solve(A, mp.matrix(list(phi)))
    gam = deriv([mu[j] for j in range(N)])
    hg = hilbert(gam)
    return [hg[i] / 2 + sum(G[i, j] * gam[j] for j in range(N)) for i in range(N)], ex


def test_dtn_high_precision_tiny_n():
    """Same discrete operator evaluated in 40-digit arithmetic (mpmath: its own
    cot, its own elimination and an explicit DFT) at N = 8 and 16."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for N, h in ((8, 1.0), (16, 1.0), (16, math.inf)):
        x = x_grid(N)
        eta = (0.0 if math.isinf(h) else h) + 0.1 * np.cos(x) - 0.04 * np.cos(2 * x)
        phi = 0.3 * np.cos(x) + 0.1 * np.sin(3 * x)
        got = O.dtn(eta, phi, h)
        ref, _ = _mp_dtn(mp, N, h, [mp.mpf(v) for v in eta], [mp.mpf(v) for v in phi])
        ref = np.array([float(v) for v in ref])
        assert np.max(np.abs(got - ref)) < 5e-15 * max(1.0, np.max(np.abs(ref))), (N, h)


def test_shot_high_precision_tiny_n():
    """A whole shot (Eq. ww with Eq. uv:from:G, the filter and P, classic RK4
    with the step filter; r = phi(T/4)/sqrt(N), f = r.r/2) in 40-digit
    arithmetic at N = 8, against the FP64 oracle: the time loop, the right-hand
    side and the objective, not only the DtN."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    N, h, g, steps = 8, 1.0, 1.0, 4
    deriv, _, filt, proj = _mp_tools(mp, N)
    x = x_grid(N)
    c = np.array([7.2, 0.05, 0.01, -0.004])
    prob, _ = O.make_problem(N, 3, g=g, h=h, steps=steps)
    r64, f64 = O.shoot(prob, c)

    def rhs(e, p):
        gp, ex = _mp_dtn(mp, N, h, e, p)
        pp = deriv(p)
        u = [(pp[i] - ex[i] * gp[i]) / (1 + ex[i] ** 2) for i in range(N)]
        v = [(ex[i] * pp[i] + gp[i]) / (1 + ex[i] ** 2) for i in range(N)]
        pt = [v[i] * gp[i] - u[i] ** 2 / 2 - v[i] ** 2 / 2 - g * e[i] for i in range(N)]
        return filt(gp), filt(proj(pt))

    e = [mp.mpf(h) + sum(mp.mpf(c[k]) * mp.cos(k * 2 * mp.pi * j / N) for k in range(1, 4)) for j in range(N)]
    p = [mp.mpf(0)] * N
    dt = mp.mpf(c[0]) / 4 / steps
    for _ in range(steps):
        k1 = rhs(e, p)
        k2 = rhs([e[i] + dt / 2 * k1[0][i] for i in range(N)], [p[i] + dt / 2 * k1[1][i] for i in range(N)])
        k3 = rhs([e[i] + dt / 2 * k2[0][i] for i in range(N)], [p[i] + dt / 2 * k2[1][i] for i in range(N)])
        k4 = rhs([e[i] + dt * k3[0][i] for i in range(N)], [p[i] + dt * k3[1][i] for i in range(N)])
        e = filt([e[i] + dt / 6 * (k1[0][i] + 2 * k2[0][i] + 2 * k3[0][i] + k4[0][i]) for i in range(N)])
        p = filt([p[i] + dt / 6 * (k1[1][i] + 2 * k2[1][i] + 2 * k3[1][i] + k4[1][i]) for i in range(N)])
    rq = np.array([float(v / mp.sqrt(N)) for v in p])
    fq = float(sum(v * v for v in p) / N / 2)
    assert np.max(np.abs(r64 - rq)) < 1e-14 * np.max(np.abs(rq))
    assert abs(f64 - fq) < 1e-14 * fq


# ----------------------------------------------------------------- evolution pins
def _evolve_linear(h, tau, eps, N=32, steps=128):
    T = W.linear_period(1.0, tau, h)
    x = x_grid(N)
    prob, _ = O.make_problem(N, 0, g=1.0, tau=tau, h=h, steps=steps)
    q0 = np.concatenate([np.full(N, 0.0 if math.isinf(h) else h), eps * np.cos(x)])
    q1 = O.evolve(prob, T, q0)
    return q1, x


@pytest.mark.parametrize("h,tau", [(1.0, 0.0), (0.5, 0.0), (math.inf, 0.1)])
def test_linear_dispersion_quarter_period(h, tau):
    """Eq. (lin:soln): phi0 = eps cos x at T = 2 pi / omega comes to rest at T/4
    up to O(eps^2); eta amplitude / eps -> omega / (g+tau) k ... i.e.
    sqrt(tanh h / g) at tau = 0, 1/sqrt(1.1) for deep water with tau = 0.1."""
    res = []
    for eps in (1e-3, 5e-4):
        q1, x = _evolve_linear(h, tau, eps)
        N = len(x)
        phi_end = q1[N:]
        mean = 0.0 if math.isinf(h) else h
        amp = 2 * np.mean((q1[:N] - mean) * np.cos(x))
        res.append((np.max(np.abs(phi_end)) / eps, amp / eps))
    ratio = math.sqrt(math.tanh(h)) if not math.isinf(h) else 1.0 / math.sqrt(1.0 + tau)
    for rest, a in res:
        assert rest < 5e-3          # comes to rest (relative to eps)
        assert abs(a - ratio) < 5e-3
    # the residual motion is nonlinear: it shrinks with eps
    assert res[1][0] < 0.7 * res[0][0]


def _wave_state(N, h=1.0):
    x = x_grid(N)
    eta = (0.0 if math.isinf(h) else h) + 0.08 * np.cos(x) + 0.02 * np.cos(2 * x)
    phi = 0.05 * np.cos(x) - 0.01 * np.cos(3 * x)
    return np.concatenate([eta, phi])


@pytest.mark.parametrize("h,tau", [(1.0, 0.0), (math.inf, 0.1)])
def test_energy_conserved_fourth_order(h, tau):
    """Energy monitor of Sec. 4: conserved; the drift falls like dt^4 (RK4)."""
    N = 32
    q0 = _wave_state(N, h)
    Tend = 2.0  # integrate over t in [0, 0.5]
    drifts = []
    for steps in (32, 64):
        prob, _ = O.make_problem(N, 0, g=1.0, tau=tau, h=h, steps=steps)
        e0 = O.energy(prob, q0)
        q1 = O.evolve(prob, Tend, q0)
        drifts.append(abs(O.energy(prob, q1) - e0) / abs(e0))
    assert drifts[1] < 1e-10
    assert drifts[0] / drifts[1] > 8  # ~16 for a 4th-order method


def test_time_reversal_and_evenness():
    """Sec. 2.3: (eta, phi) -> (eta, -phi) reverses time; even data stay even."""
    N = 64  # resolved: the filter (irreversible) acts only at roundoff level
    q0 = _wave_state(N)
    errs = []
    for steps in (32, 64):
        prob, _ = O.make_problem(N, 0, h=1.0, steps=steps)
        q1 = O.evolve(prob, 4.0, q0)
        back = O.evolve(prob, 4.0, np.concatenate([q1[:N], -q1[N:]]))
        back = np.concatenate([back[:N], -back[N:]])
        errs.append(np.max(np.abs(back - q0)))
    # RK4 is not symmetric: the round trip returns to truncation level, O(dt^4)
    assert errs[1] < 1e-10 and errs[0] / errs[1] > 8
    # evenness: f(x) = f(-x)  <=>  f[j] = f[N - j]
    for f in (q1[:N], q1[N:]):
        assert np.max(np.abs(f[1:] - f[1:][::-1])) < 1e-14


@pytest.mark.parametrize("h,tau", [(1.0, 0.0), (math.inf, 0.1), (0.6, 0.05)])
def test_variational_rhs_matches_directional_difference(h, tau):
    """App. B, Eqs. (l5a), (l6a): DF(q) qdot equals the central directional
    difference [F(q + e qdot) - F(q - e qdot)] / 2e of the filtered RHS up to
    O(e^2) and the (spectrally small) gap between continuum and discrete
    linearisation of the DtN."""
    N = 64
    x = x_grid(N)
    prob, _ = O.make_problem(N, 0, g=1.0, tau=tau, h=h)
    q = _wave_state(N, h)
    rng = np.random.default_rng(3)
    qd = np.concatenate([
        sum(rng.uniform(-1, 1) * np.cos(k * x + rng.uniform(0, 6)) / k**2 for k in range(1, 8)),
        sum(rng.uniform(-1, 1) * np.cos(k * x + rng.uniform(0, 6)) / k**2 for k in range(1, 8)),
    ])
    T = 7.0
    lin = O.rhs(prob, T, np.stack([q, qd]), 1, 0)[1]
    eps = 1e-5
    fp = O.rhs(prob, T, q + eps * qd, 0)[0]
    fm = O.rhs(prob, T, q - eps * qd, 0)[0]
    fd = (fp - fm) / (2 * eps)
    assert np.max(np.abs(lin - fd)) < 1e-8 * max(1.0, np.max(np.abs(fd)))
    # each half of the pair is exercised (non-trivial)
    assert np.max(np.abs(fd[:N])) > 1e-2 and np.max(np.abs(fd[N:])) > 1e-2


@pytest.mark.slow
def test_jacobian_columns_match_central_differences():
    """Eq. (Jik): J columns (T column by reading R2) against central differences
    of the objective r(c), eps = 1e-6 max(1, |c_k|)."""
    w = W.shrink(W.MEDIUM, N=64, n=6, steps=24)
    c, _ = W.coefficients(w)
    c[1] = 0.1
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    r, J, f = O.shoot_jacobian(prob, c)
    r2, f2 = O.shoot(prob, c)
    assert np.max(np.abs(r - r2)) < 1e-15 and abs(f - 0.5 * r @ r) < 1e-18
    for k in range(w.n + 1):
        e = 1e-6 * max(1.0, abs(c[k]))
        cp, cm = c.copy(), c.copy()
        cp[k] += e
        cm[k] -= e
        fd = (O.shoot(prob, cp)[0] - O.shoot(prob, cm)[0]) / (2 * e)
        scale = max(np.max(np.abs(fd)), 1e-3)
        assert np.max(np.abs(J[:, k] - fd)) < 1e-7 * scale, k


def test_T_column_agrees_with_phi_t_to_order_dt4():
    """Reading R2 against Eq. (Jik): dr/dT of the discrete map and
    (1/4) phi_t(T/4) / sqrt(N) differ by O(dt^4) only."""
    w = W.shrink(W.MEDIUM, N=32, n=2, steps=16)
    c, _ = W.coefficients(w)
    c[1] = 0.1
    gaps = []
    for steps in (16, 32):
        prob, _ = O.make_problem(w.N, w.n, h=w.h, steps=steps)
        r, J, f = O.shoot_jacobian(prob, c)
        qT = O.evolve(prob, c[0], O.initial(prob, c))
        F = O.rhs(prob, c[0], qT, 0)[0]
        phit = 0.25 * F[w.N:] / math.sqrt(w.N)
        gaps.append(np.max(np.abs(J[:, 0] - phit)))
    assert gaps[1] < 1e-7
    assert gaps[0] / gaps[1] > 8


# ----------------------------------------------------------------- adjoint gradient
def _adjoint_case(N, n, steps, h, tau, amp, phi_basis=False):
    w = W.Workload("adj", N=N, n=n, steps=steps, h=h, tau=tau, amp=amp)
    c, _ = W.coefficients(w)
    basis = None
    if phi_basis:
        # the paper's convention (Eq. init:stand): even k on eta, odd k on phi
        x = x_grid(N)
        basis = np.zeros((2 * N, n))
        for k in range(1, n + 1):
            basis[(0 if k % 2 == 0 else N):(N if k % 2 == 0 else 2 * N), k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, g=w.g, tau=tau, h=h, steps=steps, basis=basis)
    return prob, keep, c


@pytest.mark.parametrize("h,tau,phi_basis", [(0.3, 0.05, False), (math.inf, 0.1, False), (1.0, 0.0, True)])
def test_adjoint_gradient_equals_JT_r(h, tau, phi_basis):
    """Reading R18: the discrete adjoint's gradient is J^T r of the discrete map,
    where J comes from the forward variational columns (Eq. Jik)."""
    prob, keep, c = _adjoint_case(32, 10, 24, h, tau, 0.05, phi_basis)
    r, J, f = O.shoot_jacobian(prob, c)
    f2, g = O.objective_and_grad(prob, c)
    jtr = J.T @ r
    assert abs(f2 - f) <= 1e-15 * f
    assert np.linalg.norm(g - jtr) < 1e-13 * np.linalg.norm(jtr)
    # every component carries information (the T entry included)
    assert np.min(np.abs(jtr[:4])) > 1e-8 * np.linalg.norm(jtr)


def test_adjoint_gradient_matches_central_differences():
    """Sec. 3.2: df/dc_k and df/dT against central differences of f, eps =
    1e-6 max(1, |c_k|); agreement to the linearisation's accuracy (reading R6)."""
    prob, keep, c = _adjoint_case(32, 6, 16, 0.5, 0.05, 0.08)
    f, g = O.objective_and_grad(prob, c)
    fd = np.empty_like(g)
    for k in range(len(c)):
        e = 1e-6 * max(1.0, abs(c[k]))
        cp, cm = c.copy(), c.copy()
        cp[k] += e
        cm[k] -= e
        fd[k] = (O.shoot(prob, cp)[1] - O.shoot(prob, cm)[1]) / (2 * e)
    assert np.max(np.abs(g - fd)) < 1e-6 * np.max(np.abs(fd))


def test_transposed_dtn_and_self_adjointness():
    """The transposed DtN equals the transpose of the assembled operator; the
    discrete DtN is nearly symmetric (App. C: Green's identity makes the
    continuous map self-adjoint), with the asymmetry falling as N grows."""
    gaps = []
    for N in (32, 64):
        x = x_grid(N)
        eta = 1.0 + 0.12 * np.cos(x) + 0.03 * np.sin(2 * x)
        Gm = np.array([O.dtn(eta, e, 1.0) for e in np.eye(N)]).T   # column j = G e_j
        v = np.random.default_rng(N).standard_normal(N)
        gt = O.dtn_T(eta, v, 1.0)
        assert np.max(np.abs(gt - Gm.T @ v)) < 1e-13 * np.max(np.abs(Gm.T @ v))
        gaps.append(np.linalg.norm(Gm - Gm.T) / np.linalg.norm(Gm))
    assert gaps[1] < 1e-8 and gaps[1] < 0.1 * gaps[0]


def test_lu_transposed_solve():
    """A^{-T} b from the pivoted LU factors against a library solve with A^T."""
    import ctypes as C
    rng = np.random.default_rng(3)
    N = 40
    A = rng.standard_normal((N, N)) + 0.1 * np.eye(N)
    b = rng.standard_normal(N)
    LU = np.ascontiguousarray(A.copy())
    piv = np.zeros(N, dtype=np.int32)
    assert O.lib().orc_lu(N, O._p(LU), piv.ctypes.data_as(C.POINTER(C.c_int))) == 0
    assert np.any(piv != np.arange(N))   # interchanges happened
    x = np.empty(N)
    O.lib().orc_lu_solve_T(N, O._p(LU), piv.ctypes.data_as(C.POINTER(C.c_int)), O._p(b), O._p(x))
    ref = np.linalg.solve(A.T, b)
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["N64_n12_steps64_h1", "N512_n128_steps512_h1", "N2048_n512_steps1024_h1",
                                  "N1024_n256_steps2048_h0.05", "N1024_n256_steps2048_deep_tau0.1"])
def test_partial_pivoting_never_swaps_on_the_workloads(name):
    """Reading R9: A = 1/2 I + K is a second-kind operator, so the GPU factors it
    without pivoting.  On every workload's initial surface (and, for the small
    one, the surface at T/4 and an RK4 stage state) partial pivoting makes no
    row interchange, so the pivoted factors are the unpivoted ones, and the
    growth max|U| / max|A| stays at 1."""
    import ctypes as C
    w = W.ALL[name]
    c, _ = W.coefficients(w)
    N = w.N
    x = 2 * np.pi * np.arange(N) / N
    surfaces = [(0.0 if math.isinf(w.h) else w.h) + np.cos(np.outer(x, np.arange(1, w.n + 1))) @ c[1:]]
    if N <= 64:
        prob, _ = O.make_problem(N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
        q0 = O.initial(prob, c)
        q1 = O.evolve(prob, c[0], q0)
        k1 = O.rhs(prob, c[0], q0, 0)[0]
        surfaces += [q1[:N], q0[:N] + 0.5 * (c[0] / 4 / w.steps) * k1[:N]]
    for eta in surfaces:
        A, _ = O.dtn_matrices(eta, w.h)
        LU = np.ascontiguousarray(A.copy())
        piv = np.zeros(N, dtype=np.int32)
        assert O.lib().orc_lu(N, O._p(LU), piv.ctypes.data_as(C.POINTER(C.c_int))) == 0
        assert np.array_equal(piv, np.arange(N, dtype=np.int32)), name
        assert np.max(np.abs(np.triu(LU))) / np.max(np.abs(A)) <= 1.0 + 1e-12


def test_adjoint_identity_at_every_step():
    """Sec. 3.2: <q~(T/4 - t), qdot(t)> is constant in time.  For the discrete
    adjoint, the pairing lam_n . w_n of the adjoint state with an unforced
    variational column is the same at every step boundary (each transposed
    step is exactly the transpose of its forward step), and equals that
    column's gradient entry."""
    prob, keep, c = _adjoint_case(32, 6, 16, 0.5, 0.05, 0.08)
    N = prob.N
    lam = O.adjoint_trajectory(prob, c)
    f, g = O.objective_and_grad(prob, c)
    q0 = O.initial(prob, c)
    x = x_grid(N)
    for k in (1, 4):
        col = np.concatenate([np.cos(k * x), np.zeros(N)])    # the default basis column of c_k
        w = O.trajectory_columns(prob, c[0], q0, col)[:, 1, :]
        pair = np.einsum("ni,ni->n", lam, w)
        # rounding of each inner product scales with |lam_n| |w_n| (Cauchy-Schwarz)
        scale = np.linalg.norm(lam, axis=1) * np.linalg.norm(w, axis=1)
        assert np.all(np.abs(pair - g[k]) <= 1e-13 * scale), (k, pair, g[k])
        assert abs(g[k]) > 1e-6 * scale.max()   # far above the rounding bound: the identity is not vacuous
    # the final adjoint state is the gradient of f = r.r/2 with respect to the final state
    qT = O.evolve(prob, c[0], q0)
    assert np.array_equal(lam[-1][:N], np.zeros(N))
    assert np.allclose(lam[-1][N:], qT[N:] / N, rtol=0, atol=1e-18)
