"""Pins of the oracle's time segments, adaptive meshes and general explicit
Runge-Kutta schemes (Sec. 2.2: Eq. (xi), Eq. (rho:def), respacing between
segments, DOP853), no GPU.

What each pin catches:
* mesh closed forms -- E(0), E(pi) are the printed 8/(5+3 rho) and
  8 rho/(5+3 rho) (Eq. rho:def), rho = min/max, E has mean 1 (P in Eq. xi),
  xi' = E and xi'' = E' by an independent spectral derivative of xi - alpha:
  a wrong coefficient or sign in the integrated trigonometric polynomial;
* Newton inverse -- xi(xi^-1(x)) = x down to rho = 0.05, both centres;
* interpolant -- exact on trigonometric polynomials, returns the grid values;
* DtN on a mesh -- the analytic potentials Re cos(kz) (finite depth) and
  Re e^{-ikz} (deep water) on a non-flat surface: the 1/xi' of Eq. (G), the
  mesh in zeta of Eq. (zeta) and its derivatives in the kernels;
* RHS on a mesh -- equals the uniform RHS of the same smooth state at the
  mesh points: d/dx as d/dalpha over xi', P as the x-mean (reading R22), the
  surface-tension term;
* tableaux -- the linear order conditions b^T A^(k-1) 1 = 1/k! (k <= 8 for
  DOP853, 4 for RK4) and row sums; DOP853's measured order 8 and RK4's 4 on a
  resolved shot, and the two converge to the same state;
* segments -- two uniform segments are one run; a refined, finer last
  segment agrees with a uniform fine run at its points; J of a segmented,
  refined DOP853 shot matches central differences (T column included);
* validation -- rho_1 != 1, M_1 != N, theta not summing to 1 are refused.
"""
import math

import numpy as np
import pytest

import oracle as O


def x_grid(N):
    return 2 * np.pi * np.arange(N) / N


def spectral_derivative(f):
    """numpy FFT derivative of a periodic sample (Nyquist dropped)."""
    N = f.size
    k = np.fft.fftfreq(N, 1.0 / N)
    k[N // 2] = 0.0
    return np.real(np.fft.ifft(1j * k * np.fft.fft(f)))


# ----------------------------------------------------------------- mesh
@pytest.mark.parametrize("rho", [1.0, 0.6, 0.25, 0.05])
@pytest.mark.parametrize("centre", [1, 0])
def test_mesh_closed_forms(rho, centre):
    M = 64
    x, E, E1 = O.mesh(rho, M, centre)
    emin, emax = 8 * rho / (5 + 3 * rho), 8 / (5 + 3 * rho)
    at_pi, at_0 = E[M // 2], E[0]
    refined, other = (at_pi, at_0) if centre else (at_0, at_pi)
    assert abs(refined - emin) < 1e-15 and abs(other - emax) < 1e-15
    assert abs(min(E) - emin) < 1e-15 and abs(max(E) - emax) < 1e-15
    assert abs(min(E) / max(E) - rho) < 1e-15                          # Eq. (rho:def)
    assert abs(E.mean() - 1.0) < 1e-15                                 # P in Eq. (xi)
    a = x_grid(M)
    assert np.max(np.abs(spectral_derivative(x - a) + 1.0 - E)) < 1e-13   # xi' = E
    assert np.max(np.abs(spectral_derivative(E) - E1)) < 1e-13            # xi'' = E'
    assert x[0] == 0.0 and np.all(np.diff(x) > 0) and x[-1] < 2 * np.pi
    if rho == 1.0:
        assert np.array_equal(x, a) and np.all(E == 1.0) and np.all(E1 == 0.0)


@pytest.mark.parametrize("rho", [0.05, 0.3, 1.0])
@pytest.mark.parametrize("centre", [1, 0])
def test_mesh_inverse(rho, centre):
    """xi(xi^-1(x)) = x.  xi - alpha is a trigonometric polynomial of degree 2,
    so the interpolant of its values on the 8-point mesh gives it anywhere."""
    xs = np.linspace(0.0, 2 * np.pi, 101)[:-1]
    al = O.mesh_inverse(rho, xs, centre)
    x8, _, _ = O.mesh(rho, 8, centre)
    back = al + O.interp(x8 - x_grid(8), al)
    assert np.max(np.abs(back - xs)) < 1e-14


def test_interpolant_is_exact_on_trigonometric_polynomials():
    rng = np.random.default_rng(3)
    M = 32
    a = x_grid(M)
    ks = np.arange(0, M // 2)
    ca, cb = rng.standard_normal(ks.size), rng.standard_normal(ks.size)
    f = lambda t: sum(ca[k] * np.cos(k * t) + cb[k] * np.sin(k * t) for k in ks)
    beta = rng.uniform(0, 2 * np.pi, 40)
    assert np.max(np.abs(O.interp(f(a), beta) - f(beta))) < 1e-13
    g = rng.standard_normal(M)                                 # any data: grid values come back
    assert np.max(np.abs(O.interp(g, a) - g)) < 1e-14


# ----------------------------------------------------------------- DtN and RHS on a mesh
def _surface(x, h):
    return h + 0.15 * np.cos(x) + 0.03 * np.cos(2 * x) - 0.02 * np.cos(3 * x), \
        -0.15 * np.sin(x) - 0.06 * np.sin(2 * x) + 0.06 * np.sin(3 * x)


@pytest.mark.parametrize("rho", [0.5, 0.2])
@pytest.mark.parametrize("deep", [False, True])
def test_dtn_on_a_mesh_analytic_potential(rho, deep):
    """Phi harmonic below the surface with phi_y = 0 on the bottom y = 0
    (cos kz) or decaying (e^{-ikz}); G phi = phi_y - eta' phi_x at x = xi(alpha_j)."""
    N, k, h = 64, 2, 1.0
    x, _, _ = O.mesh(rho, N)
    eta, ex = _surface(x, 0.0 if deep else h)
    z = x + 1j * eta
    if deep:
        W = np.exp(-1j * k * z)
        d = -1j * k * W
    else:
        W = np.cos(k * z)
        d = -k * np.sin(k * z)
    u, v = d.real, -d.imag
    G = O.dtn_segment((N, 1, 1.0, rho), math.inf if deep else h, eta, W.real)
    assert np.max(np.abs(G - (v - ex * u))) < 5e-12


@pytest.mark.parametrize("h,tau", [(1.0, 0.05), (math.inf, 0.1)])
def test_rhs_on_a_mesh_matches_uniform(h, tau):
    """The same smooth state stored on a mesh and on a uniform grid: the mesh
    RHS equals the uniform RHS interpolated to the mesh points."""
    base = 0.0 if math.isinf(h) else h
    eta_f = lambda s: base + 0.08 * np.cos(s) + 0.02 * np.cos(2 * s) - 0.01 * np.sin(3 * s)
    phi_f = lambda s: 0.05 * np.cos(s) - 0.01 * np.cos(3 * s) + 0.004 * np.sin(2 * s)
    N, Nu = 64, 128
    prob, _ = O.make_problem(N, 0, h=h, tau=tau)
    probu, _ = O.make_problem(Nu, 0, h=h, tau=tau)
    xu = x_grid(Nu)
    Fu = O.rhs(probu, 7.0, np.concatenate([eta_f(xu), phi_f(xu)]), 0)[0]
    # the state is band-limited in x, not in alpha: at rho = 0.15 the coarse side
    # of the mesh is 1.47 x the uniform spacing and truncation shows at 1e-12
    for rho, tol in ((0.4, 2e-12), (0.15, 1e-11)):
        x, _, _ = O.mesh(rho, N)
        F = O.rhs_segment(prob, (N, 1, 1.0, rho), 7.0, np.concatenate([eta_f(x), phi_f(x)]))[0]
        ref = np.concatenate([O.interp(Fu[:Nu], x), O.interp(Fu[Nu:], x)])
        assert np.max(np.abs(F - ref)) < tol, rho


# ----------------------------------------------------------------- tableaux
@pytest.mark.parametrize("name,order", [("rk4", 4), ("dop853", 8)])
def test_tableau_linear_order_conditions(name, order):
    a, b = O.tableau(name)
    s = b.size
    assert np.all(np.triu(a) == 0.0)                              # explicit
    one = np.ones(s)
    v = one.copy()
    for k in range(1, order + 1):                                  # b^T A^(k-1) 1 = 1/k!
        assert abs(b @ v - 1.0 / math.factorial(k)) < 1e-14 * max(1.0, 1.0 / math.factorial(k)) + 1e-16, k
        v = a @ v
    if name == "dop853":
        assert s == 12
        # the stability polynomial is not exp(z) beyond order 8
        assert abs(b @ v - 1.0 / math.factorial(order + 1)) > 1e-8


def _resolved_shot(N=64):
    prob, keep = O.make_problem(N, 3, h=1.0, steps=16)
    c = np.array([7.2, 0.06, 0.01, -0.004])
    return prob, keep, c, O.initial(prob, c)


def test_dop853_and_rk4_orders_on_a_resolved_shot():
    """N = 64 resolves this state to roundoff below the filter's band, so the
    step filter does not depend on the step count and the schemes show their
    orders: error ratios 2^8 and 2^4 on halving dt; both reach the same state."""
    prob, keep, c, q0 = _resolved_shot()
    N = prob.N
    ev = lambda tab, s: O.evolve_segments(prob, [(N, s, 1.0, 1.0)], tab, c[0], q0)
    ref8 = ev("dop853", 64)
    e4, e8 = (np.max(np.abs(ev("dop853", s) - ref8)) for s in (4, 8))
    assert 7.5 < math.log2(e4 / e8) < 8.7, (e4, e8)
    ref4 = ev("rk4", 512)
    e16, e32 = (np.max(np.abs(ev("rk4", s) - ref4)) for s in (16, 32))
    assert 3.8 < math.log2(e16 / e32) < 4.2, (e16, e32)
    assert np.max(np.abs(ref8 - ref4)) < 5e-13


# ----------------------------------------------------------------- segments
def test_two_uniform_segments_are_one_run():
    N, n = 32, 4
    prob, _ = O.make_problem(N, n, h=1.0, steps=16)
    c = np.array([7.2, 0.06, 0.01, -0.004, 0.001])
    r1, J1, f1 = O.shoot_jacobian(prob, c)
    r2, J2, f2 = O.shoot_jacobian_segments(prob, [(N, 8, 0.5, 1.0), (N, 8, 0.5, 1.0)], "rk4", c)
    assert np.max(np.abs(r1 - r2)) < 1e-15 and np.max(np.abs(J1 - J2)) < 1e-14
    assert abs(f1 - f2) < 1e-14 * f1


def test_refined_last_segment_matches_a_uniform_fine_run():
    """Segment 2 on twice the points with the mesh refined near x = pi (rho =
    0.3, allowed since M2/M1 = 2 >= (5+3)/(5+0.9)) against one uniform run on
    the fine grid: the same PDE, both resolved, so phi agrees at the mesh
    points to spectral accuracy."""
    prob, keep, c, q0 = _resolved_shot()
    N = prob.N
    probf, _ = O.make_problem(2 * N, 0, h=1.0)
    segs = [(N, 24, 0.5, 1.0), (2 * N, 24, 0.5, 0.3, 1)]
    q = O.evolve_segments(prob, segs, "dop853", c[0], q0)
    q0f = np.concatenate([O.interp(q0[:N], x_grid(2 * N)), O.interp(q0[N:], x_grid(2 * N))])
    qf = O.evolve_segments(probf, [(2 * N, 48, 1.0, 1.0)], "dop853", c[0], q0f)
    x, E, _ = O.mesh(0.3, 2 * N)
    M = 2 * N
    assert np.max(np.abs(q[:M] - O.interp(qf[:M], x))) < 1e-11
    assert np.max(np.abs(q[M:] - O.interp(qf[M:], x))) < 1e-11
    r, f = O.shoot_segments(prob, segs, "dop853", c)
    assert np.allclose(r, np.sqrt(E / M) * q[M:], rtol=0, atol=1e-16)     # weights sqrt(E/M)


def test_segmented_jacobian_matches_central_differences():
    """As the uniform pin: J is the continuum linearisation with the shared
    discrete DtN (reading R6), so it matches differences of the discrete map to
    spectral truncation, 1e-7 of the column's size at N = 64."""
    N, n = 64, 4
    x = x_grid(N)
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):                 # Eq. (init:stand): even k on eta, odd k on phi
        basis[(N if k % 2 else 0):(2 * N if k % 2 else N), k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, h=1.0, basis=basis)
    c = np.array([7.1, 0.03, 0.004, 0.002, -0.001])
    segs = [(N, 6, 0.4, 1.0), (N, 6, 0.35, 0.5, 1), (2 * N, 6, 0.25, 0.3, 0)]
    r, J, f = O.shoot_jacobian_segments(prob, segs, "dop853", c)
    assert J.shape == (2 * N, n + 1)
    r0, f0 = O.shoot_segments(prob, segs, "dop853", c)
    assert np.array_equal(r, r0) and f == f0
    for k in range(n + 1):
        eps = 1e-6 * max(1.0, abs(c[k]))
        cp, cm = c.copy(), c.copy()
        cp[k] += eps
        cm[k] -= eps
        fd = (O.shoot_segments(prob, segs, "dop853", cp)[0] - O.shoot_segments(prob, segs, "dop853", cm)[0]) / (2 * eps)
        assert np.max(np.abs(J[:, k] - fd)) < 1e-7 * max(np.max(np.abs(fd)), 1e-3), k


def test_invalid_segments_are_refused():
    prob, _ = O.make_problem(32, 2, h=1.0)
    c = np.array([7.2, 0.01, 0.0])
    for segs in ([(32, 4, 1.0, 0.5)],                        # rho_1 != 1
                 [(64, 4, 1.0, 1.0)],                        # M_1 != N
                 [(32, 4, 0.5, 1.0), (32, 4, 0.4, 1.0)],     # theta sums to 0.9
                 [(32, 4, 0.5, 1.0), (48, 4, 0.5, 1.0)],     # M not a power of two
                 [(32, 4, 0.5, 1.0), (32, 4, 0.5, 0.0)]):    # rho out of (0, 1]
        with pytest.raises(ValueError):
            O.shoot_segments(prob, segs, "rk4", c)


# ----------------------------------------------------------------- the adjoint on segments
@pytest.mark.parametrize("rho,h,tau", [(0.4, 1.0, 0.05), (1.0, 1.0, 0.0), (0.3, math.inf, 0.1)])
def test_transposed_rhs_on_a_mesh_is_the_transpose(rho, h, tau):
    """DF(q)^T kb on a mesh against the explicit transpose of the variational RHS
    (its 2M columns from unit initial data): P^T, -D_x^T and the DtN transpose
    with diag(1/xi'); and kb . F(q) for the T forcing."""
    M = 32
    prob, _ = O.make_problem(M, 0, h=h, tau=tau)
    x, _, _ = O.mesh(rho, M)
    base = 0.0 if math.isinf(h) else h
    q = np.concatenate([base + 0.08 * np.cos(x) + 0.02 * np.cos(2 * x) - 0.01 * np.sin(3 * x),
                        0.05 * np.cos(x) - 0.01 * np.cos(3 * x)])
    y = np.zeros((2 * M + 1, 2 * M))
    y[0] = q
    y[1:] = np.eye(2 * M)
    out = O.rhs_segment(prob, (M, 1, 1.0, rho), 7.0, y, ncol=2 * M)
    kb = np.random.default_rng(1).standard_normal(2 * M)
    got, fd = O.rhs_T_segment(prob, (M, 1, 1.0, rho), q, kb)
    ref = out[1:] @ kb
    assert np.max(np.abs(got - ref)) < 5e-15 * np.max(np.abs(ref))
    assert abs(fd - kb @ out[0]) < 1e-15 * np.abs(kb) @ np.abs(out[0])


def test_segmented_gradient_is_J_transpose_r():
    """The discrete adjoint of the segmented shot (three segments, meshes refined
    near pi then near 0, M doubled, DOP853, surface tension) against J^T r of
    the segmented Jacobian, an independent algorithm; one uniform RK4 segment
    reproduces the RK4 adjoint."""
    N, n = 32, 4
    x = x_grid(N)
    basis = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        basis[(N if k % 2 else 0):(2 * N if k % 2 else N), k - 1] = 2 * np.cos(k * x)
    prob, keep = O.make_problem(N, n, h=1.0, tau=0.02, basis=basis, steps=12)
    c = np.array([7.1, 0.03, 0.004, 0.002, -0.001])
    segs = [(N, 6, 0.4, 1.0), (N, 6, 0.35, 0.5, 1), (2 * N, 6, 0.25, 0.3, 0)]
    f, g = O.objective_and_grad_segments(prob, segs, "dop853", c)
    r, J, f2 = O.shoot_jacobian_segments(prob, segs, "dop853", c)
    jtr = J.T @ r
    assert f == f2
    assert np.linalg.norm(g - jtr) < 1e-13 * np.linalg.norm(jtr)
    f1, g1 = O.objective_and_grad_segments(prob, [(N, 12, 1.0, 1.0)], "rk4", c)
    f0, g0 = O.objective_and_grad(prob, c)
    assert abs(f1 - f0) < 1e-13 * f0 and np.max(np.abs(g1 - g0)) < 1e-12 * np.max(np.abs(g0))


@pytest.mark.parametrize("h,tau,N,steps", [(1.0, 0.0, 64, 8), (math.inf, 0.05, 32, 24), (0.5, 0.02, 32, 24)])
def test_energy_is_conserved_across_segments_and_meshes(h, tau, N, steps):
    """The energy monitor of Sec. 4 (integrals in x by the mesh's own quadrature,
    weights xi') before and after three segments: refined near pi, then near 0,
    twice the points, DOP853 (steps chosen inside its stability region).  The
    paper reports energy conserved to about 14 digits in double precision."""
    prob, _ = O.make_problem(N, 3, h=h, tau=tau)
    c = np.array([6.5, 0.05, 0.01, -0.004])
    q0 = O.initial(prob, c)
    E0 = O.energy(prob, q0)
    assert O.energy_segment(prob, (N, 1, 1.0, 1.0), q0) == E0
    segs = [(N, steps, 0.4, 1.0), (2 * N, steps, 0.3, 0.4, 1), (2 * N, steps, 0.3, 0.3, 0)]
    q = O.evolve_segments(prob, segs, "dop853", c[0], q0)
    assert abs(O.energy_segment(prob, segs[-1], q) - E0) < 1e-13 * E0


def test_evenness_is_preserved_across_segments_and_meshes():
    """Sec. 2.3: even initial data stay even.  The meshes of Eq. (xi) are odd
    about x = 0 (x_{M-j} = 2 pi - x_j), so the stored values of an even state
    satisfy q_j = q_{M-j} on every segment, through respacing, to roundoff."""
    N = 32
    prob, _ = O.make_problem(N, 3, h=1.0, tau=0.01)
    c = np.array([6.8, 0.05, 0.01, -0.004])
    q0 = O.initial(prob, c)
    segs = [(N, 12, 0.4, 1.0), (2 * N, 12, 0.3, 0.4, 1), (2 * N, 12, 0.3, 0.3, 0)]
    q = O.evolve_segments(prob, segs, "dop853", c[0], q0)
    M = 2 * N
    x, _, _ = O.mesh(0.3, M, 0)
    j = np.arange(1, M)
    assert np.max(np.abs(x[M - j] - (2 * np.pi - x[j]))) < 1e-14
    for part in (q[:M], q[M:]):           # roundoff of an O(1) state over 36 steps
        assert np.max(np.abs(part[j] - part[M - j])) < 5e-14


def test_the_segmented_workload_runs_through_the_oracle():
    """The segmented workload's structure (four segments, rho down to 0.1, M
    doubling twice, DOP853), shrunk 16x in M and 4x in steps, is a valid input
    to the oracle, and energy is conserved through it."""
    from paper_1210_5672_gb300 import workloads as W
    w = W.SEGMENTED
    segs = [(M // 16, max(1, s // 4), th, rho, ctr) for (M, s, th, rho, ctr) in w.meta["segments"]]
    N = segs[0][0]
    c, _ = W.coefficients(W.Workload("seg_small", N=N, n=N // 3, steps=1, amp=0.05))
    prob, _ = O.make_problem(N, N // 3, h=w.h)
    q0 = O.initial(prob, c)
    q = O.evolve_segments(prob, segs, w.meta["tableau"], c[0], q0)
    assert q.shape == (2 * segs[-1][0],) and np.all(np.isfinite(q))
    E0 = O.energy(prob, q0)
    assert abs(O.energy_segment(prob, segs[-1], q) - E0) < 1e-11 * E0
