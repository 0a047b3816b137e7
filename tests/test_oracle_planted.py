"""The oracle pins catch planted mistakes.  Each variant of ww_oracle.c is
compiled with one deliberate error (ORC_PLANT, on the CPU only) and the pin
that targets it must fail, while the unmodified oracle passes it."""
import math

import numpy as np
import pytest

import oracle as O


def x_grid(N):
    return 2 * np.pi * np.arange(N) / N


def flat_symbol_error(L, h=1.0, k=3, N=64):
    x = x_grid(N)
    eta = np.full(N, h)
    phi = np.cos(k * x)
    out = np.empty(N)
    L.orc_dtn(N, h, O._p(eta), O._p(phi), 1, O._p(out))
    return np.max(np.abs(out - k * math.tanh(k * h) * phi))


def analytic_error(L, N=64, k=2):
    x = x_grid(N)
    eta = 1.0 + 0.15 * np.cos(x) + 0.03 * np.cos(2 * x) - 0.02 * np.cos(3 * x)
    z = x + 1j * eta
    phi = np.ascontiguousarray(np.cos(k * z).real)
    d = -k * np.sin(k * z)
    u, v = d.real, -d.imag
    ex = np.empty(N)
    L.orc_spectral(N, O.MUL_DERIV, O._p(eta), O._p(ex))
    out = np.empty(N)
    L.orc_dtn(N, 1.0, O._p(eta), O._p(phi), 1, O._p(out))
    return np.max(np.abs(out - (v - ex * u)))


def dispersion_rest(L, eps=1e-3, N=32, steps=128):
    h = 1.0
    T = 2 * math.pi / math.sqrt(math.tanh(h))
    prob, _ = O.make_problem(N, 0, h=h, steps=steps)
    q0 = np.concatenate([np.full(N, h), eps * np.cos(x_grid(N))])
    q1 = np.empty(2 * N)
    import ctypes as C
    L.orc_evolve(C.byref(prob), T, O._p(q0), O._p(q1))
    return np.max(np.abs(q1[N:])) / eps


def linearisation_gap(L, N=64):
    import ctypes as C
    x = x_grid(N)
    prob, _ = O.make_problem(N, 0, h=1.0)
    q = np.concatenate([1.0 + 0.08 * np.cos(x) + 0.02 * np.cos(2 * x), 0.05 * np.cos(x) - 0.01 * np.cos(3 * x)])
    qd = np.concatenate([0.3 * np.cos(2 * x + 0.4), 0.2 * np.cos(x + 1.0) + 0.1 * np.cos(3 * x)])
    y = np.stack([q, qd])
    out = np.empty_like(y)
    L.orc_rhs(C.byref(prob), 7.0, O._p(y), 1, 0, O._p(out))
    eps = 1e-5
    fp, fm = np.empty(2 * N), np.empty(2 * N)
    a, b = q + eps * qd, q - eps * qd
    L.orc_rhs(C.byref(prob), 7.0, O._p(a), 0, 0, O._p(fp))
    L.orc_rhs(C.byref(prob), 7.0, O._p(b), 0, 0, O._p(fm))
    return np.max(np.abs(out[1] - (fp - fm) / (2 * eps)))


def adjoint_gap(L, N=32, n=6, steps=12):
    """|grad (discrete adjoint) - J^T r| / |J^T r| (reading R18)."""
    import ctypes as C
    prob, _ = O.make_problem(N, n, h=0.5, tau=0.05, steps=steps)
    c = np.zeros(n + 1)
    c[0] = 2 * math.pi / math.sqrt(1.05 * math.tanh(0.5))
    c[1:] = 0.08 * 0.5 ** np.arange(n)
    r, f = np.empty(N), np.empty(1)
    Jc = np.empty((n + 1, N))
    L.orc_shoot_jacobian(C.byref(prob), O._p(c), O._p(r), O._p(Jc), O._p(f))
    g = np.empty(n + 1)
    L.orc_objective_and_grad(C.byref(prob), O._p(c), O._p(f), O._p(g))
    jtr = Jc @ r
    return np.linalg.norm(g - jtr) / np.linalg.norm(jtr)


def mesh_dtn_error(L, N=64, rho=0.3, k=2):
    """The DtN on a mesh against the analytic potential cos(kz) (finite depth)."""
    x = np.empty(N); e = np.empty(N); e1 = np.empty(N)
    L.orc_mesh_eval(rho, 1, N, O._p(x), O._p(e), O._p(e1))
    eta = 1.0 + 0.15 * np.cos(x) + 0.03 * np.cos(2 * x) - 0.02 * np.cos(3 * x)
    ex = -0.15 * np.sin(x) - 0.06 * np.sin(2 * x) + 0.06 * np.sin(3 * x)
    z = x + 1j * eta
    phi = np.ascontiguousarray(np.cos(k * z).real)
    d = -k * np.sin(k * z)
    out = np.empty(N)
    L.orc_dtn_segment(O._segments([(N, 1, 1.0, rho)]), 1.0, O._p(eta), O._p(phi), O._p(out))
    return np.max(np.abs(out - (d.imag * -1.0 - ex * d.real)))


def mesh_rhs_gap(L, N=64, rho=0.4):
    """The RHS on a mesh against the uniform RHS (N = 128) interpolated to the mesh."""
    import ctypes as C
    eta_f = lambda s: 1.0 + 0.08 * np.cos(s) + 0.02 * np.cos(2 * s) - 0.01 * np.sin(3 * s)
    phi_f = lambda s: 0.05 * np.cos(s) - 0.01 * np.cos(3 * s) + 0.004 * np.sin(2 * s)
    Nu = 128
    probu, _ = O.make_problem(Nu, 0, h=1.0, tau=0.05)
    xu = x_grid(Nu)
    yu = np.concatenate([eta_f(xu), phi_f(xu)])
    Fu = np.empty(2 * Nu)
    L.orc_rhs(C.byref(probu), 7.0, O._p(yu), 0, 0, O._p(Fu))
    x = np.empty(N); e = np.empty(N); e1 = np.empty(N)
    L.orc_mesh_eval(rho, 1, N, O._p(x), O._p(e), O._p(e1))
    prob, _ = O.make_problem(N, 0, h=1.0, tau=0.05)
    y = np.concatenate([eta_f(x), phi_f(x)])
    F = np.empty(2 * N)
    L.orc_rhs_segment(C.byref(prob), O._segments([(N, 1, 1.0, rho)]), 7.0, O._p(y), 0, 0, O._p(F))
    ref = np.concatenate([O.interp(Fu[:Nu], x), O.interp(Fu[Nu:], x)])
    return np.max(np.abs(F - ref))


def mesh_adjoint_gap(L, M=32, rho=0.4):
    """The transposed variational RHS on a mesh against the explicit transpose."""
    import ctypes as C
    prob, _ = O.make_problem(M, 0, h=1.0, tau=0.05)
    x = np.empty(M); e = np.empty(M); e1 = np.empty(M)
    L.orc_mesh_eval(rho, 1, M, O._p(x), O._p(e), O._p(e1))
    q = np.concatenate([1.0 + 0.08 * np.cos(x) + 0.02 * np.cos(2 * x), 0.05 * np.cos(x) - 0.01 * np.cos(3 * x)])
    y = np.zeros((2 * M + 1, 2 * M))
    y[0] = q
    y[1:] = np.eye(2 * M)
    out = np.empty_like(y)
    seg = O._segments([(M, 1, 1.0, rho)])
    L.orc_rhs_segment(C.byref(prob), seg, 7.0, O._p(y), 2 * M, 0, O._p(out))
    kb = np.random.default_rng(1).standard_normal(2 * M)
    got, fd = np.empty(2 * M), np.empty(1)
    L.orc_rhs_T_segment(C.byref(prob), seg, O._p(q), O._p(kb), O._p(got), O._p(fd))
    ref = out[1:] @ kb
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.fixture(scope="module")
def good():
    return O.load(O.build())


@pytest.mark.parametrize("plant,probe,bound", [
    (1, flat_symbol_error, 1e-12),      # image sign as printed
    (2, analytic_error, 1e-11),         # zeta'(alpha) for zeta'(beta) in K1
    (3, dispersion_rest, 5e-3),         # gravity dropped
    (4, linearisation_gap, 1e-8),       # u psi' dropped from Eq. (l6a)
    (5, adjoint_gap, 1e-13),            # forward DtN used as its own transpose
    (6, mesh_dtn_error, 5e-12),         # 1/|xi'| of Eq. (G) dropped on a mesh
    (7, mesh_rhs_gap, 2e-12),           # P as the alpha-mean on a mesh
    (8, mesh_adjoint_gap, 1e-14),       # P taken for its own transpose on a mesh
])
def test_pin_catches_planted_mistake(good, plant, probe, bound):
    assert probe(good) < bound
    bad = O.load(O.build(plant=plant))
    assert probe(bad) > 10 * bound
