"""The segmented shot on the GPU (Sec. 2.2: time segments, the adaptive meshes
of Eq. (xi), respacing, DOP853) against the oracle's segmented shot
(orc_shoot_jacobian_segments), both forms, element by element at 1e-11
relative for r and f; each Jacobian column (per-column measure with the 1e-4
floor of the other parity tests) at max(1e-11, 4 x the oracle's own one-ulp
spread of that column).

Cases: one uniform RK4 segment (the same discrete map as the plain shot);
three segments with meshes refined near x = 0 and a doubled grid, DOP853, in
finite depth and deep water; two segments with surface tension; and the
segmented workload (four segments, rho down to 0.1, M doubling twice) shrunk
8x in M and 4x in steps so that the oracle finishes in seconds.

The segmented gradient by the GPU's discrete adjoint
(objective_and_grad_segments) on the same cases against the oracle's
(orc_objective_and_grad_segments) and against J^T r of the GPU's segmented
Jacobian."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def ww():
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as m
    return m


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def col_errs(J, J0):
    """per column ||dJ_k|| / max(||J_k||, 1e-4 max_j ||J_j||); J, J0 are M x (n+1)."""
    norms = np.linalg.norm(J0, axis=0)
    return np.array([np.linalg.norm(J[:, k] - J0[:, k]) / max(norms[k], 1e-4 * norms.max())
                     for k in range(J0.shape[1])])


def col_err(J, J0):
    return float(col_errs(J, J0).max())


def gpu_segments(ww, segs, scheme, N0, n, c, precision, g=1.0, tau=0.0, h=1.0, basis=None):
    """segs: [(M, steps, theta, rho, centre)]; one context per segment."""
    import torch
    ctxs = []
    try:
        for i, (M, steps, theta, rho, centre) in enumerate(segs):
            ctx = ww.Context(M, n, g=g, tau=tau, h=h, steps=steps, precision=precision,
                             basis=basis if i == 0 else None)
            ctxs.append(ctx)
            ww.set_segment(ctx, steps, theta, rho, centre, scheme)
        last = ctxs[-1]
        r = torch.empty(last.N, dtype=torch.float64, device="cuda")
        J = torch.empty(n + 1, last.N, dtype=torch.float64, device="cuda")
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        ww.shoot_jacobian_segments(ctxs, dev(c), r, J, f)
        out = (r.cpu().numpy(), J.cpu().numpy().T.copy(), float(f.item()))
        ww.shoot_jacobian_segments(ctxs, dev(c), r, J, f)     # a second call: captured programs, cached respacing
        again = (r.cpu().numpy(), J.cpu().numpy().T.copy(), float(f.item()))
        assert np.array_equal(out[0], again[0]) and np.array_equal(out[1], again[1]) and out[2] == again[2]
        return out
    finally:
        for ctx in ctxs:
            ctx.close()


_SPREAD = {}
_ORACLE = {}


def check(ww, segs, scheme, n, c, precision, **kw):
    """Every output against the oracle.  r and f at 1e-11; each column of J at
    max(1e-11, 4 x the oracle's one-ulp spread of that column): how far the
    oracle's own column moves when c_1 moves by one ulp, i.e. when only its
    rounding changes (the variational columns amplify rounding over the
    segments, as at the full uniform size)."""
    r, J, f = gpu_segments(ww, segs, scheme, segs[0][0], n, c, precision, **kw)
    prob, keep = O.make_problem(segs[0][0], n, g=kw.get("g", 1.0), tau=kw.get("tau", 0.0), h=kw.get("h", 1.0),
                                basis=kw.get("basis"))
    key = (tuple(segs), scheme, n, tuple(c), tuple(sorted((k, str(v)) for k, v in kw.items())))
    if key not in _ORACLE:
        _ORACLE[key] = O.shoot_jacobian_segments(prob, segs, scheme, c)
    r0, J0, f0 = _ORACLE[key]
    if key not in _SPREAD:
        cp = c.copy()
        cp[1] = np.nextafter(c[1], np.inf)
        _, Jp, _ = O.shoot_jacobian_segments(prob, segs, scheme, cp)
        _SPREAD[key] = col_errs(Jp, J0)
    spread = _SPREAD[key]
    er = np.linalg.norm(r - r0) / np.linalg.norm(r0)
    ef = abs(f - f0) / abs(f0)
    ej = col_errs(J, J0)
    tol = np.maximum(TOL, 4.0 * spread)
    k = int(np.argmax(ej / tol))
    print(f"\nsegments {[s[:4] for s in segs]} {scheme} precision={precision}: r {er:.2e} f {ef:.2e} "
          f"J worst {ej.max():.2e} (column {int(ej.argmax())}), median {np.median(ej):.2e}; oracle one-ulp "
          f"spread median {np.median(spread):.2e}, worst ratio error/tolerance {ej[k] / tol[k]:.2f} (column {k})")
    assert er < TOL and ef < TOL
    assert np.all(ej < tol), [(int(i), float(ej[i]), float(tol[i])) for i in np.nonzero(ej >= tol)[0]]
    return r, J, f


def test_one_uniform_rk4_segment_is_the_plain_shot(ww):
    """The general-tableau path with the RK4 tableau on one uniform segment
    computes the plain shot's discrete map (its stage sums round differently)."""
    import torch
    N, n, steps = 64, 8, 16
    w = W.Workload("seg1", N=N, n=n, steps=steps, amp=0.05)
    c, _ = W.coefficients(w)
    for precision in (ww.WW_FP64, ww.WW_MIXED):
        with ww.Context(N, n, steps=steps, precision=precision) as ctx:
            r, J, f = ctx.empty_outputs()
            ww.shoot_jacobian(ctx, dev(c), r, J, f)
            plain = (r.cpu().numpy(), J.cpu().numpy().T.copy(), float(f.item()))
        rs, Js, fs = gpu_segments(ww, [(N, steps, 1.0, 1.0, 1)], "rk4", N, n, c, precision)
        assert np.linalg.norm(rs - plain[0]) / np.linalg.norm(plain[0]) < 1e-13
        # the small T column (1e-5 of the others) moves by ~1e-11 of itself with the rounding
        assert abs(fs - plain[2]) / plain[2] < 1e-13 and col_err(Js, plain[1]) < TOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("h,tau,segs", [
    # finite and infinite depth, meshes refined near x = 0, the grid doubled
    (1.0, 0.0, [(64, 5, 0.375, 1.0, 0), (128, 8, 0.375, 0.4, 0), (128, 6, 0.25, 0.2, 0)]),
    (math.inf, 0.0, [(64, 5, 0.375, 1.0, 0), (128, 8, 0.375, 0.4, 0), (128, 6, 0.25, 0.2, 0)]),
    # surface tension (its capillary modes are stiff: a mild mesh, more steps), near x = pi
    (0.5, 0.01, [(64, 8, 0.5, 1.0, 1), (128, 24, 0.5, 0.7, 1)]),
])
def test_segments_with_meshes_match_oracle(ww, precision, h, tau, segs):
    N, n = segs[0][0], 12
    w = W.Workload("seg3", N=N, n=n, steps=1, h=h, tau=tau, amp=0.05)
    c, _ = W.coefficients(w)
    check(ww, segs, "dop853", n, c, precision, h=h, tau=tau)


@pytest.mark.parametrize("precision", [0, 1])
def test_segmented_workload_shrunk_matches_oracle(ww, precision):
    """The segmented workload's structure, shrunk: M = 64, 128, 256, 256 (8x
    fewer points), rho = 1, 0.4, 0.1, 0.1 refined near x = 0, DOP853 steps in
    the workload's proportions (4x fewer), n = M_1 / 3 modes + T."""
    wl = W.SEGMENTED
    segs = [(M // 8, max(2, s // 4), th, rho, ctr) for (M, s, th, rho, ctr) in wl.meta["segments"]]
    N, n = segs[0][0], segs[0][0] // 3
    w = W.Workload("seg_wl", N=N, n=n, steps=1, h=wl.h, amp=0.05)
    c, _ = W.coefficients(w)
    check(ww, segs, wl.meta["tableau"], n, c, precision, h=wl.h)


@pytest.mark.parametrize("precision", [0, 1])
def test_segmented_workload_quarter_size_at_its_amplitude(ww, precision):
    """The segmented workload at a quarter of its points (M = 128, 256, 512,
    512: the base transforms of the last segments take the 8-CTA cluster path)
    with all of its DOP853 steps and its own amplitude c_1 = 0.2, 42 modes + T."""
    wl = W.SEGMENTED
    segs = [(M // 4, s, th, rho, ctr) for (M, s, th, rho, ctr) in wl.meta["segments"]]
    N, n = segs[0][0], 42
    w = W.Workload("seg_q", N=N, n=n, steps=1, h=wl.h, amp=wl.amp)
    c, _ = W.coefficients(w)
    check(ww, segs, wl.meta["tableau"], n, c, precision, h=wl.h)


def test_paper_basis_and_bad_segments(ww):
    """The paper's initial-data basis (Eq. init:stand: phi components) through
    segments, and invalid segment lists refused before any work."""
    import torch
    N, n = 64, 6
    x = 2 * np.pi * np.arange(N) / N
    B = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        B[(0 if k % 2 == 0 else N):(N if k % 2 == 0 else 2 * N), k - 1] = 2 * np.cos(k * x)
    c = np.array([7.1, 0.03, 0.004, 0.002, -0.001, 0.0005, 0.0002])
    segs = [(N, 6, 0.5, 1.0, 1), (2 * N, 6, 0.5, 0.5, 1)]
    check(ww, segs, "dop853", n, c, 0, basis=B)
    with ww.Context(N, n) as a, ww.Context(N, n) as b:
        ww.set_segment(a, 4, 0.5, 0.5, 1)                 # a refined FIRST segment
        ww.set_segment(b, 4, 0.5, 1.0, 1)
        r = torch.empty(N, dtype=torch.float64, device="cuda")
        J = torch.empty(n + 1, N, dtype=torch.float64, device="cuda")
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        with pytest.raises(ww.WWError):
            ww.shoot_jacobian_segments([a, b], dev(c), r, J, f)
        ww.set_segment(a, 4, 0.5, 1.0, 1)
        ww.set_segment(b, 4, 0.4, 1.0, 1)                 # thetas sum to 0.9
        with pytest.raises(ww.WWError):
            ww.shoot_jacobian_segments([a, b], dev(c), r, J, f)


def gpu_grad_segments(ww, segs, scheme, n, c, precision, g=1.0, tau=0.0, h=1.0, basis=None):
    """f and grad of the segmented shot by the GPU's discrete adjoint (called
    twice: bitwise the same), and J^T r of the GPU's segmented Jacobian through
    the same contexts afterwards."""
    import torch
    ctxs = []
    try:
        for i, (M, steps, theta, rho, centre) in enumerate(segs):
            ctx = ww.Context(M, n, g=g, tau=tau, h=h, steps=steps, precision=precision,
                             basis=basis if i == 0 else None)
            ctxs.append(ctx)
            ww.set_segment(ctx, steps, theta, rho, centre, scheme)
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        grad = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        ww.objective_and_grad_segments(ctxs, dev(c), f, grad)
        out = (float(f.item()), grad.cpu().numpy())
        ww.objective_and_grad_segments(ctxs, dev(c), f, grad)
        assert float(f.item()) == out[0] and np.array_equal(grad.cpu().numpy(), out[1])
        last = ctxs[-1]
        r = torch.empty(last.N, dtype=torch.float64, device="cuda")
        J = torch.empty(n + 1, last.N, dtype=torch.float64, device="cuda")
        fj = torch.empty(1, dtype=torch.float64, device="cuda")
        ww.shoot_jacobian_segments(ctxs, dev(c), r, J, fj)
        jtr = J.cpu().numpy() @ r.cpu().numpy()
        return out[0], out[1], jtr, float(fj.item())
    finally:
        for ctx in ctxs:
            ctx.close()


_GSPREAD = {}


def check_grad(ww, segs, scheme, n, c, precision, **kw):
    """f at 1e-11 and grad (norm-wise) at max(1e-11, 4 x the oracle's one-ulp
    spread of its own gradient) against the oracle's discrete adjoint, and
    against J^T r of the GPU's segmented Jacobian in the same form."""
    f, g, jtr, fj = gpu_grad_segments(ww, segs, scheme, n, c, precision, **kw)
    prob, keep = O.make_problem(segs[0][0], n, g=kw.get("g", 1.0), tau=kw.get("tau", 0.0), h=kw.get("h", 1.0),
                             basis=kw.get("basis"))
    key = (tuple(segs), scheme, n, tuple(c), tuple(sorted((k, str(v)) for k, v in kw.items())))
    f0, g0 = O.objective_and_grad_segments(prob, segs, scheme, c)
    if key not in _GSPREAD:
        cp = c.copy()
        cp[1] = np.nextafter(c[1], np.inf)
        _, gp = O.objective_and_grad_segments(prob, segs, scheme, cp)
        _GSPREAD[key] = np.linalg.norm(gp - g0) / np.linalg.norm(g0)
    tol = max(TOL, 4.0 * _GSPREAD[key])
    eg = np.linalg.norm(g - g0) / np.linalg.norm(g0)
    ej = np.linalg.norm(g - jtr) / np.linalg.norm(jtr)
    ef = abs(f - f0) / abs(f0)
    print(f"\ngradient {[s[:4] for s in segs]} {scheme} precision={precision}: f {ef:.2e}, grad vs oracle {eg:.2e}, "
          f"vs J^T r {ej:.2e} (tolerance {tol:.2e}; oracle one-ulp spread {_GSPREAD[key]:.2e})")
    assert ef < TOL and abs(f - fj) <= 1e-14 * abs(fj)
    assert eg < tol and ej < tol


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("h,tau,segs", [
    (1.0, 0.0, [(64, 5, 0.375, 1.0, 0), (128, 8, 0.375, 0.4, 0), (128, 6, 0.25, 0.2, 0)]),
    (math.inf, 0.0, [(64, 5, 0.375, 1.0, 0), (128, 8, 0.375, 0.4, 0), (128, 6, 0.25, 0.2, 0)]),
    (0.5, 0.01, [(64, 8, 0.5, 1.0, 1), (128, 24, 0.5, 0.7, 1)]),
])
def test_segmented_gradient_matches_oracle(ww, precision, h, tau, segs):
    """The discrete adjoint of the segmented shot (meshes, respacing, DOP853)
    against the oracle's (orc_objective_and_grad_segments)."""
    N, n = segs[0][0], 12
    w = W.Workload("seg3", N=N, n=n, steps=1, h=h, tau=tau, amp=0.05)
    c, _ = W.coefficients(w)
    check_grad(ww, segs, "dop853", n, c, precision, h=h, tau=tau)


@pytest.mark.parametrize("precision", [0, 1])
def test_segmented_workload_gradient_shrunk(ww, precision):
    """The segmented workload's structure shrunk as in the Jacobian test above."""
    wl = W.SEGMENTED
    segs = [(M // 8, max(2, s // 4), th, rho, ctr) for (M, s, th, rho, ctr) in wl.meta["segments"]]
    N, n = segs[0][0], segs[0][0] // 3
    w = W.Workload("seg_wl", N=N, n=n, steps=1, h=wl.h, amp=0.05)
    c, _ = W.coefficients(w)
    check_grad(ww, segs, wl.meta["tableau"], n, c, precision, h=wl.h)


def test_one_uniform_rk4_segment_gradient_is_the_plain_adjoint(ww):
    """One uniform RK4 segment: the segmented adjoint equals the plain
    objective_and_grad (the same transposed map; its sums round differently)."""
    import torch
    N, n, steps = 64, 8, 16
    w = W.Workload("seg1", N=N, n=n, steps=steps, amp=0.05)
    c, _ = W.coefficients(w)
    for precision in (ww.WW_FP64, ww.WW_MIXED):
        with ww.Context(N, n, steps=steps, precision=precision) as ctx:
            f = torch.empty(1, dtype=torch.float64, device="cuda")
            g = torch.empty(n + 1, dtype=torch.float64, device="cuda")
            ww.objective_and_grad(ctx, dev(c), f, g)
            plain = (float(f.item()), g.cpu().numpy())
        fs, gs, jtr, _ = gpu_grad_segments(ww, [(N, steps, 1.0, 1.0, 1)], "rk4", n, c, precision)
        assert abs(fs - plain[0]) <= 1e-13 * abs(plain[0])
        assert np.linalg.norm(gs - plain[1]) / np.linalg.norm(plain[1]) < 1e-12


def test_contexts_created_largest_first(ww):
    """Kernels shared by contexts of different sizes keep the largest
    shared-memory limit any context asked for: a 2048-point segment set up
    before a 512-point one still runs, with the same result as in the other
    order of creation."""
    import torch
    n = 4
    segs = [(512, 2, 0.5, 1.0, 0), (2048, 2, 0.5, 0.4, 0)]
    w = W.Workload("seg_order", N=512, n=n, steps=1, amp=0.05)
    c, _ = W.coefficients(w)
    c[0] *= 1.0 / 256   # a short shot: two DOP853 steps stay stable on the 2048-point mesh
    results = []
    for order in ((0, 1), (1, 0)):
        made = {}
        try:
            for i in order:
                M, steps, th, rho, ctr = segs[i]
                made[i] = ww.Context(M, n, steps=steps, precision=ww.WW_FP64)
                ww.set_segment(made[i], steps, th, rho, ctr, "dop853")
            ctxs = [made[0], made[1]]
            r = torch.empty(2048, dtype=torch.float64, device="cuda")
            J = torch.empty(n + 1, 2048, dtype=torch.float64, device="cuda")
            f = torch.empty(1, dtype=torch.float64, device="cuda")
            ww.shoot_jacobian_segments(ctxs, dev(c), r, J, f)
            results.append((r.cpu().numpy(), J.cpu().numpy()))
        finally:
            for x in made.values():
                x.close()
    assert np.array_equal(results[0][0], results[1][0]) and np.array_equal(results[0][1], results[1][1])
