"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerance: 1e-11 relative in the FP64 form, measured as ||d r||/||r||,
|d f|/|f| and, per Jacobian column, ||d J_k|| / max(||J_k||, 1e-4 max_j ||J_j||)
(max over k).  The two sides use different summation orders, FFTs, cotangent
formulas and solvers (no pivoting on the GPU, partial pivoting in the
oracle), so agreement is at the roundoff floor of the method, not bitwise.
The column floor 1e-4 max_j ||J_j|| covers columns that are small through
cancellation (the d/dT column of a near-linear wave is 1e-5 of the others);
their roundoff is set by the size of the terms that cancel: perturbing c by
one ulp moves that column of the ORACLE itself by 2e-11 of its norm.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def ww():
    import torch
    assert torch.cuda.is_available()
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as m
    m.lib()
    return m


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def x_grid(N):
    return 2 * np.pi * np.arange(N) / N


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def col_rel(J, J0):
    norms = np.linalg.norm(J0, axis=0)
    floor = 1e-4 * norms.max()
    return max(np.linalg.norm(J[:, k] - J0[:, k]) / max(norms[k], floor) for k in range(J0.shape[1]))


def stable_T(N, steps, g=1.0, tau=0.0, h=1.0, cfl=1.2):
    """A period T whose RK4 step dt = T / (4 steps) keeps omega_max dt = cfl, with
    omega_max^2 = (g k + tau k^3) tanh(k h) at k = N/2 (RK4 is stable to 2.83):
    parity is compared on the same discrete map, so T is just a parameter."""
    k = N / 2
    wmax = math.sqrt((g * k + tau * k**3) * (1.0 if math.isinf(h) else math.tanh(k * h)))
    return 4 * steps * cfl / wmax


def gpu_jacobian(ww, w, c, precision=0, basis=None, verify=0, **kw):
    with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, basis=basis, precision=precision,
                    **kw) as ctx:
        if verify:
            ctx.set_verify(verify)
        r, J, f = ctx.empty_outputs()
        ww.shoot_jacobian(ctx, dev(c), r, J, f)
        st = ctx.stats()
        return r.cpu().numpy(), J.cpu().numpy().T.copy(), float(f.item()), st


# ------------------------------------------------------------------ DtN
@pytest.mark.parametrize("N,h", [(64, 1.0), (256, 0.3), (64, math.inf), (1024, 0.05)])
def test_dtn_flat_symbol(ww, N, h):
    x = x_grid(N)
    eta = np.full(N, 0.0 if math.isinf(h) else h)
    ks = [1, 2, 5, N // 4 - 1]
    phi = np.stack([np.cos(k * x) for k in ks])
    with ww.Context(N, len(ks) + 2, h=h) as ctx:
        ww.dtn_setup(ctx, dev(eta))
        out = ww.dtn_apply(ctx, dev(phi)).cpu().numpy()
    for row, k in zip(out, ks):
        sym = k if math.isinf(h) else k * math.tanh(k * h)
        assert np.max(np.abs(row - sym * np.cos(k * x))) < 2e-12 * max(1, sym), k


@pytest.mark.parametrize("N,h,nrhs", [(64, 1.0, 7), (512, 1.0, 37), (128, math.inf, 5), (512, 0.4, 1)])
def test_dtn_apply_matches_oracle(ww, N, h, nrhs):
    """Random smooth surface and data; nrhs spans several 64-column tiles with a ragged tail."""
    rng = np.random.default_rng(N + nrhs)
    x = x_grid(N)
    eta = (0.0 if math.isinf(h) else h) + sum(0.1 / k**2 * rng.uniform(-1, 1) * np.cos(k * x) for k in range(1, 9))
    phi = np.stack([sum(rng.uniform(-1, 1) / k**2 * np.cos(k * x + rng.uniform(0, 6)) for k in range(1, 12))
                    for _ in range(nrhs)])
    with ww.Context(N, nrhs, h=h) as ctx:
        ww.dtn_setup(ctx, dev(eta))
        got = ww.dtn_apply(ctx, dev(phi)).cpu().numpy()
    ref = O.dtn(eta, phi, h)
    for a, b in zip(got, ref):
        assert rel(a, b) < 1e-12


def test_dtn_geometry_error(ww):
    N = 64
    x = x_grid(N)
    with ww.Context(N, 2, h=1.0) as ctx:
        with pytest.raises(ww.WWError) as ei:
            ww.dtn_setup(ctx, dev(0.5 * np.cos(x)))   # touches the bottom (eta <= 0)
        assert ei.value.code == -2
        eta = np.full(N, 1.0)
        eta[3] = np.nan
        with pytest.raises(ww.WWError):
            ww.dtn_setup(ctx, dev(eta))
        with pytest.raises(ww.WWError) as ei:
            ww.dtn_apply(ctx, dev(np.zeros((1, N))))   # no valid setup
        assert ei.value.code == -1


def test_bad_sizes_rejected(ww):
    for kw in ({"N": 100, "n": 4}, {"N": 8, "n": 4}, {"N": 64, "n": -1}, {"N": 64, "n": 4, "steps": 0},
               {"N": 64, "n": 4, "h": -1.0}, {"N": 64, "n": 4, "precision": 7}):
        with pytest.raises(ww.WWError) as ei:
            ww.Context(**kw)
        assert ei.value.code == -1


# ------------------------------------------------------------------ Jacobian
def test_small_workload_jacobian(ww):
    """N = 64, 12 modes + T, 64 RK4 steps, h = 1 (the small benchmark shape)."""
    w = W.SMALL
    c, _ = W.coefficients(w)
    r, J, f, _ = gpu_jacobian(ww, w, c)
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    assert rel(r, r0) < TOL and abs(f - f0) / f0 < TOL
    assert col_rel(J, J0) < TOL


@pytest.mark.parametrize("N,n,steps,h,tau,amp", [
    (256, 70, 8, 1.0, 0.0, 0.2),       # several 64-wide tiles, ragged tail (71 columns)
    (128, 20, 16, math.inf, 0.1, 0.1),  # deep water with surface tension
    (512, 33, 4, 0.3, 0.05, 0.05),      # shallower, tension, odd column count
])
def test_jacobian_matches_oracle(ww, N, n, steps, h, tau, amp):
    w = W.Workload("t", N=N, n=n, steps=steps, h=h, tau=tau, amp=amp)
    c, _ = W.coefficients(w)
    c[0] = min(c[0], stable_T(N, steps, tau=tau, h=h))
    r, J, f, _ = gpu_jacobian(ww, w, c)
    prob, _ = O.make_problem(N, n, g=w.g, tau=tau, h=h, steps=steps)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    assert rel(r, r0) < TOL and abs(f - f0) / f0 < TOL
    assert col_rel(J, J0) < TOL


def test_custom_basis_and_phi_initial_data(ww):
    """Paper's own parameterisation (Eq. init:stand): even modes on eta, odd on phi."""
    N, n, steps = 64, 6, 12
    x = x_grid(N)
    B = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        if k % 2 == 0:
            B[:N, k - 1] = 2 * np.cos(k * x)
        else:
            B[N:, k - 1] = 2 * np.cos(k * x)
    c = np.array([7.2, 0.01, 0.02, -0.003, 0.001, 0.0004, -0.0001])
    w = W.Workload("t", N=N, n=n, steps=steps)
    r, J, f, _ = gpu_jacobian(ww, w, c, basis=B)
    prob, keep = O.make_problem(N, n, steps=steps, basis=B)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    assert rel(r, r0) < TOL and abs(f - f0) / f0 < TOL and col_rel(J, J0) < TOL


def test_shoot_and_gradient_consistent(ww):
    import torch
    w = W.shrink(W.MEDIUM, N=128, n=16, steps=8)
    c, _ = W.coefficients(w)
    with ww.Context(w.N, w.n, h=w.h, steps=w.steps) as ctx:
        ct = dev(c)
        r, J, f = ctx.empty_outputs()
        ww.shoot_jacobian(ctx, ct, r, J, f)
        r2 = torch.empty_like(r)
        f2 = torch.empty_like(f)
        ww.shoot(ctx, ct, r2, f2)
        grad = torch.empty(w.n + 1, dtype=torch.float64, device="cuda")
        f3 = torch.empty_like(f)
        ww.objective_and_grad(ctx, ct, f3, grad)
        cg = ct.clone().requires_grad_(True)
        fa = ww.shooting_objective(cg, ctx)
        fa.backward()
    r, J, r2 = r.cpu().numpy(), J.cpu().numpy().T, r2.cpu().numpy()
    assert np.array_equal(r, r2) and f.item() == f2.item() == f3.item()
    jtr = J.T @ r
    assert rel(grad.cpu().numpy(), jtr) < 1e-13
    assert rel(cg.grad.cpu().numpy(), jtr) < 1e-13 and fa.item() == f.item()


def gpu_gradient(ww, w, c, precision=0, basis=None):
    import torch
    with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, basis=basis, precision=precision) as ctx:
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        grad = torch.empty(w.n + 1, dtype=torch.float64, device="cuda")
        ww.objective_and_grad(ctx, dev(c), f, grad)
        return float(f.item()), grad.cpu().numpy(), ctx.stats()


def paper_basis(N, n):
    # Eq. (init:stand): even k on eta, odd k on phi
    x = x_grid(N)
    B = np.zeros((2 * N, n))
    for k in range(1, n + 1):
        B[(0 if k % 2 == 0 else N):(N if k % 2 == 0 else 2 * N), k - 1] = 2 * np.cos(k * x)
    return B


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("h,tau,amp,phi_basis", [
    (0.3, 0.05, 0.05, False),          # shallow with surface tension
    (math.inf, 0.1, 0.05, False),      # deep water with surface tension
    (1.0, 0.0, 0.05, True),            # phi components in the basis
])
def test_adjoint_gradient_matches_oracle(ww, precision, h, tau, amp, phi_basis):
    """objective_and_grad (the discrete adjoint, reading R18) against the oracle's
    discrete adjoint, f and every gradient entry (the T entry included)."""
    N, n, steps = 64, 12, 24
    w = W.Workload("adj", N=N, n=n, steps=steps, h=h, tau=tau, amp=amp)
    c, _ = W.coefficients(w)
    c[0] = stable_T(N, steps, w.g, tau, h)   # RK4 inside its stability region at this N
    B = paper_basis(N, n) if phi_basis else None
    f, g, st = gpu_gradient(ww, w, c, precision, B)
    prob, keep = O.make_problem(N, n, g=w.g, tau=tau, h=h, steps=steps, basis=B)
    f0, g0 = O.objective_and_grad(prob, c)
    assert abs(f - f0) / f0 < TOL
    assert rel(g, g0) < TOL
    assert np.max(np.abs(g - g0)) < TOL * np.max(np.abs(g0))
    assert st["stages"] == 8 * steps and st["launches"] > 0


@pytest.mark.slow
@pytest.mark.parametrize("wl", ["N1024_n256_steps2048_h0.05", "N1024_n256_steps2048_deep_tau0.1"])
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_full_size_two_steps(ww, wl, precision):
    """The gradient workloads at full size (N = 1024, 256 modes + T) in the
    launch configuration the benchmark times, for TWO RK4 steps of the full
    run's dt (T scaled by 2/2048; the oracle cannot run 2048 steps at N = 1024),
    against the oracle's discrete adjoint."""
    full = W.ALL[wl]
    w = W.shrink(full, steps=2)
    c, _ = W.coefficients(full)
    c[0] *= 2 / full.steps
    f, g, _ = gpu_gradient(ww, w, c, precision)
    if wl not in _ADJ_ORACLE:
        prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
        _ADJ_ORACLE[wl] = O.objective_and_grad(prob, c)
    f0, g0 = _ADJ_ORACLE[wl]
    assert abs(f - f0) / f0 < TOL
    assert rel(g, g0) < TOL


_ADJ_ORACLE = {}


@pytest.mark.slow
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_jacobian_workload_one_step(ww, precision):
    """The gradient at the Jacobian benchmark's size (N = 2048, 512 modes + T)
    for ONE RK4 step of the full run's dt, against the oracle's discrete adjoint."""
    w = W.shrink(W.LARGE, steps=1)
    c, _ = W.coefficients(W.LARGE)
    c[0] /= W.LARGE.steps
    f, g, _ = gpu_gradient(ww, w, c, precision)
    if "large1" not in _ADJ_ORACLE:
        prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=1)
        _ADJ_ORACLE["large1"] = O.objective_and_grad(prob, c)
    f0, g0 = _ADJ_ORACLE["large1"]
    assert abs(f - f0) / f0 < TOL
    assert rel(g, g0) < TOL


def test_adjoint_two_chain_sweep_matches_one_chain_sweep(ww):
    """The mixed form's reverse sweep on the context's own stream runs as two
    chains (each stage's DtN setup one stage ahead, operands double-buffered by
    stage parity); on the legacy default stream it runs as one chain without
    graphs.  Both refine every solve to 1e-13, so the gradients agree to that
    level (their approximate inverses start from different surfaces), and both
    match the oracle.  N = 512 takes the cluster kernels."""
    import torch
    w = W.Workload("adj2", N=512, n=24, steps=6, h=math.inf, tau=0.1, amp=0.05, law="decay")
    c, _ = W.coefficients(w)
    c[0] = stable_T(w.N, w.steps, w.g, w.tau, w.h)
    out = []
    for legacy in (False, True):
        with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=ww.WW_MIXED) as ctx:
            if legacy:
                ctx.set_stream(None)
            f = torch.empty(1, dtype=torch.float64, device="cuda")
            g = torch.empty(w.n + 1, dtype=torch.float64, device="cuda")
            ww.objective_and_grad(ctx, dev(c), f, g)
            torch.cuda.synchronize()
            out.append((f.item(), g.cpu().numpy()))
    (f1, g1), (f2, g2) = out
    assert f1 == f2
    assert rel(g1, g2) < 1e-12
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    f0, g0 = O.objective_and_grad(prob, c)
    assert rel(g1, g0) < TOL and rel(g2, g0) < TOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N,h,tau,legacy", [
    (64, 0.3, 0.05, False),            # one-CTA transforms, shallow with tension
    (512, math.inf, 0.1, False),       # 8-CTA cluster transforms, deep water with tension
    (64, 1.0, 0.0, True),              # legacy default stream: one chain, no graphs
])
def test_adjoint_checkpointed_matches_resident(ww, precision, N, h, tau, legacy):
    """objective_and_grad with the base state checkpointed every K steps and each
    segment's records recomputed (Sec. 3.2's mile-markers; 18 steps, K = 4: four
    full segments and a ragged last one of 2 steps) against the resident
    record of every stage: bitwise in the FP64 form, to the refinement's level
    in the mixed form (each recomputed segment restarts its approximate
    inverse), and both against the oracle's discrete adjoint.  The workspace
    shrinks from 4 x 18 stage records to 4 x 4 plus 5 checkpoints."""
    import torch
    steps, K, n = 18, 4, 12
    w = W.Workload("ckpt", N=N, n=n, steps=steps, h=h, tau=tau, amp=0.05,
                   law="power" if N < 512 else "decay")
    c, _ = W.coefficients(w)
    c[0] = stable_T(N, steps, w.g, tau, h)
    out = []
    for every in (0, K):
        with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=precision) as ctx:
            if legacy:
                ctx.set_stream(None)
            ctx.set_checkpoint(every)
            f = torch.empty(1, dtype=torch.float64, device="cuda")
            g = torch.empty(w.n + 1, dtype=torch.float64, device="cuda")
            ww.objective_and_grad(ctx, dev(c), f, g)
            g_first = g.cpu().numpy()
            ww.objective_and_grad(ctx, dev(c), f, g)    # a second call reuses the workspace and graphs
            torch.cuda.synchronize()
            st = ctx.stats()
            assert np.array_equal(g.cpu().numpy(), g_first)
            out.append((f.item(), g.cpu().numpy(), st))
    (f1, g1, s1), (f2, g2, s2) = out
    rec = 4 * 6 * N * 8                      # bytes of one step's records
    assert s1["adjoint_bytes"] - s2["adjoint_bytes"] >= (steps - K) * rec - 5 * 2 * N * 8
    if precision == 0:
        assert f1 == f2 and np.array_equal(g1, g2)
    else:
        assert f1 == f2 and rel(g1, g2) < 1e-12
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    f0, g0 = O.objective_and_grad(prob, c)
    assert abs(f2 - f0) / f0 < TOL and rel(g2, g0) < TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_of_uneven_shots_matches_single_shots(ww, precision):
    """shoot_jacobian_batch: independent shots of uneven size and step count
    (the uneven-batch recipe at N = 128..512, 5..8 steps of each shot's own dt,
    every other shot on a non-default schedule) run as ONE graph launch give
    bitwise the results of shoot_jacobian on each context, also on a second
    call (the cached batch graph); one shot is also checked against the
    oracle."""
    shots = W.uneven_shots(n_shots=6, seed=5, step_cap=8, sizes=(128, 256, 512))
    shots = [(W.shrink(w, steps=w.steps - (i % 4), name=w.name), c * np.r_[(w.steps - (i % 4)) / w.steps,
                                                                         np.ones(w.n)])
             for i, (w, c) in enumerate(shots)]
    assert len({w.N for w, _ in shots}) > 1 and len({w.n for w, _ in shots}) > 1
    assert len({w.steps for w, _ in shots}) > 1
    ctxs = [ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=precision) for w, _ in shots]
    try:
        for i, ctx in enumerate(ctxs[1::2]):
            if precision == ww.WW_MIXED:
                ctx.set_schedule(**[dict(overlap=0), dict(corr_bn=32, inv_bn=64), dict(ns_every=1, corr_bn=128)][i % 3])
            else:
                ctx.set_schedule(lu_nb=32)
        cs = [dev(c) for _, c in shots]
        single = []
        for ctx, c in zip(ctxs, cs):
            r, J, f = ctx.empty_outputs()
            ww.shoot_jacobian(ctx, c, r, J, f)
            single.append((r.cpu().numpy(), J.cpu().numpy(), f.item()))
        outs = [ctx.empty_outputs() for ctx in ctxs]
        for _ in range(2):
            for o in outs:
                for t in o:
                    t.fill_(float("nan"))
            ww.shoot_jacobian_batch(ctxs, cs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
            for (r0, J0, f0), (r, J, f) in zip(single, outs):
                assert np.array_equal(r.cpu().numpy(), r0) and np.array_equal(J.cpu().numpy(), J0)
                assert f.item() == f0
        st = ctxs[0].stats()
        assert st["stages"] == 4 * shots[0][0].steps and st["launches"] > 8 * st["stages"]
        with pytest.raises(ww.WWError) as ei:   # a context may appear once
            dup = [outs[0], outs[1], outs[0]]
            ww.shoot_jacobian_batch(ctxs[:2] + ctxs[:1], cs[:2] + cs[:1], [o[0] for o in dup],
                                    [o[1] for o in dup], [o[2] for o in dup])
        assert ei.value.code == -1
    finally:
        for ctx in ctxs:
            ctx.close()
    i = min(range(len(shots)), key=lambda k: shots[k][0].N)
    w, c = shots[i]
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    r, J, f = outs[i]
    assert rel(r.cpu().numpy(), r0) < TOL and abs(f.item() - f0) / f0 < TOL
    assert col_rel(J.cpu().numpy().T, J0) < TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_schedules_agree_and_autotune_caches(ww, precision, tmp_path):
    """Every schedule computes the same Jacobian (to the refinement's level in
    the mixed form: other tiles round the FP32 corrections differently, and
    bitwise in the FP64 form across LU block sizes up to the LU's rounding);
    ww_autotune picks one, appends it to its cache file, and takes it from
    there without timing on the next call."""
    w = W.Workload("sched", N=256, n=40, steps=6, h=0.8, amp=0.1)
    c, _ = W.coefficients(w)
    c[0] = stable_T(w.N, w.steps, h=w.h)
    prob, _ = O.make_problem(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    if precision == ww.WW_MIXED:
        variants = [dict(), dict(overlap=0), dict(ns_every=1), dict(corr_bn=32), dict(corr_bn=128),
                    dict(inv_bn=64), dict(inv_bn=256, inv_ctas=1), dict(inv_ctas=1), dict(inv_bn=64, inv_ctas=1),
                    dict(prio=0), dict(ns_every=0)]
    else:
        variants = [dict(), dict(lu_nb=32)]
    with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=precision) as ctx:
        default = ctx.schedule()
        for v in variants:
            ctx.set_schedule(**{**default, **v})
            r, J, f = ctx.empty_outputs()
            ww.shoot_jacobian(ctx, dev(c), r, J, f)
            assert rel(r.cpu().numpy(), r0) < TOL and abs(f.item() - f0) / f0 < TOL, v
            assert col_rel(J.cpu().numpy().T, J0) < TOL, v
        with pytest.raises(ww.WWError):
            ctx.set_schedule(corr_bn=48)
        with pytest.raises(ww.WWError):
            ctx.set_schedule(inv_bn=256, inv_ctas=2)
        cache = tmp_path / "tune.txt"
        ms = ctx.autotune(dev(c), probe_steps=2, cache_path=str(cache))
        chosen = ctx.schedule()
        lines = cache.read_text().splitlines()
        assert ms > 0 and len(lines) == 1
        assert lines[0].split()[:4] == ["v2", str(w.N), str(w.n + 1), "mixed" if precision else "fp64"]
        ctx.set_schedule(**default)
        assert ctx.autotune(dev(c), probe_steps=2, cache_path=str(cache)) == 0.0   # from the cache
        assert ctx.schedule() == chosen and len(cache.read_text().splitlines()) == 1
        r, J, f = ctx.empty_outputs()
        ww.shoot_jacobian(ctx, dev(c), r, J, f)
        assert col_rel(J.cpu().numpy().T, J0) < TOL


def test_column_split_engine_on_gpu(ww):
    """The column split's sub-problems on the library (single rank: all mode
    columns through the combined-shape basis) give the unsharded Jacobian."""
    from paper_1210_5672_gb300.sharding import gpu_engine, sharded_jacobian
    N, n, steps = 128, 12, 8
    w = W.Workload("shard", N=N, n=n, steps=steps, amp=0.05)
    c, _ = W.coefficients(w)
    basis = np.zeros((2 * N, n))
    x = x_grid(N)
    for k in range(1, n + 1):
        basis[:N, k - 1] = np.cos(k * x)
    r, J, f = sharded_jacobian(c, basis, gpu_engine(N, h=w.h, steps=steps), 0, 1)
    r0, J0, f0, _ = gpu_jacobian(ww, w, c, basis=basis)
    # the initial states differ by rounding (the shape is summed once on the host)
    assert rel(r, r0) < 1e-13 and abs(f - f0) <= 1e-13 * f0
    assert col_rel(J, J0) < TOL


def test_host_entry_point_matches_device(ww):
    w = W.shrink(W.MEDIUM, N=128, n=10, steps=4)
    c, _ = W.coefficients(w)
    with ww.Context(w.N, w.n, h=w.h, steps=w.steps) as ctx:
        r, J, f = ctx.empty_outputs()
        ww.shoot_jacobian(ctx, dev(c), r, J, f)
        rh, Jh, fh = np.empty(w.N), np.empty((w.n + 1, w.N)), np.empty(1)
        ww.shoot_jacobian_host(ctx, np.ascontiguousarray(c), rh, Jh, fh)
    assert np.array_equal(rh, r.cpu().numpy()) and np.array_equal(Jh, J.cpu().numpy()) and fh[0] == f.item()


def test_geometry_failure_in_shot_reports_status(ww):
    """Initial surface below the bottom: the shot returns WW_ERR_GEOMETRY (read
    from the device status word) instead of producing garbage."""
    N, n = 64, 2
    c = np.array([8.0, 1.2, 0.0])
    with ww.Context(N, n, h=1.0, steps=4) as ctx:
        r, J, f = ctx.empty_outputs()
        with pytest.raises(ww.WWError) as ei:
            ww.shoot_jacobian(ctx, dev(c), r, J, f)
        assert ei.value.code == -2


@pytest.mark.slow
def test_large_workload_one_step_sampled(ww):
    """Full-size shape (N = 2048, 512 modes + T) in the benchmark's launch
    configuration for ONE RK4 step of the full run's dt (T scaled by 1/1024;
    the oracle cannot run 1024 steps); every column compared, plus r and f."""
    w = W.shrink(W.LARGE, steps=1)
    c, _ = W.coefficients(W.LARGE)
    c[0] /= W.LARGE.steps
    r, J, f, _ = gpu_jacobian(ww, w, c)
    prob, _ = O.make_problem(w.N, w.n, h=w.h, steps=1)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    assert rel(r, r0) < TOL and abs(f - f0) / f0 < TOL
    assert col_rel(J, J0) < TOL


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("N,n,steps,h,tau,amp", [
    (64, 12, 64, 1.0, 0.0, 0.01),       # the small workload shape
    (256, 70, 8, 1.0, 0.0, 0.2),        # several tiles, ragged tail
    (128, 20, 16, math.inf, 0.1, 0.1),  # deep water with surface tension
])
def test_mixed_jacobian_matches_oracle(ww, N, n, steps, h, tau, amp):
    """WW_MIXED: FP32-accurate tensor-core inverse + FP64-accurate digit
    residuals and G products, refined to 1e-13; same 1e-11 bar as FP64."""
    w = W.Workload("t", N=N, n=n, steps=steps, h=h, tau=tau, amp=amp)
    c, _ = W.coefficients(w)
    c[0] = min(c[0], stable_T(N, steps, tau=tau, h=h))
    r, J, f, st = gpu_jacobian(ww, w, c, precision=1)
    prob, _ = O.make_problem(N, n, g=w.g, tau=tau, h=h, steps=steps)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    assert st["refine_resid_max"] <= 1e-13
    assert rel(r, r0) < TOL and abs(f - f0) / f0 < TOL
    assert col_rel(J, J0) < TOL
    # the refinement's residual MEASURED after its last correction (every stage
    # sampled): R = Psi - A M recomputed, FP64-accurate, relative to
    # max|Psi_j| + max|M_j|; the measurement only reads, so the results are
    # bitwise those of the unmeasured program
    rv, Jv, fv, sv = gpu_jacobian(ww, w, c, precision=1, verify=1)
    print(f"\nN={N} n={n}: estimated residual {st['refine_resid_max']:.2e}, measured "
          f"{sv['refine_resid_measured']:.2e} over {sv['verified_solves']} solves")
    assert sv["verified_solves"] == 4 * steps
    assert 0 <= sv["refine_resid_measured"] <= 1e-13
    assert np.array_equal(rv, r) and np.array_equal(Jv, J) and fv == f


def test_mixed_dtn_apply_matches_oracle(ww):
    N, nrhs, h = 512, 37, 1.0
    rng = np.random.default_rng(5)
    x = x_grid(N)
    eta = h + sum(0.1 / k**2 * rng.uniform(-1, 1) * np.cos(k * x) for k in range(1, 9))
    phi = np.stack([sum(rng.uniform(-1, 1) / k**2 * np.cos(k * x + rng.uniform(0, 6)) for k in range(1, 12))
                    for _ in range(nrhs)])
    with ww.Context(N, nrhs, h=h, precision=1) as ctx:
        ww.dtn_setup(ctx, dev(eta))
        got = ww.dtn_apply(ctx, dev(phi)).cpu().numpy()
    ref = O.dtn(eta, phi, h)
    for a, b in zip(got, ref):
        assert rel(a, b) < 1e-12


@pytest.mark.parametrize("mixed", [False, True])
def test_phase_timing_and_launch_count(ww, mixed):
    """Every phase is timed once per RK stage; the product-kernel phase sits inside
    the G-apply phase; the library's launch count covers all stages."""
    w = W.shrink(W.SMALL, N=128, n=12, steps=4)
    c, _ = W.coefficients(w)
    c[0] = stable_T(w.N, w.steps)
    prec = ww.WW_MIXED if mixed else ww.WW_FP64
    with ww.Context(w.N, w.n, g=w.g, tau=w.tau, h=w.h, steps=w.steps, precision=prec) as ctx:
        ctx.set_timing(True)
        r, J, f = ctx.empty_outputs()
        ww.shoot_jacobian(ctx, dev(c), r, J, f)
        t, st = ctx.timing(), ctx.stats()
        ww.shoot(ctx, dev(c), r, f)
        st_shoot = ctx.stats()
    stages = 4 * w.steps
    for p in ww.PHASES:
        if p == "inverse":
            # the FP64 form has no inverse update; the mixed form's default schedule
            # times the guaranteed updates of the even stages (the odd ones run only
            # when the inverse drifted, decided on the device)
            assert t[p][1] == (0 if not mixed else stages // 2), (p, t[p])
            continue
        assert t[p][1] == stages, p
        assert t[p][0] > 0, p
    assert t["gkernel"][0] <= t["gapply"][0]
    if mixed:
        assert t["inverse"][0] <= t["factor"][0]
    assert st["stages"] == stages
    # at least geometry, assembly, the factor/inverse, base chain and column work per stage
    assert st["launches"] >= 8 * stages
    assert 0 < st_shoot["launches"] < st["launches"]
