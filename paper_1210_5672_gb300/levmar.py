"""Levenberg-Marquardt with delayed Jacobian updates (App. D, "Levenberg-Marquardt
implementation with delayed Jacobian updates"): the nonlinear least-squares solver
around the shooting Jacobian, minimising f(c) = r(c).r(c)/2 over the unknown
parameters.

Each step minimises the quadratic model f + g.p + p.B.p/2 (g = J^T r, B = J^T J)
over the trust region |p| <= Delta, written as the damped least-squares problem
min |[J; sqrt(lam) I] p + [r; 0]| with lam >= 0, lam (|p| - Delta) = 0.  With the
thin SVD J = U S V^T (computed once per Jacobian) the problem is diagonal:
p~ = V^T p, r~ = U^T r, p~_i(lam) = -s_i r~_i / (s_i^2 + lam), and lam solves
tau(lam) = 1/|p~| - 1/Delta = 0 by Newton's iteration from lam = 0, which
increases monotonically to the root because tau is increasing and concave.

The Jacobian is kept for several steps and recomputed only when it stops
paying (the delayed updates of the same appendix): the design decisions 1-4
there (termination, radius update, when to recompute J, when to compute r only)
are implemented literally, with the parameters printed there as defaults.

Reading (the printed Newton update is garbled): the update is
  lam <- lam + (p~.p~ / sum_i p~_i^2 / (s_i^2 + lam)) (|p~| - Delta) / Delta,
i.e. the denominator is p~^T (S^T S + lam I)^{-1} p~, the derivative of tau;
the printed form lacks the inverse, which would not be Newton's method for tau.

The solver is generic: `levmar` takes two callables (residual, and residual
with Jacobian) on numpy vectors.  `solve_standing_wave` drives it with the GPU
library's `shoot` and `shoot_jacobian` for the standing-wave problem of Sec. 3
with some parameters held fixed (the amplitude of a continuation step), and
`continue_branch` follows a family of solutions in one parameter.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class LMOptions:
    f_tol: float = 1e-26
    g_tol: float = 1e-13
    max_stepsJ: int = 10
    df_tol: float = 1e-5
    rho0: float = 0.25
    alpha0: float = 0.375
    rho1: float = 0.85
    alpha1: float = 1.875
    alpha2: float = 0.2
    lam_tol: float = 1e-12
    max_steps: int = 200


@dataclass
class LMResult:
    c: np.ndarray
    r: np.ndarray
    f: float
    jacobians: int          # Jacobian evaluations
    residuals: int          # residual-only evaluations
    steps: int              # trial steps
    accepted: int
    reason: str
    history: list = field(default_factory=list)   # (f, Delta, accepted, stepsJ) per trial step


def trust_region_step(U, s, V, r, delta, lam_tol=1e-12, max_newton=200):
    """Minimise f + g.p + p.B.p/2 over |p| <= delta from the thin SVD of J.
    Returns (p, lam, df) with df = g.p + p.B.p/2 the predicted change of f."""
    rt = U.T @ r
    s = np.asarray(s, dtype=np.float64)
    ok = s > 0
    pt = np.zeros_like(s)
    pt[ok] = -rt[ok] / s[ok]            # lam = 0: the Gauss-Newton step
    lam = 0.0
    nrm = np.linalg.norm(pt)
    if nrm > delta:
        for _ in range(max_newton):
            if abs((nrm - delta) / delta) <= lam_tol:
                break
            q2 = np.sum(pt[ok] ** 2 / (s[ok] ** 2 + lam))     # p~^T (S^2 + lam)^-1 p~
            lam += (nrm * nrm / q2) * (nrm - delta) / delta
            pt = np.zeros_like(s)
            pt[ok] = -s[ok] * rt[ok] / (s[ok] ** 2 + lam)
            nrm = np.linalg.norm(pt)
    p = V @ pt
    df = float(np.sum(s * rt * pt) + 0.5 * np.sum((s * pt) ** 2))
    return p, lam, df


def levmar(residual, residual_and_jacobian, c0, delta0, opts: LMOptions | None = None) -> LMResult:
    """Minimise f(c) = |r(c)|^2 / 2 from c0 with initial trust radius delta0.
    residual(c) -> r; residual_and_jacobian(c) -> (r, J) (J: len(r) x len(c))."""
    o = opts or LMOptions()
    c = np.array(c0, dtype=np.float64)
    delta = float(delta0)
    r, J = residual_and_jacobian(c)
    f = 0.5 * float(r @ r)
    U, s, Vt = np.linalg.svd(J, full_matrices=False)
    V = Vt.T
    nJ, nr, nsteps, nacc = 1, 0, 0, 0
    stepsJ = 0
    roundoff = False
    accepted_since_J = False
    first_rejected = None          # the first rejected radius after (or with) an accepted step
    trigger = None                 # alpha2 * first_rejected
    history = []
    reason = "max_steps"
    while nsteps < o.max_steps:
        if f == 0.0:
            reason = "f == 0"
            break
        p, lam, df = trust_region_step(U, s, V, r, delta, o.lam_tol)
        if stepsJ == 0:
            g = V @ (s * (U.T @ r))
            if np.linalg.norm(g) < o.g_tol or abs(df) / f < o.df_tol:
                roundoff = True
        c_new = c + p
        if np.array_equal(c_new, c):
            reason = "c unchanged"
            break
        r_new = residual(c_new)
        nr += 1
        nsteps += 1
        f_new = 0.5 * float(r_new @ r_new)
        rho = (f_new - f) / df if df != 0.0 else -1.0
        accepted = rho > 0.0
        pn = float(np.linalg.norm(p))
        # radius: shrink on a rejected radius, grow on a good full step
        if rho < o.rho0:
            if first_rejected is None and (accepted_since_J or accepted):
                first_rejected = delta
                trigger = o.alpha2 * first_rejected
            delta = o.alpha0 * pn
        elif rho > o.rho1 and pn > 0.9 * delta:
            delta *= o.alpha1
        if accepted:
            c, r, f = c_new, r_new, f_new
            stepsJ += 1
            nacc += 1
            accepted_since_J = True
        history.append((f, delta, accepted, stepsJ))
        if f < o.f_tol or delta < o.g_tol:
            roundoff = True
        if f == 0.0:
            reason = "f == 0"
            break
        if roundoff and (not accepted or stepsJ >= o.max_stepsJ):
            reason = "roundoff regime"
            break
        recompute = (not roundoff) and (stepsJ >= o.max_stepsJ
                                        or (stepsJ > 0 and trigger is not None and delta < trigger)
                                        or (stepsJ > 0 and abs(df) / f < o.df_tol))
        if recompute:
            if first_rejected is not None:
                delta = first_rejected / o.alpha1
            r, J = residual_and_jacobian(c)
            f = 0.5 * float(r @ r)
            U, s, Vt = np.linalg.svd(J, full_matrices=False)
            V = Vt.T
            nJ += 1
            stepsJ = 0
            accepted_since_J = False
            first_rejected = None
            trigger = None
    return LMResult(c=c, r=r, f=f, jacobians=nJ, residuals=nr, steps=nsteps, accepted=nacc, reason=reason,
                    history=history)


def continue_branch(solve, c_a, c_b, index, values):
    """Numerical continuation of a solution family in the parameter c[index]
    (the bifurcation parameter, held fixed in each solve; Sec. 4 follows the
    families of standing waves this way): each next solution is predicted by
    linear extrapolation in that parameter from the last two solutions and
    corrected by solve(c_guess) -> LMResult (with the full c in .c).  With small
    enough steps the prediction is close enough that one Jacobian per solution
    suffices (the delayed updates of App. D).  Returns the LMResults at `values`."""
    prev = np.array(c_a, dtype=np.float64)
    cur = np.array(c_b, dtype=np.float64)
    out = []
    for v in values:
        dp = cur[index] - prev[index]
        guess = cur + (cur - prev) * ((v - cur[index]) / dp)
        guess[index] = v
        res = solve(guess)
        out.append(res)
        prev, cur = cur, np.array(res.c, dtype=np.float64)
    return out


def solve_standing_wave(ctx, c0, free, delta0=1e-2, opts: LMOptions | None = None) -> LMResult:
    """Solve for a standing wave on the GPU: minimise f over the entries of c
    listed in `free` (indices into c = (T, c_1..c_n)), the others held at c0's
    values (e.g. the amplitude c_1 of a continuation step).  ctx is a
    paper_1210_5672_gb300.Context whose basis and physics define the problem."""
    import torch

    import paper_1210_5672_gb300 as ww

    c0 = np.asarray(c0, dtype=np.float64)
    free = np.asarray(free, dtype=np.int64)
    dev = torch.device("cuda")
    r_d = torch.empty(ctx.N, dtype=torch.float64, device=dev)
    f_d = torch.empty(1, dtype=torch.float64, device=dev)
    J_d = torch.empty((ctx.n + 1, ctx.N), dtype=torch.float64, device=dev)

    def full(x):
        c = c0.copy()
        c[free] = x
        return torch.tensor(c, dtype=torch.float64, device=dev)

    def residual(x):
        ww.shoot(ctx, full(x), r_d, f_d)
        return r_d.cpu().numpy()

    def residual_and_jacobian(x):
        ww.shoot_jacobian(ctx, full(x), r_d, J_d, f_d)
        J = J_d.cpu().numpy().T            # N x (n + 1), column k = d r / d c_k
        return r_d.cpu().numpy(), np.ascontiguousarray(J[:, free])

    res = levmar(residual, residual_and_jacobian, c0[free], delta0, opts)
    c = c0.copy()
    c[free] = res.c
    res.c = c
    return res
