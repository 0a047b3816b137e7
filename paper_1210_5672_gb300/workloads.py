"""Seeded synthetic standing-wave inputs shared by the tests, the benchmark and
the oracle checks.

This module holds only the input recipe: sizes, physical parameters, the
seeded Fourier coefficients c_k and the initial period.  It contains none of
the method's arithmetic (no DtN, no time stepping) and imports neither the
CUDA binding nor the oracle.

Recipe (the paper's workloads are Tables param:small / param:large, Sec. 4.6,
where n is about M/3 to M/5; no public dataset exists, so these seeded
shapes stand in for the paper's standing-wave runs):

* grid alpha_j = 2 pi j / N (uniform, xi = alpha), N a power of two;
* eta_0 = hbar + sum_k c_k cos(k x) (hbar = mean depth, 0 in deep water),
  phi_0 = 0; Jacobian column k has initial data (cos(k x), 0);
* c_1 = a, c_k = a^k u_k for k >= 2 (or amp * decay^k * u_k), with
  u_k ~ U(-1, 1) drawn by numpy's PCG64 ``default_rng(seed)``;
* if the depth is finite and min eta_0 < hbar / 2 the draw is repeated with
  seed + 1, seed + 2, ... (the seed actually used is returned);
* T from the linear dispersion relation at k = 1, omega^2 = (g + tau) tanh(h)
  (Eq. lin:soln), or omega^2 = g + tau in deep water;
* the uneven batch (`uneven_shots`): 32 independent shots with N in
  {256, ..., 4096}, 8 to 64 columns, h ~ U(0.1, 2), tau in {0, 0.05},
  c_1 ~ U(0.01, 0.5), steps = max(N/2, (T/4) omega(0.9 N/2) / 2.5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    n: int
    steps: int
    g: float = 1.0
    tau: float = 0.0
    h: float = 1.0               # math.inf => deep water
    amp: float = 0.01            # c_1
    law: str = "power"           # "power": c_k = amp^k u_k; "decay": c_k = amp * decay^k * u_k
    decay: float = 0.8
    seed: int = 0
    meta: dict = field(default_factory=dict, compare=False)


# The five shapes of the benchmark family; the first is small enough for the
# CPU oracle to finish in seconds, the third is the headline workload.
SMALL = Workload("N64_n12_steps64_h1", N=64, n=12, steps=64, amp=0.01)
MEDIUM = Workload("N512_n128_steps512_h1", N=512, n=128, steps=512, amp=0.2)
LARGE = Workload("N2048_n512_steps1024_h1", N=2048, n=512, steps=1024, amp=0.4)
# the gradient workloads.  The shallow one (a wave as tall as the depth) has its
# trough reach the bottom before T/8: only its first 512 steps (T/16 at the
# full dt) can be evaluated; the deep-water one with surface tension runs in full.
SHALLOW = Workload("N1024_n256_steps2048_h0.05", N=1024, n=256, steps=2048, h=0.05,
                   amp=0.05, law="decay")
DEEP_TENSION = Workload("N1024_n256_steps2048_deep_tau0.1", N=1024, n=256, steps=2048,
                        h=math.inf, tau=0.1, amp=0.05, law="decay")

ALL = {w.name: w for w in (SMALL, MEDIUM, LARGE, SHALLOW, DEEP_TENSION)}

# Time segments with adaptive meshes (Sec. 2.2), shaped like the paper's double
# precision run of solution O (Table param:OA): four segments with theta = (0.2,
# 0.3, 0.3, 0.2) of T/4, rho = (1, 0.4, 0.1, 0.1), n about M_1 / 3, steps in the
# printed proportions 192 : 432 : 576 : 480 scaled by M_1 / 4608, for DOP853.
# The grids are powers of two that keep the coarsest spacing from growing (the
# paper's rule M_{l+1} / M_l >= (5 + 3 rho_l) / (5 + 3 rho_{l+1}) when rho
# decreases); the printed last rho of 0.09 would need M_4 slightly above M_3, so
# the last segment keeps rho = 0.1.  Meshes are refined near x = 0, where the
# initial crest of eta_0 = h + sum c_k cos(kx) sits.  Not part of ALL: the RK4
# benchmark never selects it.
SEGMENTED = Workload("N512_n170_segments4_h1", N=512, n=170, steps=186, amp=0.2,
                     meta={"segments": ((512, 21, 0.2, 1.0, 0), (1024, 48, 0.3, 0.4, 0),
                                        (2048, 64, 0.3, 0.1, 0), (2048, 53, 0.2, 0.1, 0)),
                           "tableau": "dop853"})


def spacing_rule_ok(segments) -> bool:
    """Sec. 2.2's rule: where rho decreases from one segment to the next, M
    grows at least by (5 + 3 rho_l) / (5 + 3 rho_{l+1}), so the coarsest spacing
    8 / ((5 + 3 rho) M) never grows."""
    for (Ma, _, _, ra, *_), (Mb, _, _, rb, *_) in zip(segments, segments[1:]):
        if rb < ra and Mb * (5 + 3 * rb) < Ma * (5 + 3 * ra):
            return False
    return True


def linear_period(g: float, tau: float, h: float) -> float:
    """T = 2 pi / omega with omega^2 = (g + tau) tanh(h) at k = 1 (Eq. lin:soln)."""
    w2 = (g + tau) * (1.0 if math.isinf(h) else math.tanh(h))
    return 2.0 * math.pi / math.sqrt(w2)


def grid(N: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(N) / N


def _draw(w: Workload, seed: int) -> np.ndarray:
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, w.n)
    k = np.arange(1, w.n + 1, dtype=np.float64)
    if w.law == "power":
        c = np.power(w.amp, k) * u
        c[0] = w.amp
    else:
        c = w.amp * np.power(w.decay, k) * u
    return c


def coefficients(w: Workload, seed: int | None = None, max_redraw: int = 1000):
    """Return (c, seed_used): c[0] = T, c[1..n] the Fourier coefficients."""
    s0 = w.seed if seed is None else seed
    x = grid(w.N)
    for s in range(s0, s0 + max_redraw):
        ck = _draw(w, s)
        if not math.isinf(w.h):
            # geometry check of the recipe: the surface must stay well above the bottom
            surf = w.h + np.cos(np.outer(x, np.arange(1, w.n + 1))) @ ck
            if surf.min() < 0.5 * w.h:
                continue
        c = np.empty(w.n + 1)
        c[0] = linear_period(w.g, w.tau, w.h)
        c[1:] = ck
        return c, s
    raise RuntimeError(f"no admissible draw for {w.name} within {max_redraw} seeds")


def stable_steps(N: int, g: float, tau: float, h: float, T: float) -> int:
    """Step count of a shot of the uneven batch: max(N/2, ceil((T/4) omega(k_eff) / 2.5)),
    k_eff = 0.9 N/2, omega^2 = (g k + tau k^3) tanh(k h) (RK4's imaginary-axis
    stability limit is ~2.83)."""
    k = 0.9 * N / 2
    om = math.sqrt((g * k + tau * k**3) * (1.0 if math.isinf(h) else math.tanh(k * h)))
    return max(N // 2, math.ceil(0.25 * T * om / 2.5))


def uneven_shots(n_shots: int = 32, seed: int = 0, step_cap: int | None = None,
                 sizes=(256, 512, 1024, 2048, 4096)):
    """The batch of independent shots of uneven size: N drawn from `sizes`,
    n + 1 columns in [8, 64], h ~ U(0.1, 2), tau in {0, 0.05}, c_1 ~ U(0.01, 0.5)
    (c_k = c_1^k u_k), steps by `stable_steps`.  A shot whose c_1 would put the
    surface near the bottom (c_1 >= 0.45 h) draws its depth and c_1 again; the
    coefficient draw then follows `coefficients` (its own redraw rule).
    step_cap bounds the step count (T scaled so dt stays that of the full shot),
    for measurements that must end in minutes.  Returns [(Workload, c)]."""
    rng = np.random.default_rng(seed)
    shots = []
    for i in range(n_shots):
        N = int(rng.choice(sizes))
        n = int(rng.integers(7, 64))          # n + 1 columns in [8, 64]
        tau = float(rng.choice([0.0, 0.05]))
        while True:
            h = float(rng.uniform(0.1, 2.0))
            amp = float(rng.uniform(0.01, 0.5))
            if amp < 0.45 * h:
                break
        w = Workload(f"shot{i}_N{N}_n{n}_h{h:.3f}_tau{tau}", N=N, n=n, steps=1, tau=tau, h=h, amp=amp,
                     seed=1000 * (seed + 1) + i)
        c, _ = coefficients(w)
        steps = stable_steps(N, w.g, tau, h, c[0])
        if step_cap is not None and steps > step_cap:
            c[0] *= step_cap / steps
            steps = step_cap
        shots.append((shrink(w, steps=steps, name=w.name), c))
    return shots


def shrink(w: Workload, N: int | None = None, n: int | None = None, steps: int | None = None,
           name: str | None = None) -> Workload:
    """Same physics and coefficient law at other sizes (tests)."""
    N = w.N if N is None else N
    n = w.n if n is None else n
    steps = w.steps if steps is None else steps
    return Workload(name or f"{w.name}->N{N}_n{n}_s{steps}", N=N, n=n, steps=steps, g=w.g,
                    tau=w.tau, h=w.h, amp=w.amp, law=w.law, decay=w.decay, seed=w.seed)
