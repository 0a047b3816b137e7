"""Levenberg-Marquardt with delayed Jacobian updates (App. D) driven by the GPU
library (`solve_standing_wave`: shoot and shoot_jacobian through the C ABI),
against the same solver driven by the CPU oracle on the same discrete problem:
a standing wave of amplitude c_1 = 0.02 in the paper's basis (even k on eta,
odd k on phi), N = 64, 16 modes, h = 1."""
import math
import time

import numpy as np
import pytest

import oracle as O
from paper_1210_5672_gb300.levmar import LMOptions, levmar, solve_standing_wave

pytestmark = pytest.mark.gpu

N, NMODES, STEPS, EPS, H = 64, 16, 96, 0.02, 1.0


@pytest.fixture(scope="module")
def ww():
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as m
    m.lib()
    return m


def _basis():
    x = 2 * np.pi * np.arange(N) / N
    B = np.zeros((2 * N, NMODES))
    for k in range(1, NMODES + 1):
        if k % 2 == 0:
            B[:N, k - 1] = 2 * np.cos(k * x)
        else:
            B[N:, k - 1] = 2 * np.cos(k * x)
    return B


def _start():
    c0 = np.zeros(NMODES + 1)
    c0[0] = 2 * math.pi / math.sqrt(math.tanh(H))
    c0[1] = EPS
    free = np.array([0] + list(range(2, NMODES + 1)))
    return c0, free


@pytest.fixture(scope="module")
def oracle_solution():
    prob, keep = O.make_problem(N, NMODES, h=H, steps=STEPS, basis=_basis())
    c0, free = _start()

    def full(z):
        c = c0.copy()
        c[free] = z
        return c

    out = levmar(lambda z: O.shoot(prob, full(z))[0],
                 lambda z: (lambda rJ: (rJ[0], rJ[1][:, free]))(O.shoot_jacobian(prob, full(z))),
                 c0[free], 0.1 * c0[0], LMOptions())
    assert out.f < 1e-24
    c = c0.copy()
    c[free] = out.c
    return c


@pytest.mark.parametrize("precision", [0, 1])
def test_standing_wave_solve_on_gpu(ww, oracle_solution, precision):
    c0, free = _start()
    with ww.Context(N, NMODES, h=H, steps=STEPS, basis=_basis(), precision=precision) as ctx:
        t0 = time.perf_counter()
        res = solve_standing_wave(ctx, c0, free, delta0=0.1 * c0[0])
        dt = time.perf_counter() - t0
    print(f"\nprecision {precision}: f {res.f:.2e}, T {res.c[0]!r}, {res.jacobians} Jacobians, "
          f"{res.residuals} residuals, {res.accepted} accepted steps, {dt:.2f} s ({res.reason})")
    assert res.f < 1e-24
    assert res.jacobians < res.accepted
    T0 = oracle_solution[0]
    assert abs(res.c[0] - T0) < 1e-10 * T0
    # the free Fourier coefficients, against the amplitude scale c_1
    assert np.max(np.abs(res.c[2:] - oracle_solution[2:])) < 1e-9 * EPS
