"""dtn_apply_static: the DtN operator in one call that allocates no memory.

Some callers cannot allocate device memory when they need the operator: code
under a memory-pool or allocator policy that forbids cudaMalloc, plug-ins of a
host application that owns every allocation, loops that must not touch the
allocator.  This entry point runs the same kernels as dtn_setup + dtn_apply on
a fixed workspace inside the library.

The tests call it through the C ABI and compare it with the context-based
entry points on calls in a row (different surfaces, sizes and data, so a
stale workspace from one call would show in the next), and with the CPU
oracle's DtN.  The cases cover the full static layout (N = WW_STATIC_MAX_N,
nrhs = WW_STATIC_MAX_RHS), a caller's stream, and the one-column solve.  The
file is collected last so that a run stopping at the first failure has run
everything else.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ww():
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as m
    m.lib()
    return m


def case(N, nrhs, h, seed):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(N) / N
    eta = (0.0 if math.isinf(h) else h) + sum(0.1 / k**2 * rng.uniform(-1, 1) * np.cos(k * x) for k in range(1, 9))
    phi = np.stack([sum(rng.uniform(-1, 1) / k**2 * np.cos(k * x + rng.uniform(0, 6)) for k in range(1, 12))
                    for _ in range(nrhs)])
    return eta, phi


def col_err(got, ref):
    return max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(got, ref))


# (N, nrhs, h, seed, on a stream of its own): the whole static layout on a
# caller's stream, a finite-depth and a deep-water case on the legacy stream,
# and the one-column solve (the narrow product path)
CASES = ((256, 40, 1.0, 11, False), (128, 7, math.inf, 12, False), (256, 64, 0.5, 13, True),
         (64, 1, 2.0, 14, True))


def test_static_workspace_matches_context_entry_points_and_oracle(ww):
    import torch

    import oracle as O
    assert ww.STATIC_MAX_N >= 256 and ww.STATIC_MAX_RHS >= 64
    for (N, nrhs, h, seed, own_stream) in CASES:
        eta, phi = case(N, nrhs, h, seed)
        e_d = torch.tensor(eta, dtype=torch.float64, device="cuda")
        p_d = torch.tensor(phi, dtype=torch.float64, device="cuda")
        with ww.Context(N, nrhs, h=h) as ctx:
            ww.dtn_setup(ctx, e_d)
            ref = ww.dtn_apply(ctx, p_d).cpu().numpy()
        out = torch.full_like(p_d, float("nan"))
        if own_stream:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            ww.dtn_apply_static(e_d, p_d, h, out, stream=s)
            s.synchronize()
        else:
            ww.dtn_apply_static(e_d, p_d, h, out)
        got = out.cpu().numpy()
        e_ctx = col_err(got, ref)
        e_orc = col_err(got, O.dtn(eta, phi, h))
        print(f"N={N} nrhs={nrhs} h={h} stream={own_stream}: vs context {e_ctx:.2e}, vs oracle {e_orc:.2e}")
        assert e_ctx < TOL, (N, nrhs, e_ctx)
        assert e_orc < TOL, (N, nrhs, e_orc)


def test_static_rejects_oversize(ww):
    import torch
    N = 2 * ww.STATIC_MAX_N
    e_d = torch.ones(N, dtype=torch.float64, device="cuda")
    p_d = torch.zeros(1, N, dtype=torch.float64, device="cuda")
    with pytest.raises(ww.WWError) as ei:
        ww.dtn_apply_static(e_d, p_d, 1.0, torch.empty_like(p_d))
    assert ei.value.code == -1
    N = ww.STATIC_MAX_N
    e_d = torch.ones(N, dtype=torch.float64, device="cuda")
    p_d = torch.zeros(ww.STATIC_MAX_RHS + 1, N, dtype=torch.float64, device="cuda")
    with pytest.raises(ww.WWError) as ei:
        ww.dtn_apply_static(e_d, p_d, 1.0, torch.empty_like(p_d))
    assert ei.value.code == -1
