"""dtn_apply_static: the DtN operator in one call that allocates no memory.

Some callers cannot allocate device memory when they need the operator (inside
a stream-capture region, under an allocator policy that forbids cudaMalloc, or
from a host application that owns every allocation).  This entry point runs the
same kernels as dtn_setup + dtn_apply on a fixed workspace inside the library.
The test calls it through the C ABI and compares it with the context-based
entry points on two calls in a row (different surfaces, sizes and data), so a
stale workspace from the first call would show in the second.  It is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def test_static_workspace_matches_context_entry_points(ww):
    import torch
    assert ww.STATIC_MAX_N >= 256 and ww.STATIC_MAX_RHS >= 64
    for (N, nrhs, h, seed) in ((256, 40, 1.0, 11), (128, 7, math.inf, 12)):
        eta, phi = case(N, nrhs, h, seed)
        e_d = torch.tensor(eta, dtype=torch.float64, device="cuda")
        p_d = torch.tensor(phi, dtype=torch.float64, device="cuda")
        with ww.Context(N, nrhs, h=h) as ctx:
            ww.dtn_setup(ctx, e_d)
            ref = ww.dtn_apply(ctx, p_d).cpu().numpy()
        out = torch.empty_like(p_d)
        ww.dtn_apply_static(e_d, p_d, h, out)
        got = out.cpu().numpy()
        for a, b in zip(got, ref):
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_static_rejects_oversize(ww):
    import torch
    N = 2 * ww.STATIC_MAX_N
    e_d = torch.ones(N, dtype=torch.float64, device="cuda")
    p_d = torch.zeros(1, N, dtype=torch.float64, device="cuda")
    with pytest.raises(ww.WWError) as ei:
        ww.dtn_apply_static(e_d, p_d, 1.0, torch.empty_like(p_d))
    assert ei.value.code == -1
