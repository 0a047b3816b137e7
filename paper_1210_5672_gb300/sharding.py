"""Column sharding of one Jacobian over ranks (one GPU each).

The variational columns are independent given the base trajectory (Eq. q:qdot:
each column solves the same linear system along the same base state), so one
Jacobian splits by columns with no exchange until the end.  Every rank
integrates the full base trajectory and its own contiguous block of mode
columns; one all-gather assembles J on every rank.

A rank's sub-problem keeps the full initial state with a basis of its own:
  basis_r = [sum_k c_k b_k, b_s, ..., b_{e-1}],   c_r = [T, 1, 0, ..., 0],
so q0 = hbar + 1 * (sum_k c_k b_k) is the full problem's initial state (the sum
is formed once on the host, so it agrees with the unsharded one to rounding),
J_r's column 0 is the T column, column 1 the direction of the initial shape
(dropped), and columns 2.. the full problem's mode columns s..e-1.  The T
column is computed on every rank (one column) and taken from rank 0.

The per-rank engine is a callable engine(c_r, basis_r) -> (r, J_r, f) with J_r
of shape N x (len(c_r)); `gpu_engine` builds it on the library's
shoot_jacobian.  The gather uses torch.distributed: on a NCCL group the
gathered blocks travel as CUDA tensors of the current device, on a gloo group
(the CPU tests) as CPU tensors.

Failure detection is on the host.  Through a key-value store (by default the
process group's own), every rank reports its status ("ok", or its engine's
error) before the collective and waits, for at most `timeout` seconds, for
every other rank's report.  A rank that failed or never reported (it died or
hangs) turns into a ShardFailure on every surviving rank, naming the ranks,
and no rank enters a collective that could not complete.
"""
from __future__ import annotations

import time

import numpy as np


class ShardFailure(RuntimeError):
    """A rank of the column split failed or did not report in time."""


def _await_ranks(store, tag: str, world: int, timeout: float):
    keys = [f"{tag}/{q}" for q in range(world)]
    deadline = time.monotonic() + timeout
    missing = keys
    while True:
        missing = [k for k in keys if not store.check([k])]
        if not missing or time.monotonic() > deadline:
            break
        time.sleep(0.02)
    if missing:
        ranks = [int(k.rsplit("/", 1)[1]) for k in missing]
        raise ShardFailure(f"ranks {ranks} did not report within {timeout} s")
    bad = {q: store.get(k).decode() for q, k in enumerate(keys)}
    bad = {q: v for q, v in bad.items() if v != "ok"}
    if bad:
        raise ShardFailure("; ".join(f"rank {q}: {v}" for q, v in sorted(bad.items())))


def column_ranges(n: int, world: int):
    """Mode columns 1..n split into `world` contiguous blocks [s, e) of near-equal size."""
    base, extra = divmod(n, world)
    out, s = [], 1
    for r in range(world):
        e = s + base + (1 if r < extra else 0)
        out.append((s, e))
        s = e
    return out


def shard_problem(c, basis, rank: int, world: int):
    """(c_r, basis_r, (s, e)) of rank's sub-problem; basis is 2N x n (column k-1 = b_k)."""
    c = np.asarray(c, dtype=np.float64)
    basis = np.asarray(basis, dtype=np.float64)
    n = basis.shape[1]
    s, e = column_ranges(n, world)[rank]
    shape = basis @ c[1:]
    basis_r = np.concatenate([shape[:, None], basis[:, s - 1:e - 1]], axis=1)
    c_r = np.zeros(2 + (e - s))
    c_r[0] = c[0]
    c_r[1] = 1.0
    return c_r, basis_r, (s, e)


def sharded_jacobian(c, basis, engine, rank: int, world: int, group=None, store=None, tag: str = "jacobian",
                     timeout: float = 60.0):
    """The full (r, J, f) of the problem (c, basis) on every rank, each rank
    computing its block of columns with engine(c_r, basis_r) and one all-gather.
    With world > 1 the ranks first report to each other through `store` (the
    default process group's store when None; `tag` unique per call), and a
    failed or silent rank raises ShardFailure on every surviving rank."""
    import torch
    import torch.distributed as dist

    if world > 1 and store is None:
        from torch.distributed import distributed_c10d as c10d
        store = c10d._get_default_store()
    n = np.asarray(basis).shape[1]
    c_r, basis_r, (s, e) = shard_problem(c, basis, rank, world)
    try:
        r, J_r, f = engine(c_r, basis_r)
        status = "ok"
    except Exception as exc:              # reported to the other ranks, then raised here
        if world == 1:
            raise
        status = f"engine failed: {type(exc).__name__}: {exc}"
    if world > 1:
        store.set(f"{tag}/{rank}", status)
        _await_ranks(store, tag, world, timeout)
    N = J_r.shape[0]
    ranges = column_ranges(n, world)
    width = 1 + max(b - a for a, b in ranges)          # T column + the widest block
    local = np.zeros((width, N))
    local[0] = J_r[:, 0]
    local[1:1 + (e - s)] = J_r[:, 2:].T
    t = torch.tensor(local, dtype=torch.float64)
    if world > 1:
        if dist.get_backend(group) == "nccl":      # NCCL gathers device tensors only
            t = t.to(torch.device("cuda", torch.cuda.current_device()))
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        parts = [p.cpu() for p in parts]
    else:
        parts = [t]
    J = np.empty((N, n + 1))
    J[:, 0] = parts[0][0].numpy()
    for q, (a, b) in enumerate(ranges):
        J[:, a:b] = parts[q][1:1 + (b - a)].numpy().T
    return np.asarray(r), J, float(f)


def gpu_engine(N, g=1.0, tau=0.0, h=1.0, steps=64, precision=0):
    """engine(c_r, basis_r) on the library: a context per call (the basis is part
    of the problem description), shoot_jacobian, results as numpy."""
    import torch

    import paper_1210_5672_gb300 as ww

    def engine(c_r, basis_r):
        with ww.Context(N, basis_r.shape[1], g=g, tau=tau, h=h, steps=steps, basis=basis_r,
                        precision=precision) as ctx:
            ct = torch.tensor(c_r, dtype=torch.float64, device="cuda")
            r, J, f = ctx.empty_outputs()
            ww.shoot_jacobian(ctx, ct, r, J, f)
            return r.cpu().numpy(), J.cpu().numpy().T, float(f.item())

    return engine
