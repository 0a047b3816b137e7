"""Column sharding of one Jacobian (paper_1210_5672_gb300.sharding) on CPU ranks:
world sizes 2 and 3 over gloo, each rank computing its block of columns with
the CPU oracle as the engine (the library's engine takes its place on GPUs),
then one all-gather.  The gathered J must equal the unsharded oracle J: the
sub-problems carry the same initial state (formed once as one basis column,
so equal up to rounding) and the columns do not interact."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, NMODES, STEPS, H = 32, 10, 8, 1.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sys.path.insert(0, ROOT)
    from paper_1210_5672_gb300 import workloads as W
    w = W.Workload("shard", N=N, n=NMODES, steps=STEPS, h=H, amp=0.05)
    c, _ = W.coefficients(w)
    x = 2 * np.pi * np.arange(N) / N
    basis = np.zeros((2 * N, NMODES))
    for k in range(1, NMODES + 1):
        basis[:N, k - 1] = np.cos(k * x)
        if k % 3 == 0:
            basis[N:, k - 1] = 0.5 * np.cos(k * x)   # some columns with phi parts
    return c, basis


def _oracle_engine():
    import oracle as O

    def engine(c_r, basis_r):
        prob, keep = O.make_problem(N, basis_r.shape[1], h=H, steps=STEPS, basis=basis_r)
        r, J, f = O.shoot_jacobian(prob, c_r)
        return r, J, f

    return engine


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1210_5672_gb300.sharding import sharded_jacobian
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        c, basis = _problem()
        r, J, f = sharded_jacobian(c, basis, _oracle_engine(), rank, ws)
        q.put((rank, r, J, f))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_jacobian_matches_unsharded(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0] * ws
    sys.path.insert(0, ROOT)
    import oracle as O
    c, basis = _problem()
    prob, keep = O.make_problem(N, NMODES, h=H, steps=STEPS, basis=basis)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    norms = np.linalg.norm(J0, axis=0)
    for rank, r, J, f in outs:
        assert J.shape == J0.shape
        assert np.linalg.norm(r - r0) <= 1e-13 * np.linalg.norm(r0) and abs(f - f0) <= 1e-13 * f0
        for k in range(NMODES + 1):
            assert np.linalg.norm(J[:, k] - J0[:, k]) <= 1e-12 * norms[k], (rank, k)
    # every rank holds the same gathered J
    assert all(np.array_equal(outs[0][2], o[2]) for o in outs)


def test_column_ranges_and_single_rank():
    sys.path.insert(0, ROOT)
    from paper_1210_5672_gb300.sharding import column_ranges, sharded_jacobian
    assert column_ranges(10, 3) == [(1, 5), (5, 8), (8, 11)]
    assert column_ranges(2, 4) == [(1, 2), (2, 3), (3, 3), (3, 3)]
    c, basis = _problem()
    r, J, f = sharded_jacobian(c, basis, _oracle_engine(), 0, 1)
    import oracle as O
    prob, keep = O.make_problem(N, NMODES, h=H, steps=STEPS, basis=basis)
    r0, J0, f0 = O.shoot_jacobian(prob, c)
    norms = np.linalg.norm(J0, axis=0)
    assert max(np.linalg.norm(J[:, k] - J0[:, k]) / norms[k] for k in range(NMODES + 1)) < 1e-12


def _failing_rank_main(rank, ws, port, q, mode):
    """Rank 1 fails: its engine raises ("raise"; "raise-default" passes no store,
    so the process group's own store carries the reports), or it leaves between
    steps without reporting ("exit"); the others must learn of it on the host
    through the store and raise ShardFailure, never entering the all-gather."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    from datetime import timedelta

    import torch.distributed as dist

    from paper_1210_5672_gb300.sharding import ShardFailure, sharded_jacobian
    store = dist.TCPStore("127.0.0.1", port, ws, is_master=(rank == 0), timeout=timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=ws, timeout=timedelta(seconds=30))
    c, basis = _problem()
    engine = _oracle_engine()
    if rank == 1 and mode.startswith("raise"):
        def engine(c_r, basis_r):
            raise RuntimeError("planted engine failure")
    if rank == 1 and mode == "exit":
        q.put((rank, "left"))
        q.close()
        q.join_thread()                 # the queue's feeder thread writes before the exit
        os._exit(0)
    try:
        sharded_jacobian(c, basis, engine, rank, ws, store=None if mode == "raise-default" else store, tag="t",
                         timeout=3.0)
        q.put((rank, "no error"))
    except ShardFailure as e:
        q.put((rank, f"ShardFailure: {e}"))
    store.set(f"done/{rank}", "1")
    if rank == 0:                       # the store lives here: keep it up for the others
        import time
        deadline = time.monotonic() + 10.0
        live = [r for r in range(ws) if not (mode == "exit" and r == 1)]
        while time.monotonic() < deadline and not all(store.check([f"done/{r}"]) for r in live):
            time.sleep(0.02)
    q.close()
    q.join_thread()
    os._exit(0)


@pytest.mark.parametrize("mode,ws", [("raise", 2), ("raise-default", 2), ("exit", 2), ("exit", 3)])
def test_a_failed_rank_is_detected_on_the_host(mode, ws):
    import time
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    t0 = time.monotonic()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, ws, port, q, mode)) for r in range(ws)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0] * ws
    assert time.monotonic() - t0 < 90
    for rank, msg in outs.items():
        if mode == "exit" and rank == 1:
            assert msg == "left"
        elif mode == "exit":
            assert msg.startswith("ShardFailure") and "[1]" in msg and "did not report" in msg, msg
        else:
            assert msg.startswith("ShardFailure") and "rank 1: engine failed" in msg and "planted" in msg, msg
