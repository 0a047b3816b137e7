"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

The shooting Jacobian has no exchange step, so N GPUs run N independent
replicas (each its own seeded problem); the only collectives are the barrier
and the max over ranks of the step time.  These tests run that logic with
world_size 2 on the gloo backend, with no GPU.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1210_5672_gb300 import workloads as W
    try:
        r, n, local = bench.dist_init()
        assert (r, n, local) == (rank, ws, rank)
        bench.barrier(n)
        # rank k "took" 1 + k seconds per step: the job's step time is the slowest
        t, value = bench.replica_rate(1.0 + rank, n, 513)
        w = W.LARGE
        c, seed = W.coefficients(w, seed=w.seed + rank)
        q.put((rank, t, value, seed, float(c[1]), float(c[2])))
        bench.barrier(n)
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    out = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, t, value, _, _, _ in out:
        assert t == pytest.approx(2.0)                 # max over ranks
        assert value == pytest.approx(2 * 513 / 2.0)   # all ranks' columns / slowest time
    # replicas are independent problems: different seeds, different coefficients
    assert out[0][3] != out[1][3]
    assert out[0][5] != out[1][5]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(0.5, 1, 100) == (0.5, 200.0)
