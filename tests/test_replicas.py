"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.  Each rank
solves its own seeded batch (weak scaling, no collective on the data path;
the oracle stands in for the GPU solve here) and the whole-job figures are
the slowest rank's time and the LPs solved by all ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    import oracle

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.rank_workload("sb_small", 0, rank)
        sp = w.specs.subset(range(4))
        r = oracle.solve(w.lp, sp, tol=1e-4, max_iter=100000, threads=1, lockstep=0, want_xy=False)
        solved = int(np.sum(r.status <= 2))
        elapsed = 10.0 * (rank + 1)
        t, total = bench.reduce_over_ranks(dist, elapsed, solved, "cpu")
        out.put((rank, t, total, solved, w.lp.vals[:8].tolist(), r.obj.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_with_gloo():
    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, t0, tot0, s0, v0, o0), (r1, t1, tot1, s1, v1, o1) = got
    # the slowest rank's time and the sum of the LPs solved, on every rank
    assert t0 == t1 == 20.0
    assert tot0 == tot1 == s0 + s1
    # independent batches: each rank generated its own matrix and solved it
    assert v0 != v1 and o0 != o1


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(None, 12.5, 7, "cpu") == (12.5, 7)
