"""The multi-process path of bench.py on CPU (gloo, world size 2).

The solve does not shard ("replicas only"): each rank solves its own system
and no data moves between ranks.  What the ranks share is host logic: the
per-rank problem seeds, the barrier and max-over-ranks timing, and the
reference arm that runs on rank 0 alone.  These run here as two gloo ranks.
"""
import argparse
import io
import contextlib
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # the slowest rank sets the job time
        t = bench.max_over_ranks(1.5 * (rank + 1), world, device="cpu")
        # each rank its own system
        p = bench.make_problem("tiny", rank)
        # reference arm: ranks other than 0 exit without work or output
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            if rank != 0:
                bench.run_reference(argparse.Namespace(workload="tiny"), rank, world)
        dist.barrier()
        q.put((rank, t, p.seed, float(p.noise[0]), out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, t0, s0, m0, o0), (r1, t1, s1, m1, o1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 3.0                 # max over ranks, seen by both
    assert s0 != s1 and m0 != m1           # distinct seeded systems per rank
    assert o1 == ""                        # rank 1: no reference line


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
