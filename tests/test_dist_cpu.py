"""bench.py's multi-rank path on CPU: two gloo ranks on 127.0.0.1.

Each rank computes its own plan (independent problems, weak scaling); the job's
throughput is every rank's evaluations over the slowest rank's time, and the
reference arm runs on rank 0 only.  The ranks here report made-up counts and
times, so the test checks the aggregation and the rendezvous, not a plan.
"""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse
    import torch
    import bench
    w, r, _, pg = bench.dist_setup(argparse.Namespace(impl="reference"))
    try:
        assert pg is not None and pg.get_backend() == "gloo"
        bench.barrier(pg, torch)
        # rank r: (r + 1) * 1000 evaluations in (r + 1) * 10 ms
        value, t_ms = bench.aggregate_throughput(pg, torch, 1000.0 * (r + 1), 10.0 * (r + 1))
        ran_reference = bench.run_reference(argparse.Namespace(steps=1, warmup=0), w, r, pg) if r != 0 else None
        q.put((r, w, value, t_ms, ran_reference))
    finally:
        pg.destroy_process_group()


def test_two_gloo_ranks_aggregate_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, t_ms, ran in out:
        assert w == 2
        assert t_ms == 20.0                        # the slowest rank's time
        assert abs(value - 3000.0 / 0.020) < 1e-6  # all ranks' evaluations / that time
    assert out[1][4] is None                       # rank 1 leaves the reference arm at once


def test_single_process_is_rank_zero():
    sys.path.insert(0, ROOT)
    import argparse
    import torch
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    w, r, _, pg = bench.dist_setup(argparse.Namespace(impl="ours"))
    assert (w, r, pg) == (1, 0, None)
    value, t_ms = bench.aggregate_throughput(pg, torch, 500.0, 4.0)
    assert t_ms == 4.0 and abs(value - 500.0 / 0.004) < 1e-9
