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


def _split_rank(rank, world, port, q):
    # one plan split by beam over gloo ranks; each rank's partial dose from the
    # FP64 oracle on its share of the beams, then the library's exchange
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import oracle
    from paper_1103_1164_gb300 import beam_split, synth
    dist.init_process_group("gloo")
    try:
        p = synth.small_plan(88, n=(12, 10, 8), vox=0.5, n_beams=3, couch=True)

        def all_gather(x):
            t = torch.from_numpy(np.ascontiguousarray(x))
            out = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(out, t)
            return [o.numpy() for o in out]

        got = beam_split.dose_split(p, lambda sp: oracle.OraclePlan(sp, threads=1).dose(), rank, world, all_gather)
        q.put((rank, got, beam_split.beam_shares(p.beamlets_per_beam, world)))
    finally:
        dist.destroy_process_group()


def test_beam_split_dose_equals_whole_plan():
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import oracle
    from paper_1103_1164_gb300 import beam_split, synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    plan = synth.small_plan(88, n=(12, 10, 8), vox=0.5, n_beams=3, couch=True)
    want = oracle.OraclePlan(plan, threads=1).dose().reshape(-1)
    shares = out[0][2]
    assert sorted(b for s in shares for b in s) == [0, 1, 2] and all(s for s in shares)
    for r, got, _ in out:
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()   # eq. (1) is additive over beams
    assert np.array_equal(out[0][1], out[1][1])                          # every rank: the same sums


def test_beam_shares_balance_beamlets():
    sys.path.insert(0, ROOT)
    from paper_1103_1164_gb300 import beam_split
    assert beam_split.beam_shares([100, 100, 100, 100], 2) == [[0, 1], [2, 3]]
    assert beam_split.beam_shares([10, 300, 10, 10], 2) == [[0, 1], [2, 3]]   # 310 / 20: no cut does better
    assert beam_split.beam_shares([300, 10, 10, 10, 300], 2) == [[0, 1], [2, 3, 4]]
    sh = beam_split.beam_shares([5, 6], 4)
    assert sorted(b for s in sh for b in s) == [0, 1] and len(sh) == 4
