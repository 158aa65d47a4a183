"""Benchmark of the GB300 DC-FSPB dose engine.

One step = the whole hot path of one plan on synthetic inputs resident in HBM:
  Algorithm A1 steps 1-6 for the plan's density (smoothing, beamlet geometry,
  FP64 Siddon trace, depth tables; dc_fspb_set_density),
  the row pattern of the dose-deposition matrix (pair tests, per-voxel counts
  and their scan; dc_fspb_pair_count),
  eq. (1) and the FP32 CSR matrix from ONE evaluation of each (voxel, beamlet)
  pair (dc_fspb_dose_and_matrix).
The metric counts each pair once: evaluations = pairs of the plan.

Default workload: the 9-field coplanar thorax plan on a 128 x 128 x 96 grid of
0.25 cm voxels (0.5 cm beamlets, fields 8-15 cm, ROI 5 cm).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank computes its
own plan (independent problems: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-beamlet evals/s (full plan: steps 1-6 + eq. 1 dose and FP32 dose matrix, one evaluation per pair)"
UNIT = "evals/s"
# Algorithmic work of one (voxel, beamlet) evaluation of eqs. (2)-(4) with the
# lookups of Algorithm A1 steps 9-11, counted from the method's definition:
# 8 exponentials (four profiles p of eq. 4, two each) and 1 reciprocal
# (SAD/|r_a|) on the special-function units, and about 65 FP32 add/mul/fma
# (geometry ~20, five linear lookups ~15, the bilinear A ~8, eqs. 3-4 ~16,
# fluence weight and accumulation ~3).  16 SFU lanes per SM against 9
# operations bind before 128 FP32 lanes against 65.
ALG_FP32_PER_PAIR = 65
ALG_MUFU_PER_PAIR = 9
# The kernel's own operation count (index arithmetic, clamps and the rounding
# trick of its table coordinates included), reported beside the primary figure.
IMPL_FP32_PER_PAIR = 98
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# a pair kernel on the thorax9 plan, from an ncu capture of the kernel built
# from the sources with these SHA-256 digests (the kernel and the structures it
# reads; the summaries are under profiles/); reported only while they are unchanged.
KERNEL_TRAFFIC = {
    # k_pairs<kFill, 1> (the step's fill + eq. 1) and k_pairs<kDose> on thorax9
    "fill": (1182519296 + 5323322624, {
        "paper_1103_1164_gb300/csrc/k_dose.cu": "5d055c97e41799cec66cb70fd651222cfbbc9d1e055d0292647a3f3c08c35e5d",
        "paper_1103_1164_gb300/csrc/dc_views.cuh": "786376aaf34c342ec1f8614b14b49cfb72da1465ac3fd3094fb0956611314095",
    }),
    "dose": (110442240 + 20924416, {
        "paper_1103_1164_gb300/csrc/k_dose.cu": "5d055c97e41799cec66cb70fd651222cfbbc9d1e055d0292647a3f3c08c35e5d",
        "paper_1103_1164_gb300/csrc/dc_views.cuh": "786376aaf34c342ec1f8614b14b49cfb72da1465ac3fd3094fb0956611314095",
    }),
}


def kernel_traffic(kernel, scale):
    """The captured per-launch DRAM traffic of `kernel`, or None if there is no
    capture, the kernel's sources changed since it, or the workload is not the
    captured one."""
    import hashlib
    if scale != 1.0 or kernel not in KERNEL_TRAFFIC:
        return None
    nbytes, sources = KERNEL_TRAFFIC[kernel]
    for rel, digest in sources.items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return nbytes


def pair_peak(sms, mhz, fp32_ops=ALG_FP32_PER_PAIR):
    """Pairs/s bound of the direct evaluation: the tighter of the FP32 lanes and
    the special-function lanes at the given SM clock."""
    return sms * mhz * 1e6 * min(FP32_LANES_PER_SM / fp32_ops, MUFU_LANES_PER_SM / ALG_MUFU_PER_PAIR)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="the step only (quick runs)")
    ap.add_argument("--scale", type=float, default=1.0, help="grid scale of the thorax plan")
    ap.add_argument("--profile", default=None, choices=["count", "dose", "fill", "fused", "mlp", "prep", "spmm", "step", "table1", "train"],
                    help="small fixed run of one stage for profiler captures (prints no bench line)")
    return ap.parse_args()


def run_profile(args):
    """A short, fixed sequence of one stage's launches for ncu captures: the
    plan is built once, then the stage runs warmup + steps times."""
    import torch
    from paper_1103_1164_gb300 import build, dc_fspb as dc, synth
    build.build()
    if args.profile in ("mlp", "train"):
        # the network's factor pass on slab64 (weights from the initialiser:
        # its cost does not depend on them), or the BF16 training gradient on
        # 8192 stencil samples
        from paper_1103_1164_gb300 import surrogate
        if args.profile == "mlp":
            p1 = synth.config1()
            plan = dc.dc_fspb_create_from(p1, lateral_mode=dc.DC_LATERAL_AXIS)
            dc.dc_fspb_set_surrogate(plan, surrogate.init_params(1), surrogate.RHO_LO, surrogate.RHO_HI)
            for _ in range(args.warmup + args.steps):
                dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP)
            torch.cuda.synchronize()
            print(f"profile run done: mlp factor pass, {dc.dc_fspb_list_entries(plan)} entries")
        else:
            X, T = surrogate.generate_samples(n_phantoms=2, per_phantom=4096, seed=5)
            net = dc.Mlp(surrogate.init_params(2), precision=dc.DC_PRECISION_BF16)
            for _ in range(args.warmup + args.steps):
                net.gradient(X, T)
            print(f"profile run done: BF16 training gradient, {X.shape[0]} samples")
        return
    if args.profile == "spmm":
        p1 = synth.config1()
        plan = dc.dc_fspb_create_from(p1)
        dc.dc_fspb_spmm_prepare(plan)
        F = torch.rand(plan.n_beamlets, 64, device="cuda")
        Y = torch.empty(plan.n_voxels, 64, device="cuda")
        for _ in range(args.warmup + args.steps):
            dc.dc_fspb_spmm(plan, F, Y)
        dc.dc_fspb_device_status(plan)
        print(f"profile run done: spmm, {plan.n_voxels} voxels, {plan.n_beamlets} beamlets")
        return
    p = synth.table1_case("H5") if args.profile == "table1" else synth.config2(args.scale)
    rho_d = torch.from_numpy(p.rho).cuda()
    flu_d = torch.from_numpy(p.fluence).cuda()
    plan = dc.dc_fspb_create_from(p, device_density=rho_d)
    dose_d = torch.empty(plan.shape, device="cuda")
    if args.profile in ("step", "fused"):
        # "step": the benchmark's step after the same plan set-up (autotuned
        # binning); "fused": its dose-and-matrix pass alone (pattern known)
        dc.dc_fspb_autotune(plan, flu_d)
        pairs = dc.dc_fspb_pair_count(plan)
        rowptr = torch.empty(plan.n_voxels + 1, dtype=torch.int64, device="cuda")
        cols = torch.empty(pairs, dtype=torch.int32, device="cuda")
        vals = torch.empty(pairs, dtype=torch.float32, device="cuda")
        n0 = dc.dc_fspb_launch_count()
        for _ in range(args.warmup + args.steps):
            if args.profile == "step":
                dc.dc_fspb_set_density(plan, rho_d)
                dc.dc_fspb_pair_count(plan)
            dc.dc_fspb_dose_and_matrix(plan, flu_d, dose_d, dc.DC_F32, rowptr, cols, vals)
        torch.cuda.synchronize()
        per_step = (dc.dc_fspb_launch_count() - n0) // (args.warmup + args.steps)
        print(f"profile run done: {args.profile}, {per_step} library launches per step")
        return
    if args.profile == "fill":
        pairs = dc.dc_fspb_pair_count(plan)
        rowptr = torch.empty(plan.n_voxels + 1, dtype=torch.int64, device="cuda")
        cols = torch.empty(pairs, dtype=torch.int32, device="cuda")
        vals = torch.empty(pairs, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup + args.steps):
        if args.profile == "dose":
            dc.dc_fspb_dose(plan, flu_d, dose_d)
        elif args.profile == "table1":
            # the largest Table 1 case: density-dependent steps + dose
            dc.dc_fspb_set_density(plan, rho_d)
            dc.dc_fspb_dose(plan, flu_d, dose_d)
        elif args.profile == "fill":
            dc.dc_fspb_dose_matrix(plan, dc.DC_F32, rowptr, cols, vals)
        elif args.profile == "count":
            dc.dc_fspb_set_density(plan, rho_d)      # forgets the pattern: the next call counts again
            dc.dc_fspb_pair_count(plan)
        else:
            dc.dc_fspb_set_density(plan, rho_d)
    torch.cuda.synchronize()
    print(f"profile run done: {args.profile}, {plan.n_voxels} voxels, {plan.n_beamlets} beamlets")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args, backend=None):
    """One process per GPU (torchrun): ranks from the environment; NCCL for
    our arm on GPUs, gloo for the CPU reference arm (and CPU tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        if backend is None:
            backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def _on_gpu(pg):
    return pg.get_backend() == "nccl"


def barrier(pg, torch):
    if pg is not None:
        if _on_gpu(pg):
            pg.barrier(device_ids=[torch.cuda.current_device()])
        else:
            pg.barrier()


def _all_reduce(pg, torch, x, op):
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda" if _on_gpu(pg) else "cpu")
    pg.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(pg, torch, x):
    return x if pg is None else _all_reduce(pg, torch, x, pg.ReduceOp.MAX)


def sum_over_ranks(pg, torch, x):
    return x if pg is None else _all_reduce(pg, torch, x, pg.ReduceOp.SUM)


def aggregate_throughput(pg, torch, evals_rank, t_rank_ms):
    """Weak scaling over independent plans: every rank's evaluations over the
    slowest rank's time.  Returns (evaluations/s of the whole job, that time in ms)."""
    t_ms = max_over_ranks(pg, torch, t_rank_ms)
    total = sum_over_ranks(pg, torch, evals_rank)
    return total / (t_ms * 1e-3), t_ms


# ---------------------------------------------------------------------------
# CPU oracle timings (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_rate(plan_in, budget_s=4.0, seed=3, threads=None, op=None):
    """Times the FP64 oracle on a seeded sample of voxels of the workload.

    The sample grows until one pass takes about budget_s / 2; the pass is then
    repeated and the best of 3 kept.  Returns the oracle's plan set-up time
    (steps 1-6, measured in full) and its dose + matrix time on the sample."""
    from oracle import oracle
    threads = threads or oracle.default_threads()
    t_create = None
    if op is None:
        t0 = time.perf_counter()
        op = oracle.OraclePlan(plan_in, threads=threads)
        t_create = time.perf_counter() - t0
    op.threads = threads
    rng = np.random.default_rng(seed)
    n = 64
    while True:
        vox = np.sort(rng.choice(op.V, size=min(n, op.V), replace=False))
        t0 = time.perf_counter()
        op.dose_voxels(vox)
        op.matrix(vox)
        dt = time.perf_counter() - t0
        if dt >= 0.4 * budget_s or n >= op.V:
            break
        n = int(min(op.V, n * max(2.0, 0.5 * budget_s / max(dt, 1e-3))))
    best = dt
    for _ in range(2):
        t0 = time.perf_counter()
        op.dose_voxels(vox)
        op.matrix(vox)
        best = min(best, time.perf_counter() - t0)
    pairs_sample = int(op.pairs_voxels(vox).sum())
    return dict(op=op, t_create=t_create, t_sample=best, n_vox=int(vox.size), pairs_sample=pairs_sample,
                threads=threads)


def cpu_baseline(p, pairs):
    """The FP64 oracle (as it stands) on the host cores, all threads and one
    thread, best of 3 on bounded voxel samples, scaled by pair count to the
    whole plan (plan set-up timed in full, with all threads)."""
    est = oracle_sample_rate(p)
    one = oracle_sample_rate(p, threads=1, op=est["op"], budget_s=3.0, seed=5)
    out = {}
    for key, e in (("all", est), ("one", one)):
        t_step = est["t_create"] + e["t_sample"] * pairs / max(e["pairs_sample"], 1)
        out[key] = dict(value=pairs / t_step, threads=e["threads"], n_vox=e["n_vox"],
                        pairs_sample=e["pairs_sample"], t_sample=e["t_sample"])
    a = out["all"]
    return {"value": a["value"], "unit": UNIT, "cores": a["threads"], "kind": "oracle",
            "one_thread": {"value": out["one"]["value"], "cores": 1},
            "sample": f"FP64 oracle, best of 3: plan set-up timed in full ({est['t_create']:.2f} s), dose + "
                      f"matrix rows timed on {a['n_vox']} seeded voxels ({a['pairs_sample']} pairs, "
                      f"{a['t_sample']:.2f} s, {a['threads']} threads) and on {out['one']['n_vox']} voxels "
                      f"({out['one']['pairs_sample']} pairs, {out['one']['t_sample']:.2f} s, 1 thread), "
                      f"scaled by pair count to the {pairs} pairs of the plan"}


# ---------------------------------------------------------------------------

def run_reference(args, world, rank, pg):
    """The FP64 oracle as the reference arm (host cores, bounded samples)."""
    if rank != 0:
        return
    from paper_1103_1164_gb300 import synth
    from oracle import oracle
    p = synth.config2(args.scale)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    op = oracle.OraclePlan(p, threads=threads)
    t_create = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    vox = np.sort(rng.choice(op.V, size=min(4096, op.V), replace=False))
    pairs = int(op.pairs_voxels(vox).sum())
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        op.dose_voxels(vox)
        op.matrix(vox)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = pairs * len(times) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"thorax9 {p.grid.nx}x{p.grid.ny}x{p.grid.nz} @0.25cm, 9 fields, "
                                   f"{p.n_beamlets} beamlets (0.5 cm), ROI 5 cm",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{vox.size} seeded voxels of the plan per step "
                                       f"({pairs} pairs; dose + matrix rows); plan set-up "
                                       f"{t_create:.2f} s not in the step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1103_1164_gb300 import build, dc_fspb, synth
    build.build()
    dc = dc_fspb
    dc.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()

    p = synth.config2(args.scale)
    rho_d = torch.from_numpy(p.rho).to(dev)
    flu_d = torch.from_numpy(p.fluence).to(dev)
    plan = dc.dc_fspb_create_from(p, stream=stream.cuda_stream, device_density=rho_d)
    V, B = plan.n_voxels, plan.n_beamlets
    dose_d = torch.empty(plan.shape, device=dev)
    tuned = dc.dc_fspb_autotune(plan, flu_d)          # plan set-up, outside the timed region
    pairs = dc.dc_fspb_pair_count(plan)
    rowptr_d = torch.empty(V + 1, dtype=torch.int64, device=dev)
    cols_d = torch.empty(max(pairs, 1), dtype=torch.int32, device=dev)
    vals_d = torch.empty(max(pairs, 1), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(ev=None):
        if ev: ev[0].record(stream)
        dc.dc_fspb_set_density(plan, rho_d)
        if ev: ev[1].record(stream)
        n = dc.dc_fspb_pair_count(plan)               # row pattern: pair tests, counts, scan
        assert n == pairs
        if ev: ev[2].record(stream)
        dc.dc_fspb_dose_and_matrix(plan, flu_d, dose_d, dc.DC_F32, rowptr_d, cols_d, vals_d)
        if ev: ev[3].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = dc.dc_fspb_launch_count()
    barrier(pg, torch)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                  # L2 flushed before every step (not timed)
            step(evs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    barrier(pg, torch)
    launches = dc.dc_fspb_launch_count() - launches0
    stage = np.array([[evs[k][j].elapsed_time(evs[k][j + 1]) for j in range(3)] for k in range(args.steps)])
    step_ms = stage.sum(1)
    evals_step = pairs
    value, t_total_ms = aggregate_throughput(pg, torch, evals_step * args.steps, float(step_ms.sum()))
    ms_per_step = t_total_ms / args.steps
    clocks = clk.summary()

    # roofline of the step's dominant kernel: the fill pass, which evaluates
    # every pair (eqs. 2-4), accumulates eq. (1) and writes the matrix
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_med = float(clocks.get("sm_mhz") or sm_max)
    t_fill = float(stage[:, 2].mean()) * 1e-3
    achieved = pairs / t_fill
    peak_max = pair_peak(sms, sm_max)
    peak_med = pair_peak(sms, sm_med)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bytes_matrix = pairs * 8 + (V + 1) * 8 + V * 4     # cols + values, row pointers, dose
    roofline = {"kernel": "k_pairs<fill> (eqs. 1-4 + FP32 CSR emit, one evaluation per pair)",
                "bound": "alu", "achieved": achieved / 1e9, "peak": peak_max / 1e9, "unit": "Gpair/s",
                "frac": achieved / peak_max, "traffic": kernel_traffic("fill", args.scale),
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_basis": f"{sms} SMs x {sm_max:.0f} MHz x min(128/{ALG_FP32_PER_PAIR} FP32 lanes, "
                              f"16/{ALG_MUFU_PER_PAIR} SFU lanes) pairs per cycle and SM: the SFU binds",
                "at_median_clock": {"sm_mhz": sm_med, "peak": peak_med / 1e9, "frac": achieved / peak_med},
                "impl_count_peak": {"fp32_ops_per_pair": IMPL_FP32_PER_PAIR,
                                    "peak": pair_peak(sms, sm_max, IMPL_FP32_PER_PAIR) / 1e9,
                                    "frac": achieved / pair_peak(sms, sm_max, IMPL_FP32_PER_PAIR)},
                "hbm_write": {"bytes": bytes_matrix, "achieved_GBps": bytes_matrix / t_fill / 1e9,
                              "peak_GBps": hbm, "frac": bytes_matrix / t_fill / 1e9 / hbm},
                "fill_ms": t_fill * 1e3,
                "timing": "CUDA events on the plan's stream around dc_fspb_dose_and_matrix in every timed "
                          "step: the fill kernel plus a row-pointer copy and the per-beam dose sum"}

    # the other forms of the path; one that fails is reported as such and does
    # not take the benchmark line with it
    def form(fn, *fa):
        try:
            return fn(*fa)
        except Exception as exc:                      # noqa: BLE001 (reported in the line)
            torch.cuda.synchronize()
            return {"error": f"{type(exc).__name__}: {exc}"[:300]}

    # the end-to-end step right after the device-timed one, before the other
    # forms fill the host's memory (measured after them, the FP32 variant has
    # taken 44 ms per step, against 32.5 ms measured here)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, dc, p, plan, pairs, torch)
    if args.no_forms:
        forms = {}
    else:
        forms = run_all_forms(form, args, dc, torch, stream, peaks, plan, p, rho_d, flu_d, dose_d, rowptr_d,
                              cols_d, vals_d, flush, step_ms, pairs, sms, sm_max, sm_med, peak_max)
    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline(p, pairs)
        if not args.no_forms:
            forms["plan_error_vs_oracle"] = form(plan_error_vs_oracle, p, dose_d.cpu().numpy())
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"thorax9 {p.grid.nx}x{p.grid.ny}x{p.grid.nz} @0.25cm, 9 fields "
                                   f"8-15 cm, {B} beamlets (0.5 cm), ROI 5 cm, density correction on",
                       "pairs": pairs, "voxels": V, "beamlets": B,
                       "l2": f"flushed before each step ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                       "ranks": "independent plans (one per GPU)",
                       "autotuned_bev_cell_cm": {"tile": tuned[0], "slab": tuned[1]}},
            "stages_ms": {"steps_1_6": float(stage[:, 0].mean()), "pair_count": float(stage[:, 1].mean()),
                          "dose_and_matrix": float(stage[:, 2].mean())},
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "roofline": roofline, "peaks": peak_kind, "forms": forms,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_all_forms(form, args, dc, torch, stream, peaks, plan, p, rho_d, flu_d, dose_d, rowptr_d, cols_d, vals_d,
                  flush, step_ms, pairs, sms, sm_max, sm_med, peak_max):
    """Every other form of the path; one that fails is reported as such and
    does not take the benchmark line with it."""
    forms = form(run_forms, args, dc, torch, stream, peaks)
    forms["dose_only"] = form(run_dose_form, args, dc, torch, stream, plan, p, flu_d, dose_d, flush, pairs,
                              sms, sm_max, sm_med)
    forms["two_pass_plan"] = form(run_two_pass_form, args, dc, torch, stream, plan, rho_d, flu_d, dose_d,
                                  rowptr_d, cols_d, vals_d, flush, float(step_ms.mean()), pairs)
    forms["surrogate"] = form(run_surrogate_form, args, dc, torch, stream, peaks)
    forms["batch"] = form(run_batch_form, args, dc, torch, stream, peak_max)
    forms["gamma"] = form(run_gamma_form, args, dc, torch, stream, p, rho_d, flu_d)
    forms["commissioning"] = form(run_commission_form, args, dc, torch, stream)
    forms["table1"] = form(run_table1_form, args, dc, torch, stream, flush)
    forms["leaf_sequences"] = form(run_leaf_form, args, dc, torch, stream, flush)
    return forms


def run_two_pass_form(args, dc, torch, stream, plan, rho_d, flu_d, dose_d, rowptr_d, cols_d, vals_d, flush,
                      step_ms, pairs):
    """The same plan with the dose and the matrix from two evaluation passes
    (dc_fspb_dose, which also records the row pattern, then the FP32 fill):
    full-plan device time against the benchmark step's single pass, and the
    check that both give the same dose bit for bit."""
    def two_pass():
        dc.dc_fspb_set_density(plan, rho_d)
        dc.dc_fspb_dose(plan, flu_d, dose_d)
        dc.dc_fspb_pair_count(plan)
        dc.dc_fspb_dose_matrix(plan, dc.DC_F32, rowptr_d, cols_d, vals_d)

    ref = dose_d.clone()
    two_pass()
    torch.cuda.synchronize()
    same = bool(torch.equal(ref, dose_d))
    reps = max(3, min(args.steps, 5))
    t = time_on_stream(torch, stream, two_pass, reps, flush)
    return {"workload": "thorax9 plan, dose pass then FP32 matrix fill (each pair evaluated twice)",
            "full_plan_ms": t, "benchmark_step_ms": step_ms, "step_speedup_over_two_pass": t / step_ms,
            "dose_identical_to_step": same}


def run_dose_form(args, dc, torch, stream, plan, p, flu_d, dose_d, flush, pairs, sms, sm_max, sm_med):
    """Eq. (1) alone on the thorax9 plan (dc_fspb_dose: the dose kernel, the
    per-beam sum, two small clears), with the roofline of the dose kernel."""
    reps = max(5, args.steps)
    dc.dc_fspb_dose(plan, flu_d, dose_d)
    t = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose(plan, flu_d, dose_d), reps, flush) * 1e-3
    ach = pairs / t
    return {"workload": "thorax9 plan, eq. (1) only", "ms": t * 1e3, "evals_per_s": ach,
            "roofline": {"kernel": "k_pairs<dose>", "bound": "alu", "achieved": ach / 1e9,
                         "peak": pair_peak(sms, sm_max) / 1e9, "unit": "Gpair/s",
                         "frac": ach / pair_peak(sms, sm_max),
                         "at_median_clock": {"sm_mhz": sm_med, "frac": ach / pair_peak(sms, sm_med)},
                         "traffic": kernel_traffic("dose", args.scale)}}


def plan_error_vs_oracle(p, dose, n_vox=1500, seed=12):
    """The step's dose against the FP64 oracle on seeded voxels of the plan:
    max |D_gpu - D_oracle| over the GPU dose maximum, the same with the dose of
    pairs whose ROI or depth decision lies within rounding taken out, and the
    voxels past the 0.5 % bar."""
    from oracle import oracle
    op = oracle.OraclePlan(p)
    rng = np.random.default_rng(seed)
    d = np.asarray(dose, np.float64).ravel()
    vox = np.sort(rng.choice(d.size, size=min(n_vox, d.size), replace=False))
    want, amb = op.dose_voxels(vox, with_amb=True)
    dmax = float(d.max())
    err = np.abs(d[vox] - want)
    return {"voxels": int(vox.size), "max_err_over_dmax": float(err.max() / dmax),
            "max_err_beyond_ambiguous_over_dmax": float(np.maximum(err - amb, 0).max() / dmax),
            "voxels_over_0p5pct": int((err > 5e-3 * dmax + amb).sum()),
            "normaliser": "GPU dose maximum over the whole plan"}


def time_on_stream(torch, stream, fn, reps, flush):
    """Mean device time (ms) of fn() over reps calls, L2 flushed before each (untimed)."""
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))


def run_forms(args, dc, torch, stream, peaks, k=64):
    """Multi-fluence dose of the single-beam slab plan (64 x 64 x 64 voxels, 400
    beamlets, 64 fluence vectors U[0, 1]): plain FP32 direct evaluation
    (dc_fspb_dose_batch) against the BF16 block-sparse tensor-core SpMM
    (dc_fspb_spmm) on the matrix built once per plan."""
    from paper_1103_1164_gb300 import synth
    p1 = synth.config1()
    rho = torch.from_numpy(p1.rho).cuda()
    plan = dc.dc_fspb_create_from(p1, stream=stream.cuda_stream, device_density=rho)
    F = torch.from_numpy(np.random.default_rng(synth.FLUENCE_SEED).uniform(0, 1, (plan.n_beamlets, k))
                         .astype(np.float32)).cuda()
    Ft = F.t().contiguous()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dose = torch.empty((k, plan.n_voxels), device="cuda")
    Y = torch.empty((plan.n_voxels, k), device="cuda")
    dc.dc_fspb_autotune(plan, F[:, 0].contiguous())
    t0 = time.perf_counter()
    dc.dc_fspb_spmm_prepare(plan)
    prep_s = time.perf_counter() - t0
    chunks, rbs = dc.dc_fspb_spmm_info(plan)
    pairs = dc.dc_fspb_pair_count(plan)
    reps = max(3, args.steps)
    for _ in range(2):
        dc.dc_fspb_dose_batch(plan, Ft, dose)
        dc.dc_fspb_spmm(plan, F, Y)
    t_plain = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose_batch(plan, Ft, dose), reps, flush)
    t_spmm = time_on_stream(torch, stream, lambda: dc.dc_fspb_spmm(plan, F, Y), reps, flush)
    dc.dc_fspb_device_status(plan)
    err = float(((Y.t() - dose).abs().max(1).values / dose.abs().max(1).values).max())
    oracle_err = None
    if not args.no_cpu:
        # per fluence column: max over voxels of |result - M_oracle F| / max of M_oracle F
        want = oracle_multi_fluence(p1, F.cpu().numpy())
        oracle_err = {"bf16_spmm": column_error(Y.cpu().numpy(), want),
                      "plain_fp32": column_error(dose.t().cpu().numpy(), want)}
    # the SpMM's algorithmic bytes: the BF16 matrix (2 B value + 4 B column per
    # nonzero), the FP32 output, the BF16 fluences; the tile bytes the kernel actually streams
    # (128 x 16 BF16 tiles with their zero fill, tile indices, FP32 fluences) beside it
    bytes_alg = pairs * 6 + plan.n_voxels * k * 4 + plan.n_beamlets * k * 2
    bytes_tiles = chunks * 4096 + chunks * 4 + plan.n_voxels * k * 4 + plan.n_beamlets * k * 4
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return {"workload": f"slab64 64^3 @0.25cm, 1 beam, {plan.n_beamlets} beamlets, ROI 3 cm, {k} fluences U[0,1]",
            "pairs": pairs,
            "plain_fp32": {"ms": t_plain, "evals_per_s": pairs * k / (t_plain * 1e-3)},
            "bf16_spmm": {"ms": t_spmm, "evals_per_s": pairs * k / (t_spmm * 1e-3),
                          "tiles_128x16": chunks, "row_blocks": rbs,
                          "tile_fill": pairs / (chunks * 2048.0), "prepare_s": prep_s,
                          "roofline": {"bound": "hbm", "achieved": bytes_alg / (t_spmm * 1e-3) / 1e9,
                                       "peak": hbm, "unit": "GB/s",
                                       "frac": bytes_alg / (t_spmm * 1e-3) / 1e9 / hbm,
                                       "bytes": bytes_alg,
                                       "tile_bytes": bytes_tiles,
                                       "tile_bytes_frac": bytes_tiles / (t_spmm * 1e-3) / 1e9 / hbm},
                          "max_err_vs_fp32_over_colmax": err},
            "max_err_vs_fp64_oracle_over_colmax": oracle_err,
            "speedup_bf16_over_fp32": t_plain / t_spmm}


def oracle_multi_fluence(p, F, lateral_mode=0, voxels=None):
    """M_oracle F in FP64: the oracle's dose-deposition matrix (all voxels, or
    the listed ones) times the fluence columns F [B, k]."""
    from scipy import sparse
    from oracle import oracle
    op = oracle.OraclePlan(p, lateral_mode=lateral_mode)
    rowptr, cols, vals, flags = op.matrix(voxels)
    inside = (flags & 1).astype(bool)
    n = op.V if voxels is None else len(voxels)
    M = sparse.csr_matrix((np.where(inside, vals, 0.0), cols, rowptr), shape=(n, op.B))
    return M @ np.asarray(F, np.float64)


def column_error(got, want):
    """max over columns of max_v |got - want| / max_v |want| (got, want: [V, k])."""
    got = np.asarray(got, np.float64)
    return float((np.abs(got - want).max(0) / (np.abs(want).max(0) + 1e-300)).max())


def run_surrogate_form(args, dc, torch, stream, peaks, k=64):
    """The learned lateral correction: 2M (nearest-tap stencil, plain axis
    densities) samples from 200 random slab/sphere phantoms, trained with the
    library's kernels, then the slab plan's 64-fluence dose with the network's
    correction and the BF16 tensor-core SpMM, against the plain FP32 form (axis
    stencils, direct evaluation), which is also the reference for its error."""
    from paper_1103_1164_gb300 import surrogate, synth
    net = trained_network(dc)
    params, loss, held, n_tr, t_gen, t_train = (net[k] for k in ("params", "loss", "held", "n_train",
                                                                   "generate_s", "train_s"))

    p1 = synth.config1()
    rho = torch.from_numpy(p1.rho).cuda()
    plan = dc.dc_fspb_create_from(p1, stream=stream.cuda_stream, device_density=rho,
                                  lateral_mode=dc.DC_LATERAL_AXIS)
    F = torch.from_numpy(np.random.default_rng(synth.FLUENCE_SEED).uniform(0, 1, (plan.n_beamlets, k))
                         .astype(np.float32)).cuda()
    Ft = F.t().contiguous()
    dose = torch.empty((k, plan.n_voxels), device="cuda")
    Y = torch.empty((plan.n_voxels, k), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dc.dc_fspb_autotune(plan, F[:, 0].contiguous())
    reps = max(3, args.steps)
    # plain FP32 form: axis-stencil factors (per density) + direct 64-fluence evaluation
    t_set_axis = time_on_stream(torch, stream, lambda: dc.dc_fspb_set_density(plan, rho), reps, flush)
    dc.dc_fspb_dose_batch(plan, Ft, dose)
    t_plain = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose_batch(plan, Ft, dose), reps, flush)
    plain = dose.clone()
    # surrogate + BF16 form: network factors (per density), BF16 matrix, tensor-core SpMM
    dc.dc_fspb_set_surrogate(plan, params, surrogate.RHO_LO, surrogate.RHO_HI)
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP)
    t_set_mlp = time_on_stream(torch, stream, lambda: dc.dc_fspb_set_density(plan, rho), reps, flush)
    dc.dc_fspb_spmm_prepare(plan)
    torch.cuda.synchronize()
    preps = []
    for _ in range(3):
        # the BF16 matrix and its tiles, rebuilt for the current density (host wall clock:
        # the call synchronises to learn the pattern's size)
        dc.dc_fspb_set_density(plan, rho)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dc.dc_fspb_spmm_prepare(plan)
        torch.cuda.synchronize()
        preps.append((time.perf_counter() - t0) * 1e3)
    t_prep = float(np.median(preps))
    dc.dc_fspb_spmm(plan, F, Y)
    t_spmm = time_on_stream(torch, stream, lambda: dc.dc_fspb_spmm(plan, F, Y), reps, flush)
    dc.dc_fspb_device_status(plan)
    err = float(((Y.t() - plain).abs().max(1).values / plain.abs().max(1).values).max())
    # the direct tensor-core form (no matrix): the BF16 pair values and
    # fluences of every pair multiplied on the tensor cores, per set of 64
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_BF16)
    dose_tc = torch.empty_like(dose)
    dc.dc_fspb_dose_batch(plan, Ft, dose_tc)
    t_direct = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose_batch(plan, Ft, dose_tc), reps, flush)
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_FP32)
    dc.dc_fspb_device_status(plan)
    # the network's factor pass alone (k_mlp_factors: 48 nearest taps and the
    # network per (voxel, beam) entry), against the BF16 tensor peak
    entries = dc.dc_fspb_list_entries(plan)
    t_fac = time_on_stream(torch, stream, lambda: dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP), reps, flush)
    t_axis_fac = time_on_stream(torch, stream, lambda: dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_AXIS),
                                reps, flush)
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP)
    bf_peak = float(peaks.get("bf16_tflops", 1900.0))
    samples = 8 * n_tr
    net32 = net["fp32"]
    mlp = {"factor_pass": {"kernel": "k_mlp_factors (mma.sync BF16)", "entries": entries, "ms": t_fac,
                           "axis_stencil_pass_ms": t_axis_fac,
                           "tflops": entries * MLP_FWD_FLOP / (t_fac * 1e-3) / 1e12,
                           "frac_of_bf16_peak": entries * MLP_FWD_FLOP / (t_fac * 1e-3) / 1e12 / bf_peak},
           "training_bf16": {"kernel": "k_mlp_grad_bf16 + k_mlp_adam (8 epochs, host wall clock, staging included)",
                             "s": t_train, "samples_per_s": samples / t_train,
                             "tflops": samples * MLP_TRAIN_FLOP / t_train / 1e12,
                             "frac_of_bf16_peak": samples * MLP_TRAIN_FLOP / t_train / 1e12 / bf_peak},
           "training_fp32": {"s": net32["train_s"], "samples_per_s": samples / net32["train_s"],
                             "held_out_p50": float(np.median(net32["held"])),
                             "held_out_p99": float(np.percentile(net32["held"], 99))}}
    oracle_err = None
    if not args.no_cpu:
        # against the FP64 oracle's axis-stencil form (the method the network
        # stands in for) on seeded voxels, all 64 fluence columns
        vox = np.sort(np.random.default_rng(21).choice(plan.n_voxels, 3000, replace=False))
        want = oracle_multi_fluence(p1, F.cpu().numpy(), lateral_mode=1, voxels=vox)
        oracle_err = {"surrogate_bf16": column_error(Y.cpu().numpy()[vox], want),
                      "surrogate_bf16_direct": column_error(dose_tc.t().cpu().numpy()[vox], want),
                      "plain_fp32_axis": column_error(plain.t().cpu().numpy()[vox], want),
                      "voxels": int(vox.size)}

    def surrogate_ms(n):
        # the faster surrogate + BF16 form for n sets of 64 fluences per density
        return min(t_set_mlp + t_prep + n * t_spmm, t_set_mlp + n * t_direct)

    sets_3x = next((n for n in range(1, 1001) if t_set_axis + n * t_plain >= 3.0 * surrogate_ms(n)), None)
    return {"workload": f"slab64 64^3 @0.25cm, 1 beam, {plan.n_beamlets} beamlets, {k} fluences U[0,1]; "
                        f"network 48-64-64-3 SiLU trained on {n_tr} stencils from 200 random phantoms",
            "samples_generate_s": t_gen, "train_s": t_train, "train_loss": loss,
            "held_out_abs_err_density": {"p50": float(np.median(held)), "p99": float(np.percentile(held, 99))},
            "plain_fp32_axis": {"set_density_ms": t_set_axis, "dose_64_ms": t_plain},
            "surrogate_bf16": {"set_density_ms": t_set_mlp, "spmm_prepare_ms": t_prep, "spmm_64_ms": t_spmm,
                               "fallbacks": dc.dc_fspb_lateral_fallbacks(plan)},
            "surrogate_bf16_direct": {"set_density_ms": t_set_mlp, "dose_64_ms": t_direct},
            "speedup_one_set_of_64": (t_set_axis + t_plain) / surrogate_ms(1),
            "speedup_one_set_by_form": {"matrix_spmm": (t_set_axis + t_plain) / (t_set_mlp + t_prep + t_spmm),
                                        "direct_tensor_core": (t_set_axis + t_plain) / (t_set_mlp + t_direct)},
            "speedup_per_further_set_of_64": t_plain / min(t_spmm, t_direct),
            "sets_of_64_for_3x": sets_3x,
            "accounting": "per density: factors (+ matrix build for the matrix form); per set of 64 "
                          "fluences: the direct batch, the SpMM or the direct tensor-core pass; the "
                          "surrogate figures take the faster form for the number of sets",
            "max_err_vs_plain_over_colmax": err,
            "max_err_vs_fp64_oracle_over_colmax": oracle_err,
            "network_kernels": mlp}


_NETWORK = {}


MLP_FWD_FLOP = 2 * (48 * 64 + 64 * 64 + 64 * 3)      # 14,720 per sample
MLP_TRAIN_FLOP = 3 * MLP_FWD_FLOP                     # forward + the two products of the backward pass


def trained_network(dc):
    """The surrogate network of config 4, trained once per process: 2M
    (nearest-tap stencil, plain axis densities) samples from 200 random
    slab/sphere phantoms, 90 % trained with the library's BF16 tensor-core
    kernels (8 epochs, batch 4096, Adam, FP32 master parameters), 10 % held
    out; the same schedule with the FP32 kernels for comparison."""
    if not _NETWORK:
        from paper_1103_1164_gb300 import surrogate
        t0 = time.perf_counter()
        X, T = surrogate.generate_samples(n_phantoms=200, per_phantom=10000, seed=2024)
        t_gen = time.perf_counter() - t0
        n_tr = int(0.9 * X.shape[0])
        res = {}
        for name, prec in (("bf16", dc.DC_PRECISION_BF16), ("fp32", dc.DC_PRECISION_FP32)):
            import torch
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            params, loss = surrogate.train(X[:n_tr], T[:n_tr], epochs=8, batch=4096, lr=2e-3, seed=17,
                                           precision=prec)
            t_train = time.perf_counter() - t0
            held = np.abs(dc.dc_mlp_predict(params, X[n_tr:]) - T[n_tr:]).max(1)
            res[name] = dict(params=params, loss=loss, held=held, train_s=t_train)
        b = res["bf16"]
        _NETWORK.update(params=b["params"], loss=b["loss"], held=b["held"], n_train=n_tr, generate_s=t_gen,
                        train_s=b["train_s"], fp32=res["fp32"])
    return _NETWORK


def run_commission_form(args, dc, torch, stream, iterations=400):
    """The commissioning fit of Section 2.1 on the synthetic model: reference
    doses of the six slab phantoms (30 cm water cube, 15 cm slab of density
    0.1-2.0 at 8 cm, 10 x 10 cm2 field, SSD 90 cm, 0.5 cm voxels and beamlets)
    computed with the seeded model; the fit starts 20 % away and runs Adam on
    the model's twelve parameters with gradients from the backward-pass kernel,
    then Levenberg-Marquardt from the same start.
    Device time of one backward pass, host wall time per iteration (six
    plans: new tables, density steps, dose, backward pass), the loss and the
    recovered parameters."""
    from paper_1103_1164_gb300 import commission as cmn, synth
    true = synth.model_params()
    cm = synth.make_commissioning(roi_radius=5.0)
    dens = (0.1, 0.25, 0.5, 1.0, 1.5, 2.0)
    inputs = [cmn.slab_phantom(r, vox=0.5, comm=cm) for r in dens]
    refp = [dc.dc_fspb_create_from(q, stream=stream.cuda_stream) for q in inputs]
    ref = [dc.dc_fspb_dose(pl, q.fluence) for pl, q in zip(refp, inputs)]
    pairs = sum(dc.dc_fspb_pair_count(pl) for pl in refp)
    for pl in refp:
        dc.dc_fspb_destroy(pl)
    fit = cmn.CommissioningFit(inputs, ref, stream=stream.cuda_stream)
    rng = np.random.default_rng(3)
    th0 = {k: (true[k] + 0.006 if k in cmn.LINEAR else true[k] * float(rng.uniform(0.8, 1.2))) for k in cmn.PARAMS}
    # device time of the backward pass on one phantom (device buffers)
    q0, pl0 = inputs[3], fit.plans[3]
    w_n, f_n = cm.water.shape[1], cm.dens.shape[1]
    flu = torch.from_numpy(q0.fluence).cuda()
    wv = torch.rand(pl0.n_voxels, device="cuda")
    out = (torch.empty(4, w_n, device="cuda"), torch.empty(4, f_n, device="cuda"), torch.empty(2, device="cuda"))
    dummy = torch.empty(1, device="cuda")
    vjp = lambda: dc.dc_fspb_dose_vjp(pl0, flu, wv, w_n, f_n, out=out)
    vjp()
    t_vjp = time_on_stream(torch, stream, vjp, 5, dummy)
    t_dose = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose(pl0, flu, wv), 5, dummy)
    pairs0 = dc.dc_fspb_pair_count(pl0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fit.fit(th0, iterations=iterations, lr=0.02)
    wall = time.perf_counter() - t0
    t0 = time.perf_counter()
    rl = fit.fit_lm(th0, iterations=25)
    wall_lm = time.perf_counter() - t0
    fit.destroy()
    rel = {k: (r.theta[k] - true[k]) / abs(true[k]) for k in cmn.PARAMS}
    rel_lm = {k: (rl.theta[k] - true[k]) / abs(true[k]) for k in cmn.PARAMS}
    return {"workload": "6 slab phantoms (Section 2.1 geometry), 60^3 voxels of 0.5 cm, 400 beamlets each, "
                        f"{pairs} pairs in all; 12 model parameters from 20 % away",
            "iterations": r.iterations, "fit_s": wall, "ms_per_iteration": 1e3 * wall / r.iterations,
            "loss_first": r.loss[0], "loss_last": r.loss[-1],
            "param_rel_err": rel,
            "levenberg_marquardt": {"iterations": rl.iterations, "fit_s": wall_lm,
                                    "ms_per_iteration": 1e3 * wall_lm / rl.iterations,
                                    "loss_last": rl.loss[-1], "param_rel_err": rel_lm,
                                    "max_abs_rel_err": max(abs(v) for v in rel_lm.values()),
                                    "jacobian": "gradient from the backward-pass kernel; J^T J from forward "
                                                "differences of the doses (one set of doses per parameter and iteration)"},
            "backward_pass": {"ms": t_vjp, "pairs": pairs0, "pairs_per_s": pairs0 / (t_vjp * 1e-3),
                              "forward_dose_ms": t_dose},
            "reference": "doses of the seeded model computed by the library (a synthetic reference)"}


def run_gamma_form(args, dc, torch, stream, p, rho_d, flu_d):
    """The 3 %-3 mm gamma index of plain FSPB (no density correction) against
    DC-FSPB on the thorax plan (dc_gamma_index, device buffers), the paper's
    accuracy statistics of the density correction's effect; the FP64 oracle
    on seeded voxels gives its CPU rate."""
    import dataclasses
    from oracle import gamma as og
    ref = torch.empty(p.grid.shape, device="cuda")
    ev = torch.empty(p.grid.shape, device="cuda")
    pq = dataclasses.replace(p, comm=dataclasses.replace(p.comm, density_correction=0))
    for inp, out in ((p, ref), (pq, ev)):
        plan = dc.dc_fspb_create_from(inp, stream=stream.cuda_stream, device_density=rho_d)
        dc.dc_fspb_dose(plan, flu_d, out)
        del plan
    gamma = torch.empty_like(ref)
    with torch.cuda.stream(stream):
        for _ in range(2):
            dc.dc_gamma_index(ref, ev, p.grid, gamma=gamma, stream=stream.cuda_stream)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = dc.dc_gamma_index(ref, ev, p.grid, gamma=gamma, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    V = p.grid.n_voxels
    out = {"workload": f"FSPB vs DC-FSPB doses of thorax9 ({V} voxels), 3 %-3 mm, search 1.5 cm",
           "ms": ms, "voxels_per_s": V / (ms * 1e-3), **st}
    if not args.no_cpu:
        r, e = ref.cpu().numpy(), ev.cpu().numpy()
        vox = np.random.default_rng(4).choice(V, 4000, replace=False)
        t0 = time.perf_counter()
        want = og.gamma_at(r, e, (p.grid.dx, p.grid.dy, p.grid.dz), vox)
        dt = time.perf_counter() - t0
        out["oracle_voxels_per_s"] = vox.size / dt
        out["max_abs_diff_vs_oracle"] = float(np.abs(gamma.cpu().numpy().ravel()[vox] - want).max())
    return out


# Table 4: g-DC-FSPB GPU computation time T_gpu (s) per case on a Tesla C1060
# (the paper's hardware; context for the synthetic stand-ins, not a target).
TABLE4_TGPU_S = {"H1": 0.64, "H2": 0.40, "H3": 0.38, "H4": 0.35, "H5": 1.31,
                 "L1": 0.22, "L2": 0.40, "L3": 0.30, "L4": 0.25, "L5": 0.33}


def run_table1_form(args, dc, torch, stream, flush):
    """The ten synthetic Table 1 cases (128 x 128 x 72-103 at 0.4 x 0.4 x 0.25 cm,
    5-8 coplanar or non-coplanar beams, 637-10,369 beamlets of 0.2 x 0.5 cm):
    per case the GPU time of the density-dependent steps plus the dose (the
    paper's T_gpu: smoothing, beamlet geometry, ray tracing, tables, binning,
    eq. 1) with the default binning cell and again after dc_fspb_autotune; then,
    on the tuned plan, the same through pinned host buffers (density and
    fluence in, dose out: T_gpu + T_tr, host wall clock) and all ten cases as
    one batch graph."""
    from paper_1103_1164_gb300 import synth
    inputs = synth.table1_plans()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    cases, plans, flus = [], [], []
    reps = max(3, min(args.steps, 5))
    for p in inputs:
        rho_d = torch.from_numpy(p.rho).cuda()
        flu_d = torch.from_numpy(p.fluence).cuda()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        plan = dc.dc_fspb_create_from(p, stream=stream.cuda_stream, device_density=rho_d)
        torch.cuda.synchronize()
        t_create = (time.perf_counter() - w0) * 1e3
        dose_d = torch.empty(plan.shape, device="cuda")

        def gpu_step():
            dc.dc_fspb_set_density(plan, rho_d)
            dc.dc_fspb_dose(plan, flu_d, dose_d)

        gpu_step()
        t_gpu = time_on_stream(torch, stream, gpu_step, reps, flush)
        t_dose = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose(plan, flu_d, dose_d), reps, flush)
        tuned = dc.dc_fspb_autotune(plan, flu_d)
        t_gpu_tuned = time_on_stream(torch, stream, gpu_step, reps, flush)
        t_dose_tuned = time_on_stream(torch, stream, lambda: dc.dc_fspb_dose(plan, flu_d, dose_d), reps, flush)
        pairs = dc.dc_fspb_pair_count(plan)
        rho_h, flu_h = pin(p.rho), pin(p.fluence)
        dose_h = torch.empty(plan.shape, dtype=torch.float32).pin_memory()
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            dc.dc_fspb_set_density(plan, rho_h.numpy())
            dc.dc_fspb_dose(plan, flu_h.numpy(), dose_h.numpy())
            ts.append((time.perf_counter() - w0) * 1e3)
        diff = float((dose_h.cuda() - dose_d).abs().max() / dose_d.abs().max())
        cases.append({"case": p.name, "beams": len(p.beams),
                      "non_coplanar": any(b.couch_deg != 0.0 for b in p.beams),
                      "beamlets": plan.n_beamlets, "voxels": plan.n_voxels, "pairs": pairs,
                      "create_ms": t_create, "t_gpu_ms": t_gpu, "dose_ms": t_dose,
                      "autotuned": {"tile_cm": tuned[0], "slab_cm": tuned[1], "t_gpu_ms": t_gpu_tuned,
                                    "dose_ms": t_dose_tuned},
                      "t_tot_host_buffers_ms": float(np.median(ts)),
                      "evals_per_s": 2 * pairs / (t_gpu * 1e-3),
                      "paper_t_gpu_ms_c1060": 1e3 * TABLE4_TGPU_S[p.name],
                      "host_vs_device_max_diff_over_max": diff})
        plans.append(plan)
        flus.append(flu_d)
    batch = dc.dc_fspb_batch_create(plans, stream=stream.cuda_stream)
    for j, pl in enumerate(plans):
        fptr, _ = dc.dc_fspb_batch_buffers(batch, j)
        dc_view(torch, fptr, pl.n_beamlets).copy_(flus[j])
    for _ in range(2):
        dc.dc_fspb_batch_run(batch, density=True)
    t_batch = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch, density=True), reps, flush)
    t_batch_dose = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch), reps, flush)
    tg = [c["t_gpu_ms"] for c in cases]
    pairs = sum(c["pairs"] for c in cases)
    return {"workload": "10 synthetic Table 1 cases (H1-H5 head-and-neck, L1-L5 lung), "
                        "128x128x72-103 @0.4x0.4x0.25 cm, 0.2x0.5 cm beamlets, ROI 5 cm, "
                        "density correction on",
            "cases": cases, "pairs": pairs,
            "sum_t_gpu_ms": float(sum(tg)), "median_t_gpu_ms": float(np.median(tg)),
            "paper_median_t_gpu_ms_c1060": 1e3 * float(np.median(list(TABLE4_TGPU_S.values()))),
            "batch_graph": {"full_plans_ms": t_batch, "dose_ms": t_batch_dose,
                            "evals_per_s": 2 * pairs / (t_batch * 1e-3),
                            "kernels_per_replay": dc.dc_fspb_batch_kernels(batch)}}


def run_leaf_form(args, dc, torch, stream, flush, n_cp=128):
    """Replanning loop on the largest Table 1 case (H5, 7 non-coplanar beams,
    10,369 beamlets of 0.2 x 0.5 cm): each iteration turns new sliding-window
    leaf sequences (n_cp control points per beam, host memory) into the
    fluence (dc_fluence_from_leaves) and the dose of the cached plan.  Device
    time of the fluence step and of fluence + dose; host wall time of an
    iteration through host buffers (sequences in, dose out)."""
    from paper_1103_1164_gb300 import synth
    p = synth.table1_case("H5")
    seqs = [synth.plan_sequences(p, 2000 + k, "sliding", n_cp=n_cp, transmission=0.015) for k in range(4)]
    rho_d = torch.from_numpy(p.rho).cuda()
    plan = dc.dc_fspb_create_from(p, stream=stream.cuda_stream, device_density=rho_d)
    flu_d = torch.empty(plan.n_beamlets, device="cuda")
    dose_d = torch.empty(plan.shape, device="cuda")
    dc.dc_fspb_autotune(plan, torch.from_numpy(p.fluence).cuda())
    reps = max(3, min(args.steps, 5))
    it = iter(range(1 << 30))
    nxt = lambda: seqs[next(it) % len(seqs)]
    for _ in range(2):
        dc.dc_fluence_from_leaves(plan, nxt(), flu_d)
        dc.dc_fspb_dose(plan, flu_d, dose_d)
    torch.cuda.synchronize()
    t_flu = time_on_stream(torch, stream, lambda: dc.dc_fluence_from_leaves(plan, nxt(), flu_d), reps, flush)

    def flu_dose():
        dc.dc_fluence_from_leaves(plan, nxt(), flu_d)
        dc.dc_fspb_dose(plan, flu_d, dose_d)

    t_both = time_on_stream(torch, stream, flu_dose, reps, flush)
    dose_h = torch.empty(plan.shape, dtype=torch.float32).pin_memory().numpy()
    flu_h = np.empty(plan.n_beamlets, np.float32)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        dc.dc_fluence_from_leaves(plan, nxt(), flu_h)
        dc.dc_fspb_dose(plan, flu_h, dose_h)
        ts.append((time.perf_counter() - w0) * 1e3)
    out = {"workload": f"H5 ({plan.n_beamlets} beamlets, 7 non-coplanar beams), sliding-window sequences "
                       f"of {n_cp} control points per beam, 0.5 cm leaves, 1.5 % transmission",
           "fluence_ms": t_flu, "fluence_plus_dose_ms": t_both,
           "iteration_host_buffers_ms": float(np.median(ts)),
           "beamlet_intervals_per_s": plan.n_beamlets * (n_cp - 1) / (t_flu * 1e-3)}
    if not args.no_cpu:
        from oracle import fluence as ofl
        t0 = time.perf_counter()
        fo = ofl.plan_fluence(p, seqs[0])
        out["oracle_fluence_ms"] = (time.perf_counter() - t0) * 1e3
        dc.dc_fluence_from_leaves(plan, seqs[0], flu_h)
        out["max_diff_vs_oracle_over_mu"] = float(np.abs(flu_h - fo).max() / 100.0)
    return out


def run_batch_form(args, dc, torch, stream, peak_pairs):
    """The 16 uneven head-and-neck plans (grids 112 x 112 x 64 to 256 x 256 x 192
    at 0.2-0.3 cm, 5-9 beams, 0.25 cm beamlets, ROI 5 cm), each plan's binning
    cell autotuned at set-up: one persistent
    graph-replayed launch over all plans (dc_fspb_batch_run) against the plans'
    own launches one after another, dose only and whole plans (density-dependent
    steps + dose), in the paper's lateral form.  Then the cross-form
    comparison on the same batch: the plain form (axis-stencil lateral
    densities, FP32 evaluation) against the surrogate + BF16 form (the trained
    network's lateral densities, packed-BF16 exponentials), whole plans and
    dose only, each with its error against the FP64 oracle's axis form on
    seeded voxels of the largest and the smallest plan."""
    from paper_1103_1164_gb300 import surrogate, synth
    t0 = time.perf_counter()
    inputs = synth.config5_plans()
    t_gen = time.perf_counter() - t0
    rhos = [torch.from_numpy(p.rho).cuda() for p in inputs]
    flus = [torch.from_numpy(p.fluence).cuda() for p in inputs]
    plans = [dc.dc_fspb_create_from(p, stream=stream.cuda_stream, device_density=r) for p, r in zip(inputs, rhos)]
    doses = [torch.empty(pl.n_voxels, device="cuda") for pl in plans]
    t0 = time.perf_counter()
    cells = [dc.dc_fspb_autotune(pl, f)[:2] for pl, f in zip(plans, flus)]   # plan set-up, untimed
    t_cells = time.perf_counter() - t0
    pairs = [dc.dc_fspb_pair_count(pl) for pl in plans]
    batch = dc.dc_fspb_batch_create(plans, stream=stream.cuda_stream)
    for j, pl in enumerate(plans):
        fptr, _ = dc.dc_fspb_batch_buffers(batch, j)
        dc_view(torch, fptr, pl.n_beamlets).copy_(flus[j])
    variant, tune_ms = dc.dc_fspb_batch_autotune(batch)
    reps = max(3, min(args.steps, 5))
    dummy = torch.empty(1, device="cuda")   # inputs far exceed L2: no flush needed

    def seq_dose():
        for pl, f, d in zip(plans, flus, doses):
            dc.dc_fspb_dose(pl, f, d)

    def seq_full():
        for pl, r, f, d in zip(plans, rhos, flus, doses):
            dc.dc_fspb_set_density(pl, r)
            dc.dc_fspb_dose(pl, f, d)

    for _ in range(2):
        dc.dc_fspb_batch_run(batch)
        dc.dc_fspb_batch_run(batch, density=True)
        seq_dose()
    torch.cuda.synchronize()
    l0 = dc.dc_fspb_launch_count()
    t_batch = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch), reps, dummy)
    launches = (dc.dc_fspb_launch_count() - l0) / reps
    t_full = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch, density=True), reps, dummy)
    t_seq = time_on_stream(torch, stream, seq_dose, reps, dummy)
    t_seq_full = time_on_stream(torch, stream, seq_full, reps, dummy)
    err = 0.0
    for j, d in enumerate(doses):
        _, dptr = dc.dc_fspb_batch_buffers(batch, j)
        b = dc_view(torch, dptr, plans[j].n_voxels)
        err = max(err, float((b - d).abs().max() / d.abs().max()))
    total = int(sum(pairs))
    ach = total / (t_batch * 1e-3)
    out = {"workload": f"{len(plans)} head-and-neck plans, {sum(pl.n_voxels for pl in plans)} voxels, "
                       f"{sum(len(p.beams) for p in inputs)} beams, {sum(pl.n_beamlets for pl in plans)} "
                       f"beamlets (0.25 cm), ROI 5 cm, density correction on",
           "pairs": total, "generate_s": t_gen,
           "bev_cells_cm": {"autotune_s": t_cells,
                            "chosen": sorted({f"{t:g}x{sl:g}" for t, sl in cells})},
           "batch_graph": {"dose_ms": t_batch, "full_plans_ms": t_full, "evals_per_s": ach,
                           "kernels_per_replay": launches,
                           "autotuned_variant": ("persistent, 4 CTAs per SM", "persistent, 5 CTAs per SM",
                                                 "per-plan launches in the graph")[variant],
                           "autotune_ms": tune_ms,
                           "roofline": {"bound": "alu", "achieved": ach / 1e9, "peak": peak_pairs / 1e9,
                                        "unit": "Gpair/s", "frac": ach / peak_pairs}},
           "sequential_plans": {"dose_ms": t_seq, "full_plans_ms": t_seq_full,
                                "evals_per_s": total / (t_seq * 1e-3)},
           "speedup_batch_over_sequential": {"dose": t_seq / t_batch, "full_plans": t_seq_full / t_full},
           "max_diff_batch_vs_sequential_over_max": err}

    # the cross-form comparison: plain (axis stencils, FP32) against surrogate + BF16
    net = trained_network(dc)
    big = int(np.argmax([pl.n_voxels for pl in plans]))
    small = int(np.argmin([pl.n_voxels for pl in plans]))
    forms = {}
    for name, mode, prec in (("plain_fp32_axis", dc.DC_LATERAL_AXIS, dc.DC_PRECISION_FP32),
                             ("surrogate_bf16", dc.DC_LATERAL_MLP, dc.DC_PRECISION_BF16)):
        for pl in plans:
            if mode == dc.DC_LATERAL_MLP:
                dc.dc_fspb_set_surrogate(pl, net["params"], surrogate.RHO_LO, surrogate.RHO_HI)
            dc.dc_fspb_set_lateral_mode(pl, mode)
            dc.dc_fspb_set_precision(pl, prec)
        for _ in range(2):
            dc.dc_fspb_batch_run(batch, density=True)
        torch.cuda.synchronize()
        t_f = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch, density=True), reps, dummy)
        t_d = time_on_stream(torch, stream, lambda: dc.dc_fspb_batch_run(batch), reps, dummy)
        r = {"full_plans_ms": t_f, "dose_ms": t_d, "evals_per_s_dose": total / (t_d * 1e-3),
             "fallbacks": int(sum(dc.dc_fspb_lateral_fallbacks(pl) for pl in plans)) if mode == dc.DC_LATERAL_MLP
             else 0}
        if not args.no_cpu:
            errs = {}
            for tag, j in (("largest", big), ("smallest", small)):
                _, dptr = dc.dc_fspb_batch_buffers(batch, j)
                errs[tag] = batch_plan_error(inputs[j], dc_view(torch, dptr, plans[j].n_voxels).cpu().numpy())
            r["error_vs_fp64_oracle_axis"] = errs
        forms[name] = r
    p_, s_ = forms["plain_fp32_axis"], forms["surrogate_bf16"]
    out["cross_form"] = {
        "forms": forms,
        "speedup_surrogate_bf16_over_plain_fp32": {"full_plans": p_["full_plans_ms"] / s_["full_plans_ms"],
                                                   "dose_only": p_["dose_ms"] / s_["dose_ms"]},
        "target": ">= 3x at <= 1 % of max dose against the FP64 oracle",
        "fallback_rule": "stencils with a density outside the network's training range [0.05, 2.0] "
                         "(air cavities, the body surface) use the axis computation"}
    for pl in plans:
        dc.dc_fspb_set_lateral_mode(pl, dc.DC_LATERAL_ISO)
        dc.dc_fspb_set_precision(pl, dc.DC_PRECISION_FP32)
    # the same plans with 64 fluence vectors each, one plan resident at a time
    # (the BF16 matrix of the largest is tens of GB)
    del batch, plans, doses, rhos, flus
    torch.cuda.synchronize()
    out["multi_fluence_64"] = run_batch_multi_fluence(args, dc, torch, inputs, net)
    return out


def run_batch_multi_fluence(args, dc, torch, inputs, net, k=64):
    """The 16 head-and-neck plans with k fluence vectors each (uniform [0, 1],
    seeded), the two forms of the multi-fluence dose, plan after
    plan: plain = axis-stencil lateral densities and the FP32 direct
    evaluation of the k vectors (dc_fspb_dose_batch); surrogate + BF16 = the
    network's lateral densities with, either, the BF16 dose-deposition matrix
    (dc_fspb_spmm_prepare) and the tensor-core SpMM (dc_fspb_spmm), or the
    direct tensor-core form (dc_fspb_dose_batch in the reduced-precision
    setting: the pair values and fluences in BF16, their products on the
    tensor cores, no matrix).  Host wall clock around each plan's calls (all
    forms synchronise), cells autotuned at set-up.  The surrogate forms' cost
    per density (factors, + matrix) and per set of k vectors are reported
    apart, with the number of sets at which the faster of them is 3x faster;
    their error against the FP64 oracle's axis form on seeded voxels of the
    largest and the smallest plan, every column."""
    from paper_1103_1164_gb300 import surrogate
    peaks, _ = measured_peaks()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1005)
    big = int(np.argmax([p.grid.nx * p.grid.ny * p.grid.nz for p in inputs]))
    small = int(np.argmin([p.grid.nx * p.grid.ny * p.grid.nz for p in inputs]))

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0)

    acc = {"plain_ms": 0.0, "surrogate_density_ms": 0.0, "surrogate_spmm_ms": 0.0, "surrogate_factors_ms": 0.0,
           "surrogate_direct_ms": 0.0}
    errs = {}
    pairs_total = 0
    bytes_alg = bytes_tiles = 0
    for j, p in enumerate(inputs):
        rho = torch.from_numpy(p.rho).cuda()
        plan = dc.dc_fspb_create_from(p, device_density=rho)
        dc.dc_fspb_autotune(plan, torch.from_numpy(p.fluence).cuda())
        B, V = plan.n_beamlets, plan.n_voxels
        F = torch.rand(B, k, device="cuda", generator=gen)
        Ft = F.t().contiguous()
        D = torch.empty(k, V, device="cuda")
        Y = torch.empty(V, k, device="cuda")
        dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_AXIS)
        plain = lambda: (dc.dc_fspb_set_density(plan, rho), dc.dc_fspb_dose_batch(plan, Ft, D))
        plain()
        acc["plain_ms"] += wall(plain)
        dc.dc_fspb_set_surrogate(plan, net["params"], surrogate.RHO_LO, surrogate.RHO_HI)
        dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP)
        per_density = lambda: (dc.dc_fspb_set_density(plan, rho), dc.dc_fspb_spmm_prepare(plan))
        per_density()
        dc.dc_fspb_spmm(plan, F, Y)
        acc["surrogate_density_ms"] += wall(per_density)
        acc["surrogate_spmm_ms"] += wall(lambda: dc.dc_fspb_spmm(plan, F, Y))
        npairs = dc.dc_fspb_pair_count(plan)
        pairs_total += npairs
        chunks, _ = dc.dc_fspb_spmm_info(plan)
        # per set of k: the matrix's algorithmic bytes (2 B value + 4 B column per
        # nonzero), the FP32 output, the BF16 fluences; the bytes the SpMM streams
        # (4 KB tiles and their indices, the FP32 partial rows of every beam
        # written and read back, the output)
        bytes_alg += npairs * 6 + V * k * 4 + B * k * 2
        items = dc.dc_fspb_list_entries(plan) if len(p.beams) > 1 else 0
        bytes_tiles += chunks * (4096 + 4) + 2 * items * k * 4 + V * k * 4 + B * k * 4
        # the direct tensor-core form (after the matrix's figures: a new density
        # drops the tiles): per density the network's factors, per
        # set the BF16 evaluation of every pair for the k vectors
        acc["surrogate_factors_ms"] += wall(lambda: dc.dc_fspb_set_density(plan, rho))
        dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_BF16)
        Dt = torch.empty(k, V, device="cuda")
        dc.dc_fspb_dose_batch(plan, Ft, Dt)
        acc["surrogate_direct_ms"] += wall(lambda: dc.dc_fspb_dose_batch(plan, Ft, Dt))
        dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_FP32)
        if not args.no_cpu and j in (big, small):
            # seeded voxels, half of them above 10 % of the first column's maximum
            d0 = D[0].cpu().numpy()
            rng = np.random.default_rng(41)
            hot = np.flatnonzero(d0 > 0.1 * d0.max())
            vox = np.unique(np.concatenate([rng.integers(0, V, 150), rng.choice(hot, 150)]))
            want = oracle_multi_fluence(p, F.cpu().numpy(), lateral_mode=1, voxels=vox)
            # per column: max over the voxels of |error| over the column's maximum dose (GPU plain form)
            colmax = D.abs().max(1).values.cpu().numpy().astype(np.float64)
            e = np.abs(Y.cpu().numpy()[vox].astype(np.float64) - want).max(0) / colmax
            ep = np.abs(D.t().cpu().numpy()[vox].astype(np.float64) - want).max(0) / colmax
            et = np.abs(Dt.t().cpu().numpy()[vox].astype(np.float64) - want).max(0) / colmax
            errs["largest" if j == big else "smallest"] = {"voxels": int(vox.size),
                                                           "surrogate_bf16": float(e.max()),
                                                           "surrogate_bf16_direct": float(et.max()),
                                                           "plain_fp32_axis": float(ep.max())}
        del plan, D, Dt, Y, F, Ft, rho
        torch.cuda.empty_cache()
    sur_one = acc["surrogate_density_ms"] + acc["surrogate_spmm_ms"]
    per_set = acc["surrogate_spmm_ms"]
    direct_one = acc["surrogate_factors_ms"] + acc["surrogate_direct_ms"]

    def surrogate_ms(n):
        # the faster surrogate + BF16 form for n sets of k vectors per density
        return min(acc["surrogate_density_ms"] + n * per_set,
                   acc["surrogate_factors_ms"] + n * acc["surrogate_direct_ms"])

    sets_3x = None
    for n in range(1, 1001):
        if n * acc["plain_ms"] >= 3.0 * surrogate_ms(n):
            sets_3x = n
            break
    return {"workload": f"the 16 plans, {k} fluence vectors U[0,1] each ({pairs_total} pairs per vector)",
            "plain_fp32_axis_ms": acc["plain_ms"],
            "surrogate_bf16": {"per_density_ms": acc["surrogate_density_ms"],
                               "per_set_of_64_ms": per_set, "one_set_ms": sur_one},
            "surrogate_bf16_direct": {"per_density_ms": acc["surrogate_factors_ms"],
                                      "per_set_of_64_ms": acc["surrogate_direct_ms"], "one_set_ms": direct_one},
            "speedup_one_set": acc["plain_ms"] / surrogate_ms(1),
            "speedup_one_set_by_form": {"matrix_spmm": acc["plain_ms"] / sur_one,
                                        "direct_tensor_core": acc["plain_ms"] / direct_one},
            "speedup_per_further_set": acc["plain_ms"] / min(per_set, acc["surrogate_direct_ms"]),
            "sets_of_64_for_3x": sets_3x,
            "evals_per_s": {"plain": pairs_total * k / (acc["plain_ms"] * 1e-3),
                            "surrogate_bf16_one_set": pairs_total * k / (sur_one * 1e-3)},
            "spmm_roofline": {"bound": "hbm", "achieved": bytes_alg / (per_set * 1e-3) / 1e9,
                              "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                              "frac": bytes_alg / (per_set * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
                              "bytes": bytes_alg, "streamed_bytes": bytes_tiles,
                              "streamed_frac": bytes_tiles / (per_set * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
                              "timing": "host wall clock per plan around dc_fspb_spmm (fluence packing, "
                                        "the tensor-core product, the per-beam reduction)"},
            "timing": "host wall clock, synchronised, around each plan's calls; cells autotuned at set-up",
            "max_err_vs_fp64_oracle_axis_over_colmax": errs or None}


def batch_plan_error(p, dose, n_vox=800, seed=31):
    """A batch plan's dose against the FP64 oracle's axis-form dose on seeded
    voxels: max |D - D_oracle| over the dose maximum of the plan (GPU), with
    the dose of ambiguous pairs allowed on top."""
    from oracle import oracle
    op = oracle.OraclePlan(p, lateral_mode=1)
    d = np.asarray(dose, np.float64).ravel()
    rng = np.random.default_rng(seed)
    hot = np.flatnonzero(d > 0.1 * d.max())       # half the sample above 10 % of the maximum
    vox = np.unique(np.concatenate([rng.integers(0, d.size, n_vox // 2), rng.choice(hot, n_vox // 2)]))
    want, amb = op.dose_voxels(vox, with_amb=True)
    dmax = float(d.max())
    e = np.abs(d[vox] - want)
    return {"voxels": int(vox.size), "max_err_over_dmax": float(e.max() / dmax),
            "max_err_beyond_ambiguous_over_dmax": float(np.maximum(e - amb, 0).max() / dmax)}


def dc_view(torch, ptr, n):
    """torch view (no copy) of a float32 device buffer owned by the library."""
    class _A:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                    "strides": None}
    return torch.as_tensor(_A(), device="cuda")


def run_e2e(args, dc, p, plan, pairs, torch):
    """The benchmark step through the C ABI with page-locked host buffers (from
    PyTorch's pinned allocator): every H2D/D2H copy of the step's inputs and
    results is inside the timed region (host wall clock over the same number
    of steps as the device-timed value).  Variants: the matrix values in BF16,
    and the dose alone (no matrix)."""
    V, B = plan.n_voxels, plan.n_beamlets
    dtypes = {np.float32: torch.float32, np.int32: torch.int32, np.int64: torch.int64, np.uint16: torch.int16}

    def pin(shape, dt):
        return torch.empty(shape, dtype=dtypes[dt], pin_memory=True).numpy().view(dt)

    rho_h = pin(p.rho.shape, np.float32)
    rho_h[...] = p.rho
    flu_h = pin((B,), np.float32)
    flu_h[...] = p.fluence
    dose_h = pin(plan.shape, np.float32)
    rowptr_h = pin((V + 1,), np.int64)
    cols_h = pin((max(pairs, 1),), np.int32)
    vals_h = pin((max(pairs, 1),), np.float32)
    vals16_h = pin((max(pairs, 1),), np.uint16)

    def full(vals, dtype):
        def step():
            dc.dc_fspb_set_density(plan, rho_h)
            dc.dc_fspb_pair_count(plan)
            dc.dc_fspb_dose_and_matrix(plan, flu_h, dose_h, dtype, rowptr_h, cols_h, vals)
        return step

    def dose_only():
        dc.dc_fspb_set_density(plan, rho_h)
        dc.dc_fspb_dose(plan, flu_h, dose_h)

    def timed(step):
        for _ in range(max(1, min(args.warmup, 2))):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / args.steps

    h2d = 4 * V + 4 * B
    dt = timed(full(vals_h, dc.DC_F32))
    out = {"value": pairs / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": 4 * V + 8 * (V + 1) + 8 * pairs + 8, "ms_per_step": dt * 1e3,
           "steps": args.steps}
    dt16 = timed(full(vals16_h, dc.DC_BF16))
    dtd = timed(dose_only)
    out["variants"] = {
        "bf16_matrix": {"value": pairs / dt16, "ms_per_step": dt16 * 1e3, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": 4 * V + 8 * (V + 1) + 6 * pairs + 8},
        "dose_only": {"value": pairs / dtd, "ms_per_step": dtd * 1e3, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": 4 * V}}
    return out


def main():
    args = parse()
    if args.profile:
        run_profile(args)
        return
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
