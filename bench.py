"""Benchmark of the GB300 DC-FSPB dose engine.

One step = the whole hot path of one plan on synthetic inputs resident in HBM:
  Algorithm A1 steps 1-6 for the plan's density (smoothing, beamlet geometry,
  FP64 Siddon trace, depth tables; dc_fspb_set_density),
  eq. (1) direct dose (dc_fspb_dose),
  the dose-deposition matrix: pair count, row pointers and FP32 CSR fill
  (dc_fspb_pair_count + dc_fspb_dose_matrix).
Every pair of the plan is evaluated twice per step (once for the dose, once for
its matrix entry), so the metric counts 2 x pairs voxel-beamlet evaluations.

Default workload: the 9-field coplanar thorax plan on a 128 x 128 x 96 grid of
0.25 cm voxels (0.5 cm beamlets, fields 8-15 cm, ROI 5 cm).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank computes its
own plan (independent problems: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-beamlet evals/s (full plan: steps 1-6 + eq. 1 dose + FP32 dose matrix)"
UNIT = "evals/s"
# Algorithmic work of one (voxel, beamlet) evaluation of eqs. (2)-(4) with the
# lookups of Algorithm A1 steps 9-11 (counted from the method's definition):
ALG_FP32_PER_PAIR = 98     # FP32 add/mul/fma/compare/round operations (itemised in the design doc)
ALG_MUFU_PER_PAIR = 9      # 8 exponentials (four p() of eq. 4) + 1 reciprocal (SAD/|r_a|)
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dose kernel on the thorax9 plan, from an ncu capture of the kernel built
# from the sources with these SHA-256 digests (the kernel and the structures it
# reads; profiles/k_pairs_dose_thorax9.md); reported only while they are unchanged.
DOSE_TRAFFIC_BYTES = 110389248 + 20729344
DOSE_TRAFFIC_SOURCES = {
    "paper_1103_1164_gb300/csrc/k_dose.cu": "70ece8998f2945e076ecef028daaf234232d4b3e7fd3d9d6e96961a68bf3742f",
    "paper_1103_1164_gb300/csrc/dc_views.cuh": "604f1c61d84a82494049db8c574ff1384cee296c4ebbe27db75ba78b5c54a772",
}


def dose_traffic(scale):
    """The captured per-launch DRAM traffic, or None if the kernel's sources
    changed since the capture or the workload is not the captured one."""
    import hashlib
    if scale != 1.0:
        return None
    for rel, digest in DOSE_TRAFFIC_SOURCES.items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return DOSE_TRAFFIC_BYTES


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0, help="grid scale of the thorax plan")
    ap.add_argument("--profile", default=None, choices=["dose", "fill", "prep", "spmm", "step", "table1"],
                    help="small fixed run of one stage for profiler captures (prints no bench line)")
    return ap.parse_args()


def run_profile(args):
    """A short, fixed sequence of one stage's launches for ncu captures: the
    plan is built once, then the stage runs warmup + steps times."""
    import torch
    from paper_1103_1164_gb300 import build, dc_fspb as dc, synth
    build.build()
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
    if args.profile == "step":
        # the benchmark's step after the same plan set-up (autotuned binning)
        dc.dc_fspb_autotune(plan, flu_d)
        pairs = dc.dc_fspb_pair_count(plan)
        rowptr = torch.empty(plan.n_voxels + 1, dtype=torch.int64, device="cuda")
        cols = torch.empty(pairs, dtype=torch.int32, device="cuda")
        vals = torch.empty(pairs, dtype=torch.float32, device="cuda")
        n0 = dc.dc_fspb_launch_count()
        for _ in range(args.warmup + args.steps):
            dc.dc_fspb_set_density(plan, rho_d)
            dc.dc_fspb_dose(plan, flu_d, dose_d)
            dc.dc_fspb_pair_count(plan)
            dc.dc_fspb_dose_matrix(plan, dc.DC_F32, rowptr, cols, vals)
        torch.cuda.synchronize()
        per_step = (dc.dc_fspb_launch_count() - n0) // (args.warmup + args.steps)
        print(f"profile run done: step, {per_step} library launches per step")
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

def oracle_sample_rate(plan_in, budget_s=12.0, seed=3):
    """Times the FP64 oracle on a seeded sample of voxels of the workload.

    Returns per-step CPU estimates: the oracle's plan set-up time (steps 1-6,
    measured in full) and its dose + matrix time scaled from the sample by the
    ratio of pair counts."""
    from oracle import oracle
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    op = oracle.OraclePlan(plan_in, threads=threads)
    t_create = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    n = 256
    while True:
        vox = np.sort(rng.choice(op.V, size=min(n, op.V), replace=False))
        t0 = time.perf_counter()
        op.dose_voxels(vox)
        op.matrix(vox)
        dt = time.perf_counter() - t0
        if dt >= 0.4 * budget_s or n >= op.V:
            break
        n = int(min(op.V, n * max(2.0, 0.5 * budget_s / max(dt, 1e-3))))
    pairs_sample = int(op.pairs_voxels(vox).sum())
    return dict(op=op, t_create=t_create, t_sample=dt, n_vox=int(vox.size), pairs_sample=pairs_sample,
                threads=threads)


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
    value = 2 * pairs * len(times) / t
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
        dc.dc_fspb_dose(plan, flu_d, dose_d)
        if ev: ev[2].record(stream)
        n = dc.dc_fspb_pair_count(plan)
        assert n == pairs
        if ev: ev[3].record(stream)
        dc.dc_fspb_dose_matrix(plan, dc.DC_F32, rowptr_d, cols_d, vals_d)
        if ev: ev[4].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
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
    stage = np.array([[evs[k][j].elapsed_time(evs[k][j + 1]) for j in range(4)] for k in range(args.steps)])
    step_ms = stage.sum(1)
    evals_step = 2 * pairs
    value, t_total_ms = aggregate_throughput(pg, torch, evals_step * args.steps, float(step_ms.sum()))
    ms_per_step = t_total_ms / args.steps

    # roofline of the dominant kernel: the direct dose kernel (ALU bound)
    t_dose = float(stage[:, 1].mean()) * 1e-3
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # the tighter of the FP32 lanes and the MUFU lanes (issue slots do not bound
    # the method: packed FP32 instructions issue two of its operations at once)
    peak_pairs = props.multi_processor_count * sm_max * 1e6 * min(
        FP32_LANES_PER_SM / ALG_FP32_PER_PAIR, MUFU_LANES_PER_SM / ALG_MUFU_PER_PAIR)
    achieved = pairs / t_dose
    roofline = {"kernel": "k_dose<dose,1> (eqs. 1-4)", "bound": "alu",
                "achieved": achieved / 1e9, "peak": peak_pairs / 1e9, "unit": "Gpair/s",
                "frac": achieved / peak_pairs, "traffic": dose_traffic(args.scale),
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_basis": f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz x "
                              f"min(128/{ALG_FP32_PER_PAIR} FP32 lanes, 16/{ALG_MUFU_PER_PAIR} MUFU lanes) "
                              f"pairs per cycle and SM",
                "dose_kernel_ms": t_dose * 1e3,
                "timing": "CUDA events around dc_fspb_dose on the plan's stream: the pair kernel plus "
                          "the per-beam sum and two small memsets (the pair kernel alone is ~2 % shorter)"}
    fill_ms = float(stage[:, 3].mean())
    bytes_matrix = pairs * 8 + (V + 1) * 8
    matrix = {"fill_ms": fill_ms, "fill_GBps": bytes_matrix / (fill_ms * 1e-3) / 1e9,
              "hbm_peak_GBps": peaks.get("hbm_gbs"), "count_scan_ms": float(stage[:, 2].mean()),
              "nnz": pairs, "bytes": bytes_matrix}

    # the other forms of the path; one that fails is reported as such and does
    # not take the benchmark line with it
    def form(fn, *fa):
        try:
            return fn(*fa)
        except Exception as exc:                      # noqa: BLE001 (reported in the line)
            torch.cuda.synchronize()
            return {"error": f"{type(exc).__name__}: {exc}"[:300]}

    forms = form(run_forms, args, dc, torch, stream, peaks)
    forms["fused_plan"] = form(run_fused_form, args, dc, torch, stream, plan, rho_d, flu_d, dose_d, rowptr_d,
                               cols_d, vals_d, flush, float(step_ms.mean()), pairs)
    forms["surrogate"] = form(run_surrogate_form, args, dc, torch, stream)
    forms["batch"] = form(run_batch_form, args, dc, torch, stream, peak_pairs)
    forms["gamma"] = form(run_gamma_form, args, dc, torch, stream, p, rho_d, flu_d)
    forms["table1"] = form(run_table1_form, args, dc, torch, stream, flush)
    forms["leaf_sequences"] = form(run_leaf_form, args, dc, torch, stream, flush)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, dc, p, plan, pairs, torch)
    cpu = None
    if not args.no_cpu and rank == 0:
        est = oracle_sample_rate(p)
        scale_pairs = pairs / max(est["pairs_sample"], 1)
        t_cpu_step = est["t_create"] + est["t_sample"] * scale_pairs
        cpu = {"value": evals_step / t_cpu_step, "unit": UNIT, "cores": est["threads"], "kind": "oracle",
               "sample": f"FP64 oracle: plan set-up timed in full ({est['t_create']:.2f} s), dose + "
                         f"matrix rows timed on {est['n_vox']} seeded voxels ({est['pairs_sample']} pairs, "
                         f"{est['t_sample']:.2f} s) and scaled by pair count to the {pairs} pairs of the plan"}
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
            "stages_ms": {"steps_1_6": float(stage[:, 0].mean()), "dose": float(stage[:, 1].mean()),
                          "pair_count": float(stage[:, 2].mean()), "matrix_fill": fill_ms},
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "roofline": roofline, "peaks": peak_kind, "dose_matrix": matrix, "forms": forms,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_fused_form(args, dc, torch, stream, plan, rho_d, flu_d, dose_d, rowptr_d, cols_d, vals_d, flush,
                   step_ms, pairs):
    """The same plan (thorax9: steps 1-6, dose and FP32 matrix) with the dose
    accumulated by the matrix fill (dc_fspb_dose_and_matrix): one evaluation
    of each pair instead of two, after a pair-count pass for the row pattern.
    Full-plan device time against the benchmark step's."""
    def fused():
        dc.dc_fspb_set_density(plan, rho_d)
        dc.dc_fspb_dose_and_matrix(plan, flu_d, dose_d, dc.DC_F32, rowptr_d, cols_d, vals_d)

    ref = dose_d.clone()
    fused()
    torch.cuda.synchronize()
    same = bool(torch.equal(ref, dose_d))
    reps = max(3, min(args.steps, 5))
    t = time_on_stream(torch, stream, fused, reps, flush)
    return {"workload": "thorax9 plan, dose + FP32 matrix from one pass (after a pair-count pass)",
            "full_plan_ms": t, "benchmark_step_ms": step_ms, "speedup": step_ms / t,
            "pairs_per_s": pairs / (t * 1e-3), "dose_identical_to_step": same}


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
    bytes_alg = chunks * 4096 + chunks * 4 + plan.n_voxels * k * 4 + plan.n_beamlets * k * 4
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
                                       "bytes": bytes_alg},
                          "max_err_vs_fp32_over_colmax": err},
            "speedup_bf16_over_fp32": t_plain / t_spmm}


def run_surrogate_form(args, dc, torch, stream, k=64):
    """The learned lateral correction: 2M (nearest-tap stencil, plain axis
    densities) samples from 200 random slab/sphere phantoms, trained with the
    library's kernels, then the slab plan's 64-fluence dose with the network's
    correction and the BF16 tensor-core SpMM, against the plain FP32 form (axis
    stencils, direct evaluation), which is also the judge of its error."""
    from paper_1103_1164_gb300 import surrogate, synth
    t0 = time.perf_counter()
    X, T = surrogate.generate_samples(n_phantoms=200, per_phantom=10000, seed=2024)
    t_gen = time.perf_counter() - t0
    n_tr = int(0.9 * X.shape[0])
    t0 = time.perf_counter()
    params, loss = surrogate.train(X[:n_tr], T[:n_tr], epochs=8, batch=4096, lr=2e-3, seed=17)
    t_train = time.perf_counter() - t0
    held = np.abs(dc.dc_mlp_predict(params, X[n_tr:]) - T[n_tr:]).max(1)

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
    t0 = time.perf_counter()
    dc.dc_fspb_spmm_prepare(plan)
    t_prep = time.perf_counter() - t0
    dc.dc_fspb_spmm(plan, F, Y)
    t_spmm = time_on_stream(torch, stream, lambda: dc.dc_fspb_spmm(plan, F, Y), reps, flush)
    dc.dc_fspb_device_status(plan)
    err = float(((Y.t() - plain).abs().max(1).values / plain.abs().max(1).values).max())
    return {"workload": f"slab64 64^3 @0.25cm, 1 beam, {plan.n_beamlets} beamlets, {k} fluences U[0,1]; "
                        f"network 48-64-64-3 SiLU trained on {n_tr} stencils from 200 random phantoms",
            "samples_generate_s": t_gen, "train_s": t_train, "train_loss": loss,
            "held_out_abs_err_density": {"p50": float(np.median(held)), "p99": float(np.percentile(held, 99))},
            "plain_fp32_axis": {"set_density_ms": t_set_axis, "dose_64_ms": t_plain},
            "surrogate_bf16": {"set_density_ms": t_set_mlp, "spmm_prepare_s": t_prep, "spmm_64_ms": t_spmm,
                               "fallbacks": dc.dc_fspb_lateral_fallbacks(plan)},
            "speedup_64_fluences": t_plain / t_spmm,
            "max_err_vs_plain_over_colmax": err}


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
    at 0.2-0.3 cm, 5-9 beams, 0.25 cm beamlets, ROI 5 cm): one persistent
    graph-replayed launch over all plans (dc_fspb_batch_run) against the plans'
    own launches one after another, dose only and whole plans (density-dependent
    steps + dose)."""
    from paper_1103_1164_gb300 import synth
    t0 = time.perf_counter()
    inputs = synth.config5_plans()
    t_gen = time.perf_counter() - t0
    rhos = [torch.from_numpy(p.rho).cuda() for p in inputs]
    flus = [torch.from_numpy(p.fluence).cuda() for p in inputs]
    plans = [dc.dc_fspb_create_from(p, stream=stream.cuda_stream, device_density=r) for p, r in zip(inputs, rhos)]
    doses = [torch.empty(pl.n_voxels, device="cuda") for pl in plans]
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
    return {"workload": f"{len(plans)} head-and-neck plans, {sum(pl.n_voxels for pl in plans)} voxels, "
                        f"{sum(len(p.beams) for p in inputs)} beams, {sum(pl.n_beamlets for pl in plans)} "
                        f"beamlets (0.25 cm), ROI 5 cm, density correction on",
            "pairs": total, "generate_s": t_gen,
            "batch_graph": {"dose_ms": t_batch, "full_plans_ms": t_full, "evals_per_s": ach,
                            "kernels_per_replay": launches,
                            "autotuned_ctas_per_sm": 4 + variant, "autotune_ms": tune_ms,
                            "roofline": {"bound": "alu", "achieved": ach / 1e9, "peak": peak_pairs / 1e9,
                                         "unit": "Gpair/s", "frac": ach / peak_pairs}},
            "sequential_plans": {"dose_ms": t_seq, "full_plans_ms": t_seq_full,
                                 "evals_per_s": total / (t_seq * 1e-3)},
            "speedup_batch_over_sequential": {"dose": t_seq / t_batch, "full_plans": t_seq_full / t_full},
            "max_diff_batch_vs_sequential_over_max": err}


def dc_view(torch, ptr, n):
    """torch view (no copy) of a float32 device buffer owned by the library."""
    class _A:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                    "strides": None}
    return torch.as_tensor(_A(), device="cuda")


def run_e2e(args, dc, p, plan, pairs, torch):
    """The same step through the C ABI with pinned host buffers: every H2D/D2H
    copy of the step's inputs and results is inside the timed region."""
    V, B = plan.n_voxels, plan.n_beamlets
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    rho_h = pin(p.rho.shape, torch.float32)
    rho_h[...] = p.rho
    flu_h = pin((B,), torch.float32)
    flu_h[...] = p.fluence
    dose_h = pin(plan.shape, torch.float32)
    rowptr_h = pin((V + 1,), torch.int64)
    cols_h = pin((max(pairs, 1),), torch.int32)
    vals_h = pin((max(pairs, 1),), torch.float32)

    def step():
        dc.dc_fspb_set_density(plan, rho_h)
        dc.dc_fspb_dose(plan, flu_h, dose_h)
        n = dc.dc_fspb_pair_count(plan)
        dc.dc_fspb_dose_matrix(plan, dc.DC_F32, rowptr_h, cols_h, vals_h)
        return n

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    h2d = 4 * V + 4 * B
    d2h = 4 * V + 8 * (V + 1) + 8 * pairs + 8
    return {"value": 2 * pairs / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": k}


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
