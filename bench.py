"""Benchmark: pair interactions per second of the direct-summation hot path.

Workload (default): a Plummer cluster (M = 1, a = 1), N = 65536, on a circular
orbit at R = 50 in the Miyamoto-Nagai disk + Plummer bulge field, softening
eps = 0.005 / N^{1/3}, sixth-order SI6A steps of dt = 1/256, mixed precision
(float pairs, double-single accumulation).  One timed step is one SI6A step:
seven all-pairs force evaluations (7 N^2 interactions, 20 flops each by the
paper's convention) plus the fused FP64 kick/drift/field kernels.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the library's stream, with a 512 MB L2 flush between steps (outside the
events); barrier + synchronize around the timed region; max over ranks.
Under torchrun each rank integrates its own independent cluster (seed =
rank): no collective on the data path (weak scaling).

``--impl reference`` times the CPU oracle on the host cores instead, on a
bounded sample of the same workload (bodies x all N sources per step); with
``--workload`` it does the same for that workload (bench_workloads.py).
Under torchrun only rank 0 runs it.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpair-interactions/s & % FP32 peak vs plain FP64 kernel; p50/p99 solve latency"
UNIT = "Gpair-interactions/s"
FLOPS_PER_PAIR = 20


def workload(n: int, seed: int):
    from paper_1003_3896_gb300 import ics
    pos, vel, m = ics.plummer(n, seed)
    pos, vel = ics.place_on_orbit(pos, vel)
    return pos, vel, m, ics.paper_softening(n)


def config_dict(args, n_gpus):
    return {"workload": f"plummer_N{args.n}_orbit_R50_disk_bulge_si6a_dt1/256",
            "n": args.n, "order": 6, "dt": 1.0 / 256, "evals_per_step": 7,
            "precision": args.precision, "eps": "0.005/N^(1/3)",
            "l2": "flushed between timed steps (512 MB write)",
            "parallelism": f"independent clusters x{n_gpus}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(),
                                 f"nbsym_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[3 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM bytes (read + write) per launch of the mixed pair kernel on this
# workload, from one `ncu --set full` capture (profiles/ has the summary and the
# command).  Reported only for the captured launch shape and while pair.cu's
# code is the captured code (first 16 hex digits of the SHA-256 of the source
# with comments and whitespace removed, pair_source_digest); any change to the
# kernel's code or its shape makes the figure stale and the bench then reports
# null.
PAIR_TRAFFIC = {"source_sha256": "dd3a4816a22b3fe1", "n": 65536, "precision": "ds",
                "bodies_per_thread": 8, "blocks_per_sm": 12, "bytes_per_launch": 3259904.0}


# The paper's own throughput (Table 3, GFLOPS at 20 flops per pair, leapfrog)
# on its hardware, quoted beside the headline as context, not as a target:
# NBSympleC runs the pair sum on one Tesla C1060, NBSympleE on two, hosted by
# two quad-core 2.00 GHz Xeons (Sect. 4.1); per Sect. 5.1 the two-GPU version
# takes about a minute per leapfrog step at N = 1,536,000.
PAPER_CONTEXT = {
    "source": "paper Table 3 (GFLOPS, 20 flops per pair, leapfrog) and Sect. 5.1",
    "hardware": "Tesla C1060 (1 GPU: NBSympleC; 2 GPUs: NBSympleE), host 2x quad-core "
                "Xeon 2.00 GHz, 2010",
    "n": [480, 30720, 1536000],
    "sp_gflops_1gpu": [5.97, 409.0, 423.0], "dp_gflops_1gpu": [3.36, 21.9, 22.0],
    "sp_gflops_2gpu": [11.29, 797.0, 846.0], "dp_gflops_2gpu": [3.37, 43.8, 44.0],
    "two_gpu_leapfrog_step_s_at_n_1536000": 60.0,
    "note": "other hardware: context only",
}


def code_digest(text: str) -> str:
    """First 16 hex digits of the SHA-256 of C/C++ source with its comments
    and whitespace removed: equal across comment and layout edits, different
    for any change of the code."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()[:16]


def pair_source_digest() -> str | None:
    """code_digest of pair.cu: the recorded traffic stays valid across
    comment edits and lapses with any change of the kernel's code."""
    path = os.path.join(ROOT, "paper_1003_3896_gb300", "csrc", "pair.cu")
    try:
        return code_digest(open(path).read())
    except OSError:
        return None


def pair_traffic(n: int, precision: str, shape: dict):
    digest = pair_source_digest()
    if digest is None:
        return None
    t = PAIR_TRAFFIC
    if (digest != t["source_sha256"] or n != t["n"] or precision != t["precision"]
            or shape.get("bodies_per_thread") != t["bodies_per_thread"]
            or shape.get("blocks_per_sm") != t["blocks_per_sm"]):
        return None
    return t["bytes_per_launch"]


# ---- multi-rank host logic (one process per GPU; no data-path collective) ----

def rank_env():
    """(world, rank, local_rank) of this process as torchrun sets them."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _reduce(value: float, op: str, device) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device="cpu") -> float:
    """The sum of every rank's value (work done by the whole job)."""
    return _reduce(value, "sum", device)


def shard_clusters(sizes, world: int):
    """Whole clusters per rank for an ensemble: longest-processing-time
    assignment by N_k^2 (the pair work), ties to the lower rank; each
    cluster goes to exactly one rank, every rank's list ascending."""
    sizes = np.asarray(sizes, dtype=np.int64)
    order = sorted(range(sizes.size), key=lambda k: (-int(sizes[k]) ** 2, k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(sizes[k]) ** 2
    return [np.array(sorted(o), dtype=np.int64) for o in out]


FP64_PEAK_TFLOPS = 1.25   # GB300 nominal dense FP64


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA peak from unit counts: 128 FP32 lanes per SM, 2 flops per FMA."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def cpu_baseline(pos, m, eps, budget_s: float = 12.0):
    """The oracle as it stands, on the host cores: eq. 5 sums for a sample of
    target bodies against all N sources, repeated up to ~budget_s."""
    import oracle
    oracle.build()
    n = m.size
    cores = oracle.max_threads()
    rng = np.random.default_rng(0)
    k = min(n, 4096)
    idx = np.sort(rng.choice(n, k, replace=False))
    t0 = time.perf_counter()
    oracle.accel_int_at(pos, m, idx, 1.0, eps)
    dt1 = time.perf_counter() - t0
    reps = max(1, min(20, int(budget_s / max(dt1, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.accel_int_at(pos, m, idx, 1.0, eps)
    dt = time.perf_counter() - t0
    pairs = reps * k * n
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} x ({k} target bodies x {n} sources), FP64, "
                      f"{dt:.1f} s on {cores} host threads"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle timed on the same workload's metric."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    pos, vel, m, eps = workload(args.n, 0)
    n = m.size
    k = min(n, 2048)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, k, replace=False))
    for _ in range(args.warmup):
        oracle.accel_int_at(pos, m, idx, 1.0, eps)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.accel_int_at(pos, m, idx, 1.0, eps)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * k * n / tot / 1e9
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "device": "host cores (no GPU work)",
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step {k} target bodies x {n} sources (eq. 5, FP64)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_strong(args):
    """One cluster shared by all ranks, each owning a range of bodies (the
    paper's multi-GPU scheme, Sect. 4.2; paper_1003_3896_gb300/isplit.py):
    the paper's uniform sphere (Q = 0.3) of N = --strong-n bodies, leapfrog
    steps of dt = 5e-4, mixed precision; positions all-gathered over NCCL
    between substeps.  Total work is fixed as ranks are added (strong
    scaling); value = N^2 per evaluation x evaluations / slowest rank's time."""
    world, rank, local = rank_env()
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1003_3896_gb300 import build as nbbuild
    if rank == 0:
        nbbuild.build()
    if world > 1:
        dist.barrier()
    from paper_1003_3896_gb300 import ics, isplit, nbsym
    n = args.strong_n
    pos, vel, m = ics.uniform_sphere(n, 0, q_vir=0.3)
    eps = ics.paper_softening(n)
    dt = 5e-4
    ctx = nbsym.Context(n, eps=eps, precision=args.precision, device=local)
    ctx.load(pos, vel, m)
    rg, chunk = isplit.ranges(n, world)
    i0, i1 = rg[rank]
    me = isplit.Rank(isplit.ContextBackend(ctx, dev), i0, i1, chunk)
    ex = isplit.DistExchange() if world > 1 else isplit.LocalExchange()
    w = nbsym.stage_weights(2)
    isplit.run([me], ex, w, dt, args.warmup)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        isplit.run([me], ex, w, dt, args.steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    t_max = max_over_ranks(t, dev)
    value = args.steps * float(n) * n / t_max / 1e9
    peak = fp32_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count, 2070.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32-pair/ds-acc" if args.precision == "ds" else args.precision,
            "data": "synthetic",
            "config": {"workload": f"uniform_sphere_Q0.3_N{n}_leapfrog_dt5e-4_isplit",
                       "n": n, "order": 2, "dt": dt, "precision": args.precision,
                       "eps": "0.005/N^(1/3)", "l2": "inputs far larger than L2",
                       "parallelism": f"i-split x{world} (positions all-gathered per substep)"},
            "frac_of_fp32_peak_per_gpu": 20 * value / 1e3 / world / peak,
            "clocks": clk.summary(),
            "paper_context": {"source": "paper Table 3 / Sect. 5.1, N = 1536000, 2 x Tesla C1060",
                              "sp_gflops_2gpu": 846.0, "two_gpu_leapfrog_step_s": 60.0}}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--precision", default="ds", choices=["ds", "ds_full", "fp32", "fp64", "dd"])
    ap.add_argument("--near-frac", type=float, default=0.0,
                    help="mixed mode near-pair radius in units of R_rms / N^(1/3) (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the pair-kernel shape autotuner (nb_tune) before timing")
    ap.add_argument("--tune-save", default="",
                    help="write the tuned-shape table (nb_tune_save) to this file after tuning")
    ap.add_argument("--tune-load", default="",
                    help="load a tuned-shape table (nb_tune_load) and skip tuning, so a "
                         "profiled run times the same kernel shapes as the run that saved it")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "c4", "c5", "paper", "plunge", "sym"],
                    help="c2 (default): the headline line; the others print their own "
                         "labelled lines (see bench_workloads.py)")
    ap.add_argument("--jobs", type=int, default=32,
                    help="c5: jobs in the bounded trace (the first arrivals)")
    ap.add_argument("--steps-cap", type=int, default=1000,
                    help="c5: cap on steps per job (1000, the trace's own upper bound: none)")
    ap.add_argument("--n-cap", type=int, default=131072,
                    help="c5: cap on bodies per job (131072, the trace's own upper bound: none)")
    ap.add_argument("--fp64-kernel", action="store_true",
                    help="c5: run FP64 jobs on the plain FP64 kernel instead of float-float")
    ap.add_argument("--rates", default="",
                    help="c5: comma-separated arrival rates (jobs/s) to replay the trace at "
                         "after the 200/s run, e.g. 2,4,8 (the rate sweep)")
    ap.add_argument("--strong", action="store_true",
                    help="one cluster split by body range over the ranks (strong scaling)")
    ap.add_argument("--strong-n", type=int, default=1536000,
                    help="--strong: bodies of the shared cluster")
    args = ap.parse_args()
    if args.strong and args.impl != "reference":
        return run_strong(args)
    if args.workload != "c2":
        import bench_workloads
        return bench_workloads.run(args)

    world, rank, local = rank_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1003_3896_gb300 import build as nbbuild
    if rank == 0:
        nbbuild.build()
    if world > 1:
        dist.barrier()
    from paper_1003_3896_gb300 import nbsym

    pos, vel, m, eps = workload(args.n, seed=rank)
    n = m.size
    dt = 1.0 / 256
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = nbsym.Context(n, eps=eps, precision=args.precision, ext_on=True, device=local,
                        stream=stream.cuda_stream, near_frac=args.near_frac)
    if args.tune_load:
        nbsym.tune_load(args.tune_load)
    ctx.load(pos, vel, m)
    tune = not args.no_tune and not args.tune_load
    tuning = ctx.tune(reps=3) if tune else None
    for _ in range(args.warmup):
        ctx.step(6, dt, 1)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.prof_enable(True)
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                ctx.step(6, dt, 1)
                ends[k].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    prof = ctx.prof_read()
    shape = ctx.pair_shape()
    ctx.prof_enable(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = max_over_ranks(sum(step_ms), dev)
    if world > 1:
        dist.barrier()
    pairs_all = sum_over_ranks(7 * args.steps * n * n, dev)
    value = pairs_all / (t_ms * 1e-3) / 1e9

    # end-to-end through the public API: host buffers in pinned memory, the
    # state uploaded before and read back after every step
    pin_p = torch.from_numpy(pos).pin_memory().numpy()
    pin_v = torch.from_numpy(vel).pin_memory().numpy()
    pin_m = torch.from_numpy(m).pin_memory().numpy()
    out_p = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    out_v = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    e_ms = []
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.load(pin_p, pin_v, pin_m)
            ctx.step(6, dt, 1)
            nbsym.check(nbsym.nb_get_state(ctx.handle, nbsym._p(out_p), nbsym._p(out_v)))
            e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = max_over_ranks(statistics.mean(e_ms), dev)
    e2e_value = sum_over_ranks(7 * n * n, dev) / (e2e_ms * 1e-3) / 1e9

    # plain FP64 kernel on the same state and configuration
    ctx.set_precision("fp64")
    tuning64 = ctx.tune(reps=1) if tune else None
    if args.tune_save:
        nbsym.tune_save(args.tune_save)
    ctx.prof_enable(True)
    for _ in range(2):
        ctx.accel()
    p64 = ctx.prof_read()
    ctx.prof_enable(False)
    fp64_rate = p64["interactions"] / (p64["pair_ms"] * 1e-3) / 1e9

    clocks = clk.summary()
    peaks = nbsym.measure_peaks(local)
    achieved = FLOPS_PER_PAIR * prof["interactions"] / (prof["pair_ms"] * 1e-3) / 1e12
    sustained_mhz = clocks.get("sm_mhz") or 2070.0
    kernel = {"fp64": "pair_fp64_kernel", "dd": "pair_ff_kernel"}.get(args.precision,
                                                                       "pair_sp_kernel")
    if args.precision == "fp64":
        # the FP64 pipe: the DFMA rate measured in the same run is the
        # ceiling (this GPU's DFMA issue measures ~83% of the nominal 1.25
        # TFLOP/s); the nominal fraction is reported beside it
        peak = peaks["dfma_tflops"]
        peak_basis = (f"FP64 DFMA measured in this run ({peak:.3f} TFLOP/s; nominal "
                      f"{FP64_PEAK_TFLOPS} TFLOP/s gives frac_of_nominal_fp64)")
        frac_clock = achieved / FP64_PEAK_TFLOPS * 2070.0 / sustained_mhz
        frac_meas = achieved / FP64_PEAK_TFLOPS
    else:
        peak = fp32_peak_tflops(sms, 2070.0)
        peak_basis = f"{sms} SMs x 128 FP32 lanes x 2 flops x 2070 MHz (max clock)"
        frac_clock = achieved / fp32_peak_tflops(sms, sustained_mhz)
        frac_meas = achieved / max(peaks["ffma_tflops"], peaks["ffma2_tflops"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"ds": "f32-pair/ds-acc", "ds_full": "f32-pair/ds-acc",
                  "fp32": "f32", "fp64": "f64", "dd": "f32x2-pair/f32x2-acc"}[args.precision],
        "data": "synthetic", "config": config_dict(args, world),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": pair_traffic(n, args.precision, shape),
                     "traffic_unit": "bytes per launch (dram read + write)",
                     "kernel": f"{kernel} ({args.precision})",
                     "peak_basis": peak_basis,
                     "frac_at_sampled_clock": frac_clock,
                     ("frac_of_nominal_fp64" if args.precision == "fp64"
                      else "frac_of_measured_fp32"): frac_meas,
                     "measured_peaks": peaks,
                     "pair_kernel_ms_mean": prof["pair_ms"] / max(1, prof["pair_launches"]),
                     "pair_launches": prof["pair_launches"]},
        "pair_shape": {"timed": shape, "tuning": tuning},
        "fp64_kernel": {"value": fp64_rate, "unit": UNIT, "tuned": tuning64},
        "vs_fp64_kernel": value / fp64_rate if fp64_rate > 0 else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 7 * 8,
                "d2h_bytes_per_step": n * 6 * 8, "steps": e2e_steps},
        "gpu_launches": prof["kernel_launches"],
        "clocks": clocks, "wall_s_timed": wall,
        "paper_context": PAPER_CONTEXT,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pos, m, eps)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
