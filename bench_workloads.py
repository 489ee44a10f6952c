"""Secondary benchmark workloads of bench.py (``--workload c1|c3|c4|c5``).

Each prints one labelled JSON line; the headline line (``c2``) stays in
bench.py.  Inputs are seeded and synthetic (paper_1003_3896_gb300.ics).
With ``--impl reference`` each instead times the CPU oracle on the same
workload's inputs and metric (run_reference); the serving workload has no
counterpart there.

  c1  N = 1024 Plummer in Henon units, eps = 1e-3, FP64, leapfrog DKD,
      dt = 1/1024, 64 steps: latency per step and |dE/E| against the oracle's
      own on the same initial conditions.
  c3  N = 262144 Plummer with Salpeter masses, eps = 1e-4: one force
      evaluation in FP64 / mixed / FP32 with its accuracy against the oracle
      on sampled bodies, then 20 leapfrog steps (dt = 1/512) in mixed
      precision.
  c4  512 independent Plummer clusters (Henon units, N log-uniform on
      [256, 8192], cluster seed k, eps by the paper's rule), SI6A, dt = 1/512,
      mixed precision, one persistent launch per force evaluation.
  c5  Serving: Poisson arrivals at 200/s of jobs with N log-uniform on
      [1024, 131072], order uniform on {2, 6}, precision uniform on
      {FP64, mixed}, step count log-uniform on [10, 1000], admitted under a
      150 GB budget; a bounded trace of the first ``--jobs`` arrivals (32:
      about 50 s of GPU work; the stream offers ~75x what one GPU serves, so
      its first 2000 arrivals would take ~50 min); FP64 jobs in float-float
      (the server's default; ``--fp64-kernel`` for the FP64 pipe); latency
      includes queueing.  Also the pair kernels' fraction of the FP32 peak
      inside the mix (server pair-launch events).
  plunge  Sect. 6.2's quasi-radial collisions with a massive black hole at the
      galactic centre: a Plummer cluster (N = 15360, M = 1, a = 1) released at
      (10, 0, 0) with velocity 0.001 v_c, black hole masses 0.1, 1, 50 and 105
      times the cluster's (static, softened by 0.05 so the passages through
      it are resolvable), disk + bulge field, SI6A with dt = 2e-4 over
      t in [0, 4] (NB_PLUNGE_STEPS steps, default 20000), mixed precision: relative
      energy and angular momentum changes (the quantities of Table 8) and
      the external torque of eq. 8 at the start and the end.
  sym  The N(N-1)/2 variant (each unordered pair once, Newton's third law;
      float class) against the full N x N float kernel on Plummer spheres of
      N = 16384, 65536, 262144: pair-kernel time and N^2 / time for both.
  paper  The paper's own test workload (Sect. 3, Sect. 5.1): a uniform sphere
      (R = 1, M = 1, virial ratio Q = 0.3) at the sizes of its Table 3,
      N = 480, 30720 and 1536000, one leapfrog step per precision (FP64 only
      up to N = 30720: at 1536000 one FP64 evaluation takes over a minute),
      in GFLOPS at 20 flops per pair beside the single-GPU figures that table
      reports for its Tesla C1060 (context, other hardware).
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

import numpy as np

from paper_1003_3896_gb300 import ics

UNIT = "Gpair-interactions/s"


def _ctx(nbsym, n, **kw):
    return nbsym.Context(n, **kw)


def _rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())


def _err_stats(a, ref) -> dict:
    """The global relative RMS (the measure the tolerances apply to) and, as
    diagnostics, the median and 99th percentile of the per-body relative error
    |a_i - ref_i| / |ref_i| (bodies whose reference is exactly zero left out:
    near the centre |a| ~ 0 makes the per-body ratio ill-defined)."""
    num = np.linalg.norm(a - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    per = num[den > 0] / den[den > 0]
    return {"rel_rms": _rel_rms(a, ref),
            "per_body_median": float(np.median(per)) if per.size else 0.0,
            "per_body_p99": float(np.percentile(per, 99)) if per.size else 0.0}


def _cpu_baseline_c1(pos, vel, m, eps, dt, nsteps):
    """CPU baseline leg of C1: the oracle's full run on the host cores (timed),
    with the energies of its initial and final states."""
    import oracle
    oracle.build()
    p = oracle.Params(eps=eps)
    t0 = time.perf_counter()
    rx, rv = oracle.run(pos, vel, m, p, 2, dt, nsteps)
    wall = time.perf_counter() - t0
    e0 = oracle.energy(pos, vel, m, p).E
    e1 = oracle.energy(rx, rv, m, p).E
    cores = oracle.max_threads()
    # the same run on one host core (the protocol's second CPU figure)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.run(pos, vel, m, p, 2, dt, nsteps)
    wall1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return rx, abs((e1 - e0) / e0), {
        "value": 1e6 * wall / nsteps, "unit": "us/step", "cores": cores, "kind": "oracle",
        "one_core_us_per_step": 1e6 * wall1 / nsteps,
        "sample": f"the full run ({nsteps} steps of N = {pos.shape[0]}), FP64, "
                  f"{wall:.2f} s on {cores} host threads ({wall1:.2f} s on one)"}


def c1(args, nbsym, torch):
    n, eps, dt, nsteps = 1024, 1e-3, 1.0 / 1024, 64
    pos, vel, m = ics.henon_plummer(n, 0)
    rx, de_ref, cpu = _cpu_baseline_c1(pos, vel, m, eps, dt, nsteps)
    out = {}
    for prec in ("fp64", "ds", "dd"):
        with _ctx(nbsym, n, eps=eps, precision=prec) as c:
            c.load(pos, vel, m)
            tuning = None if args.no_tune else c.tune(reps=5)
            c.step(2, dt, 3)             # warm-up (graph capture)
            c.load(pos, vel, m)
            e0 = c.energy().E
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.step(2, dt, nsteps)
            wall = time.perf_counter() - t0
            x, v = c.get_state()
            de = abs((c.energy().E - e0) / e0)
            # the paper's timing protocol: the mean over 1000 cycles
            c.load(pos, vel, m)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.step(2, dt, 1000)
            wall1000 = time.perf_counter() - t0
        out[prec] = {"us_per_step": 1e6 * wall / nsteps,
                     "us_per_step_mean_of_1000": 1e6 * wall1000 / 1000,
                     "value": nsteps * n * n / wall / 1e9,
                     "dE_over_E": de, "dE_over_E_oracle": de_ref,
                     "max_pos_err_vs_oracle": float(np.abs(x - rx).max()),
                     "tuning": tuning}
    return {"metric": "leapfrog step latency, N=1024", "workload":
            "plummer_N1024_henon_eps1e-3_dkd_dt1/1024_64steps", "unit": "us/step",
            "value": out["fp64"]["us_per_step"], "higher_is_better": False,
            "detail": out, "cpu_baseline": cpu}


def _cpu_baseline_c3(pos, m, idx, eps):
    """CPU baseline leg of C3: the oracle's sums for the sampled bodies
    against all N sources on the host cores (timed)."""
    import oracle
    oracle.build()
    n = m.size
    t0 = time.perf_counter()
    ref = oracle.accel_int_at(pos, m, idx, 1.0, eps)
    wall = time.perf_counter() - t0
    cores = oracle.max_threads()
    return ref, {"value": idx.size * n / wall / 1e9, "unit": UNIT, "cores": cores,
                 "kind": "oracle",
                 "sample": f"{idx.size} target bodies x {n} sources, FP64, {wall:.2f} s "
                           f"on {cores} host threads"}


def c3(args, nbsym, torch):
    n, eps = 262144, 1e-4
    pos, vel, m = ics.plummer(n, 0, masses=ics.salpeter_masses(n, 0))
    idx = np.unique(np.random.default_rng(2).choice(n, 256, replace=False))
    ref, cpu = _cpu_baseline_c3(pos, m, idx, eps)
    sweep = {}
    with _ctx(nbsym, n, eps=eps, precision="ds") as c:
        c.load(pos, vel, m)
        tunings = {}
        for prec in ("fp64", "ds", "fp32", "dd"):
            c.set_precision(prec)
            # the FP64 kernel takes seconds per launch here: tuned only by request
            if not args.no_tune and prec != "fp64":
                tunings[prec] = c.tune(reps=2)
            c.accel()
            c.prof_enable(True)
            a = c.accel()
            pr = c.prof_read()
            c.prof_enable(False)
            sweep[prec] = {**_err_stats(a[idx], ref),
                           "pair_ms": pr["pair_ms"],
                           "value": n * n / (pr["pair_ms"] * 1e-3) / 1e9}
        c.set_precision("ds")
        c.step(2, 1.0 / 512, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.step(2, 1.0 / 512, 20)
        wall = time.perf_counter() - t0
    return {"metric": "accuracy sweep and leapfrog throughput, N=262144 Salpeter",
            "workload": "plummer_salpeter_N262144_eps1e-4", "unit": UNIT,
            "value": 20 * n * n / wall / 1e9, "higher_is_better": True,
            "sweep": sweep, "tolerance": {"fp64": 1e-12, "ds": 1e-6, "fp32": 1e-5, "dd": 1e-12},
            "tuning": tunings, "cpu_baseline": cpu}


def c4(args, nbsym, torch):
    import bench
    world, rank, local = bench.rank_env()
    all_sizes = ics.ensemble_sizes(512, 256, 8192, seed=0)
    # under torchrun each rank integrates its share of whole clusters (no
    # data-path collective); the job's time is its slowest rank's
    mine = bench.shard_clusters(all_sizes, world)[rank]
    sizes = all_sizes[mine]
    pos, vel, mass, eps = [], [], [], []
    for k, n in zip(mine, sizes):
        p, v, m = ics.henon_plummer(int(n), int(k))
        pos.append(p)
        vel.append(v)
        mass.append(m)
        eps.append(ics.paper_softening(int(n)))
    pos, vel, mass = np.concatenate(pos), np.concatenate(vel), np.concatenate(mass)
    dt = 1.0 / 512
    pairs = float((sizes.astype(np.float64) ** 2).sum())
    with nbsym.Context(sizes=sizes, precision="ds") as b:
        b.set_cluster_params(eps=eps)
        b.load(pos, vel, mass)
        tuning = None if args.no_tune else b.tune(reps=2)
        b.step(6, dt, max(1, args.warmup))
        steps = args.steps
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        b.prof_enable(True)
        t0 = time.perf_counter()
        b.step(6, dt, steps)
        wall = time.perf_counter() - t0
        pr = b.prof_read()
    wall = bench.max_over_ranks(wall, "cuda")
    pairs_all = bench.sum_over_ranks(pairs, "cuda")
    value = 7 * steps * pairs_all / wall / 1e9
    achieved = 20 * pr["interactions"] / (pr["pair_ms"] * 1e-3) / 1e12
    return {"metric": "batched ensemble throughput", "unit": UNIT, "value": value,
            "higher_is_better": True, "n_gpus": world,
            "scaling": "strong" if world > 1 else "weak",
            "workload": "512_plummer_clusters_N256-8192_henon_si6a_dt1/512_ds",
            "clusters": int(all_sizes.size), "clusters_rank0": int(sizes.size),
            "bodies": int(all_sizes.sum()),
            "sum_N2_per_eval": pairs_all, "steps": steps, "ms_per_step": 1e3 * wall / steps,
            "pair_kernel_tflops": achieved, "pair_launches": pr["pair_launches"],
            "pair_kernel_ms_mean": pr["pair_ms"] / max(1, pr["pair_launches"]),
            "gpu_launches": pr["kernel_launches"], "tuning": tuning}


def _serve_trace(args, nbsym, rate_hz, n_cap, fp64_via_dd=1, all_mixed=False):
    """Replay the first args.jobs arrivals at rate_hz through one server;
    per-job latency is submission to completion (queueing included).
    all_mixed: every job in the mixed arithmetic (the served form of the
    FP32-pipe kernel alone)."""
    # the first args.jobs arrivals of the one 2000-arrival stream (the
    # generator draws each field for all jobs at once, so a shorter stream
    # would not be this one's prefix)
    trace = ics.serving_trace(n_jobs=2000, rate_hz=rate_hz, seed=0, n_hi=n_cap)[:args.jobs]
    dt = 1.0 / 512
    prepared = []
    for j in trace:
        p, v, m = ics.henon_plummer(j.n, j.seed)
        prepared.append((j, p, v, m, ics.paper_softening(j.n)))
    with nbsym.Server(hbm_budget_bytes=150e9, max_jobs=256, fp64_via_dd=fp64_via_dd) as srv:
        t0 = time.perf_counter()
        ids = []
        for j, p, v, m, e in prepared:
            delay = j.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            steps = min(j.nsteps, args.steps_cap)
            prec = "fp64" if j.precision == 0 and not all_mixed else "ds"
            ids.append((srv.submit(p, v, m, j.order, dt, steps, precision=prec, eps=e),
                        j, steps))
        lat = []
        pairs = 0.0
        for jid, j, steps in ids:
            st = srv.wait(jid, 3600)
            if st["state"] == nbsym.JOB_DONE:
                lat.append(st["t_done"] - st["t_submit"])
            pairs += j.n * j.n * steps * (7 if j.order == 6 else 1)
        makespan = time.perf_counter() - t0
        stats = srv.stats()
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    # pair kernels inside the mix: interactions over the device time during
    # which at least one launch of that arithmetic ran (the union of their
    # event intervals; concurrent groups' launches counted together)
    served = {}
    for a, name in ((0, "fp64_kernel"), (1, "ds"), (2, "dd")):
        if stats["pair_busy_ms"][a] > 0:
            rate = stats["pair_interactions"][a] / (stats["pair_busy_ms"][a] * 1e-3)
            served[name] = {"gpairs_s": rate / 1e9, "tflops_20": 20 * rate / 1e12,
                            "busy_ms": stats["pair_busy_ms"][a],
                            "event_ms_summed": stats["pair_ms"][a],
                            "interactions": stats["pair_interactions"][a]}
    return {"rate_hz": rate_hz, "p50_s": q(0.5), "p99_s": q(0.99), "jobs_done": len(lat),
            "throughput_gpairs_s": pairs / makespan / 1e9, "makespan_s": makespan,
            "offered_gpairs_s": pairs / max(trace[-1].arrival_s, 1e-9) / 1e9,
            "completed": stats["completed"], "failed": stats["failed"],
            "pair_kernels_in_mix": served}


def c5(args, nbsym, torch):
    n_cap = args.n_cap
    via_dd = 0 if args.fp64_kernel else 1
    r = _serve_trace(args, nbsym, 200.0, n_cap, fp64_via_dd=via_dd)
    sweep = []
    for rate in [float(x) for x in args.rates.split(",") if x.strip()]:
        sweep.append(_serve_trace(args, nbsym, rate, n_cap, fp64_via_dd=via_dd))
    # the pair kernels' fraction of the FP32 peak inside the mix (unit counts
    # at the maximum clock, as the headline line), and the served form of the
    # mixed arithmetic alone: the same arrivals with every job mixed, whose
    # throughput over the makespan (queueing gaps, small jobs and every
    # non-pair kernel included) is the served form's fraction of the peak
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    frac = {k: v["tflops_20"] / peak for k, v in r["pair_kernels_in_mix"].items()
            if k != "fp64_kernel"}
    r_ds = _serve_trace(args, nbsym, 200.0, n_cap, all_mixed=True)
    served_ds = {"throughput_gpairs_s": r_ds["throughput_gpairs_s"],
                 "frac_of_fp32_peak": 20 * r_ds["throughput_gpairs_s"] / 1e3 / peak,
                 "p50_s": r_ds["p50_s"], "p99_s": r_ds["p99_s"],
                 "makespan_s": r_ds["makespan_s"], "completed": r_ds["completed"],
                 "pair_kernels": r_ds["pair_kernels_in_mix"],
                 "pair_kernel_frac_of_fp32_peak": (
                     r_ds["pair_kernels_in_mix"]["ds"]["tflops_20"] / peak
                     if "ds" in r_ds["pair_kernels_in_mix"] else None)}
    caps = []
    if n_cap < 131072:
        caps.append(f"N <= {n_cap}")
    if args.steps_cap < 1000:
        caps.append(f"steps <= {args.steps_cap}")
    return {"metric": "serving latency p50/p99 (bounded trace)", "unit": "s",
            "value": r["p50_s"], "p99_s": r["p99_s"], "higher_is_better": False,
            "workload": f"poisson200hz_first{args.jobs}_N1024-{n_cap}_steps10-{args.steps_cap}"
                        "_order2or6_fp64orDS_dt1/512",
            "fp64_jobs": "float-float (NB_DD)" if via_dd else "FP64 kernel",
            "jobs_done": r["jobs_done"], "throughput_gpairs_s": r["throughput_gpairs_s"],
            "makespan_s": r["makespan_s"], "completed": r["completed"],
            "failed": r["failed"], "pair_kernels_in_mix": r["pair_kernels_in_mix"],
            "pair_frac_of_fp32_peak_in_mix": frac,
            "all_mixed_replay": served_ds,
            "rate_sweep": sweep,
            "note": "latency includes queueing; bounded to the first "
                    f"{args.jobs} arrivals of the 200/s stream ("
                    + (", ".join(caps) if caps else "full N and step ranges")
                    + "): the stream offers ~75x what one GPU serves, its first 2000 "
                    "arrivals would take ~50 min; rate_sweep replays the same jobs at "
                    "lower arrival rates; pair-kernel rates in the mix are interactions "
                    "over the union of each arithmetic's launch intervals (groups' "
                    "launches overlap on the device and are counted together)"}


# Table 3 of the paper, one Tesla C1060, leapfrog, GFLOPS at 20 flops per
# pair: single precision and double precision at N = 480, 30720, 1536000.
PAPER_TABLE3_SP = {480: 5.97, 30720: 409.0, 1536000: 423.0}
PAPER_TABLE3_DP = {480: 3.36, 30720: 21.9, 1536000: 22.0}


def paper(args, nbsym, torch):
    eps = ics.paper_softening  # eps = 0.005 R / N^(1/3), R = 1
    rows = []
    for n in (480, 30720, 1536000):
        pos, vel, m = ics.uniform_sphere(n, 0, q_vir=0.3)
        for prec in ("fp32", "ds", "fp64"):
            if prec == "fp64" and n > 30720:
                continue
            with nbsym.Context(n, eps=eps(n), precision=prec) as c:
                c.load(pos, vel, m)
                if not args.no_tune and n <= 30720:
                    c.tune(reps=3)
                c.step(2, 5e-4, 1)          # warm-up (graph capture)
                c.load(pos, vel, m)
                torch.cuda.synchronize()
                c.prof_enable(True)
                t0 = time.perf_counter()
                c.step(2, 5e-4, 1)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
                pr = c.prof_read()
            pair_rate = n * n / (pr["pair_ms"] * 1e-3)
            ref = (PAPER_TABLE3_DP if prec == "fp64" else PAPER_TABLE3_SP)[n]
            rows.append({"n": n, "precision": prec, "step_ms": 1e3 * wall,
                         "pair_ms": pr["pair_ms"], "gpairs_s": pair_rate / 1e9,
                         "gflops": 20 * pair_rate / 1e9,
                         "paper_c1060_gflops": ref,
                         "paper_table": "Table 3 " + ("DP" if prec == "fp64" else "SP")})
    best = max(r["gpairs_s"] for r in rows if r["precision"] == "ds")
    return {"metric": "paper workload series (uniform sphere Q = 0.3, leapfrog)",
            "unit": UNIT, "value": best, "higher_is_better": True,
            "workload": "uniform_sphere_Q0.3_N480_30720_1536000_leapfrog_dt5e-4",
            "rows": rows,
            "note": "paper figures are context (Tesla C1060, 2010), not targets"}


# Table 8 of the paper (N = 15360, its own units and field): |dE/E0| and
# |dL/L0| over its run, per black hole to cluster mass ratio.
PAPER_TABLE8 = {0.1: (3.06e-7, 5.90e-4), 1.0: (7.75e-6, 1.06e-2), 50.0: (9.23e-5, 2.65),
                105.0: (5.63e-3, 3.91)}


def plunge(args, nbsym, torch):
    n = 15360
    eps = ics.paper_softening(n)
    eps_bh = 0.05
    nsteps = int(os.environ.get("NB_PLUNGE_STEPS", "20000"))
    dt = 4.0 / nsteps
    pos, vel, m = ics.plunge_cluster(n, 0)
    rows = []
    total_pairs = 0.0
    total_wall = 0.0
    for q in (0.1, 1.0, 50.0, 105.0):
        with nbsym.Context(n, eps=eps, precision="ds", ext_on=True, Mbh=q,
                           eps_bh=eps_bh) as c:
            c.load(pos, vel, m)
            if not args.no_tune:
                c.tune(reps=3)
            e0 = c.energy()
            tq0 = c.torque()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.step(6, dt, nsteps)
            wall = time.perf_counter() - t0
            e1 = c.energy()
            tq1 = c.torque()
            x, _ = c.get_state()
        L0 = np.linalg.norm(e0.L)
        rows.append({"mbh_over_m": q, "dE_over_E0": abs((e1.E - e0.E) / e0.E),
                     "dL_over_L0": float(np.linalg.norm(e1.L - e0.L) / L0),
                     "torque_start": tq0.tolist(), "torque_end": tq1.tolist(),
                     "barycentre_end": (m @ x / m.sum()).tolist(),
                     "s_per_run": wall,
                     "paper_table8": {"dE_over_E0": PAPER_TABLE8[q][0],
                                      "dL_over_L0": PAPER_TABLE8[q][1]}})
        total_pairs += 7.0 * nsteps * n * n
        total_wall += wall
    return {"metric": "black-hole collision runs (Sect. 6.2)", "unit": UNIT,
            "value": total_pairs / total_wall / 1e9, "higher_is_better": True,
            "workload": f"plunge_plummer_N{n}_r0_10_v0.001vc_epsbh0.05_si6a_t4_{nsteps}steps_ds",
            "rows": rows,
            "note": "Table 8 values are context only: another field, other units"}


def sym(args, nbsym, torch):
    rows = []
    for n in (16384, 65536, 262144):
        pos, vel, m = ics.henon_plummer(n, 0)
        eps = ics.paper_softening(n)
        with nbsym.Context(n, eps=eps, precision="fp32") as c:
            c.load(pos, vel, m)
            if not args.no_tune:
                c.tune(reps=3)
            c.accel()
            c.prof_enable(True)
            full = c.accel()
            pr = c.prof_read()
            c.prof_enable(False)
            c.accel_symmetric()
            times = []
            for _ in range(3):
                a, ms = c.accel_symmetric()
                times.append(ms)
        ms = sorted(times)[1]
        rows.append({"n": n, "full_ms": pr["pair_ms"], "sym_ms": ms,
                     "full_gpairs_s": n * n / (pr["pair_ms"] * 1e-3) / 1e9,
                     "sym_gpairs_s": n * n / (ms * 1e-3) / 1e9,
                     "sym_over_full": pr["pair_ms"] / ms,
                     "rel_diff": float(np.sqrt(((a - full) ** 2).sum() / (full ** 2).sum()))})
    return {"metric": "N(N-1)/2 variant vs full N^2 sum (float class)", "unit": UNIT,
            "value": rows[-1]["sym_gpairs_s"], "higher_is_better": True,
            "workload": "henon_plummer_N16384_65536_262144_fp32", "rows": rows,
            "note": "interactions counted as N^2 for both, so the rates compare time"}


def _timed_steps(args, fn) -> float:
    """args.warmup untimed calls of fn, then the seconds args.steps calls take."""
    for _ in range(args.warmup):
        fn()
    wall = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        fn()
        wall += time.perf_counter() - t0
    return wall


def run_reference(args):
    """Reference arm of a secondary workload: the CPU oracle as it stands, on
    the host cores, timed on that workload's own inputs and metric.  Each step
    is a bounded sample: the whole 64-step run for c1, whole clusters (in
    index order) for c4, otherwise a sample of target bodies against all N
    sources (eq. 5, FP64).  The serving workload (c5) has no counterpart: the
    oracle has no serving loop.  Under torchrun rank 0 alone runs."""
    import bench
    import oracle
    world, rank, _ = bench.rank_env()
    if rank != 0:
        return 0
    w = args.workload
    if w == "c5":
        print(json.dumps({"impl": "reference", "workload": "c5",
                          "unavailable": "the CPU oracle has no serving loop: the p50/p99 "
                                         "latency of a job stream is defined for the GPU "
                                         "server only"}), flush=True)
        return 0
    oracle.build()
    rng = np.random.default_rng(1)
    pairs_per_step = None

    def targets(pos, m, eps, k):
        nonlocal pairs_per_step
        n = m.size
        k = min(k, n)
        idx = np.sort(rng.choice(n, k, replace=False))
        pairs_per_step = k * n
        return (lambda: oracle.accel_int_at(pos, m, idx, 1.0, eps),
                f"per step {k} target bodies x {n} sources (eq. 5, FP64)")

    hib, unit = True, UNIT
    if w == "c1":
        n, eps, dt, nsteps = 1024, 1e-3, 1.0 / 1024, 64
        pos, vel, m = ics.henon_plummer(n, 0)
        prm = oracle.Params(eps=eps)
        fn = lambda: oracle.run(pos, vel, m, prm, 2, dt, nsteps)
        sample = f"per step the full run: {nsteps} DKD steps of N = {n} (FP64)"
        metric, workload = ("leapfrog step latency, N=1024",
                            "plummer_N1024_henon_eps1e-3_dkd_dt1/1024_64steps")
        hib, unit = False, "us/step"
    elif w == "c3":
        n = 262144
        pos, _, m = ics.plummer(n, 0, masses=ics.salpeter_masses(n, 0))
        fn, sample = targets(pos, m, 1e-4, 256)
        metric, workload = ("accuracy sweep and leapfrog throughput, N=262144 Salpeter",
                            "plummer_salpeter_N262144_eps1e-4")
    elif w == "c4":
        sizes = ics.ensemble_sizes(512, 256, 8192, seed=0)
        chosen, tot = [], 0.0
        for k, n in enumerate(sizes):
            chosen.append((k, int(n)))
            tot += float(n) * float(n)
            if tot >= 1e8:
                break
        systems = []
        for k, n in chosen:
            p, _, m = ics.henon_plummer(n, k)
            systems.append((p, m, ics.paper_softening(n)))
        fn = lambda: [oracle.accel_int(p, m, 1.0, e) for p, m, e in systems]
        pairs_per_step = tot
        sample = (f"per step the full sums of clusters 0-{len(chosen) - 1} of the 512 "
                  f"({int(sum(n for _, n in chosen))} bodies, eq. 5, FP64)")
        metric, workload = ("batched ensemble throughput",
                            "512_plummer_clusters_N256-8192_henon_si6a_dt1/512_ds")
    elif w == "paper":
        n = 30720
        pos, _, m = ics.uniform_sphere(n, 0, q_vir=0.3)
        fn, sample = targets(pos, m, ics.paper_softening(n), 2048)
        metric, workload = ("paper workload series (uniform sphere Q = 0.3, leapfrog)",
                            "uniform_sphere_Q0.3_N480_30720_1536000_leapfrog_dt5e-4")
    elif w == "plunge":
        n = 15360
        pos, _, m = ics.plunge_cluster(n, 0)
        fn, sample = targets(pos, m, ics.paper_softening(n), 2048)
        metric, workload = ("black-hole collision runs (Sect. 6.2)",
                            f"plunge_plummer_N{n}_r0_10_v0.001vc_epsbh0.05_si6a_t4_"
                            f"{int(os.environ.get('NB_PLUNGE_STEPS', '20000'))}steps_ds")
    elif w == "sym":
        n = 262144
        pos, _, m = ics.henon_plummer(n, 0)
        fn, sample = targets(pos, m, ics.paper_softening(n), 1024)
        metric, workload = ("N(N-1)/2 variant vs full N^2 sum (float class)",
                            "henon_plummer_N16384_65536_262144_fp32")
    else:
        raise ValueError(f"unknown workload {w}")
    wall = _timed_steps(args, fn)
    if unit == "us/step":
        value = 1e6 * wall / (args.steps * nsteps)
    else:
        value = args.steps * pairs_per_step / wall / 1e9
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit,
            "n_gpus": args.gpus, "device": "host cores (no GPU work)",
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": hib,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "workload": workload, "config": {"workload": workload},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    """One workload line.  Under torchrun only the ensemble (c4) shards across
    ranks (whole clusters per rank); the single-system workloads run on rank
    0 alone and the other ranks exit without work."""
    if getattr(args, "impl", "ours") == "reference":
        return run_reference(args)
    import bench
    import torch
    world, rank, local = bench.rank_env()
    if world > 1 and args.workload != "c4":
        if rank != 0:
            return 0
        world = 1
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", init_method="env://")
    from paper_1003_3896_gb300 import build as nbbuild
    if rank == 0:
        nbbuild.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1003_3896_gb300 import nbsym
    if args.tune_load:
        # replay saved shapes instead of tuning (profiled runs time the
        # bench's shapes without tuning under the profiler)
        nbsym.tune_load(args.tune_load)
        args.no_tune = True
    fn = {"c1": c1, "c3": c3, "c4": c4, "c5": c5, "paper": paper,
          "plunge": plunge, "sym": sym}[args.workload]
    line = fn(args, nbsym, torch)
    if args.tune_save and rank == 0:
        nbsym.tune_save(args.tune_save)
    line["impl"] = "ours"
    line["data"] = "synthetic"
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0
