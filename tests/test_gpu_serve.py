"""Serving loop: jobs of different size, order and precision admitted by
budget and slots, batched while others run, each result the same alone and
in the mix (within the parity tolerances), failures isolated to their job."""
import time

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nbs():
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import nbsym
    return nbsym


JOBS = [  # n, order, precision, dt, nsteps
    (1500, 6, "ds", 1 / 512, 5),
    (3000, 2, "fp64", 1 / 1024, 9),
    (700, 2, "ds", 1 / 256, 12),
    (2200, 6, "fp64", 1 / 512, 3),
    (5000, 6, "ds", 1 / 512, 4),
    (400, 6, "ds", 1 / 128, 7),
]


def ic(n, seed):
    pos, vel, m = ics.henon_plummer(n, seed)
    return pos, vel, m, ics.paper_softening(n)


def test_each_result_same_alone_and_in_mix(nbs):
    with nbs.Server(hbm_budget_bytes=2e9, max_jobs=16) as srv:
        ids = []
        for k, (n, order, prec, dt, steps) in enumerate(JOBS):
            pos, vel, m, eps = ic(n, 500 + k)
            ids.append(srv.submit(pos, vel, m, order, dt, steps, precision=prec, eps=eps))
        st = [srv.wait(j, 300) for j in ids]
        assert all(s["state"] == nbs.JOB_DONE for s in st), st
        # work overlapped: some job was admitted before another finished
        overlap = any(a["t_admit"] < b["t_done"] and b["t_admit"] < a["t_done"]
                      for i, a in enumerate(st) for b in st[i + 1:])
        assert overlap
        stats = srv.stats()
        assert stats["completed"] == len(JOBS) and stats["interactions"] > 0
        # pair launches timed by arithmetic: mixed jobs, and the FP64 jobs in
        # float-float (the default); none on the FP64 kernel
        assert stats["pair_ms"][1] > 0 and stats["pair_interactions"][1] > 0
        assert stats["pair_ms"][2] > 0 and stats["pair_interactions"][2] > 0
        assert stats["pair_interactions"][0] == 0
        assert sum(stats["pair_interactions"]) == stats["interactions"]
        # busy time: the union of launch intervals, at most their sum (the
        # intervals are float milliseconds after a reference event: allow a
        # few of their ulps)
        slack = 1e-3
        for a in (1, 2):
            assert 0 < stats["pair_busy_ms"][a] <= stats["pair_ms"][a] * (1 + 1e-4) + slack
        assert (max(stats["pair_busy_ms"]) <= stats["pair_busy_ms_any"] + slack
                and stats["pair_busy_ms_any"] <= sum(stats["pair_busy_ms"]) + slack)
        results = [srv.result(j) for j in ids]
    for k, ((n, order, prec, dt, steps), (x, v)) in enumerate(zip(JOBS, results)):
        pos, vel, m, eps = ic(n, 500 + k)
        with nbs.Context(n, eps=eps, precision=prec) as c:
            c.load(pos, vel, m)
            c.step(order, dt, steps)
            xa, va = c.get_state()
        # alone, a small job may get a different launch shape (narrower
        # j-ranges), which moves where per-tile float sums are cut: the mixed
        # bar is its stated tolerance, FP64 agrees to rounding
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.abs(x - xa).max() <= tol, (k, np.abs(x - xa).max())
        assert np.abs(v - va).max() <= 10 * tol


def test_two_pass_group_same_alone_and_in_mix(nbs, orc):
    """A 12000-body mixed job makes its group's set large enough (sum of N^2
    above 2^27) for the two-pass form, so the served step graph runs the
    near-pair pass; the other jobs of the group share it while they last.
    Every result equals the job run alone (its own context) within the mixed
    bar, and the large job matches the oracle's 3 SI6A steps."""
    jobs = [(12000, 6, 1 / 512, 3), (900, 6, 1 / 512, 5), (2500, 6, 1 / 256, 2)]
    with nbs.Server(hbm_budget_bytes=2e9, max_jobs=8) as srv:
        ids = []
        for k, (n, order, dt, steps) in enumerate(jobs):
            pos, vel, m, eps = ic(n, 950 + k)
            ids.append(srv.submit(pos, vel, m, order, dt, steps, precision="ds", eps=eps))
        st = [srv.wait(j, 300) for j in ids]
        assert all(s["state"] == nbs.JOB_DONE for s in st), st
        results = [srv.result(j) for j in ids]
    for k, ((n, order, dt, steps), (x, v)) in enumerate(zip(jobs, results)):
        pos, vel, m, eps = ic(n, 950 + k)
        with nbs.Context(n, eps=eps, precision="ds") as c:
            c.load(pos, vel, m)
            c.step(order, dt, steps)
            xa, _ = c.get_state()
        assert np.abs(x - xa).max() <= 1e-6, (k, np.abs(x - xa).max())
        if k == 0:
            rx, _ = orc.run(pos, vel, m, orc.Params(eps=eps), order, dt, steps)
            assert np.abs(x - rx).max() <= 1e-6, np.abs(x - rx).max()


def test_concurrent_groups_do_not_share_scratch(nbs):
    """Four groups (mixed and float-float, orders 2 and 6) of sizeable jobs
    step concurrently on their own streams for tens of steps: each group's
    pair-kernel partial sums and near-pair scratch are its own, so every
    result equals the job run alone."""
    jobs = [(20000, 2, "ds", 30), (18000, 6, "ds", 6), (9000, 2, "fp64", 20),
            (8000, 6, "fp64", 4), (15000, 2, "ds", 25), (7000, 6, "ds", 8)]
    with nbs.Server(hbm_budget_bytes=4e9, max_jobs=16) as srv:
        ids = []
        for k, (n, order, prec, steps) in enumerate(jobs):
            pos, vel, m, eps = ic(n, 990 + k)
            ids.append(srv.submit(pos, vel, m, order, 1 / 1024, steps, precision=prec, eps=eps))
        st = [srv.wait(j, 600) for j in ids]
        assert all(s["state"] == nbs.JOB_DONE for s in st), st
        results = [srv.result(j) for j in ids]
    for k, ((n, order, prec, steps), (x, v)) in enumerate(zip(jobs, results)):
        pos, vel, m, eps = ic(n, 990 + k)
        with nbs.Context(n, eps=eps, precision="dd" if prec == "fp64" else prec) as c:
            c.load(pos, vel, m)
            c.step(order, 1 / 1024, steps)
            xa, _ = c.get_state()
        tol = 1e-10 if prec == "fp64" else 1e-6
        assert np.abs(x - xa).max() <= tol, (k, np.abs(x - xa).max())


def test_admission_respects_budget_and_slots(nbs):
    """A budget for about two 1000-body jobs: never more than two resident,
    every job still completes in arrival order of admission."""
    with nbs.Server(hbm_budget_bytes=2200 * 460.0, max_jobs=8) as srv:
        cap = srv.stats()["capacity_bodies"]
        assert 2000 <= cap < 3000
        ids = []
        for k in range(5):
            pos, vel, m, eps = ic(1000, 600 + k)
            ids.append(srv.submit(pos, vel, m, 6, 1 / 512, 6, precision="ds", eps=eps))
        st = [srv.wait(j, 300) for j in ids]
    assert all(s["state"] == nbs.JOB_DONE for s in st)
    events = sorted([(s["t_admit"], +1) for s in st] + [(s["t_done"], -1) for s in st])
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 2
    admits = [s["t_admit"] for s in st]
    assert admits == sorted(admits)


def test_slot_limit_and_cancel(nbs):
    # the FP64 kernel keeps the long job running for seconds
    with nbs.Server(hbm_budget_bytes=1e9, max_jobs=1, fp64_via_dd=0) as srv:
        pos, vel, m, eps = ic(4000, 700)
        long_job = srv.submit(pos, vel, m, 6, 1 / 512, 400, precision="fp64", eps=eps)
        p2, v2, m2, e2 = ic(500, 701)
        queued = srv.submit(p2, v2, m2, 2, 1 / 512, 5, precision="ds", eps=e2)
        time.sleep(0.05)
        assert srv.poll(queued)["state"] == nbs.JOB_QUEUED
        srv.cancel(queued)
        srv.cancel(long_job)
        assert srv.wait(queued, 60)["state"] == nbs.JOB_CANCELLED
        assert srv.wait(long_job, 120)["state"] == nbs.JOB_CANCELLED
        with pytest.raises(nbs.NBError) as e:
            srv.result(long_job)
        assert e.value.code == nbs.NB_ESTATE
        srv.forget(queued)


def test_failure_is_isolated(nbs):
    """A job with coincident bodies and eps = 0 goes non-finite and fails; a
    job in the same group finishes normally."""
    with nbs.Server(hbm_budget_bytes=1e9, max_jobs=8) as srv:
        bad = np.zeros((3, 3))
        bad[2, 0] = 1.0
        jb = srv.submit(bad, np.zeros((3, 3)), np.ones(3), 2, 1 / 64, 3, precision="ds", eps=0.0)
        pos, vel, m, eps = ic(900, 800)
        jg = srv.submit(pos, vel, m, 2, 1 / 512, 3, precision="ds", eps=eps)
        assert srv.wait(jb, 60)["state"] == nbs.JOB_FAILED
        assert srv.wait(jg, 60)["state"] == nbs.JOB_DONE
        with pytest.raises(nbs.NBError) as e:
            srv.result(jb)
        assert e.value.code == nbs.NB_ENONFINITE
        x, _ = srv.result(jg)
        assert np.isfinite(x).all()


def test_bad_jobs_rejected(nbs):
    with nbs.Server(hbm_budget_bytes=100 * 460.0, max_jobs=2) as srv:
        pos, vel, m, eps = ic(50, 900)
        for kw in [dict(order=3), dict(dt=0.0), dict(nsteps=0), dict(precision="fp32")]:
            args = dict(order=2, dt=0.01, nsteps=1, precision="ds", eps=eps)
            args.update(kw)
            with pytest.raises(nbs.NBError) as e:
                srv.submit(pos, vel, m, **args)
            assert e.value.code == nbs.NB_EINVAL
        p2, v2, m2, _ = ic(500, 901)
        with pytest.raises(nbs.NBError):
            srv.submit(p2, v2, m2, 2, 0.01, 1)


def test_fp64_jobs_via_float_float(nbs, orc):
    """By default (fp64_via_dd = 1) the server runs FP64 jobs in float-float
    arithmetic: the result still meets the FP64 bar against the oracle (4
    steps, positions within 1e-10), and NB_DD jobs are accepted directly.
    With fp64_via_dd = 0 they run the FP64 kernel, to the same bar."""
    n, order, dt, steps = 1500, 6, 1.0 / 512, 4
    pos, vel, m, eps = ic(n, 77)
    rx, _ = orc.run(pos, vel, m, orc.Params(eps=eps), order, dt, steps)
    with nbs.Server(hbm_budget_bytes=1e9, max_jobs=8) as srv:
        a = srv.submit(pos, vel, m, order, dt, steps, precision="fp64", eps=eps)
        b = srv.submit(pos, vel, m, order, dt, steps, precision="dd", eps=eps)
        for jid in (a, b):
            assert srv.wait(jid, 300)["state"] == nbs.JOB_DONE
            x, _ = srv.result(jid)
            assert np.abs(x - rx).max() <= 1e-10, np.abs(x - rx).max()
        st = srv.stats()
        assert st["pair_interactions"][0] == 0 and st["pair_interactions"][2] > 0
    with nbs.Server(hbm_budget_bytes=1e9, max_jobs=8, fp64_via_dd=0) as srv:
        a = srv.submit(pos, vel, m, order, dt, steps, precision="fp64", eps=eps)
        assert srv.wait(a, 300)["state"] == nbs.JOB_DONE
        x, _ = srv.result(a)
        assert np.abs(x - rx).max() <= 1e-10, np.abs(x - rx).max()
        st = srv.stats()
        assert st["pair_interactions"][0] > 0 and st["pair_interactions"][2] == 0
