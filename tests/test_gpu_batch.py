"""Batched ensemble: many independent clusters of uneven size integrated by
one persistent launch per force evaluation.  Each cluster's result must equal
the same cluster run alone (its own context), within the parity tolerances,
and match the oracle."""
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

SIZES = [300, 1000, 129, 2048, 777, 4100, 256, 1]


@pytest.fixture(scope="module")
def nbs():
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import nbsym
    return nbsym


def rel_rms(a, ref):
    den = (ref ** 2).sum()
    return math.sqrt(((a - ref) ** 2).sum() / den) if den > 0 else float(np.abs(a - ref).max())


def clusters(sizes, base_seed=100):
    out = []
    for k, n in enumerate(sizes):
        pos, vel, m = ics.henon_plummer(n, base_seed + k)
        out.append((pos, vel, m, ics.paper_softening(n)))
    return out


def concat(cl):
    return (np.concatenate([c[0] for c in cl]), np.concatenate([c[1] for c in cl]),
            np.concatenate([c[2] for c in cl]))


@pytest.mark.parametrize("prec", ["fp64", "ds", "fp32", "dd"])
def test_batch_accel_matches_oracle_and_alone(nbs, orc, prec):
    cl = clusters(SIZES)
    pos, vel, m = concat(cl)
    eps = [c[3] for c in cl]
    with nbs.Context(sizes=SIZES, precision=prec) as b:
        assert b.clusters == len(SIZES)
        b.set_cluster_params(eps=eps)
        b.load(pos, vel, m)
        a = b.accel()
    tol = {"fp64": 1e-12, "ds": 1e-6, "fp32": 1e-4, "dd": 1e-12}[prec]
    off = 0
    for (p, v, mm, e), n in zip(cl, SIZES):
        ref = orc.accel_int(p, mm, 1.0, e)
        got = a[off:off + n]
        if n > 1:
            assert rel_rms(got, ref) <= tol, (n, rel_rms(got, ref))
        else:
            assert np.all(got == 0)
        with nbs.Context(n, eps=e, precision=prec) as c:
            c.load(p, v, mm)
            alone = c.accel()
        # same arithmetic, different grouping of partial sums
        assert rel_rms(got, alone) <= (1e-14 if prec in ("fp64", "dd") else 1e-6)
        off += n


def test_batch_near_pass_with_single_body_clusters(nbs, orc):
    """Single-body clusters have no near radius and stay out of the cell grid,
    so fewer than N bodies are in it; in a set large enough for the near-pair
    pass (sum of N_k^2 above 2^27) every other cluster must still match the
    oracle to the mixed tolerance and the single bodies feel no force."""
    sizes = [1, 12000, 1, 3000]
    cl = clusters(sizes, base_seed=300)
    pos, vel, m = concat(cl)
    with nbs.Context(sizes=sizes, precision="ds") as b:
        b.set_cluster_params(eps=[c[3] for c in cl])
        b.load(pos, vel, m)
        a = b.accel()
    off = 0
    for (p, v, mm, e), n in zip(cl, sizes):
        got = a[off:off + n]
        if n == 1:
            assert np.all(got == 0)
        else:
            err = rel_rms(got, orc.accel_int(p, mm, 1.0, e))
            assert err <= 1e-6, (n, err)
        off += n


@pytest.mark.parametrize("prec", ["fp64", "ds"])
def test_batch_steps_equal_alone_runs(nbs, orc, prec):
    """Four SI6A steps of the whole ensemble with per-cluster softening and
    per-cluster step scale against each cluster stepped alone.  A cluster
    alone may get a different launch shape (narrower j-ranges for small N),
    which moves where per-tile float sums are cut, so the mixed-precision bar
    is its stated tolerance (positions after 4 steps 1e-6), not bit equality."""
    cl = clusters(SIZES, base_seed=200)
    pos, vel, m = concat(cl)
    eps = [c[3] for c in cl]
    scale = [1.0 + 0.25 * (k % 3) for k in range(len(SIZES))]
    dt = 1.0 / 512
    with nbs.Context(sizes=SIZES, precision=prec) as b:
        b.set_cluster_params(eps=eps, dt_scale=scale)
        b.load(pos, vel, m)
        e_cl = b.energy_clusters()
        b.step(6, dt, 4)
        x, v = b.get_state()
    off = 0
    tol = 1e-12 if prec == "fp64" else 1e-6
    for k, ((p, vv, mm, e), n) in enumerate(zip(cl, SIZES)):
        with nbs.Context(n, eps=e, precision=prec) as c:
            c.load(p, vv, mm)
            e_alone = c.energy()
            c.step(6, dt * scale[k], 4)
            xa, va = c.get_state()
        assert np.abs(x[off:off + n] - xa).max() <= tol
        assert np.abs(v[off:off + n] - va).max() <= tol * 10
        assert abs(e_cl[k].E - e_alone.E) <= 1e-13 * abs(e_alone.E) + 1e-300
        if k == 3:
            rx, rv = orc.run(p, vv, mm, orc.Params(eps=e), 6, dt * scale[k], 4)
            assert np.abs(x[off:off + n] - rx).max() <= (1e-10 if prec == "fp64" else 1e-6)
        off += n


def test_batch_two_pass_steps_match_oracle_and_alone(nbs, orc):
    """A set above the near-pass threshold (sum of N_k^2 > 2^27: one
    12000-body cluster among small ones), so the batched step graph runs the
    two-pass mixed form (pair kernel plus near-pair pass on the side stream)
    with per-cluster frames and near radii: 4 SI6A steps with per-cluster
    softening and step scale, every cluster's positions against the oracle
    and against the cluster stepped alone, within the mixed bar 1e-6."""
    sizes = [700, 12000, 1, 3000, 129]
    cl = clusters(sizes, base_seed=250)
    pos, vel, m = concat(cl)
    eps = [c[3] for c in cl]
    scale = [1.0, 1.0, 2.0, 0.5, 1.5]
    dt = 1.0 / 512
    with nbs.Context(sizes=sizes, precision="ds") as b:
        b.set_cluster_params(eps=eps, dt_scale=scale)
        b.load(pos, vel, m)
        b.accel()
        b.prof_enable(True)
        b.accel()
        assert b.prof_read()["kernel_launches"] == 7   # pair, near pass (5), output
        b.prof_enable(False)
        b.step(6, dt, 4)
        x, v = b.get_state()
    off = 0
    for k, ((p, vv, mm, e), n) in enumerate(zip(cl, sizes)):
        rx, rv = orc.run(p, vv, mm, orc.Params(eps=e), 6, dt * scale[k], 4)
        assert np.abs(x[off:off + n] - rx).max() <= 1e-6, (k, np.abs(x[off:off + n] - rx).max())
        with nbs.Context(n, eps=e, precision="ds") as c:
            c.load(p, vv, mm)
            c.step(6, dt * scale[k], 4)
            xa, _ = c.get_state()
        assert np.abs(x[off:off + n] - xa).max() <= 1e-6
        off += n


def test_batch_energy_totals(nbs, orc):
    cl = clusters(SIZES[:5], base_seed=300)
    pos, vel, m = concat(cl)
    with nbs.Context(sizes=SIZES[:5], precision="ds", eps=0.01) as b:
        b.load(pos, vel, m)
        per = b.energy_clusters()
        tot = b.energy()
    assert abs(sum(e.E for e in per) - tot.E) <= 1e-14 * abs(tot.E)
    for (p, v, mm, _), e in zip(cl, per):
        r = orc.energy(p, v, mm, orc.Params(eps=0.01))
        assert abs(e.E - r.E) <= 1e-12 * abs(r.E)
        np.testing.assert_allclose(e.L, r.L, rtol=0, atol=1e-13)


def test_batch_rejects_bad_shapes(nbs):
    with pytest.raises(nbs.NBError):
        nbs.Context(sizes=[10, 0, 5])
    with nbs.Context(sizes=[10, 5]) as b:
        p, v, m = ics.henon_plummer(14, 0)
        with pytest.raises(nbs.NBError) as e:
            b.load(p, v, m)
        assert e.value.code == nbs.NB_EINVAL
        with pytest.raises(nbs.NBError):
            b.set_cluster_params(eps=[0.1, -1.0])


def test_c4_full_ensemble_sampled(nbs, orc):
    """The benchmark's ensemble at full size (512 Plummer clusters, N_k
    log-uniform in [256, 8192], 1.29M bodies, paper softening per cluster) in
    the launch configuration the benchmark times: accelerations of sampled
    bodies of the smallest, largest and 18 other clusters against the oracle,
    each cluster to the mixed tolerance."""
    sizes = ics.ensemble_sizes(512, 256, 8192, seed=0)
    cl = [ics.henon_plummer(int(n), k) for k, n in enumerate(sizes)]
    eps = [ics.paper_softening(int(n)) for n in sizes]
    pos, vel, m = (np.concatenate([c[i] for c in cl]) for i in range(3))
    with nbs.Context(sizes=sizes, precision="ds") as b:
        b.set_cluster_params(eps=eps)
        b.load(pos, vel, m)
        shape = b.pair_shape()
        a = b.accel()
    assert shape["grid"] > 3 * 152, shape   # the grid runs in waves, as in the benchmark
    off = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(4)
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    pick |= set(int(k) for k in rng.choice(len(sizes), 18, replace=False))
    for k in sorted(pick):
        n = int(sizes[k])
        idx = np.unique(rng.choice(n, min(n, 64), replace=False))
        ref = orc.accel_int_at(cl[k][0], cl[k][2], idx, 1.0, eps[k])
        got = a[off[k]:off[k + 1]][idx]
        err = rel_rms(got, ref)
        assert err <= 1e-6, (k, n, err)
