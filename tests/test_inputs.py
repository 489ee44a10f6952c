"""The seeded input generators (paper_1003_3896_gb300/ics.py) draw the
distributions the input recipe states, checked on the CPU: Kolmogorov-Smirnov
tests against the analytic distribution functions (each with a neighbouring
wrong recipe that the same test must reject, so the test is shown to have the
power to see a slip), frame and bulk-motion checks, the workload statistics
the ensemble and serving configurations are quoted on, and determinism."""
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

stats = pytest.importorskip("scipy.stats")

P_OK = 1e-3        # a correct recipe passes at this level (fixed seeds)
P_WRONG = 1e-6     # the neighbouring wrong recipe is rejected at this level


def _cdf_on_grid(density, lo, hi, k=200001):
    """Distribution function of an unnormalised density on [lo, hi], by the
    trapezoid rule on a fine grid (the densities here are smooth)."""
    x = np.linspace(lo, hi, k)
    f = density(x)
    c = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(x))])
    c /= c[-1]
    return lambda v: np.interp(v, x, c)


def _ks(sample, cdf):
    return stats.kstest(sample, cdf).pvalue


# ------------------------------------------------------------------ Plummer

def _plummer_mass_cdf(a, rmax):
    """Cumulative mass fraction r^3 / (r^2 + a^2)^{3/2}, renormalised to the
    truncation radius."""
    X = lambda r: r ** 3 / (r * r + a * a) ** 1.5
    return lambda r: X(np.asarray(r)) / X(rmax)


def test_plummer_radii_follow_the_truncated_mass_profile():
    a = 1.3
    pos, _, _ = ics.plummer(20000, seed=41, a=a, com_frame=False)
    r = np.linalg.norm(pos, axis=1)
    assert r.max() <= 20 * a
    assert _ks(r, _plummer_mass_cdf(a, 20 * a)) > P_OK
    # a Plummer sphere of another scale, or an untruncated profile, is seen
    assert _ks(r, _plummer_mass_cdf(1.2 * a, 20 * 1.2 * a)) < P_WRONG


def test_henon_units_scale():
    """Henon units (E = -1/4 with G = M = 1) give the Plummer scale 3 pi / 16."""
    a = 3 * math.pi / 16
    pos, _, m = ics.henon_plummer(20000, seed=42)
    assert abs(m.sum() - 1.0) < 1e-12
    r = np.linalg.norm(pos, axis=1)
    assert _ks(r, _plummer_mass_cdf(a, 20 * a)) > P_OK
    assert _ks(r, _plummer_mass_cdf(1.0, 20.0)) < P_WRONG


def test_plummer_speeds_follow_the_distribution_function():
    """q = v / v_esc(r), v_esc = sqrt(2 G M / a) (1 + r^2/a^2)^{-1/4}, has the
    density q^2 (1 - q^2)^{7/2} on [0, 1]; the rejection envelope 0.1 lies
    above its maximum."""
    a, M = 0.8, 2.0
    pos, vel, _ = ics.plummer(20000, seed=43, a=a, total_mass=M, com_frame=False)
    r = np.linalg.norm(pos, axis=1)
    q = np.linalg.norm(vel, axis=1) / (math.sqrt(2 * M / a) * (1 + (r / a) ** 2) ** -0.25)
    assert q.max() < 1.0
    g = lambda x: x * x * (1 - x * x) ** 3.5
    assert g(np.linspace(0, 1, 100001)).max() < 0.1
    assert _ks(q, _cdf_on_grid(g, 0.0, 1.0)) > P_OK
    assert _ks(q, _cdf_on_grid(lambda x: x * x * (1 - x * x) ** 2.5, 0.0, 1.0)) < P_WRONG


def test_directions_are_isotropic():
    pos, vel, _ = ics.plummer(20000, seed=44, com_frame=False)
    for v in (pos, vel):
        u = v / np.linalg.norm(v, axis=1)[:, None]
        assert _ks(u[:, 2], stats.uniform(-1, 2).cdf) > P_OK
        phi = np.arctan2(u[:, 1], u[:, 0])
        assert _ks(phi, stats.uniform(-math.pi, 2 * math.pi).cdf) > P_OK
    # directions uniform in theta (not in cos theta) would be seen
    th = np.random.default_rng(0).uniform(0, math.pi, 20000)
    assert _ks(np.cos(th), stats.uniform(-1, 2).cdf) < P_WRONG


@pytest.mark.parametrize("gen", ["plummer", "henon", "uniform", "salpeter"])
def test_centre_of_mass_frame(gen):
    if gen == "plummer":
        pos, vel, m = ics.plummer(3000, seed=45)
    elif gen == "henon":
        pos, vel, m = ics.henon_plummer(3000, seed=45)
    elif gen == "uniform":
        pos, vel, m = ics.uniform_sphere(3000, seed=45)
    else:
        pos, vel, m = ics.plummer(3000, seed=45, masses=ics.salpeter_masses(3000, 45))
    for v in (pos, vel):
        assert np.abs((m[:, None] * v).sum(0)).max() <= 1e-15 * (m[:, None] * np.abs(v)).sum()


# ------------------------------------------------------- paper's workloads

def test_uniform_sphere_positions_and_speeds():
    """Positions uniform in the ball (r/R has distribution function (r/R)^3);
    speeds uniform on [0, v_max] with v_max^2 = 3 Q |W| / M for a uniform
    sphere's W = -(3/5) G M^2 / R."""
    n, R, Q, M = 8000, 2.0, 0.3, 1.5
    pos, vel, m = ics.uniform_sphere(n, seed=46, q_vir=Q, radius=R, total_mass=M)
    np.testing.assert_array_equal(m, np.full(n, M / n))
    r = np.linalg.norm(pos, axis=1)
    assert _ks(r / R, lambda x: np.clip(x, 0, 1) ** 3) > P_OK
    vmax = math.sqrt(3 * Q * 0.6 * M / R)
    s = np.linalg.norm(vel, axis=1)
    assert _ks(s / vmax, stats.uniform(0, 1).cdf) > P_OK
    assert _ks(s / vmax, stats.uniform(0, 1.05).cdf) < P_WRONG
    # positions uniform in radius instead of in volume would be seen
    assert _ks(r / R, stats.uniform(0, 1).cdf) < P_WRONG


def test_salpeter_masses():
    """dN/dm ~ m^{-2.35} on [0.1, 100], rescaled to a total mass: the scale
    is recovered from the lightest body (within 1e-4 of the lower bound at this
    size), the shape is tested against the truncated power law."""
    n = 20000
    m = ics.salpeter_masses(n, seed=47, total=3.0)
    assert abs(m.sum() - 3.0) < 1e-12
    c = m.min() / 0.1
    mm = m / c
    assert mm.max() <= 100.0 * (1 + 1e-3)

    def cdf(slope):
        p = 1 - slope
        lo, hi = 0.1 ** p, 100.0 ** p
        return lambda x: (np.clip(x, 0.1, 100.0) ** p - lo) / (hi - lo)
    assert _ks(mm, cdf(2.35)) > P_OK
    assert _ks(mm, cdf(2.2)) < P_WRONG
    # independent of position: drawing masses leaves the phase-space draw as it is
    a = ics.plummer(500, seed=47, com_frame=False)
    b = ics.plummer(500, seed=47, com_frame=False, masses=ics.salpeter_masses(500, 47))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_paper_softening_rule():
    """eps = 0.005 R / N^{1/3}: 1.24e-4 at N = 65536 with R = 1."""
    assert abs(ics.paper_softening(65536) - 0.005 / 40.31747359663594) < 1e-18
    assert abs(ics.paper_softening(1000, radius=2.0) - 0.001) < 1e-18


def test_cluster_on_orbit_and_plunge_start():
    pos, vel, m = ics.plummer(4096, seed=48)
    p, v = ics.place_on_orbit(pos, vel)
    w = m / m.sum()
    np.testing.assert_allclose((w[:, None] * p).sum(0), [50.0, 0, 0], atol=1e-12)
    np.testing.assert_allclose((w[:, None] * v).sum(0), [0, ics.VC_R50, 0], atol=1e-14)
    p, v, m = ics.plunge_cluster(4096, seed=48)
    w = m / m.sum()
    np.testing.assert_allclose((w[:, None] * p).sum(0), [10.0, 0, 0], atol=1e-12)
    np.testing.assert_allclose((w[:, None] * v).sum(0), [0, 1e-3 * ics.VC_R10, 0], atol=1e-15)


def test_kepler_pair_elements():
    """Pericentre a(1 - e) on x, barycentre at rest at the origin, energy
    -G m1 m2 / (2a), angular momentum mu sqrt(G M a (1 - e^2)) (textbook)."""
    m1, m2, a, e = 0.6, 0.4, 1.3, 0.5
    pos, vel, m = ics.kepler_pair(m1, m2, a, e)
    np.testing.assert_allclose(m @ pos, 0, atol=1e-16)
    np.testing.assert_allclose(m @ vel, 0, atol=1e-16)
    d = pos[1] - pos[0]
    assert abs(np.linalg.norm(d) - a * (1 - e)) < 1e-15
    K = 0.5 * (m * (vel ** 2).sum(1)).sum()
    assert abs(K - m1 * m2 / np.linalg.norm(d) + m1 * m2 / (2 * a)) < 1e-14
    L = (m[:, None] * np.cross(pos, vel)).sum(0)
    mu = m1 * m2 / (m1 + m2)
    np.testing.assert_allclose(L, [0, 0, mu * math.sqrt((m1 + m2) * a * (1 - e * e))],
                               rtol=1e-14)


# ------------------------------------------------ ensemble and serving jobs

def test_ensemble_sizes_log_uniform():
    """512 sizes log-uniform on [256, 8192]; the workload figures follow:
    E[N] = (8192 - 256) / ln 32 = 2290 and E[sum N^2] = 512 (8192^2 - 256^2) /
    (2 ln 32) = 4.95e9 (the seed-0 draw has 5.73e9)."""
    n = ics.ensemble_sizes()
    assert n.shape == (512,) and n.dtype == np.int64
    assert n.min() >= 256 and n.max() <= 8192
    u = np.log(n)
    assert _ks(u, stats.uniform(math.log(256), math.log(32)).cdf) > P_OK
    assert _ks(u, stats.uniform(math.log(256), math.log(16)).cdf) < P_WRONG
    mean = (8192 - 256) / math.log(32)
    assert abs(n.mean() / mean - 1) < 4 * 0.8 / math.sqrt(512)
    # N^2 is heavy-tailed: E[N^4] / E[N^2]^2 - 1 = 2.47, a 7% standard error
    e2 = (8192 ** 2 - 256 ** 2) / (2 * math.log(32))
    e4 = (8192 ** 4 - 256 ** 4) / (4 * math.log(32))
    cv = math.sqrt(e4 / e2 ** 2 - 1)
    assert abs((n.astype(float) ** 2).sum() / (512 * e2) - 1) < 4 * cv / math.sqrt(512)
    np.testing.assert_array_equal(n, ics.ensemble_sizes())


def test_serving_trace_statistics():
    """Poisson arrivals at 200 / s (exponential gaps), N log-uniform on
    [1024, 131072], order and precision fair coins, steps log-uniform on
    [10, 1000], job k seeded with k."""
    jobs = ics.serving_trace()
    assert len(jobs) == 2000
    t = np.array([j.arrival_s for j in jobs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert _ks(gaps, stats.expon(scale=1 / 200).cdf) > P_OK
    assert _ks(gaps, stats.expon(scale=1 / 150).cdf) < P_WRONG
    n = np.array([j.n for j in jobs])
    assert n.min() >= 1024 and n.max() <= 131072
    assert _ks(np.log(n), stats.uniform(math.log(1024), math.log(128)).cdf) > P_OK
    for field, values in (("order", (2, 6)), ("precision", (0, 1))):
        x = np.array([getattr(j, field) for j in jobs])
        assert set(np.unique(x)) == set(values)
        assert abs((x == values[0]).mean() - 0.5) < 4 * 0.5 / math.sqrt(2000)
    s = np.array([j.nsteps for j in jobs])
    assert s.min() >= 10 and s.max() <= 1000
    assert _ks(np.log(s), stats.uniform(math.log(10), math.log(100)).cdf) > P_OK
    assert [j.seed for j in jobs] == list(range(2000))
    assert [j.index for j in jobs] == list(range(2000))


# -------------------------------------------------------------- determinism

def test_seeded_and_distinct():
    for gen in (lambda s: ics.plummer(300, s), lambda s: ics.uniform_sphere(300, s),
                lambda s: (ics.salpeter_masses(300, s),)):
        a, b, c = gen(7), gen(7), gen(8)
        for x, y, z in zip(a, b, c):
            np.testing.assert_array_equal(x, y)
        assert any(not np.array_equal(x, z) for x, z in zip(a, c))
    assert ics.plummer(0, 1)[0].shape == (0, 3)
