"""Pins for the CPU oracle: each check compares it with something other than
itself -- a closed form, a symmetry, an invariant, a convergence order, or a
consistency relation between two independently written functions (a force
against the derivative of a potential) -- chosen so that a dropped term, a
wrong sign, index or exponent anywhere in the oracle fails at least one.
"""
import math
import os

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics


def _params(orc, **kw):
    return orc.Params(**kw)


# ---------------------------------------------------------------- force sum

def test_two_body_closed_form(orc):
    """N = 2: a_1 = G m_2 r_12 / (r^2 + eps^2)^{3/2} and a_2 = -(m_1/m_2) a_1
    (eq. 1 with r_ij = r_j - r_i, softened as in eq. 5)."""
    rng = np.random.default_rng(1)
    for eps in (0.0, 0.3):
        pos = rng.normal(size=(2, 3))
        m = np.array([0.7, 2.9])
        G = 1.7
        a = orc.accel_int(pos, m, G, eps)
        r = pos[1] - pos[0]
        d2 = r @ r + eps * eps
        want = G * m[1] * r / d2 ** 1.5
        np.testing.assert_allclose(a[0], want, rtol=1e-14)
        np.testing.assert_allclose(a[1], -m[0] * want / m[1], rtol=1e-14)


@pytest.mark.parametrize("n,eps", [(3, 0.0), (7, 0.0), (12, 0.05), (64, 0.2)])
def test_ring_closed_form(orc, n, eps):
    """n equal masses on a tilted circle of radius R: by symmetry every
    acceleration points to the centre, with magnitude
    G m sum_k 2R sin^2(pi k/n) / ((2R sin(pi k/n))^2 + eps^2)^{3/2}
    (chord length 2R sin(pi k/n), radial projection of the chord 2R sin^2)."""
    R, m, G = 1.3, 0.25, 1.0
    th = 2 * math.pi * np.arange(n) / n
    ring = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(n)], axis=1)
    # rotate into a generic orientation and shift away from the origin
    q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(3, 3)))
    centre = np.array([3.0, -1.0, 2.0])
    pos = ring @ q.T + centre
    a = orc.accel_int(pos, np.full(n, m), G, eps)
    k = np.arange(1, n)
    s = np.sin(math.pi * k / n)
    mag = G * m * np.sum(2 * R * s * s / ((2 * R * s) ** 2 + eps * eps) ** 1.5)
    inward = (centre - pos) / R
    np.testing.assert_allclose(a, mag * inward, rtol=1e-13, atol=1e-13 * mag)


def test_cube_centre_zero_and_outside(orc):
    """Symmetric shells: zero acceleration at the centre of a cube of masses;
    on the cube's diagonal far away the field tends to G M / d^2."""
    c = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    pos = np.vstack([c, np.zeros((1, 3))])
    m = np.full(9, 0.5)
    a = orc.accel_int(pos, m, 1.0, 0.01)
    assert np.abs(a[8]).max() < 1e-15
    d = 1e4
    probe = np.vstack([c, [[d, 0.0, 0.0]]])
    m2 = np.append(np.full(8, 0.5), 1e-9)
    a = orc.accel_int(probe, m2, 1.0, 0.0)
    np.testing.assert_allclose(a[8], [-4.0 / d ** 2, 0, 0], rtol=1e-6, atol=1e-20)


def test_momentum_and_torque_free(orc):
    """Antisymmetry F_ij = -F_ji (Sect. 2): sum m_i a_i = 0 and
    sum m_i r_i x a_i = 0, with unequal masses (a sum over m_i instead of m_j
    breaks both)."""
    rng = np.random.default_rng(2)
    n = 200
    pos = rng.normal(size=(n, 3)) + np.array([50.0, 0, 0])
    m = rng.uniform(0.1, 3.0, n)
    a = orc.accel_int(pos, m, 1.0, 0.01)
    f = m[:, None] * a
    scale = np.abs(f).sum()
    assert np.abs(f.sum(0)).max() < 1e-14 * scale
    tq = np.cross(pos, f).sum(0)
    assert np.abs(tq).max() < 1e-13 * np.abs(np.cross(pos, f)).sum()


def test_translation_rotation_scaling(orc):
    """a(r + c) = a(r); a(Q r) = Q a(r); a(l r; l eps) = a(r; eps) / l^2;
    a linear in G and in the masses."""
    rng = np.random.default_rng(3)
    n = 50
    pos = rng.normal(size=(n, 3))
    m = rng.uniform(0.5, 2, n)
    a = orc.accel_int(pos, m, 1.0, 0.05)
    np.testing.assert_allclose(orc.accel_int(pos + [7.0, -3.0, 1.0], m, 1.0, 0.05), a,
                               rtol=1e-11, atol=1e-12 * np.abs(a).max())
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    np.testing.assert_allclose(orc.accel_int(pos @ q.T, m, 1.0, 0.05), a @ q.T,
                               rtol=1e-11, atol=1e-12 * np.abs(a).max())
    lam = 3.0
    np.testing.assert_allclose(orc.accel_int(lam * pos, m, 1.0, lam * 0.05), a / lam ** 2,
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(orc.accel_int(pos, 2 * m, 3.0, 0.05), 6 * a, rtol=1e-14)


def test_self_term_skipped_unsoftened(orc):
    """eps = 0 needs the j != i exclusion of eq. 2; the result is finite."""
    pos = np.array([[0.0, 0, 0], [2.0, 0, 0], [0, 3.0, 0]])
    a = orc.accel_int(pos, np.ones(3), 1.0, 0.0)
    assert np.isfinite(a).all()
    np.testing.assert_allclose(a[0], [1 / 4, 1 / 9, 0], rtol=1e-15)


def test_force_is_minus_gradient_of_pair_potential(orc):
    """Eq. 4 and eq. 5 written independently (energy routine vs force
    routine): dW/dr_i = -m_i a_i, central finite differences."""
    rng = np.random.default_rng(4)
    n = 12
    pos = rng.normal(size=(n, 3))
    vel = np.zeros((n, 3))
    m = rng.uniform(0.5, 2, n)
    p = _params(orc, G=1.3, eps=0.1)
    a = orc.accel_int(pos, m, 1.3, 0.1)
    h = 1e-5
    for i in (0, 5, 11):
        for k in range(3):
            pp = pos.copy(); pp[i, k] += h
            pm = pos.copy(); pm[i, k] -= h
            dW = (orc.energy(pp, vel, m, p).W - orc.energy(pm, vel, m, p).W) / (2 * h)
            assert abs(dW + m[i] * a[i, k]) < 1e-7 * max(1.0, abs(m[i] * a[i, k]))


def test_plummer_mean_field(orc):
    """Large sampled Plummer sphere: the mean radial acceleration at radius r
    approaches the analytic -G M r / (r^2 + a^2)^{3/2} (statistical pin on
    exponent and sign of the whole sum)."""
    n = 12000
    pos, vel, m = ics.plummer(n, seed=11)
    a = orc.accel_int(pos, m, 1.0, 0.01)
    r = np.linalg.norm(pos, axis=1)
    ar = (a * pos).sum(1) / r
    want = -r / (r * r + 1.0) ** 1.5
    for lo, hi in [(0.5, 0.8), (0.8, 1.2), (1.2, 2.0), (2.0, 4.0)]:
        sel = (r > lo) & (r < hi)
        rel = np.mean(ar[sel] - want[sel]) / np.mean(np.abs(want[sel]))
        assert abs(rel) < 0.04, (lo, hi, rel)


# ----------------------------------------------------------- external field

def _fd_grad(orc, p, x, h=2e-4):
    """Fourth-order central differences (truncation ~ (h / b_d)^4)."""
    g = np.zeros(3)
    for k in range(3):
        f = []
        for s in (-2, -1, 1, 2):
            y = x.copy(); y[k] += s * h
            f.append(orc.ext_phi(p, y))
        g[k] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
    return g


def test_ext_accel_is_minus_grad_phi(orc):
    """F_ext = grad U_ext = -grad Phi (eq. 3): the closed-form acceleration
    against central differences of the independently written potential."""
    p = _params(orc, ext_on=True)
    rng = np.random.default_rng(6)
    pts = np.vstack([[50.0, 0, 0], [49.2, 1.1, 0.3], [0.5, -0.2, 0.05],
                     rng.normal(scale=10, size=(6, 3))])
    for x in pts:
        a = orc.ext_accel(p, x)[0]
        g = _fd_grad(orc, p, x)
        np.testing.assert_allclose(a, -g, rtol=1e-7, atol=1e-9 * np.abs(a).max())


def test_ext_phi_limits(orc):
    """Miyamoto-Nagai with a_d = 0 is a Plummer sphere of scale b_d; far away
    the model tends to a point mass M_d + M_b; at the bulge centre the bulge
    potential is -G M_b / a_b."""
    x = np.array([0.3, -0.7, 0.4])
    p = _params(orc, ext_on=True, Md=2.0, ad=0.0, bd=0.8, Mb=0.0, ab=1.0)
    assert abs(orc.ext_phi(p, x) + 2.0 / math.sqrt(x @ x + 0.64)) < 1e-15
    p = _params(orc, ext_on=True)
    far = np.array([3e5, 1e5, -2e5])
    r = np.linalg.norm(far)
    assert abs(orc.ext_phi(p, far) * r / -115.0 - 1) < 1e-4
    p = _params(orc, ext_on=True, Md=0.0)
    assert abs(orc.ext_phi(p, np.zeros(3)) + 15.0 / 0.7) < 1e-14


def test_ext_symmetries(orc):
    """Axisymmetric about z and mirror-symmetric in z."""
    p = _params(orc, ext_on=True)
    x = np.array([12.0, 5.0, 0.7])
    a = orc.ext_accel(p, x)[0]
    c, s = math.cos(0.9), math.sin(0.9)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    np.testing.assert_allclose(orc.ext_accel(p, Rz @ x)[0], Rz @ a, rtol=1e-13, atol=1e-16)
    xm = x * [1, 1, -1]
    np.testing.assert_allclose(orc.ext_accel(p, xm)[0], a * [1, 1, -1], rtol=1e-14)


def test_ext_field_scaling_laws(orc):
    """Phi and a_ext are linear in G and, jointly, in the three masses;
    stretching every length (the point and a_d, b_d, a_b, eps_bh) by l divides
    Phi by l and a_ext by l^2. A dropped G, or a scale entering unsquared,
    breaks one of these."""
    base = dict(ext_on=True, Mbh=4.0, eps_bh=0.3)
    p = _params(orc, **base)
    lam, g = 2.5, 1.9
    big = _params(orc, ext_on=True, eps_bh=p.eps_bh, G=g, Md=3 * p.Md, Mb=3 * p.Mb,
                  Mbh=3 * p.Mbh)
    far = _params(orc, ext_on=True, Mbh=p.Mbh, eps_bh=lam * p.eps_bh, ad=lam * p.ad,
                  bd=lam * p.bd, ab=lam * p.ab)
    for x in ([50.0, 0.3, -0.2], [0.4, -0.1, 0.05], [7.0, 3.0, 1.5], [0.0, 0.0, 0.0]):
        x = np.array(x)
        phi, a = orc.ext_phi(p, x), orc.ext_accel(p, x)[0]
        assert abs(orc.ext_phi(big, x) - 3 * g * phi) <= 1e-14 * abs(phi) * 3 * g
        np.testing.assert_allclose(orc.ext_accel(big, x)[0], 3 * g * a,
                                   rtol=1e-14, atol=1e-15 * np.abs(a).max() * 3 * g)
        assert abs(orc.ext_phi(far, lam * x) - phi / lam) <= 1e-14 * abs(phi)
        np.testing.assert_allclose(orc.ext_accel(far, lam * x)[0], a / lam ** 2,
                                   rtol=1e-14, atol=1e-15 * np.abs(a).max())


def test_total_acceleration_is_internal_plus_field(orc):
    """Eq. 3: the right-hand side is the pair sum plus the field term; a lone
    body feels the field alone."""
    p = _params(orc, ext_on=True, eps=0.05, G=1.3, Mbh=2.0, eps_bh=0.1)
    one = np.array([[3.0, -1.0, 0.7]])
    np.testing.assert_array_equal(orc.accel(one, [2.0], p), orc.ext_accel(p, one))
    pos, _, m = ics.plummer(40, seed=12)
    pos = pos + np.array([4.0, 1.0, 0.5])
    want = orc.accel_int(pos, m, 1.3, 0.05) + orc.ext_accel(p, pos)
    np.testing.assert_allclose(orc.accel(pos, m, p), want, rtol=1e-15, atol=1e-16)
    off = _params(orc, ext_on=False, eps=0.05, G=1.3, Mbh=2.0, eps_bh=0.1)
    np.testing.assert_array_equal(orc.accel(pos, m, off), orc.accel_int(pos, m, 1.3, 0.05))


def test_circular_speed_constant(orc):
    """VC_R50 and VC_R10 (input module constants) equal sqrt(R |a_R|) at
    R = 50 and R = 10, z = 0."""
    p = _params(orc, ext_on=True)
    a = orc.ext_accel(p, np.array([50.0, 0, 0]))[0]
    assert abs(math.sqrt(50.0 * -a[0]) / ics.VC_R50 - 1) < 1e-14
    a = orc.ext_accel(p, np.array([10.0, 0, 0]))[0]
    assert abs(math.sqrt(10.0 * -a[0]) / ics.VC_R10 - 1) < 1e-14


def test_circular_orbit_stays_circular(orc):
    """A test particle started at R = 50 with v_c on the sixth-order scheme
    keeps |R - 50| < 1e-9 over one full orbital period."""
    p = _params(orc, ext_on=True, eps=0.01)
    pos = np.array([[50.0, 0, 0]])
    vel = np.array([[0.0, ics.VC_R50, 0]])
    period = 2 * math.pi * 50 / ics.VC_R50
    steps = 400
    x, v = orc.run(pos, vel, [1.0], p, 6, period / steps, steps)
    R = np.hypot(x[0, 0], x[0, 1])
    assert abs(R - 50.0) < 1e-9
    assert np.linalg.norm(x[0] - pos[0]) < 1e-6


# ------------------------------------------------------------- integrators

def _kepler_closed_form(pos0, vel0, m, t):
    """Textbook two-body solution: Kepler's equation E - e sin E = n t by
    Newton's method, starting from pericentre on +x with motion in +y."""
    mu = m.sum()
    rel0 = pos0[1] - pos0[0]
    vrel0 = vel0[1] - vel0[0]
    rp = np.linalg.norm(rel0)
    vp = np.linalg.norm(vrel0)
    a = 1.0 / (2.0 / rp - vp * vp / mu)
    e = 1.0 - rp / a
    nmot = math.sqrt(mu / a ** 3)
    M = nmot * t
    E = M if e < 0.8 else math.pi
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    rel = np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    return np.stack([-(m[1] / mu) * rel, (m[0] / mu) * rel])


def _kepler_error(orc, order, nsteps, periods=1.0):
    pos, vel, m = ics.kepler_pair(0.6, 0.4, 1.0, 0.5)
    T = 2 * math.pi * periods
    x, _ = orc.run(pos, vel, m, _params(orc, eps=0.0), order, T / nsteps, nsteps)
    return np.abs(x - _kepler_closed_form(pos, vel, m, T)).max()


def test_kepler_leapfrog_second_order(orc):
    e1 = _kepler_error(orc, 2, 2000)
    e2 = _kepler_error(orc, 2, 4000)
    assert e1 < 1e-3
    assert 3.7 < e1 / e2 < 4.3, e1 / e2


def test_kepler_sixth_order(orc):
    """Order 6: halving dt divides the error by ~64 (a wrong SI6A weight or
    a reversed sequence gives 4th order or worse)."""
    e1 = _kepler_error(orc, 6, 200)
    e2 = _kepler_error(orc, 6, 400)
    assert e1 < 1e-6
    assert 50 < e1 / e2 < 80, (e1, e2, e1 / e2)


def test_si6a_weights_consistency(orc):
    w = orc.si6a_weights()
    assert abs(w[0] + 2 * (w[1] + w[2] + w[3]) - 1) < 1e-15
    # third-order condition of a symmetric composition: sum of w^3 vanishes
    s3 = w[0] ** 3 + 2 * (w[1] ** 3 + w[2] ** 3 + w[3] ** 3)
    assert abs(s3) < 1e-12
    s5 = w[0] ** 5 + 2 * (w[1] ** 5 + w[2] ** 5 + w[3] ** 5)
    assert abs(s5) < 1e-12


@pytest.mark.parametrize("order", [2, 6])
def test_free_body_moves_in_a_straight_line(orc, order):
    """A lone body with no field feels no force, so every scheme moves it by
    t v exactly up to rounding: the drift weights of a step sum to one (for
    SI6A, w0 + 2(w1 + w2 + w3) = 1) and no kick changes v."""
    x0 = np.array([[3.0, -2.0, 0.5]])
    v0 = np.array([[0.25, 1.5, -0.75]])
    h, n = 1 / 64, 128
    x, v = orc.run(x0, v0, [1.0], _params(orc, eps=0.1), order, h, n)
    np.testing.assert_array_equal(v, v0)
    np.testing.assert_allclose(x, x0 + n * h * v0, rtol=0, atol=1e-13)


def test_results_do_not_depend_on_the_thread_count(orc):
    """OpenMP splits only the independent per-body work, and every sum keeps
    its serial order: one thread and all threads give the same bits."""
    pos, vel, m = ics.plummer(300, seed=14, masses=ics.salpeter_masses(300, 14))
    p = _params(orc, eps=0.02, ext_on=True, Mbh=2.0, eps_bh=0.1)
    pos = pos + np.array([8.0, 1.0, 0.3])
    full = orc.max_threads()
    out = []
    for t in (1, full):
        orc.set_threads(t)
        try:
            e = orc.energy(pos, vel, m, p)
            out.append((orc.accel(pos, m, p), orc.run(pos, vel, m, p, 6, 1 / 512, 3),
                        [e.K, e.W, e.W_ext, *e.P, *e.L], orc.torque(pos, m, p)))
        finally:
            orc.set_threads(full)
    (a1, (x1, v1), e1, t1), (a2, (x2, v2), e2, t2) = out
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(v1, v2)
    assert e1 == e2
    np.testing.assert_array_equal(t1, t2)


def test_degenerate_sizes_and_arguments(orc):
    """No bodies: empty accelerations and zero diagnostics; zero steps leave the
    state as it is; an order other than 2 or 6 is refused."""
    p = _params(orc, eps=0.1, ext_on=True)
    z = np.zeros((0, 3))
    assert orc.accel(z, np.zeros(0), p).shape == (0, 3)
    e = orc.energy(z, z, np.zeros(0), p)
    assert (e.K, e.W, e.W_ext, e.E) == (0.0, 0.0, 0.0, 0.0)
    assert not e.P.any() and not e.L.any()
    pos, vel, m = ics.plummer(8, seed=13)
    x, v = orc.run(pos, vel, m, p, 6, 0.01, 0)
    np.testing.assert_array_equal(x, pos)
    np.testing.assert_array_equal(v, vel)
    with pytest.raises(ValueError):
        orc.run(pos, vel, m, p, 4, 0.01, 1)


def _energy_drift(orc, order, nsteps):
    pos, vel, m = ics.kepler_pair(0.5, 0.5, 1.0, 0.5)
    p = _params(orc, eps=0.0)
    E0 = orc.energy(pos, vel, m, p).E
    T = 2 * math.pi
    h = T / nsteps
    worst = 0.0
    x, v = pos, vel
    chunk = nsteps // 8
    for _ in range(8):
        x, v = orc.run(x, v, m, p, order, h, chunk)
        worst = max(worst, abs(orc.energy(x, v, m, p).E - E0))
    return worst / abs(E0)


def test_energy_error_scaling(orc):
    """Symplectic schemes: bounded energy error scaling as dt^2 and dt^6."""
    r2 = _energy_drift(orc, 2, 4000) / _energy_drift(orc, 2, 8000)
    assert 3.5 < r2 < 4.5, r2
    r6 = _energy_drift(orc, 6, 400) / _energy_drift(orc, 6, 800)
    assert 45 < r6 < 85, r6


@pytest.mark.parametrize("order", [2, 6])
def test_time_reversal(orc, order):
    """Symmetric schemes are time reversible (Sect. 3.1): n steps, flip the
    velocities, n steps gives back the initial positions."""
    pos, vel, m = ics.plummer(32, seed=3)
    p = _params(orc, eps=0.05, ext_on=True)
    pos = pos + [50.0, 0, 0]
    vel = vel + [0, ics.VC_R50, 0]
    x, v = orc.run(pos, vel, m, p, order, 1 / 256, 40)
    x2, v2 = orc.run(x, -v, m, p, order, 1 / 256, 40)
    assert np.abs(x2 - pos).max() < 1e-12
    assert np.abs(v2 + vel).max() < 1e-12


def test_isolated_conservation(orc):
    """No external field: total momentum and angular momentum are conserved
    to round-off (Sect. 2), energy to the scheme's truncation level."""
    pos, vel, m = ics.plummer(64, seed=4, masses=ics.salpeter_masses(64, 4))
    p = _params(orc, eps=0.02)
    e0 = orc.energy(pos, vel, m, p)
    x, v = orc.run(pos, vel, m, p, 6, 1 / 512, 100)
    e1 = orc.energy(x, v, m, p)
    assert np.abs(e1.P - e0.P).max() < 1e-15
    assert np.abs(e1.L - e0.L).max() < 1e-14
    assert abs((e1.E - e0.E) / e0.E) < 1e-8


def test_axisymmetric_field_conserves_lz(orc):
    """In the axisymmetric disk + bulge field the z torque vanishes pairwise
    and each drift preserves r x v, so L_z is conserved to round-off by the
    discrete scheme (the paper's Table 2 finds L_z errors near 1e-17); L_x,
    L_y change by the external torque of eq. 8."""
    pos, vel, m = ics.plummer(64, seed=5)
    pos, vel = ics.place_on_orbit(pos, vel)
    pos[:, 2] += 0.3
    p = _params(orc, eps=0.01, ext_on=True)
    e0 = orc.energy(pos, vel, m, p)
    x, v = orc.run(pos, vel, m, p, 6, 1 / 256, 50)
    e1 = orc.energy(x, v, m, p)
    assert abs(e1.L[2] - e0.L[2]) < 1e-13 * abs(e0.L[2])
    assert abs((e1.E - e0.E) / e0.E) < 1e-10
    tq = orc.torque(pos, m, p)
    assert abs(tq[2]) < 1e-13 * np.abs(tq).max()
    assert np.abs(tq[:2]).max() > 0


def test_torque_closed_form(orc):
    """Eq. 8 for one particle at (x, 0, z): torque about y equals
    m (z a_x - x a_z), with a from the field routine; x component zero."""
    p = _params(orc, ext_on=True)
    x = np.array([[5.0, 0.0, 0.4]])
    a = orc.ext_accel(p, x[0])[0]
    t = orc.torque(x, [2.0], p)
    np.testing.assert_allclose(t, [0.0, 2.0 * (0.4 * a[0] - 5.0 * a[2]), 0.0],
                               rtol=1e-14, atol=1e-18)



# ------------------------------------------- central black hole (Sect. 6.2)

def test_black_hole_is_a_plummer_sphere_of_its_softening(orc):
    """The central point mass M_bh softened by eps_bh and a Plummer bulge with
    M_b = M_bh, a_b = eps_bh are the same field; the bulge term is pinned on
    its own above (centre value, far field, -grad Phi)."""
    rng = np.random.default_rng(21)
    bh = _params(orc, ext_on=True, Md=0.0, Mb=0.0, Mbh=7.0, eps_bh=0.4)
    bu = _params(orc, ext_on=True, Md=0.0, Mb=7.0, ab=0.4)
    for x in np.vstack([[0.0, 0, 0], [0.3, -0.2, 0.1], rng.normal(scale=3, size=(5, 3))]):
        assert abs(orc.ext_phi(bh, x) - orc.ext_phi(bu, x)) <= 1e-15 * abs(orc.ext_phi(bu, x))
        np.testing.assert_allclose(orc.ext_accel(bh, x)[0], orc.ext_accel(bu, x)[0],
                                   rtol=1e-15, atol=0)


def test_black_hole_field_is_minus_grad_phi(orc):
    """With the black hole added to disk and bulge, a_ext = -grad Phi still
    holds (fourth-order differences), including well inside eps_bh."""
    p = _params(orc, ext_on=True, Mbh=50.0, eps_bh=0.05)
    for x in ([0.02, 0.01, -0.005], [0.2, 0.1, -0.05], [3.0, -1.0, 0.5], [10.0, 0.0, 0.0]):
        x = np.array(x)
        a = orc.ext_accel(p, x)[0]
        g = _fd_grad(orc, p, x, h=1e-5 if np.linalg.norm(x) < 0.1 else 2e-4)
        np.testing.assert_allclose(a, -g, rtol=1e-7, atol=1e-9 * np.abs(a).max())


def _bh_kepler_error(orc, nsteps):
    """Test particle about an unsoftened point mass fixed at the origin (no
    disk, no bulge): e = 0.5 orbit, compared after 0.6 periods with the
    solution of Kepler's equation for mu = M_bh."""
    M, a, e = 3.0, 1.0, 0.5
    rp = a * (1 - e)
    vp = math.sqrt(M * (1 + e) / rp)
    pos0 = np.array([[0.0, 0, 0], [rp, 0, 0]])
    vel0 = np.array([[0.0, 0, 0], [0, vp, 0]])
    t = 0.6 * 2 * math.pi * math.sqrt(a ** 3 / M)
    exact = _kepler_closed_form(pos0, vel0, np.array([M, 0.0]), t)[1]
    p = _params(orc, ext_on=True, Md=0.0, Mb=0.0, Mbh=M, eps_bh=0.0)
    x, _ = orc.run(pos0[1:], vel0[1:], [1.0], p, 6, t / nsteps, nsteps)
    return np.abs(x[0] - exact).max()


def test_orbit_about_black_hole_is_keplerian(orc):
    """The point-mass term integrates to Kepler's orbit at sixth order (error
    ratio ~64 per dt halving; a wrong exponent or a missing G M fails)."""
    e1 = _bh_kepler_error(orc, 240)
    e2 = _bh_kepler_error(orc, 480)
    assert e1 < 1e-5, e1
    assert 45 < e1 / e2 < 85, (e1, e2, e1 / e2)


def test_angular_momentum_rate_is_external_torque(orc):
    """L changes only through the external torque of eq. 8 (internal forces
    are central, Sect. 5.1): (L(h) - L(-h)) / 2h from two sixth-order steps
    matches M_ext at t = 0 to O(h^2); the black hole, central about the
    origin, adds no torque of its own."""
    pos, vel, m = ics.plummer(64, seed=8)
    pos = 0.5 * pos + np.array([6.0, 1.0, 0.8])
    p = _params(orc, eps=0.01, ext_on=True, Mbh=5.0, eps_bh=0.1)
    h = 1e-3
    xf, vf = orc.run(pos, vel, m, p, 6, h, 1)
    xb, vb = orc.run(pos, vel, m, p, 6, -h, 1)
    dL = (orc.energy(xf, vf, m, p).L - orc.energy(xb, vb, m, p).L) / (2 * h)
    tq = orc.torque(pos, m, p)
    assert np.abs(tq).max() > 0
    np.testing.assert_allclose(dL, tq, rtol=0, atol=1e-6 * np.abs(tq).max())
    only_bh = _params(orc, eps=0.01, ext_on=True, Md=0.0, Mb=0.0, Mbh=5.0, eps_bh=0.1)
    assert np.abs(orc.torque(pos, m, only_bh)).max() < 1e-14 * np.abs(tq).max() * 1e3

# ------------------------------------------------------------ diagnostics

def test_energy_closed_forms(orc):
    """Two bodies: K = sum m v^2/2, W = -G m1 m2 / sqrt(r^2 + eps^2) (eq. 4),
    P = sum m v, L = sum m r x v."""
    pos = np.array([[1.0, 2.0, 0.5], [-0.5, 0.0, 1.0]])
    vel = np.array([[0.1, -0.2, 0.3], [0.0, 0.4, -0.1]])
    m = np.array([2.0, 3.0])
    p = _params(orc, G=1.5, eps=0.2)
    e = orc.energy(pos, vel, m, p)
    r2 = ((pos[0] - pos[1]) ** 2).sum()
    assert abs(e.W + 1.5 * 6.0 / math.sqrt(r2 + 0.04)) < 1e-15
    assert abs(e.K - 0.5 * (2 * 0.14 + 3 * 0.17)) < 1e-15
    np.testing.assert_allclose(e.P, [0.2, 0.8, 0.3], atol=1e-16)
    np.testing.assert_allclose(e.L, 2 * np.cross(pos[0], vel[0]) + 3 * np.cross(pos[1], vel[1]),
                               atol=1e-15)
    assert e.W_ext == 0.0


def test_ext_energy_gradient(orc):
    """W_ext = sum m Phi: its derivative in r_i is -m_i a_ext(r_i)."""
    p = _params(orc, ext_on=True, eps=0.1)
    pos = np.array([[49.0, 1.0, 0.2], [51.0, -0.5, -0.1]])
    vel = np.zeros((2, 3))
    m = np.array([0.3, 0.7])
    h = 1e-5
    ae = orc.ext_accel(p, pos)
    for i in range(2):
        for k in range(3):
            pp = pos.copy(); pp[i, k] += h
            pm = pos.copy(); pm[i, k] -= h
            d = (orc.energy(pp, vel, m, p).W_ext - orc.energy(pm, vel, m, p).W_ext) / (2 * h)
            assert abs(d + m[i] * ae[i, k]) < 1e-7 * max(1e-3, abs(m[i] * ae[i, k]))


def test_plummer_virial_and_henon_energy(orc):
    """Sampled Plummer sphere in Henon units: 2K/|W| = 1 and E = -1/4 within
    sampling noise (a few / sqrt(N))."""
    n = 8192
    pos, vel, m = ics.henon_plummer(n, seed=0)
    e = orc.energy(pos, vel, m, _params(orc, eps=1e-3))
    q = 2 * e.K / abs(e.W)
    assert abs(q - 1) < 4 / math.sqrt(n), q
    assert abs(e.E + 0.25) < 0.25 * 4 / math.sqrt(n), e.E


def test_uniform_sphere_virial_ratio(orc):
    """The paper's workload: uniform sphere with expected Q = 0.3."""
    n = 6000
    pos, vel, m = ics.uniform_sphere(n, seed=0, q_vir=0.3)
    e = orc.energy(pos, vel, m, _params(orc, eps=ics.paper_softening(n)))
    assert abs(2 * e.K / abs(e.W) - 0.3) < 0.3 * 5 / math.sqrt(n)


def test_sampled_sum_matches_full_sum(orc):
    """The sampled routine used at full size is the same sum as the full one,
    bit for bit, on the bodies it is asked for."""
    pos, vel, m = ics.plummer(700, seed=9, masses=ics.salpeter_masses(700, 9))
    full = orc.accel_int(pos, m, 1.0, 0.01)
    idx = np.array([0, 5, 699, 350, 5])
    np.testing.assert_array_equal(orc.accel_int_at(pos, m, idx, 1.0, 0.01), full[idx])


# ------------------------------------------- high-precision brute force

def _dec_accel(pos, m, eps):
    """a_i = sum_{j != i} m_j (x_j - x_i) / (r^2 + eps^2)^{3/2} (eq. 5) in
    60-digit decimal arithmetic, from the exact values of the double inputs;
    also the sum of the terms' magnitudes per body."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    P = [[Decimal(float(v)) for v in row] for row in pos]
    M = [Decimal(float(v)) for v in m]
    e2 = Decimal(float(eps)) ** 2
    n = len(M)
    out, mag = [], []
    for i in range(n):
        a = [Decimal(0)] * 3
        s = Decimal(0)
        for j in range(n):
            if j == i:
                continue
            d = [P[j][c] - P[i][c] for c in range(3)]
            r2 = sum(x * x for x in d) + e2
            w = M[j] / (r2 * r2.sqrt())
            for c in range(3):
                a[c] += w * d[c]
            s += abs(w) * r2.sqrt()
        out.append([float(x) for x in a])
        mag.append(float(s))
    return np.array(out), np.array(mag)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_force_sum_against_high_precision_brute_force(orc, n, eps):
    """The FP64 sum agrees with a 60-digit brute force of eq. 5 to within a
    rounding bound: a few ulps per term times the sum of the terms' sizes."""
    rng = np.random.default_rng(500 + n)
    pos = rng.normal(size=(n, 3))
    m = rng.uniform(0.1, 2.0, n)
    ref, mag = _dec_accel(pos, m, eps)
    got = orc.accel_int(pos, m, 1.0, eps)
    err = np.linalg.norm(got - ref, axis=1)
    bound = 8 * n * 2.0 ** -52 * mag
    assert np.all(err <= bound), (err, bound)
    # and well below the FP64 GPU bar of 1e-12 relative
    assert np.linalg.norm(got - ref) <= 1e-15 * np.linalg.norm(ref) * max(1.0, mag.max() / np.abs(ref).max())


def test_potential_energy_against_high_precision_brute_force(orc):
    """W = -G sum_{i<j} m_i m_j / sqrt(r^2 + eps^2) (eq. 4) to 1e-15 relative."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    rng = np.random.default_rng(77)
    n, eps = 7, 0.03
    pos = rng.normal(size=(n, 3))
    vel = np.zeros((n, 3))
    m = rng.uniform(0.1, 2.0, n)
    W = Decimal(0)
    for i in range(n):
        for j in range(i + 1, n):
            r2 = sum((Decimal(float(pos[j, c])) - Decimal(float(pos[i, c]))) ** 2
                     for c in range(3)) + Decimal(eps) ** 2
            W -= Decimal(float(m[i])) * Decimal(float(m[j])) / r2.sqrt()
    e = orc.energy(pos, vel, m, _params(orc, eps=eps))
    assert abs(e.W - float(W)) <= 1e-15 * abs(float(W))


def test_external_field_against_high_precision(orc):
    """The disk + bulge + black hole acceleration (closed form of -grad Phi)
    against the same closed form in 60-digit decimals, to 1e-15 relative."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    p = _params(orc, ext_on=True, Mbh=3.0, eps_bh=0.2)
    D = lambda v: Decimal(float(v))
    for x in ([50.0, 0.3, -0.2], [0.4, -0.1, 0.05], [7.0, 3.0, 1.5]):
        X, Y, Z = (D(v) for v in x)
        R2 = X * X + Y * Y
        s = (Z * Z + D(p.bd) ** 2).sqrt()
        Dd = (R2 + (D(p.ad) + s) ** 2)
        kd = D(p.Md) / (Dd * Dd.sqrt())
        rb2 = R2 + Z * Z + D(p.ab) ** 2
        kb = D(p.Mb) / (rb2 * rb2.sqrt())
        rh2 = R2 + Z * Z + D(p.eps_bh) ** 2
        kh = D(p.Mbh) / (rh2 * rh2.sqrt())
        want = np.array([float(-(kd + kb + kh) * X), float(-(kd + kb + kh) * Y),
                         float(-(kd * (D(p.ad) + s) / s + kb + kh) * Z)])
        got = orc.ext_accel(p, np.array(x))[0]
        assert np.linalg.norm(got - want) <= 1e-15 * np.linalg.norm(want) * 4


# ------------------------------------------------------------ golden fixtures

def _golden(name):
    from golden.fixture import load
    return load(name)


def test_oracle_reproduces_its_fixture(orc):
    """The oracle against the fixture tests/golden/make_golden.py wrote from it
    (a seeded 16-body cluster at R = 50 in the field): a change to the
    oracle's arithmetic shows here and must come with its reason."""
    g = _golden("oracle_plummer16_orbit.txt")
    G, eps, Md, ad, bd, Mb, ab, dt, steps = g["params"][0]
    p = orc.Params(G=G, eps=eps, ext_on=True, Md=Md, ad=ad, bd=bd, Mb=Mb, ab=ab)
    m, pos, vel = g["mass"][0], g["pos"], g["vel"]
    a = orc.accel(pos, m, p)
    np.testing.assert_allclose(a, g["acc"], rtol=1e-13, atol=1e-15 * np.abs(g["acc"]).max())
    e = orc.energy(pos, vel, m, p)
    np.testing.assert_allclose([e.K, e.W, e.W_ext, e.E, *e.P, *e.L], g["energy"][0],
                               rtol=1e-13, atol=1e-16)
    for order in (6, 2):
        x, v = orc.run(pos, vel, m, p, order, dt, int(steps))
        np.testing.assert_allclose(x, g[f"pos_order{order}"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(v, g[f"vel_order{order}"], rtol=0, atol=1e-12)


def test_fixture_is_exactly_what_its_script_writes(tmp_path):
    """The committed fixture is the byte-for-byte output of the committed
    script (which calls only the oracle and the seeded inputs), so no stored
    value has another source."""
    import importlib.util
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(here, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = tmp_path / "fixture.txt"
    mod.main(str(out))
    with open(os.path.join(here, "oracle_plummer16_orbit.txt"), "rb") as f:
        assert out.read_bytes() == f.read()


def test_paper_context_matches_the_printed_tables():
    """The paper's figures quoted in the benchmark lines (context) equal the
    transcription of its Tables 3 and 8 in tests/golden/paper_tables.txt."""
    import bench
    import bench_workloads
    t = _golden("paper_tables.txt")
    n = [int(v) for v in t["table3_n"][0]]
    assert bench.PAPER_CONTEXT["n"] == n
    for key in ("sp_gflops_1gpu", "dp_gflops_1gpu", "sp_gflops_2gpu", "dp_gflops_2gpu"):
        row = "table3_" + key.replace("_gflops", "")
        assert bench.PAPER_CONTEXT[key] == list(t[row][0]), key
    assert [bench_workloads.PAPER_TABLE3_SP[k] for k in n] == list(t["table3_sp_1gpu"][0])
    assert [bench_workloads.PAPER_TABLE3_DP[k] for k in n] == list(t["table3_dp_1gpu"][0])
    for q, de, dl in t["table8"]:
        assert bench_workloads.PAPER_TABLE8[q] == (de, dl), q
