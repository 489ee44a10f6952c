"""A massive point at the galactic centre (the black hole of Sect. 6.2's
collision runs, read as a static Plummer-softened mass in the external field):
accelerations, a close passage integrated step by step, energies and the
torque of eq. 8 against the oracle, through the C ABI."""
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ds": 1e-6}


@pytest.fixture(scope="module")
def nbs():
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import nbsym
    return nbsym


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())


def cluster_near_bh(n, seed, scale=0.2):
    """A compact Plummer cluster at (1, 0, 0) moving past the centre."""
    pos, vel, m = ics.plummer(n, seed)
    pos = scale * pos + np.array([1.0, 0.0, 0.0])
    vel = vel / math.sqrt(scale) + np.array([-3.0, 0.5, 0.0])
    return pos, vel, m


@pytest.mark.parametrize("prec", ["fp64", "ds"])
@pytest.mark.parametrize("n", [129, 3000, 16500])
def test_black_hole_accel_parity(nbs, orc, prec, n):
    pos, vel, m = cluster_near_bh(n, 40 + n)
    eps = ics.paper_softening(n)
    p = orc.Params(eps=eps, ext_on=True, Mbh=50.0, eps_bh=0.01)
    ref = orc.accel(pos, m, p)
    with nbs.Context(n, eps=eps, precision=prec, ext_on=True, Mbh=50.0, eps_bh=0.01) as c:
        c.load(pos, vel, m)
        a = c.accel()
    assert rel_rms(a, ref) <= TOL[prec], rel_rms(a, ref)


@pytest.mark.parametrize("prec", ["fp64", "ds"])
def test_black_hole_passage_steps(nbs, orc, prec):
    """40 sixth-order steps of a cluster passing 0.1 from a mass 50 times its
    own: positions against the oracle, and the energy error no worse than
    twice the oracle's."""
    n = 700
    pos, vel, m = cluster_near_bh(n, 5)
    eps = ics.paper_softening(n)
    p = orc.Params(eps=eps, ext_on=True, Mbh=50.0, eps_bh=0.01)
    dt, steps = 1e-3, 40
    rx, rv = orc.run(pos, vel, m, p, 6, dt, steps)
    e0 = orc.energy(pos, vel, m, p).E
    de_ref = abs(orc.energy(rx, rv, m, p).E - e0)
    with nbs.Context(n, eps=eps, precision=prec, ext_on=True, Mbh=50.0, eps_bh=0.01) as c:
        c.load(pos, vel, m)
        eg0 = c.energy()
        assert abs(eg0.E - e0) <= 1e-12 * abs(e0)
        c.step(6, dt, steps)
        x, v = c.get_state()
        e1 = c.energy()
    assert np.abs(x - rx).max() <= (1e-10 if prec == "fp64" else 1e-6)
    assert abs(e1.E - eg0.E) <= 2 * de_ref + 1e-13 * abs(e0)


def test_black_hole_torque_and_zero_mass_limit(nbs, orc):
    """Eq. 8's torque with the black hole on equals the oracle's; with
    M_bh = 0 the field is the plain disk + bulge one, bit for bit."""
    pos, vel, m = cluster_near_bh(500, 9)
    pos[:, 2] += 0.3
    p = orc.Params(eps=1e-3, ext_on=True, Mbh=20.0, eps_bh=0.05)
    want = orc.torque(pos, m, p)
    with nbs.Context(500, eps=1e-3, precision="fp64", ext_on=True, Mbh=20.0,
                     eps_bh=0.05) as c:
        c.load(pos, vel, m)
        got = c.torque()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    with nbs.Context(500, eps=1e-3, precision="fp64", ext_on=True) as c0, \
            nbs.Context(500, eps=1e-3, precision="fp64", ext_on=True, Mbh=0.0,
                        eps_bh=0.05) as c1:
        c0.load(pos, vel, m)
        c1.load(pos, vel, m)
        assert np.array_equal(c0.accel(), c1.accel())


def test_black_hole_parameters_checked(nbs):
    for kw in ({"Mbh": -1.0}, {"eps_bh": -0.1}, {"Mbh": float("nan")}):
        with pytest.raises(nbs.NBError):
            nbs.Context(16, eps=0.01, ext_on=True, **kw)
