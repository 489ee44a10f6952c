"""The N(N-1)/2 variant (each unordered pair once, Newton's third law): float
class, so it is held to the pure-float bar against the oracle (1e-4 on small
clusters with the paper's softening, as NB_FP32) and checked against the full
N x N float sum."""
import math

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


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())


@pytest.mark.parametrize("n,ext_on", [(2, False), (63, False), (129, True), (3000, False),
                                      (20001, True)])
def test_symmetric_matches_oracle_and_full_sum(nbs, orc, n, ext_on):
    pos, vel, m = ics.plummer(n, 90 + n)
    if ext_on:
        pos, vel = ics.place_on_orbit(pos, vel)
    eps = ics.paper_softening(n)
    ref = orc.accel(pos, m, orc.Params(eps=eps, ext_on=ext_on))
    with nbs.Context(n, eps=eps, precision="fp32", ext_on=ext_on) as c:
        c.load(pos, vel, m)
        full = c.accel()
        sym, ms = c.accel_symmetric()
        # the context's own float state is untouched by the call
        assert np.array_equal(c.accel(), full)
    ref_int = orc.accel_int(pos, m, 1.0, eps)
    field = ref - ref_int
    assert ms > 0
    assert rel_rms(sym - field, ref_int) <= 1e-4, rel_rms(sym - field, ref_int)
    assert rel_rms(sym - field, full - field) <= 1e-4


def test_symmetric_unsoftened_pair_and_errors(nbs, orc):
    pos, vel, m = ics.kepler_pair(0.6, 0.4, 1.0, 0.5)
    with nbs.Context(2, eps=0.0, precision="ds") as c:
        with pytest.raises(nbs.NBError):
            c.accel_symmetric()          # nothing loaded
        c.load(pos, vel, m)
        a, _ = c.accel_symmetric()
    ref = orc.accel_int(pos, m, 1.0, 0.0)
    assert rel_rms(a, ref) <= 1e-6
    with nbs.Context(sizes=[10, 20], precision="fp32") as b:
        p, v, mm = ics.plummer(30, 3)
        b.load(p, v, mm)
        with pytest.raises(nbs.NBError):
            b.accel_symmetric()          # one cluster only
