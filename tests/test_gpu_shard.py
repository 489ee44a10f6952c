"""One-GPU virtual shards of the paper's multi-GPU scheme (each GPU sums an
i-range against all bodies, Sect. 4.2): nb_accel_range over split ranges must
concatenate bit for bit to the whole-range result, in every precision, and
meet the oracle bar."""
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ds": 1e-6, "dd": 1e-12, "fp32": 1e-4}


@pytest.fixture(scope="module")
def nbs():
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import nbsym
    return nbsym


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())


@pytest.mark.parametrize("prec,n", [("fp64", 3001), ("ds", 3001), ("dd", 3001), ("fp32", 3001),
                                    ("ds", 12289)])
def test_split_ranges_concatenate_bit_for_bit(nbs, orc, prec, n):
    pos, vel, m = ics.plummer(n, 120 + n)
    pos, vel = ics.place_on_orbit(pos, vel)
    eps = ics.paper_softening(n)
    ref = orc.accel(pos, m, orc.Params(eps=eps, ext_on=True))
    with nbs.Context(n, eps=eps, precision=prec, ext_on=True) as c:
        c.load(pos, vel, m)
        whole = c.accel_range(0, n)
        for h in (1, 777, n // 2, n - 1):
            parts = np.concatenate([c.accel_range(0, h), c.accel_range(h, n)])
            assert np.array_equal(parts, whole), (prec, h)
        cuts = [0, n // 5, n // 3, (2 * n) // 3, n]
        four = np.concatenate([c.accel_range(a, b) for a, b in zip(cuts[:-1], cuts[1:])])
        assert np.array_equal(four, whole)
        full = c.accel()
    ref_int = orc.accel_int(pos, m, 1.0, eps)
    field = ref - ref_int
    assert rel_rms(whole - field, ref_int) <= TOL[prec]
    assert rel_rms(whole - field, full - field) <= TOL[prec]


def test_range_errors(nbs):
    pos, vel, m = ics.plummer(100, 3)
    with nbs.Context(100, eps=0.01, precision="fp64") as c:
        with pytest.raises(nbs.NBError):
            c.accel_range(0, 10)            # nothing loaded
        c.load(pos, vel, m)
        for a, b in ((-1, 5), (5, 5), (10, 101), (50, 20)):
            with pytest.raises(nbs.NBError):
                c.accel_range(a, b)
    with nbs.Context(sizes=[40, 60], precision="fp64") as b:
        b.load(pos, vel, m)
        with pytest.raises(nbs.NBError):
            b.accel_range(0, 10)
