"""The i-split on the GPU (one cluster shared by several ranks, each owning a
range of bodies, positions exchanged between substeps; Sect. 4.2): ranks
emulated in one process on one GPU, one context each, run one after another
with the exchange a concatenation (no rank waits on another's kernels).
Split runs equal the one-rank run bit for bit, and match the oracle and
nb_step within the parity tolerances."""
import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "dd": 1e-10, "ds": 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import isplit, nbsym
    return torch, nbsym, isplit


def split_run(env, pos, vel, m, eps, prec, world, order, dt, nsteps, align=1024):
    torch, nbsym, isplit = env
    n = len(m)
    rg, chunk = isplit.ranges(n, world, align)
    ctxs, ranks = [], []
    for i0, i1 in rg:
        c = nbsym.Context(n, eps=eps, precision=prec, ext_on=True)
        c.load(pos, vel, m)
        ctxs.append(c)
        ranks.append(isplit.Rank(isplit.ContextBackend(c, "cuda"), i0, i1, chunk))
    ex = isplit.LocalExchange()
    isplit.run(ranks, ex, nbsym.stage_weights(order), dt, nsteps)
    isplit.gather(ranks, ex)
    out = [c.get_state() for c in ctxs]
    for c in ctxs:
        c.close()
    return out


@pytest.mark.parametrize("prec,n", [("fp64", 3000), ("dd", 5000), ("ds", 16384)])
def test_split_ranks_equal_one_rank_and_oracle(env, orc, prec, n):
    """4 SI6A steps of dt = 1/256 on the orbit in the disk + bulge field: 2 and
    3 ranks (uneven last range) give the one-rank state bit for bit; the
    state matches the oracle's run (and nb_step's) within the tolerance."""
    pos, vel, m = ics.plummer(n, 3)
    pos, vel = ics.place_on_orbit(pos, vel)
    eps = ics.paper_softening(n)
    one = split_run(env, pos, vel, m, eps, prec, 1, 6, 1 / 256, 4)
    for world in (2, 3):
        many = split_run(env, pos, vel, m, eps, prec, world, 6, 1 / 256, 4, align=512)
        for x, v in many:
            np.testing.assert_array_equal(x, one[0][0])
            np.testing.assert_array_equal(v, one[0][1])
    rx, rv = orc.run(pos, vel, m, orc.Params(eps=eps, ext_on=True), 6, 1 / 256, 4)
    assert np.abs(one[0][0] - rx).max() <= TOL[prec], np.abs(one[0][0] - rx).max()
    _, nbsym, _ = env
    with nbsym.Context(n, eps=eps, precision=prec, ext_on=True) as c:
        c.load(pos, vel, m)
        c.step(6, 1 / 256, 4)
        xs, _ = c.get_state()
    assert np.abs(one[0][0] - xs).max() <= TOL[prec]


def test_substep_range_touches_only_its_range(env):
    """A kick-drift of bodies [i0, i1) changes those bodies only; set_state
    replaces positions and velocities without reloading."""
    torch, nbsym, _ = env
    n = 4000
    pos, vel, m = ics.plummer(n, 8)
    with nbsym.Context(n, eps=1e-3, precision="ds") as c:
        c.load(pos, vel, m)
        c.substep_range(1000, 2100, 1e-3, 1e-3)
        x, v = c.get_state()
        out = np.r_[0:1000, 2100:n]
        np.testing.assert_array_equal(x[out], pos[out])
        np.testing.assert_array_equal(v[out], vel[out])
        assert np.all(x[1000:2100] != pos[1000:2100])
        c.set_state(pos, None)
        x2, v2 = c.get_state()
        np.testing.assert_array_equal(x2, pos)
        np.testing.assert_array_equal(v2, v)
        c.set_state(None, vel)
        np.testing.assert_array_equal(c.get_state()[1], vel)
        for bad in [(-1, 10), (10, 10), (0, n + 1)]:
            with pytest.raises(nbsym.NBError) as e:
                c.substep_range(*bad, 0.1, 0.1)
            assert e.value.code == nbsym.NB_EINVAL
