"""Host logic of the i-split (one cluster shared by several ranks, each owning
a range of bodies, positions exchanged between substeps; the paper's
multi-GPU scheme, Sect. 4.2), on CPU: the per-rank force evaluation is the
oracle's sum over the rank's targets, the exchange runs over gloo with world
size 2 and 3.  The gathered state must equal the unsplit run's bit for bit,
and the oracle's own integrator to rounding."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleBackend:
    """A rank's share computed by the oracle: accelerations of its targets
    against all bodies, then v += kick a, x += drift v (the kick-drift
    kernel's operations) on its range."""

    def __init__(self, orc, pos, vel, m, p):
        import torch
        self.torch, self.orc, self.p = torch, orc, p
        self.x, self.v, self.m = pos.copy(), vel.copy(), m
        self.n = len(m)

    def substep_range(self, i0, i1, kick, drift):
        if kick != 0.0:
            idx = np.arange(i0, i1)
            a = self.orc.accel_int_at(self.x, self.m, idx, self.p.G, self.p.eps)
            if self.p.ext_on:
                a = a + self.orc.ext_accel(self.p, self.x[i0:i1])
            self.v[i0:i1] = self.v[i0:i1] + kick * a
        self.x[i0:i1] = self.x[i0:i1] + drift * self.v[i0:i1]

    def positions(self):
        return self.torch.from_numpy(self.x.copy())

    def velocities(self):
        return self.torch.from_numpy(self.v.copy())

    def set_positions(self, t):
        self.x = t.numpy().copy()

    def set_velocities(self, t):
        self.v = t.numpy().copy()


def system(n=2500):
    from paper_1003_3896_gb300 import ics
    pos, vel, m = ics.plummer(n, 5)
    pos, vel = ics.place_on_orbit(pos, vel)
    return pos, vel, m, ics.paper_softening(n)


def local_run(orc, world, order=6, dt=1 / 256, nsteps=3, align=1024):
    """All ranks in this process (LocalExchange)."""
    from paper_1003_3896_gb300 import isplit, nbsym
    pos, vel, m, eps = system()
    p = orc.Params(eps=eps, ext_on=True)
    rg, chunk = isplit.ranges(len(m), world, align)
    ranks = [isplit.Rank(OracleBackend(orc, pos, vel, m, p), i0, i1, chunk) for i0, i1 in rg]
    ex = isplit.LocalExchange()
    isplit.run(ranks, ex, nbsym.stage_weights(order), dt, nsteps)
    isplit.gather(ranks, ex)
    return [(r.b.x, r.b.v) for r in ranks]


def test_ranges_tile_the_bodies():
    from paper_1003_3896_gb300 import isplit
    for n in (1, 5, 1023, 1024, 1025, 2500, 65536, 1536000):
        for world in (1, 2, 3, 4, 8):
            rg, chunk = isplit.ranges(n, world)
            assert chunk % isplit.ALIGN == 0 and chunk * world >= n
            assert rg[0][0] == 0 and rg[-1][1] == n
            for (a0, a1), (b0, b1) in zip(rg, rg[1:]):
                assert a1 == b0 and a0 <= a1
            assert all(i1 - i0 <= chunk for i0, i1 in rg)
            # whole chunks for every rank but those at the end
            assert all(i0 % chunk == 0 for i0, _ in rg if i0 < n)


def test_schedule_is_the_merged_composition():
    """The substeps of one step: drift w0/2, then kick w_k and drift
    (w_k + w_k+1)/2; total drift = total kick = dt (weights sum to one)."""
    from paper_1003_3896_gb300 import isplit, nbsym
    for order in (2, 6):
        w = nbsym.stage_weights(order)
        subs = isplit.schedule(w, 0.5)
        assert len(subs) == len(w) + 1 and subs[0][0] == 0.0
        assert abs(sum(k for k, _ in subs) - 0.5) < 1e-15
        assert abs(sum(d for _, d in subs) - 0.5) < 1e-15
        assert [k for k, _ in subs[1:]] == [wk * 0.5 for wk in w]


def test_local_split_equals_unsplit_and_oracle(orc):
    one = local_run(orc, 1)
    for world in (2, 3):
        many = local_run(orc, world, align=512)
        for x, v in many:            # every rank ends with the whole state
            np.testing.assert_array_equal(x, one[0][0])
            np.testing.assert_array_equal(v, one[0][1])
    pos, vel, m, eps = system()
    rx, rv = orc.run(pos, vel, m, orc.Params(eps=eps, ext_on=True), 6, 1 / 256, 3)
    # the oracle composes whole leapfrogs (14 half drifts per step), the split
    # run merges adjacent half drifts: the same scheme up to rounding
    assert np.abs(one[0][0] - rx).max() <= 1e-12
    assert np.abs(one[0][1] - rv).max() <= 1e-11


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import oracle as orc
    from paper_1003_3896_gb300 import isplit, nbsym
    from test_isplit import OracleBackend, system
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    pos, vel, m, eps = system()
    p = orc.Params(eps=eps, ext_on=True)
    rg, chunk = isplit.ranges(len(m), world, 512)
    i0, i1 = rg[rank]
    me = isplit.Rank(OracleBackend(orc, pos, vel, m, p), i0, i1, chunk)
    ex = isplit.DistExchange()
    isplit.run([me], ex, nbsym.stage_weights(6), 1 / 256, 3)
    isplit.gather([me], ex)
    np.save(os.path.join(out_dir, f"x{rank}.npy"), me.b.x)
    np.save(os.path.join(out_dir, f"v{rank}.npy"), me.b.v)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_unsplit(orc, tmp_path, world):
    """world processes over gloo, each owning its range: after 3 SI6A steps
    every rank's gathered state equals the unsplit run bit for bit."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    one = local_run(orc, 1)
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"x{r}.npy"), one[0][0])
        np.testing.assert_array_equal(np.load(tmp_path / f"v{r}.npy"), one[0][1])
