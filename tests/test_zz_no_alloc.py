"""nb_accel_static: the force evaluation for callers that cannot allocate
device memory (their own pool allocator owns it all, they cannot afford the
implicit synchronisation of cudaMalloc/cudaFree, or their host forbids device
allocation after start-up).  It keeps its working memory in a fixed static
device array instead.

Checked through the C ABI against nb_accel, the context-based entry point,
and against the CPU oracle, within the tolerances of the parity tests, on two
calls in a row with different systems (so nothing left in the shared array
from one call can leak into the next), in every arithmetic mode; and checked
to leave the device's free memory unchanged over repeated calls.  Collected
last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "dd": 1e-12, "ds": 1e-6, "ds_full": 1e-6, "ds_near": 1e-6, "fp32": 1e-4}
MAX_N = 16384


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1003_3896_gb300 import build
    build.build()
    from paper_1003_3896_gb300 import nbsym
    return torch, nbsym


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())


def params(nbsym, prec, eps, ext_on, stream):
    p = nbsym.Params()
    nbsym.nb_params_default(C.byref(p))
    p.precision = nbsym.PRECISIONS[prec]
    p.eps = eps
    p.ext_on = int(ext_on)
    p.device = 0
    p.stream = stream
    return p


def static_accel(torch, nbsym, prec, pos, m, eps, ext_on, stream):
    n = len(m)
    tp = torch.from_numpy(pos).cuda()
    tm = torch.from_numpy(m).cuda()
    out = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    p = params(nbsym, prec, eps, ext_on, stream.cuda_stream)
    rc = nbsym.nb_accel_static(C.byref(p), n, tp.data_ptr(), tm.data_ptr(), out.data_ptr())
    assert rc == nbsym.NB_OK, nbsym.nb_last_error()
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "dd", "ds", "ds_full", "ds_near", "fp32"])
def test_static_matches_context_and_oracle_two_calls(env, orc, prec):
    torch, nbsym = env
    stream = torch.cuda.Stream()
    for n, seed, offset in [(3001, 1, True), (MAX_N, 2, False)]:
        pos, vel, m = ics.plummer(n, seed)
        if offset:
            pos, vel = ics.place_on_orbit(pos, vel)
        eps = ics.paper_softening(n)
        with nbsym.Context(n, eps=eps, precision=prec, ext_on=offset) as c:
            c.load(pos, vel, m)
            want = c.accel()
        got = static_accel(torch, nbsym, prec, pos, m, eps, offset, stream)
        assert np.isfinite(got).all()
        assert rel_rms(got, want) <= TOL[prec], (prec, n, rel_rms(got, want))
        # the oracle on a sample of bodies (the pair sum; the field is exact
        # FP64 on both sides)
        idx = np.unique(np.concatenate([np.arange(0, n, max(1, n // 300)), [n - 1]]))
        ref = orc.accel_int_at(pos, m, idx, 1.0, eps)
        if offset:
            ref = ref + orc.ext_accel(orc.Params(eps=eps, ext_on=True), pos[idx])
        assert rel_rms(got[idx], ref) <= TOL[prec], (prec, n, rel_rms(got[idx], ref))


def test_static_allocates_nothing(env):
    """After a first call (which loads the module and looks the array up),
    further calls in every mode leave the device's free memory unchanged."""
    torch, nbsym = env
    stream = torch.cuda.Stream()
    n = 5000
    pos, vel, m = ics.plummer(n, 3)
    eps = ics.paper_softening(n)
    tp = torch.from_numpy(pos).cuda()
    tm = torch.from_numpy(m).cuda()
    out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ps = [params(nbsym, k, eps, True, stream.cuda_stream) for k in TOL]
    for p in ps:   # warm-up: every mode's kernels loaded
        assert nbsym.nb_accel_static(C.byref(p), n, tp.data_ptr(), tm.data_ptr(),
                                     out.data_ptr()) == nbsym.NB_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for p in ps:
            assert nbsym.nb_accel_static(C.byref(p), n, tp.data_ptr(), tm.data_ptr(),
                                         out.data_ptr()) == nbsym.NB_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rejects_oversize_and_null(env):
    torch, nbsym = env
    p = params(nbsym, "ds", 0.01, False, None)
    t = torch.zeros(3 * (MAX_N + 1), dtype=torch.float64, device="cuda")
    assert nbsym.nb_accel_static(C.byref(p), MAX_N + 1, t.data_ptr(), t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
    assert b"16384" in nbsym.nb_last_error()
    assert nbsym.nb_accel_static(C.byref(p), 10, None, t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
    assert nbsym.nb_accel_static(None, 10, t.data_ptr(), t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
