"""nb_accel_static: the force evaluation for callers that cannot allocate
device memory (their own pool allocator owns it all, they cannot afford the
implicit synchronisation of cudaMalloc/cudaFree, or their host forbids device
allocation after start-up).  It keeps its working memory in a fixed static
device array instead.

Checked through the C ABI against nb_accel, the context-based entry point,
within the tolerances of the parity tests, on two calls in a row with
different systems (so nothing left in the shared array from one call can leak
into the next).  Collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1003_3896_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ds": 1e-6, "fp32": 1e-5}
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


@pytest.mark.parametrize("prec", ["fp64", "ds", "fp32"])
def test_static_matches_context_two_calls(env, prec):
    torch, nbsym = env
    stream = torch.cuda.Stream()
    systems = []
    for n, seed, offset in [(3001, 1, True), (MAX_N, 2, False)]:
        pos, vel, m = ics.plummer(n, seed)
        if offset:
            pos, vel = ics.place_on_orbit(pos, vel)
        systems.append((n, pos, vel, m, offset))
    for n, pos, vel, m, offset in systems:
        eps = ics.paper_softening(n)
        with nbsym.Context(n, eps=eps, precision=prec, ext_on=offset) as c:
            c.load(pos, vel, m)
            want = c.accel()
        tp = torch.from_numpy(pos).cuda()
        tm = torch.from_numpy(m).cuda()
        out = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        p = params(nbsym, prec, eps, offset, stream.cuda_stream)
        rc = nbsym.nb_accel_static(C.byref(p), n, tp.data_ptr(), tm.data_ptr(),
                                   out.data_ptr())
        assert rc == nbsym.NB_OK
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_rms(got, want) <= TOL[prec], (prec, n, rel_rms(got, want))


def test_static_rejects_oversize_and_null(env):
    torch, nbsym = env
    p = params(nbsym, "ds", 0.01, False, None)
    t = torch.zeros(3 * (MAX_N + 1), dtype=torch.float64, device="cuda")
    assert nbsym.nb_accel_static(C.byref(p), MAX_N + 1, t.data_ptr(), t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
    assert nbsym.nb_accel_static(C.byref(p), 10, None, t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
    assert nbsym.nb_accel_static(None, 10, t.data_ptr(), t.data_ptr(),
                                 t.data_ptr()) == nbsym.NB_EINVAL
