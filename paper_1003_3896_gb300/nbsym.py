"""ctypes binding of ``libnbsym.so`` (declared in ``include/nbsym.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads the library and raises ImportError if
it has not been built (``paper_1003_3896_gb300.build.build()``); there is no
fallback.  Device-pointer methods accept either an integer address or any
object with ``data_ptr()`` (a torch tensor), so torch is never imported here;
such objects are checked to be contiguous float64 of sufficient size before
their address reaches the library.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbsym.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1003_3896_gb300.build.build()")
_lib = C.CDLL(LIB_PATH)

NB_FP64, NB_DS, NB_FP32, NB_DS_FULL, NB_DD, NB_DS_NEAR = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": NB_FP64, "ds": NB_DS, "fp32": NB_FP32, "ds_full": NB_DS_FULL,
              "dd": NB_DD, "ds_near": NB_DS_NEAR}
NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ESTATE, NB_ETIMEOUT, NB_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "NB_OK", -1: "NB_EINVAL", -2: "NB_ENOMEM", -3: "NB_ECUDA", -4: "NB_ESTATE",
                -5: "NB_ETIMEOUT", -6: "NB_ENONFINITE"}


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("precision", C.c_int),
                ("ext_on", C.c_int), ("Md", C.c_double), ("ad", C.c_double),
                ("bd", C.c_double), ("Mb", C.c_double), ("ab", C.c_double),
                ("device", C.c_int), ("stream", C.c_void_p), ("near_frac", C.c_double),
                ("Mbh", C.c_double), ("eps_bh", C.c_double)]


class EnergyT(C.Structure):
    _fields_ = [("K", C.c_double), ("W", C.c_double), ("W_ext", C.c_double),
                ("E", C.c_double), ("P", C.c_double * 3), ("L", C.c_double * 3)]


class ProfT(C.Structure):
    _fields_ = [("pair_launches", C.c_int64), ("pair_ms", C.c_double),
                ("interactions", C.c_int64), ("kernel_launches", C.c_int64)]


class PeaksT(C.Structure):
    _fields_ = [("sm_count", C.c_int), ("ffma_tflops", C.c_double),
                ("ffma2_tflops", C.c_double), ("dfma_tflops", C.c_double),
                ("rsqrt_gops", C.c_double), ("pairmix_gpairs", C.c_double)]


class TuneT(C.Structure):
    _fields_ = [("precision", C.c_int), ("bodies_per_thread", C.c_int),
                ("blocks_per_sm", C.c_int), ("j_tile", C.c_int), ("candidates", C.c_int),
                ("grid", C.c_int64),
                ("pair_ms", C.c_double), ("default_ms", C.c_double),
                ("cost_ms", C.c_double), ("default_cost_ms", C.c_double)]


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_ctxp = C.c_void_p


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


nb_abi_version = _sig("nb_abi_version", C.c_int)
nb_last_error = _sig("nb_last_error", C.c_char_p)
nb_params_default = _sig("nb_params_default", None, C.POINTER(Params))
nb_create = _sig("nb_create", C.c_int, C.POINTER(Params), C.c_int64, C.POINTER(_ctxp))
nb_load = _sig("nb_load", C.c_int, _ctxp, C.c_int64, _dp, _dp, _dp)
nb_load_device = _sig("nb_load_device", C.c_int, _ctxp, C.c_int64, _vp, _vp, _vp)
nb_accel = _sig("nb_accel", C.c_int, _ctxp, _dp)
nb_accel_device = _sig("nb_accel_device", C.c_int, _ctxp, _vp)
nb_step = _sig("nb_step", C.c_int, _ctxp, C.c_int, C.c_double, C.c_int64)
nb_energy = _sig("nb_energy", C.c_int, _ctxp, C.POINTER(EnergyT))
nb_torque = _sig("nb_torque", C.c_int, _ctxp, _dp)
nb_get_state = _sig("nb_get_state", C.c_int, _ctxp, _dp, _dp)
nb_get_state_device = _sig("nb_get_state_device", C.c_int, _ctxp, _vp, _vp)
nb_size = _sig("nb_size", C.c_int64, _ctxp)
nb_set_precision = _sig("nb_set_precision", C.c_int, _ctxp, C.c_int)
nb_prof_enable = _sig("nb_prof_enable", C.c_int, _ctxp, C.c_int)
nb_prof_read = _sig("nb_prof_read", C.c_int, _ctxp, C.POINTER(ProfT))
nb_destroy = _sig("nb_destroy", None, _ctxp)
nb_measure_peaks = _sig("nb_measure_peaks", C.c_int, C.c_int, C.POINTER(PeaksT))
nb_create_batch = _sig("nb_create_batch", C.c_int, C.POINTER(Params), C.c_int64,
                       C.POINTER(C.c_int64), C.POINTER(_ctxp))
nb_set_cluster_params = _sig("nb_set_cluster_params", C.c_int, _ctxp, _dp, _dp)
nb_clusters = _sig("nb_clusters", C.c_int64, _ctxp)
nb_energy_clusters = _sig("nb_energy_clusters", C.c_int, _ctxp, C.POINTER(EnergyT))
nb_accel_static = _sig("nb_accel_static", C.c_int, C.POINTER(Params), C.c_int64, _vp, _vp, _vp)
nb_tune = _sig("nb_tune", C.c_int, _ctxp, C.c_int, C.POINTER(TuneT))
nb_accel_range = _sig("nb_accel_range", C.c_int, _ctxp, C.c_int64, C.c_int64, _dp)
nb_accel_symmetric = _sig("nb_accel_symmetric", C.c_int, _ctxp, _dp, C.POINTER(C.c_double))
nb_stage_weights = _sig("nb_stage_weights", C.c_int, C.c_int, _dp)
nb_substep_range = _sig("nb_substep_range", C.c_int, _ctxp, C.c_int64, C.c_int64, C.c_double,
                        C.c_double)
nb_set_state = _sig("nb_set_state", C.c_int, _ctxp, _dp, _dp)
nb_set_state_device = _sig("nb_set_state_device", C.c_int, _ctxp, _vp, _vp)
nb_tune_save = _sig("nb_tune_save", C.c_int, C.c_char_p)
nb_tune_load = _sig("nb_tune_load", C.c_int64, C.c_char_p)
nb_tune_entries = _sig("nb_tune_entries", C.c_int64)
nb_pair_shape = _sig("nb_pair_shape", C.c_int, _ctxp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                     C.POINTER(C.c_int), C.POINTER(C.c_int64))
nb_tune_clear = _sig("nb_tune_clear", None)


def tune_save(path: str):
    """Write the process-wide table of tuned pair-kernel shapes."""
    check(nb_tune_save(os.fsencode(path)))


def tune_load(path: str) -> int:
    """Merge a saved table; returns the number of entries read."""
    return int(check(nb_tune_load(os.fsencode(path))))


def tune_entries() -> int:
    return int(nb_tune_entries())


def tune_clear():
    nb_tune_clear()


def stage_weights(order: int) -> list:
    """Kick weights of one step of the given order (nb_stage_weights)."""
    w = np.empty(7)
    k = check(nb_stage_weights(int(order), _p(w)))
    return [float(x) for x in w[:k]]


def measure_peaks(device: int = 0) -> dict:
    """Measured FP32 (scalar / packed), FP64 and MUFU peaks of a device."""
    p = PeaksT()
    check(nb_measure_peaks(int(device), C.byref(p)))
    return {k: getattr(p, k) for k, _ in PeaksT._fields_}


class NBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc < 0:
        raise NBError(rc, nb_last_error().decode(errors="replace"))
    return rc


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _dev(x, count: int, what: str) -> int:
    """Address of device memory for ``count`` float64 values: an integer
    address is taken as given; an object with ``data_ptr()`` (a torch tensor)
    must be contiguous float64 with at least ``count`` elements, so that the
    library never reads or writes past it.  None passes NULL."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "dtype") and "float64" not in str(x.dtype):
        raise ValueError(f"{what}: float64 expected, got {x.dtype}")
    if hasattr(x, "is_contiguous") and not x.is_contiguous():
        raise ValueError(f"{what}: not contiguous")
    if hasattr(x, "numel") and x.numel() < count:
        raise ValueError(f"{what}: {x.numel()} elements, {count} needed")
    return int(x.data_ptr())


def _host3(a, n) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != 3 * n:
        raise ValueError(f"expected {3 * n} values, got {a.size}")
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


@dataclass
class Energy:
    K: float
    W: float
    W_ext: float
    E: float
    P: np.ndarray
    L: np.ndarray


class Context:
    """One particle system (``nb_create``) or an ensemble of independent
    clusters of fixed sizes (``sizes=...``, ``nb_create_batch``) resident on
    one GPU (``nb_ctx``)."""

    def __init__(self, capacity: int = 0, G: float = 1.0, eps: float = 0.0,
                 precision: int | str = NB_DS, ext_on: bool = False,
                 Md: float = 100.0, ad: float = 6.5, bd: float = 0.26, Mb: float = 15.0,
                 ab: float = 0.7, device: int = 0, stream=None, near_frac: float = 0.0,
                 sizes=None, Mbh: float = 0.0, eps_bh: float = 0.0):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        p = Params()
        nb_params_default(C.byref(p))
        p.G, p.eps, p.precision, p.ext_on = G, eps, int(precision), int(bool(ext_on))
        p.Md, p.ad, p.bd, p.Mb, p.ab = Md, ad, bd, Mb, ab
        p.device = device
        p.stream = _addr(stream) if stream is not None else None
        p.near_frac = near_frac
        p.Mbh, p.eps_bh = Mbh, eps_bh
        h = _ctxp()
        if sizes is None:
            check(nb_create(C.byref(p), int(capacity), C.byref(h)))
            self.capacity = int(capacity)
        else:
            sz = np.ascontiguousarray(sizes, dtype=np.int64)
            check(nb_create_batch(C.byref(p), sz.size,
                                  sz.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(h)))
            self.capacity = int(sz.sum())
        self._h = h

    @property
    def clusters(self) -> int:
        return int(check(nb_clusters(self._h)))

    def set_cluster_params(self, eps=None, dt_scale=None):
        k = self.clusters
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64).ravel()
        d = None if dt_scale is None else np.ascontiguousarray(dt_scale, dtype=np.float64).ravel()
        for name, a in (("eps", e), ("dt_scale", d)):
            if a is not None and a.size != k:
                raise ValueError(f"{name}: {a.size} values for {k} clusters")
        check(nb_set_cluster_params(self._h, None if e is None else _p(e),
                                    None if d is None else _p(d)))

    def energy_clusters(self) -> list:
        k = self.clusters
        arr = (EnergyT * k)()
        check(nb_energy_clusters(self._h, arr))
        return [Energy(e.K, e.W, e.W_ext, e.E, np.array(e.P[:]), np.array(e.L[:])) for e in arr]

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            nb_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- state
    def load(self, pos, vel, mass):
        mass = np.ascontiguousarray(mass, dtype=np.float64).ravel()
        n = mass.size
        pos = _host3(pos, n)
        vel = _host3(vel, n)
        check(nb_load(self._h, n, _p(pos), _p(vel), _p(mass)))

    def load_device(self, n: int, pos, vel, mass):
        n = int(n)
        check(nb_load_device(self._h, n, _dev(pos, 3 * n, "pos"), _dev(vel, 3 * n, "vel"),
                             _dev(mass, n, "mass")))

    @property
    def n(self) -> int:
        return int(check(nb_size(self._h)))

    def get_state(self):
        n = self.n
        pos = np.empty((n, 3))
        vel = np.empty((n, 3))
        check(nb_get_state(self._h, _p(pos), _p(vel)))
        return pos, vel

    def get_state_device(self, pos, vel):
        n = self.n
        check(nb_get_state_device(self._h, _dev(pos, 3 * n, "pos"), _dev(vel, 3 * n, "vel")))

    # -- compute
    def accel(self) -> np.ndarray:
        out = np.empty((self.n, 3))
        check(nb_accel(self._h, _p(out)))
        return out

    def accel_device(self, out):
        check(nb_accel_device(self._h, _dev(out, 3 * self.n, "out")))

    def step(self, order: int, dt: float, nsteps: int = 1):
        check(nb_step(self._h, int(order), float(dt), int(nsteps)))

    def energy(self) -> Energy:
        e = EnergyT()
        check(nb_energy(self._h, C.byref(e)))
        return Energy(e.K, e.W, e.W_ext, e.E, np.array(e.P[:]), np.array(e.L[:]))

    def torque(self) -> np.ndarray:
        out = np.empty(3)
        check(nb_torque(self._h, _p(out)))
        return out

    def set_precision(self, precision: int | str):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        check(nb_set_precision(self._h, int(precision)))

    def accel_range(self, i0: int, i1: int) -> np.ndarray:
        """Accelerations of bodies [i0, i1) against all (nb_accel_range)."""
        out = np.empty((max(int(i1) - int(i0), 1), 3))   # the library checks the range
        check(nb_accel_range(self._h, int(i0), int(i1), _p(out)))
        return out

    def substep_range(self, i0: int, i1: int, kick: float, drift: float):
        """Kick (when kick != 0) and drift bodies [i0, i1) (nb_substep_range)."""
        check(nb_substep_range(self._h, int(i0), int(i1), float(kick), float(drift)))

    def set_state(self, pos=None, vel=None):
        """Replace positions and / or velocities, host arrays (nb_set_state)."""
        p = None if pos is None else _host3(pos, self.n)
        v = None if vel is None else _host3(vel, self.n)
        check(nb_set_state(self._h, None if p is None else _p(p), None if v is None else _p(v)))

    def set_state_device(self, pos=None, vel=None):
        """Replace positions and / or velocities from device memory."""
        check(nb_set_state_device(self._h, _dev(pos, 3 * self.n, "pos"),
                                  _dev(vel, 3 * self.n, "vel")))

    def accel_symmetric(self):
        """(accelerations, pair-kernel ms) from the N(N-1)/2 float variant."""
        out = np.empty((self.n, 3))
        ms = C.c_double()
        check(nb_accel_symmetric(self._h, _p(out), C.byref(ms)))
        return out, ms.value

    def tune(self, reps: int = 3) -> dict:
        """Time every compiled pair-kernel shape on the loaded state and keep
        the fastest (``nb_tune``)."""
        t = TuneT()
        check(nb_tune(self._h, int(reps), C.byref(t)))
        return {k: getattr(t, k) for k, _ in TuneT._fields_}

    def pair_shape(self) -> dict:
        """Bodies per thread, blocks per SM and grid of the current plan."""
        i, b, j, g = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        check(nb_pair_shape(self._h, C.byref(i), C.byref(b), C.byref(j), C.byref(g)))
        return {"bodies_per_thread": i.value, "blocks_per_sm": b.value, "j_tile": j.value,
                "grid": g.value}

    def prof_enable(self, on: bool = True):
        check(nb_prof_enable(self._h, int(bool(on))))

    def prof_read(self) -> dict:
        p = ProfT()
        check(nb_prof_read(self._h, C.byref(p)))
        return {"pair_launches": p.pair_launches, "pair_ms": p.pair_ms,
                "interactions": p.interactions, "kernel_launches": p.kernel_launches}


# ---- serving loop --------------------------------------------------------------

class ServerParams(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget_bytes", C.c_double), ("max_jobs", C.c_int),
                ("G", C.c_double), ("ext_on", C.c_int), ("Md", C.c_double), ("ad", C.c_double),
                ("bd", C.c_double), ("Mb", C.c_double), ("ab", C.c_double),
                ("near_frac", C.c_double), ("Mbh", C.c_double), ("eps_bh", C.c_double),
                ("fp64_via_dd", C.c_int)]


class JobDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("order", C.c_int), ("precision", C.c_int),
                ("dt", C.c_double), ("nsteps", C.c_int64), ("eps", C.c_double)]


class JobStatus(C.Structure):
    _fields_ = [("state", C.c_int), ("steps_done", C.c_int64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("cancelled", C.c_int64), ("queued", C.c_int64),
                ("running", C.c_int64), ("interactions", C.c_double),
                ("kernel_launches", C.c_int64), ("capacity_bodies", C.c_int64),
                ("clock_s", C.c_double), ("pair_ms", C.c_double * 3),
                ("pair_interactions", C.c_double * 3), ("pair_busy_ms", C.c_double * 3),
                ("pair_busy_ms_any", C.c_double)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELLED = 0, 1, 2, 3, 4
_srvp = C.c_void_p
nb_server_params_default = _sig("nb_server_params_default", None, C.POINTER(ServerParams))
nb_server_create = _sig("nb_server_create", C.c_int, C.POINTER(ServerParams), C.POINTER(_srvp))
nb_server_submit = _sig("nb_server_submit", C.c_int, _srvp, C.POINTER(JobDesc), _dp, _dp, _dp,
                        C.POINTER(C.c_int64))
nb_server_poll = _sig("nb_server_poll", C.c_int, _srvp, C.c_int64, C.POINTER(JobStatus))
nb_server_wait = _sig("nb_server_wait", C.c_int, _srvp, C.c_int64, C.c_double,
                      C.POINTER(JobStatus))
nb_server_result = _sig("nb_server_result", C.c_int, _srvp, C.c_int64, _dp, _dp)
nb_server_cancel = _sig("nb_server_cancel", C.c_int, _srvp, C.c_int64)
nb_server_forget = _sig("nb_server_forget", C.c_int, _srvp, C.c_int64)
nb_server_stats = _sig("nb_server_stats", C.c_int, _srvp, C.POINTER(ServerStats))
nb_server_destroy = _sig("nb_server_destroy", None, _srvp)


def _status(st: JobStatus) -> dict:
    return {"state": st.state, "steps_done": st.steps_done, "t_submit": st.t_submit,
            "t_admit": st.t_admit, "t_done": st.t_done}


class Server:
    """Continuous-batching request loop (``nb_server``)."""

    def __init__(self, hbm_budget_bytes: float = 4e9, max_jobs: int = 64, device: int = 0,
                 G: float = 1.0, ext_on: bool = False, near_frac: float = 0.0, **field):
        p = ServerParams()
        nb_server_params_default(C.byref(p))
        p.device, p.hbm_budget_bytes, p.max_jobs = device, hbm_budget_bytes, max_jobs
        p.G, p.ext_on, p.near_frac = G, int(bool(ext_on)), near_frac
        for k, v in field.items():
            setattr(p, k, v)
        h = _srvp()
        check(nb_server_create(C.byref(p), C.byref(h)))
        self._h = h
        self._n = {}

    def close(self):
        if getattr(self, "_h", None):
            nb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, pos, vel, mass, order: int, dt: float, nsteps: int,
               precision: int | str = NB_DS, eps: float = 0.0) -> int:
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        mass = np.ascontiguousarray(mass, dtype=np.float64).ravel()
        n = mass.size
        pos = _host3(pos, n)
        vel = _host3(vel, n)
        d = JobDesc(n, int(order), int(precision), float(dt), int(nsteps), float(eps))
        jid = C.c_int64()
        check(nb_server_submit(self._h, C.byref(d), _p(pos), _p(vel), _p(mass), C.byref(jid)))
        self._n[jid.value] = n
        return jid.value

    def poll(self, job_id: int) -> dict:
        st = JobStatus()
        check(nb_server_poll(self._h, int(job_id), C.byref(st)))
        return _status(st)

    def wait(self, job_id: int, timeout_s: float = 600.0) -> dict:
        st = JobStatus()
        check(nb_server_wait(self._h, int(job_id), float(timeout_s), C.byref(st)))
        return _status(st)

    def result(self, job_id: int):
        n = self._n[job_id]
        pos = np.empty((n, 3))
        vel = np.empty((n, 3))
        check(nb_server_result(self._h, int(job_id), _p(pos), _p(vel)))
        return pos, vel

    def cancel(self, job_id: int):
        check(nb_server_cancel(self._h, int(job_id)))

    def forget(self, job_id: int):
        check(nb_server_forget(self._h, int(job_id)))
        self._n.pop(job_id, None)

    def stats(self) -> dict:
        s = ServerStats()
        check(nb_server_stats(self._h, C.byref(s)))
        out = {k: getattr(s, k) for k, _ in ServerStats._fields_}
        for k in ("pair_ms", "pair_interactions", "pair_busy_ms"):
            out[k] = list(out[k])
        return out
