"""CPU oracle for NBSymple's direct-summation method (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs are the only callers.  The product
path (the CUDA library and its binding) never imports this package, and this
package imports nothing from the product package.

``build()`` compiles ``nbody_oracle.c`` (plain C, FP64, -ffp-contract=off,
OpenMP over independent particles) into ``liboracle.so`` next to it; the
wrappers below pass numpy arrays through ctypes.  Every function follows one
passage of the paper, cited in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
          "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", *CFLAGS, "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("ext_on", C.c_int),
                ("Md", C.c_double), ("ad", C.c_double), ("bd", C.c_double),
                ("Mb", C.c_double), ("ab", C.c_double), ("Mbh", C.c_double),
                ("eps_bh", C.c_double)]


@dataclass
class Params:
    """Physical parameters: G, softening eps, and the optional external
    field: Miyamoto-Nagai disk (M_d, a_d, b_d), Plummer bulge (M_b, a_b) and
    a central point mass M_bh softened by eps_bh (the black hole of Sect. 6.2;
    0 = none)."""
    G: float = 1.0
    eps: float = 0.0
    ext_on: bool = False
    Md: float = 100.0
    ad: float = 6.5
    bd: float = 0.26
    Mb: float = 15.0
    ab: float = 0.7
    Mbh: float = 0.0
    eps_bh: float = 0.0

    def _c(self) -> _Params:
        return _Params(self.G, self.eps, int(self.ext_on), self.Md, self.ad,
                       self.bd, self.Mb, self.ab, self.Mbh, self.eps_bh)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(C.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Declare the argument and result types of the oracle's C entry points on
    a loaded copy of the library (the tests also bind copies built from
    deliberately altered sources, to check that the pins reject them)."""
    dp = C.POINTER(C.c_double)
    pp = C.POINTER(_Params)
    i64 = C.c_int64
    lib.orc_accel_int.argtypes = [i64, dp, dp, C.c_double, C.c_double, dp]
    lib.orc_accel_int_at.argtypes = [i64, dp, dp, C.c_double, C.c_double, i64,
                                     C.POINTER(C.c_int64), dp]
    lib.orc_ext_phi.argtypes = [pp, dp]
    lib.orc_ext_phi.restype = C.c_double
    lib.orc_ext_accel_one.argtypes = [pp, dp, dp]
    lib.orc_ext_accel.argtypes = [i64, dp, pp, dp]
    lib.orc_accel.argtypes = [i64, dp, dp, pp, dp]
    lib.orc_energy.argtypes = [i64, dp, dp, dp, pp, dp]
    lib.orc_torque.argtypes = [i64, dp, dp, pp, dp]
    lib.orc_si6a_weights.argtypes = [dp]
    lib.orc_run.argtypes = [i64, dp, dp, dp, pp, C.c_int, C.c_double, i64]
    lib.orc_run.restype = C.c_int
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_max_threads.restype = C.c_int
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    """OpenMP threads the oracle uses (results do not depend on it)."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def accel_int(pos, mass, G: float = 1.0, eps: float = 0.0) -> np.ndarray:
    """Eq. 2 / eq. 5 divided by m_i: internal accelerations, (n, 3)."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3))
    out = np.empty((n, 3))
    _load().orc_accel_int(n, _ptr(pos), _ptr(mass), float(G), float(eps), _ptr(out))
    return out


def accel_int_at(pos, mass, idx, G: float = 1.0, eps: float = 0.0) -> np.ndarray:
    """Eq. 5 accelerations of the bodies listed in ``idx`` only, (len(idx), 3)."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise IndexError("idx out of range")
    out = np.empty((idx.size, 3))
    _load().orc_accel_int_at(n, _ptr(pos), _ptr(mass), float(G), float(eps), idx.size,
                             idx.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(out))
    return out


def ext_phi(p: Params, x) -> float:
    """Potential Phi(x) per unit mass of the external field of eq. 3 (disk +
    bulge + optional central point mass); a_ext = -grad Phi."""
    x = _f64(x, (3,))
    pc = p._c()
    return float(_load().orc_ext_phi(C.byref(pc), _ptr(x)))


def ext_accel(p: Params, pos) -> np.ndarray:
    """External acceleration -grad Phi (eq. 3's field term) at each row of pos."""
    pos = _f64(pos).reshape(-1, 3)
    out = np.empty_like(pos)
    pc = p._c()
    _load().orc_ext_accel(pos.shape[0], _ptr(pos), C.byref(pc), _ptr(out))
    return out


def accel(pos, mass, p: Params) -> np.ndarray:
    """Eq. 3 right-hand side: internal plus (optional) external acceleration."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3))
    out = np.empty((n, 3))
    pc = p._c()
    _load().orc_accel(n, _ptr(pos), _ptr(mass), C.byref(pc), _ptr(out))
    return out


@dataclass
class Energy:
    K: float
    W: float
    W_ext: float
    E: float
    P: np.ndarray
    L: np.ndarray


def energy(pos, vel, mass, p: Params) -> Energy:
    """Diagnostics of Sect. 5.1: K, the softened pair energy W of eq. 4,
    W_ext = sum m Phi, E = K + W + W_ext (whose relative change is eq. 9),
    momentum P and angular momentum L (eq. 10)."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3))
    vel = _f64(vel, (n, 3))
    out = np.empty(10)
    pc = p._c()
    _load().orc_energy(n, _ptr(pos), _ptr(vel), _ptr(mass), C.byref(pc), _ptr(out))
    return Energy(out[0], out[1], out[2], out[3], out[4:7].copy(), out[7:10].copy())


def torque(pos, mass, p: Params) -> np.ndarray:
    """External torque of eq. 8, sum m_i r_i x a_ext(r_i)."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3))
    out = np.empty(3)
    pc = p._c()
    _load().orc_torque(n, _ptr(pos), _ptr(mass), C.byref(pc), _ptr(out))
    return out


def si6a_weights() -> np.ndarray:
    """Stage weights (w0, w1, w2, w3) of the sixth-order composition of
    Sect. 3.1, applied in the order w3 w2 w1 w0 w1 w2 w3."""
    w = np.empty(4)
    _load().orc_si6a_weights(_ptr(w))
    return w


def run(pos, vel, mass, p: Params, order: int, dt: float, nsteps: int):
    """Return copies of (pos, vel) advanced by ``nsteps`` steps of the order-2
    (drift-kick-drift leapfrog) or order-6 (SI6A) scheme."""
    mass = _f64(mass).ravel()
    n = mass.size
    pos = _f64(pos, (n, 3)).copy()
    vel = _f64(vel, (n, 3)).copy()
    pc = p._c()
    rc = _load().orc_run(n, _ptr(pos), _ptr(vel), _ptr(mass), C.byref(pc),
                         int(order), float(dt), int(nsteps))
    if rc != 0:
        raise ValueError("oracle: bad argument to run()")
    return pos, vel
