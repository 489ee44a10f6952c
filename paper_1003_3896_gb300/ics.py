"""Seeded synthetic initial conditions.

This module is the only code shared by the CUDA path's tests and the CPU
oracle's tests.  It draws positions, velocities and masses and holds none of
the method's arithmetic: no force, potential, energy or integrator.  Every
scaling it applies is an analytic expectation of the sampled distribution,
never a quantity measured on the sample.

Units are G = 1 throughout.  Arrays are float64, positions and velocities as
(n, 3) row-major (x, y, z interleaved per particle), masses as (n,).

Workloads (all seeded, synthetic):

* ``plummer``: Plummer sphere sampled after Aarseth, Henon & Wielen (1974),
  radii by inverse CDF of the cumulative mass r^3/(r^2+a^2)^{3/2}, truncated
  at 20 a, speeds by von Neumann rejection on q^2 (1-q^2)^{7/2}.
* ``henon_plummer``: the same in Henon units (G = M = 1, E = -1/4), which for
  the analytic Plummer model means a = 3 pi / 16.
* ``salpeter_masses``: power-law mass function dN/dm ~ m^{-2.35} on
  [0.1, 100], normalised to total mass M.
* ``uniform_sphere``: the paper's own test workload (Sect. 3 and Sect. 5.1):
  positions uniform in a sphere of radius R, velocities isotropic with a
  uniformly distributed modulus, scaled so the expected virial ratio is Q
  (Q = 0.3 in the paper).
* ``kepler_pair``: a two-body orbit started at pericentre.
* ``ensemble_sizes`` / ``serving_trace``: the batched-ensemble and serving
  workloads' job parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "paper_softening",
    "plummer",
    "henon_plummer",
    "salpeter_masses",
    "uniform_sphere",
    "kepler_pair",
    "place_on_orbit",
    "VC_R50",
    "VC_R10",
    "plunge_cluster",
    "DISK_BULGE",
    "ensemble_sizes",
    "serving_trace",
    "Job",
]

#: Miyamoto-Nagai disk + Plummer bulge used for the cluster-on-orbit workload
#: (M_d, a_d, b_d, M_b, a_b), G = 1.
DISK_BULGE = (100.0, 6.5, 0.26, 15.0, 0.7)

#: Circular speed of the DISK_BULGE model at R = 50 in its midplane,
#: v_c = sqrt(R |dPhi/dR|).  Derived by hand from the model's closed form:
#: v_c^2 = 100*2500/(2500+6.76^2)^{3/2} + 15*2500/(2500+0.49)^{3/2}.
#: tests/test_oracle_pins.py checks it against the oracle's field.
VC_R50 = 1.4987666537924513

#: The same at R = 10 (the start of the quasi-radial black-hole collision runs
#: of Sect. 6.2): v_c^2 = 100*100/(100+6.76^2)^{3/2} + 15*100/(100+0.49)^{3/2}.
VC_R10 = 2.678662467336762


def paper_softening(n: int, radius: float = 1.0) -> float:
    """Softening rule of Sect. 2: eps = 0.005 R / N^{1/3}."""
    return 0.005 * radius / float(n) ** (1.0 / 3.0)


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    """Isotropic unit vectors (uniform cos(theta), uniform phi)."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _com_frame(pos: np.ndarray, vel: np.ndarray, mass: np.ndarray):
    w = mass / mass.sum()
    pos -= (w[:, None] * pos).sum(axis=0)
    vel -= (w[:, None] * vel).sum(axis=0)
    return pos, vel


def salpeter_masses(n: int, seed: int, m_lo: float = 0.1, m_hi: float = 100.0,
                    slope: float = 2.35, total: float = 1.0) -> np.ndarray:
    """Masses drawn by inverse CDF of dN/dm ~ m^{-slope} on [m_lo, m_hi],
    independent of position, then rescaled so that their sum is ``total``."""
    rng = np.random.default_rng([seed, 0x5A1])
    p = 1.0 - slope
    u = rng.random(n)
    lo, hi = m_lo ** p, m_hi ** p
    m = (lo + u * (hi - lo)) ** (1.0 / p)
    return m * (total / m.sum())


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
            rmax: float = 20.0, masses: np.ndarray | None = None,
            com_frame: bool = True):
    """Plummer sphere of scale ``a`` and mass ``total_mass`` (G = 1).

    Returns (pos (n,3), vel (n,3), mass (n,)), float64.  Equal masses unless
    ``masses`` is given (their sum should be ``total_mass``).  The draw order
    is fixed: radii, position directions, speeds, velocity directions.
    """
    if n <= 0:
        z = np.zeros((0, 3))
        return z, z.copy(), np.zeros(0)
    rng = np.random.default_rng(seed)
    # Radii: inverse of the cumulative mass fraction X = r^3/(r^2+a^2)^{3/2}.
    radii = []
    have = 0
    while have < n:
        x = rng.random(max(16, 2 * (n - have)))
        x = x[x > 0.0]
        r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        r = r[r <= rmax * a]
        radii.append(r)
        have += r.size
    r = np.concatenate(radii)[:n]
    pos = r[:, None] * _unit_vectors(rng, n)
    # Speeds: q = v / v_esc with density q^2 (1-q^2)^{7/2} (max ~0.092 < 0.1).
    qs = []
    have = 0
    while have < n:
        m = max(16, 12 * (n - have))
        q = rng.random(m)
        y = 0.1 * rng.random(m)
        q = q[y < q * q * (1.0 - q * q) ** 3.5]
        qs.append(q)
        have += q.size
    q = np.concatenate(qs)[:n]
    vesc = math.sqrt(2.0 * total_mass / a) * (1.0 + (r / a) ** 2) ** -0.25
    vel = (q * vesc)[:, None] * _unit_vectors(rng, n)
    if masses is None:
        mass = np.full(n, total_mass / n)
    else:
        mass = np.asarray(masses, dtype=np.float64).copy()
        if mass.shape != (n,):
            raise ValueError(f"masses has shape {mass.shape}, expected ({n},)")
    if com_frame:
        pos, vel = _com_frame(pos, vel, mass)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def henon_plummer(n: int, seed: int, masses: np.ndarray | None = None):
    """Plummer sphere in Henon (virial) units: G = M = 1 and E = -1/4, i.e.
    scale a = 3 pi / 16 for the analytic model."""
    return plummer(n, seed, a=3.0 * math.pi / 16.0, total_mass=1.0, masses=masses)


def uniform_sphere(n: int, seed: int, q_vir: float = 0.3, radius: float = 1.0,
                   total_mass: float = 1.0):
    """The paper's test workload (Sect. 3, Sect. 5.1): equal masses m = M/N,
    positions uniform inside a sphere of radius R, velocities uniform in
    direction with modulus uniform on [0, v_max].

    v_max is set from the expected virial ratio Q = 2K/|W| using the
    continuum potential energy of a uniform sphere, W = -(3/5) G M^2 / R, and
    E[v^2] = v_max^2 / 3:  K = M v_max^2 / 6 = Q |W| / 2.
    """
    rng = np.random.default_rng(seed)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    pos = r[:, None] * _unit_vectors(rng, n)
    w_abs = 0.6 * total_mass * total_mass / radius
    vmax = math.sqrt(3.0 * q_vir * w_abs / total_mass)
    speed = vmax * rng.random(n)
    vel = speed[:, None] * _unit_vectors(rng, n)
    mass = np.full(n, total_mass / n)
    pos, vel = _com_frame(pos, vel, mass)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def kepler_pair(m1: float, m2: float, sma: float, ecc: float):
    """Two bodies (G = 1) on a Kepler orbit of semi-major axis ``sma`` and
    eccentricity ``ecc``, started at pericentre on the x axis, moving in +y,
    centre of mass at rest at the origin (textbook two-body elements)."""
    mu = m1 + m2
    rp = sma * (1.0 - ecc)
    vp = math.sqrt(mu * (1.0 + ecc) / rp)
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    pos = np.stack([-(m2 / mu) * rel_x, (m1 / mu) * rel_x])
    vel = np.stack([-(m2 / mu) * rel_v, (m1 / mu) * rel_v])
    return pos, vel, np.array([m1, m2], dtype=np.float64)


def place_on_orbit(pos: np.ndarray, vel: np.ndarray, radius: float = 50.0,
                   vc: float = VC_R50):
    """Move a cluster (in its centre-of-mass frame) to (radius, 0, 0) with
    bulk velocity (0, vc, 0): counter-clockwise in the x-y plane."""
    p = pos.copy()
    v = vel.copy()
    p[:, 0] += radius
    v[:, 1] += vc
    return p, v


def plunge_cluster(n: int, seed: int, r0: float = 10.0, vc: float = VC_R10,
                   vfrac: float = 1e-3):
    """Initial conditions of the quasi-radial collision runs of Sect. 6.2:
    a Plummer cluster (M = 1, a = 1) with its barycentre at (r0, 0, 0) and
    velocity (0, vfrac * v_c, 0), v_c the local circular speed, so it falls
    almost radially through the galactic centre."""
    pos, vel, m = plummer(n, seed)
    pos = pos + np.array([r0, 0.0, 0.0])
    vel = vel + np.array([0.0, vfrac * vc, 0.0])
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), m


def ensemble_sizes(n_clusters: int = 512, n_lo: int = 256, n_hi: int = 8192,
                   seed: int = 0) -> np.ndarray:
    """Cluster sizes log-uniform on [n_lo, n_hi] from a master seed."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(n_lo), math.log(n_hi), n_clusters)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), n_lo, n_hi)


@dataclass(frozen=True)
class Job:
    """One integration request of the serving workload."""
    index: int
    arrival_s: float
    n: int
    order: int          # 2 or 6
    precision: int      # 0 = FP64, 1 = double-single
    nsteps: int
    seed: int


def serving_trace(n_jobs: int = 2000, rate_hz: float = 200.0, seed: int = 0,
                  n_lo: int = 1024, n_hi: int = 131072, steps_lo: int = 10,
                  steps_hi: int = 1000) -> list[Job]:
    """Poisson arrivals at ``rate_hz``; N log-uniform on [n_lo, n_hi]; order
    uniform on {2, 6}; precision uniform on {FP64, double-single}; step count
    log-uniform integer on [steps_lo, steps_hi].  Job k's ICs use seed k."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_jobs)
    t = np.cumsum(gaps)
    n = np.clip(np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_jobs))),
                n_lo, n_hi).astype(np.int64)
    order = np.where(rng.random(n_jobs) < 0.5, 2, 6)
    prec = np.where(rng.random(n_jobs) < 0.5, 0, 1)
    steps = np.clip(np.rint(np.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi), n_jobs))),
                    steps_lo, steps_hi).astype(np.int64)
    return [Job(int(k), float(t[k]), int(n[k]), int(order[k]), int(prec[k]),
                int(steps[k]), int(k)) for k in range(n_jobs)]
