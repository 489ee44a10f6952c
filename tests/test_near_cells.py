"""The near-pair pass's candidate set is complete: every pair closer than the
near radius d_th lies within the 2 x 2 x 2 cells its first body probes.

The pass bins bodies into cubic cells of side h = CELL_SCALE d_th by their
float coordinates (q = x * (1 / h) in float, cell = floor(q), clamped to
+-CELL_MAX) and probes, per axis, the body's own cell and the neighbour on the
side of the cell half it sits in.  This restates that float arithmetic on the
CPU (numpy float32 rounds each multiply and divide to nearest, as the kernel's
default float operations do), with the constants read from csrc/near.cu, and
checks it over pairs at every scale from 1e-6 to 1e3, pairs straddling cell
boundaries and lying along an axis, and bodies far enough out to be clamped.
A cell side under 2 d_th must miss pairs, which shows the check has power."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _constants():
    src = open(os.path.join(ROOT, "paper_1003_3896_gb300", "csrc", "near.cu")).read()
    scale = float(re.search(r"constexpr float CELL_SCALE = ([0-9.]+)f;", src).group(1))
    bits = int(re.search(r"constexpr int CELL_BITS = (\d+);", src).group(1))
    cmax = (1 << (bits - 1)) - 2
    assert re.search(r"constexpr int CELL_MAX = CELL_OFF - 2;", src)
    return scale, cmax


def _cells(v, ih, cmax):
    """Cell index and neighbour side per coordinate, in float32 as the kernel."""
    q = (v.astype(np.float32) * np.float32(ih)).astype(np.float32)
    f = np.floor(q)
    side = np.where((q - f) < np.float32(0.5), -1, 1)
    c = np.clip(f, -np.float32(cmax), np.float32(cmax)).astype(np.int64)
    return c, side


def _missed(pi, pj, dth, scale, cmax):
    """Pairs (pi[k], pj[k]) whose second body is outside the first one's
    probed cells."""
    ih = np.float32(1.0) / (np.float32(scale) * np.float32(dth))
    ci, si = _cells(pi, ih, cmax)
    cj, _ = _cells(pj, ih, cmax)
    ok = (cj == ci) | (cj == ci + si)
    return ~ok.all(axis=1)


def _pairs(rng, n, dth, spread):
    """Float32 pairs closer than d_th: random centres over +-spread, random
    directions, distances up to just under d_th."""
    pi = rng.uniform(-spread, spread, (n, 3)).astype(np.float32)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    d = dth * rng.uniform(0.0, 1.0, n) ** (1 / 3)
    pj = (pi.astype(np.float64) + u * d[:, None]).astype(np.float32)
    close = ((pj.astype(np.float64) - pi.astype(np.float64)) ** 2).sum(1) < dth * dth
    return pi[close], pj[close]


def test_probe_set_holds_every_close_pair():
    scale, cmax = _constants()
    assert scale > 2.0
    rng = np.random.default_rng(0)
    for dth in (1e-6, 3.7e-4, 0.02, 1.0, 123.0):
        h = scale * dth
        for spread in (3 * h, 1000 * h, 0.9 * cmax * h, 3 * cmax * h):
            pi, pj = _pairs(rng, 40000, dth, spread)
            assert not _missed(pi, pj, dth, scale, cmax).any(), (dth, spread)


def test_pairs_across_cell_boundaries_and_along_axes():
    scale, cmax = _constants()
    rng = np.random.default_rng(1)
    dth = np.float32(0.0123)
    h = np.float64(scale) * np.float64(dth)
    cells = rng.integers(-cmax + 2, cmax - 2, (20000, 3))
    # first body within a few ulps of a cell boundary, the partner up to d_th
    # away along one axis, either way
    frac = rng.choice([1e-7, 0.25, 0.4999, 0.5, 0.5001, 0.75, 1 - 1e-7], (20000, 3))
    pi = ((cells + frac) * h).astype(np.float32)
    for axis in range(3):
        for sign in (-1.0, 1.0):
            pj = pi.astype(np.float64).copy()
            pj[:, axis] += sign * 0.999999 * float(dth)
            pj = pj.astype(np.float32)
            close = ((pj.astype(np.float64) - pi.astype(np.float64)) ** 2).sum(1) < float(dth) ** 2
            assert not _missed(pi[close], pj[close], dth, scale, cmax).any(), (axis, sign)


def test_a_cell_narrower_than_two_radii_misses_pairs():
    _, cmax = _constants()
    rng = np.random.default_rng(2)
    dth = 0.5
    pi, pj = _pairs(rng, 40000, dth, 200.0)
    assert _missed(pi, pj, dth, 1.6, cmax).any()
