"""The oracle's pins against planted mistakes (mutation testing, CPU only).

Each mutant below is one plausible slip planted in a copy of the oracle's C
source: a flipped sign, a transposed index, a dropped term or factor, a wrong
exponent, a mistyped weight, a misordered composition. Every copy is compiled
with the oracle's own flags, bound in place of the real library, and run
through every pin of ``test_oracle_pins`` except the two fixture tests (which
compare the oracle with its own earlier output and so would catch any change
trivially). The test passes only if every mutant makes at least one pin fail,
and the unaltered source, built the same way, passes them all.

Mutants that the model cannot tell apart from the original are not listed: in
the axisymmetric field the z torque is zero whatever its prefactor, and the
self term of the sum is exactly zero when eps > 0.
"""
import ctypes as C
import inspect
import itertools
import os
import subprocess
import warnings
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_oracle_pins as pins

# (name, text in the oracle's source, replacement, number of occurrences)
MUTANTS = [
    # the pair sum of eq. 5 (full and sampled routines alike)
    ("dx sign", "const double dx = pos[3 * j] - xi;", "const double dx = xi - pos[3 * j];", 2),
    ("dy reads z", "const double dy = pos[3 * j + 1] - yi;",
     "const double dy = pos[3 * j + 2] - yi;", 2),
    ("softening dropped", "dz * dz + eps2;", "dz * dz;", 2),
    ("softening not squared", "const double eps2 = eps * eps;", "const double eps2 = eps;", 2),
    ("inverse-square weight", "const double w = mass[j] / (r2 * r);",
     "const double w = mass[j] / r2;", 2),
    ("weight r^-4", "const double w = mass[j] / (r2 * r);",
     "const double w = mass[j] / (r2 * r2);", 2),
    ("mass of i", "mass[j] / (r2 * r)", "mass[i] / (r2 * r)", 2),
    ("self term kept", "            if (j == i) continue;\n", "", 2),
    ("half the pairs", "for (int64_t j = 0; j < n; ++j) {",
     "for (int64_t j = i + 1; j < n; ++j) {", 2),
    ("y accumulator sign", "ay += w * dy;", "ay -= w * dy;", 2),
    ("G dropped on z", "acc[3 * i + 2] = G * az;", "acc[3 * i + 2] = az;", 1),
    ("sampled sum reads x for z", "acc[3 * q + 2] = G * az;", "acc[3 * q + 2] = G * ax;", 1),
    # the external field (potential and closed-form acceleration)
    ("disk z factor inverted", "(p->ad + s) / s", "s / (p->ad + s)", 1),
    ("disk height not squared", "p->bd * p->bd", "p->bd", 2),
    ("bulge scale not squared", "p->ab * p->ab", "p->ab", 2),
    ("disk force power", "const double D3 = D2 * sqrt(D2);", "const double D3 = D2;", 1),
    ("bulge force sign", "- kb * x[0]", "+ kb * x[0]", 1),
    ("black hole softening not squared", "p->eps_bh * p->eps_bh", "p->eps_bh", 2),
    ("black hole force power", "const double rh3 = rh2 * sqrt(rh2);",
     "const double rh3 = rh2;", 1),
    ("field without G", "const double kd = p->G * p->Md / D3;",
     "const double kd = p->Md / D3;", 1),
    ("potential without G", "return -p->G * p->Md / D - p->G * p->Mb / rb - ph;",
     "return -p->Md / D - p->Mb / rb - ph;", 1),
    ("field ignored by the total", "    if (p->ext_on) {\n", "    if (0) {\n", 1),
    ("field z subtracted", "acc[3 * i + 2] += ae[2];", "acc[3 * i + 2] -= ae[2];", 1),
    # diagnostics of Sect. 5.1 and the torque of eq. 8
    ("kinetic energy without 1/2", "K += 0.5 * m *", "K += m *", 1),
    ("pair energy without m_i", "wi[i] = mass[i] * s;", "wi[i] = s;", 1),
    ("pair energy over all ordered pairs", "for (int64_t j = i + 1; j < n; ++j) {",
     "for (int64_t j = 0; j < n; ++j) {\n            if (j == i) continue;", 1),
    ("pair energy unsoftened", "dz * dz + eps2);", "dz * dz);", 1),
    ("field energy without m", "Wext += m * orc_ext_phi(p, x);", "Wext += orc_ext_phi(p, x);", 1),
    ("total energy without the field", "out[3] = K + W + Wext;", "out[3] = K + W;", 1),
    ("momentum without m", "P[1] += m * v[1];", "P[1] += v[1];", 1),
    ("L_z sign", "L[2] += m * (x[0] * v[1] - x[1] * v[0]);",
     "L[2] += m * (x[1] * v[0] - x[0] * v[1]);", 1),
    ("L_x transposed", "L[0] += m * (x[1] * v[2] - x[2] * v[1]);",
     "L[0] += m * (x[2] * v[1] - x[1] * v[2]);", 1),
    ("torque x transposed", "M[0] += mass[i] * (x[1] * a[2] - x[2] * a[1]);",
     "M[0] += mass[i] * (x[2] * a[1] - x[1] * a[2]);", 1),
    ("torque without mass", "M[1] += mass[i] * (", "M[1] += (", 1),
    # the integrators of Sect. 3.1
    ("kick of half weight", "kick(n, vel, acc, h);", "kick(n, vel, acc, 0.5 * h);", 1),
    ("full-step drifts", "drift(n, pos, vel, 0.5 * h);", "drift(n, pos, vel, h);", 2),
    ("first drift missing", "    drift(n, pos, vel, 0.5 * h);\n    orc_accel(",
     "    orc_accel(", 1),
    ("kick before the force", "    orc_accel(n, pos, mass, p, acc);\n    kick(n, vel, acc, h);",
     "    kick(n, vel, acc, h);\n    orc_accel(n, pos, mass, p, acc);", 1),
    ("w0 sign", "w[0] = 1.0 - 2.0 * (", "w[0] = 1.0 + 2.0 * (", 1),
    ("w1 digit", "SI6A_W1 = -1.17767998417887;", "SI6A_W1 = -1.17767998417787;", 1),
    ("w2 and w3 swapped", "w[2] = SI6A_W2;\n    w[3] = SI6A_W3;",
     "w[2] = SI6A_W3;\n    w[3] = SI6A_W2;", 1),
    ("stages misordered", "{3, 2, 1, 0, 1, 2, 3}", "{3, 1, 2, 0, 2, 1, 3}", 1),
    ("stages not symmetric", "{3, 2, 1, 0, 1, 2, 3}", "{3, 2, 1, 0, 3, 2, 1}", 1),
    ("one stage short", "for (int k = 0; k < 7; ++k)", "for (int k = 0; k < 6; ++k)", 1),
]

# pins that do not compare the oracle with something independent of it
SKIP = {"test_oracle_reproduces_its_fixture", "test_fixture_is_exactly_what_its_script_writes",
        "test_paper_context_matches_the_printed_tables"}


def _pin_calls():
    """Every pin of test_oracle_pins with each of its parameter sets expanded,
    as (label, zero-argument callable taking the oracle module)."""
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_") or name in SKIP:
            continue
        grids = []
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [a.strip() for a in mark.args[0].split(",")]
            grids.append([dict(zip(names, v if len(names) > 1 else (v,)))
                          for v in mark.args[1]])
        for combo in itertools.product(*grids) if grids else [()]:
            kw = {k: v for d in combo for k, v in d.items()}
            label = name + (str(sorted(kw.items())) if kw else "")
            out.append((label, fn, kw))
    return out


def _failing_pins(lib_path):
    """Bind the library at lib_path in place of the oracle's own and return the
    labels of the pins that fail on it."""
    saved = oracle._lib
    oracle._lib = oracle._bind(C.CDLL(lib_path))
    failed = []
    try:
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")      # a mutant's NaNs and overflows
            for label, fn, kw in _pin_calls():
                try:
                    fn(orc=oracle, **kw)
                except Exception:      # assertion or any error the slip provokes
                    failed.append(label)
    finally:
        oracle._lib = saved
    return failed


def _compile(src_text, path):
    c_path = path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    r = subprocess.run(["gcc", *oracle.CFLAGS, "-o", path, c_path, "-lm"],
                       capture_output=True, text=True)
    return r.returncode, r.stderr


@pytest.fixture(scope="module")
def built(tmp_path_factory):
    """The unaltered source and every mutant, compiled in parallel."""
    with open(oracle._SRC) as f:
        src = f.read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = [("original", src)]
    for name, old, new, count in MUTANTS:
        assert src.count(old) == count, (name, src.count(old))
        jobs.append((name, src.replace(old, new)))
    paths = {name: os.path.join(str(d), "m%02d.so" % k) for k, (name, _) in enumerate(jobs)}
    with ThreadPoolExecutor(max_workers=8) as ex:
        res = dict(zip([n for n, _ in jobs],
                       ex.map(lambda j: _compile(j[1], paths[j[0]]), jobs)))
    for name, (rc, err) in res.items():
        assert rc == 0, (name, err)
    return paths


def test_harness_passes_the_unaltered_oracle(built):
    assert _failing_pins(built["original"]) == []


def test_every_planted_mistake_fails_a_pin(built):
    survivors = []
    caught = {}
    for name, *_ in MUTANTS:
        failed = _failing_pins(built[name])
        if failed:
            caught[name] = failed
        else:
            survivors.append(name)
    assert not survivors, "mutants no pin rejects: %s" % survivors
