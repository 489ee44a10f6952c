"""Writes oracle_plummer16_orbit.txt: a seeded 16-body Plummer sphere on a
circular orbit at R = 50 in the disk + bulge field, with what the oracle
computes for it -- the accelerations of eq. 3 (pair sum eq. 5 plus the field),
the energies (the softened potential energy of eq. 4), and the state after 4
steps of the sixth-order scheme (Sect. 3.1) and of the leapfrog.  It calls only the oracle and the
seeded input generator; run it from the repository root:

    python tests/golden/make_golden.py

The fixture stores its inputs too, so a reader needs neither generator."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1003_3896_gb300 import ics  # noqa: E402

N, SEED, DT, STEPS = 16, 7, 1.0 / 64, 4


def block(f, name, a):
    f.write(f"[{name}]\n")
    for row in np.atleast_2d(a):
        f.write(" ".join(f"{v:.17e}" for v in row) + "\n")


def main(out=None):
    """Write the fixture to ``out`` (default: its place beside this script)."""
    oracle.build()
    pos, vel, m = ics.plummer(N, SEED)
    pos, vel = ics.place_on_orbit(pos, vel)
    eps = ics.paper_softening(N)
    p = oracle.Params(G=1.0, eps=eps, ext_on=True)
    acc = oracle.accel(pos, m, p)
    e = oracle.energy(pos, vel, m, p)
    x6, v6 = oracle.run(pos, vel, m, p, 6, DT, STEPS)
    x2, v2 = oracle.run(pos, vel, m, p, 2, DT, STEPS)
    if out is None:
        out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_plummer16_orbit.txt")
    with open(out, "w") as f:
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle (oracle/), FP64.\n")
        f.write("# Inputs: Plummer sphere (a = 1, M = 1, N = 16, seed 7) with its centre of mass\n")
        f.write("# moved to (50, 0, 0) on the circular orbit of the disk + bulge field of eq. 3\n")
        f.write("# (M_d = 100, a_d = 6.5, b_d = 0.26, M_b = 15, a_b = 0.7, G = 1); softening by\n")
        f.write("# the paper's rule eps = 0.005 / N^(1/3) (Sect. 2).  Outputs: accelerations of\n")
        f.write("# eq. 3 with the pair sum of eq. 5; K, W (the softened potential energy, eq. 4),\n")
        f.write("# W_ext, E = K + W + W_ext, P, L (whose relative changes are eqs. 9 and 10); the\n")
        f.write(f"# state after {STEPS} steps of dt = 1/{int(1 / DT)} of the sixth-order scheme (Sect. 3.1)\n")
        f.write("# and of the leapfrog.\n")
        block(f, "params", [[1.0, eps, 100.0, 6.5, 0.26, 15.0, 0.7, DT, STEPS]])
        block(f, "mass", m.reshape(1, -1))
        block(f, "pos", pos)
        block(f, "vel", vel)
        block(f, "acc", acc)
        block(f, "energy", [[e.K, e.W, e.W_ext, e.E, *e.P, *e.L]])
        block(f, "pos_order6", x6)
        block(f, "vel_order6", v6)
        block(f, "pos_order2", x2)
        block(f, "vel_order2", v2)
    print("wrote", out)


if __name__ == "__main__":
    main()
