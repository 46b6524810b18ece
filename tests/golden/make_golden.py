"""Writes the stored oracle fixtures under tests/golden/ (calls only oracle/ and the input generators).

gyre_ftle_32x16.txt: FTLE of the double gyre (Sec. 3.2's 2D Cartesian case; A = 0.1,
eps = 0.25, omega = 2 pi / 10, 129x65 FP32 nodes, 101 frames) on a 32x16 seed lattice over
[0,2]x[0,1], RK4 dt = 0.05, t0 = 0, T = 10, central / one-sided differences.  It guards the
oracle against unintended changes; the paper prints no FTLE values of its own.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2209_13775_gb300 import inputs  # noqa: E402


def gyre_ftle_32x16():
    g = inputs.double_gyre()
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    n, lo, hi = [32, 16], [0.0, 0.0], [2.0, 1.0]
    x0 = oracle.seed_grid(2, n, lo, hi)
    xT, st, _ = oracle.rk4(F, x0.astype(np.float64), 0.0, 10.0, 0.05)
    G = oracle.flowmap_gradient(2, n, oracle.lattice_spacing(2, n, lo, hi), [0, 0], [0, 0], xT, st)
    _, sig = oracle.ftle(oracle.cauchy_green(G), 2, 10.0)
    return sig


def main():
    sig = gyre_ftle_32x16()
    path = os.path.join(HERE, "gyre_ftle_32x16.txt")
    with open(path, "w") as f:
        f.write("# FTLE of the double gyre (2D Cartesian case, Sec. 3.2), oracle output; see make_golden.py\n")
        f.write("# 32x16 seeds on [0,2]x[0,1], seed id x-fastest; RK4 dt=0.05, t0=0, T=10\n")
        for v in sig:
            f.write("%.17g\n" % v)


if __name__ == "__main__":
    main()
