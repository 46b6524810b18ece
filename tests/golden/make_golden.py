"""Writes the stored oracle fixtures under tests/golden/ (calls only oracle/ and the input generators).

gyre_ftle_32x16.txt: FTLE of the double gyre (Sec. 3.2's 2D Cartesian case; A = 0.1,
eps = 0.25, omega = 2 pi / 10, 129x65 FP32 nodes, 101 frames) on a 32x16 seed lattice over
[0,2]x[0,1], RK4 dt = 0.05, t0 = 0, T = 10, central / one-sided differences.  It guards the
oracle against unintended changes; the paper prints no FTLE values of its own.

stenosis_ftle_24x8.txt: the triangle path (Sec. 3.1 walk, P1, Sec. 4's 2D stenosis-type data):
seed cells and FTLE on a 24x8 lattice over the body-fitted stenosis mesh (h = 0.1, L = 10, 10
frames per period 1), RK4 dt = 0.01, t0 = 0.2, T = 0.6.

kuhn_dp45_4x4x4.txt: the tetrahedral path with DP5(4) in the 32-lane shared-step mode: end positions,
statuses and accepted steps of a 4x4x4 lattice on a Kuhn mesh of [-2, 2]^3 in the unsteady field
u = (-(1 + t) y, x, 0.1 + 0.05 x y) (two frames, t in {0, 1}), rtol = atol = 1e-6, t0 = 0, T = 1.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from meshes import kuhn_mesh  # noqa: E402
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


def stenosis_ftle_24x8():
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.1, L=10.0), nframes=10, period=1.0)
    F = oracle.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
    n, lo, hi = [24, 8], [0.05, -0.96], [9.95, 0.96]
    x0 = oracle.seed_grid(2, n, lo, hi)
    cells = F.locate_seeds(x0)
    xT, st, _ = oracle.rk4(F, x0.astype(np.float64), 0.2, 0.6, 0.01, cells=cells)
    G = oracle.flowmap_gradient(2, n, oracle.lattice_spacing(2, n, lo, hi), [0, 0], [0, 0], xT, st)
    _, sig = oracle.ftle(oracle.cauchy_green(G), 2, 0.6)
    return np.column_stack([cells, sig])


def kuhn_dp45_4x4x4():
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)
    x, y = pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64)
    times = [0.0, 1.0]
    fr = np.stack([np.stack([-(1.0 + t) * y, x, 0.1 + 0.05 * x * y], -1) for t in times]).astype(np.float32)
    F = oracle.TetField(pts, tets, nbrs, fr, times)
    x0 = oracle.seed_grid(3, [4, 4, 4], [-1.2] * 3, [1.2] * 3)
    xT, st, _, ns = oracle.dp45(F, x0.astype(np.float64), 0.0, 1.0, h0=0.01, rtol=1e-6, atol=1e-6, group=32,
                                cells=F.locate_seeds(x0))
    return np.column_stack([xT.T, st, ns])


def main():
    with open(os.path.join(HERE, "stenosis_ftle_24x8.txt"), "w") as f:
        f.write("# seed cell and FTLE per seed (x-fastest) on the stenosis mesh, triangles; see make_golden.py\n")
        for c, v in stenosis_ftle_24x8():
            f.write("%d %.17g\n" % (c, v))
    with open(os.path.join(HERE, "kuhn_dp45_4x4x4.txt"), "w") as f:
        f.write("# x y z status accepted_steps per seed (x-fastest), DP5(4) 32-lane mode on tets; see make_golden.py\n")
        for r in kuhn_dp45_4x4x4():
            f.write("%.17g %.17g %.17g %d %d\n" % tuple(r))
    sig = gyre_ftle_32x16()
    path = os.path.join(HERE, "gyre_ftle_32x16.txt")
    with open(path, "w") as f:
        f.write("# FTLE of the double gyre (2D Cartesian case, Sec. 3.2), oracle output; see make_golden.py\n")
        f.write("# 32x16 seeds on [0,2]x[0,1], seed id x-fastest; RK4 dt=0.05, t0=0, T=10\n")
        for v in sig:
            f.write("%.17g\n" % v)


if __name__ == "__main__":
    main()
