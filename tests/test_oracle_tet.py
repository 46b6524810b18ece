"""Pins for the oracle's tetrahedral point location and P1 interpolation
(Sec. 3.1: tetrahedralized data, local cell search; Sec. 2 "Seed": the cell
holding each seed).

* orient3d against exact rational arithmetic (fractions.Fraction) on random
  and nearly degenerate FP32 inputs.
* The walk (with the lowest-id tie-break) against brute force over all tets,
  on a Kuhn (6 tets per cube) triangulation with integer nodes -- queried at
  vertices, edge midpoints and face points, where several tets hold the point
  -- and on a jittered Delaunay mesh.
* P1 interpolation reproduces affine fields; RK4 on them is R(hA)^N.
* A uniform stream leaves a box mesh at a time known in closed form.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2209_13775_gb300 import inputs
from meshes import kuhn_mesh, l_kuhn_mesh


def _orient_exact(a, b, c, d):
    q = [[Fraction(float(v)) for v in p] for p in (a, b, c, d)]
    u = [q[1][i] - q[0][i] for i in range(3)]
    v = [q[2][i] - q[0][i] for i in range(3)]
    w = [q[3][i] - q[0][i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
           + u[2] * (v[0] * w[1] - v[1] * w[0]))
    return (det > 0) - (det < 0)


def test_orient3d_matches_rational_arithmetic(ora):
    rng = np.random.default_rng(30)
    for _ in range(300):
        P = rng.normal(size=(4, 3)).astype(np.float32)
        assert ora.orient3d(*P) == _orient_exact(*P)
    # nearly coplanar: d on the plane of a, b, c (to FP32 rounding), then nudged by one ulp
    for _ in range(300):
        a, b, c = (rng.uniform(-1e3, 1e3, 3) for _ in range(3))
        s, t = rng.uniform(-2, 2, 2)
        d = (a + s * (b - a) + t * (c - a)).astype(np.float32)
        for dd in (d, np.nextafter(d, np.float32(np.inf)), np.nextafter(d, np.float32(-np.inf))):
            P = [a.astype(np.float32), b.astype(np.float32), c.astype(np.float32), dd]
            assert ora.orient3d(*P) == _orient_exact(*P)
    # a small tet far from the origin: the 24 raw triple products (~2^60) cancel down to a
    # determinant of a few ulps^3, so every bit of every product must be kept
    base = np.float32(2 ** 20)
    signs = set()
    for _ in range(300):
        P = base + np.float32(0.125) * rng.integers(-6, 7, (4, 3)).astype(np.float32)
        o = ora.orient3d(*P)
        assert o == _orient_exact(*P)
        signs.add(o)
    assert signs == {-1, 0, 1}
    # exactly coplanar integer points and the sign convention ((b-a) x (c-a)) . (d-a)
    assert ora.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 5, 0]) == 0
    assert ora.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]) == 1
    assert ora.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, -1]) == -1
    # tiny coordinates (subnormal FP32) still decided exactly
    t = np.float32(1e-44)
    assert ora.orient3d([0, 0, 0], [t, 0, 0], [0, t, 0], [0, 0, t]) == 1


def _field(ora, pts, tets, nbrs, frames=None, times=(0.0,)):
    if frames is None:
        frames = np.zeros((1, len(pts), 3), dtype=np.float32)
    return ora.TetField(pts, tets, nbrs, frames, times)


def test_walk_equals_brute_force_with_tie_break(ora):
    pts, tets, nbrs = kuhn_mesh(4)
    f = _field(ora, pts, tets, nbrs)
    rng = np.random.default_rng(31)
    queries = [pts[i] for i in rng.choice(len(pts), 40, replace=False)]                 # vertices
    queries += [0.5 * (pts[a] + pts[b]) for a, b in rng.choice(tets[:, :2], 40)]         # edge points
    queries += [np.float32([rng.integers(0, 4), rng.integers(0, 4) + 0.25, rng.integers(0, 4) + 0.5])
                for _ in range(40)]                                                        # on faces/planes
    queries += list(rng.uniform(0, 4, (80, 3)).astype(np.float32))                         # generic
    queries += list(rng.uniform(-1, 5, (40, 3)).astype(np.float32))                        # some outside
    n_ties = 0
    for q in queries:
        brute = f.locate_brute(q)
        holders = [t for t in range(len(tets)) if f.contains(t, q)[0]]
        assert brute == (min(holders) if holders else -1)
        n_ties += len(holders) > 1
        for start in rng.choice(len(tets), 3):
            assert f.locate_walk(q, int(start)) == brute
    assert n_ties > 60          # the tie-break path really ran


def test_walk_on_non_convex_mesh(ora):
    # an L-shaped prism: from a start in one arm, the straight walk to a point in the other arm
    # crosses the notch and meets a boundary face, yet the point is inside
    pts, tets, nbrs = l_kuhn_mesh(4)
    f = _field(ora, pts, tets, nbrs)
    rng = np.random.default_rng(34)
    arm_a = rng.uniform([2.1, 0.1, 0.1], [3.9, 1.9, 3.9], (40, 3)).astype(np.float32)   # x-arm
    arm_b = rng.uniform([0.1, 2.1, 0.1], [1.9, 3.9, 3.9], (40, 3)).astype(np.float32)   # y-arm
    notch = rng.uniform([2.1, 2.1, 0.1], [3.9, 3.9, 3.9], (20, 3)).astype(np.float32)   # outside
    start_a = f.locate_brute(np.float32([3.5, 0.5, 2.0]))
    start_b = f.locate_brute(np.float32([0.5, 3.5, 2.0]))
    for p in arm_a:
        assert f.locate_walk(p, start_b) == f.locate_brute(p) >= 0
    for p in arm_b:
        assert f.locate_walk(p, start_a) == f.locate_brute(p) >= 0
    for p in notch:
        assert f.locate_walk(p, start_a) == -1
    # the interpolation-time location too: u of an affine field from a start across the notch
    A = np.array([[0.5, -1.0, 0.25], [1.0, 0.0, -0.5], [0.125, 0.75, -0.5]])
    fr = np.stack([pts @ A.T]).astype(np.float32)
    g = _field(ora, pts, tets, nbrs, fr, (0.0,))
    for p in arm_b[:10]:
        u, c = g.velocity(p.astype(np.float64), 0.0, cell=start_a)
        np.testing.assert_allclose(u, A @ p.astype(np.float64), rtol=0, atol=1e-12)


def test_rk4_stages_across_the_notch(ora):
    # u = (1, -1, 0), one step of h = 1 from the y-arm of an L-shaped prism: every stage point is in
    # the mesh (the later ones in the x-arm), but the straight line to them crosses the notch, so a
    # walk that stopped at the boundary face would freeze the tracer; the flow map is x0 + (1, -1, 0)
    pts, tets, nbrs = l_kuhn_mesh(4)
    fr = np.zeros((2, len(pts), 3), np.float32)
    fr[..., 0], fr[..., 1] = 1.0, -1.0
    f = _field(ora, pts, tets, nbrs, fr, (0.0, 10.0))
    x0 = ora.seed_grid(3, (5, 5, 4), (1.55, 2.05, 0.5), (1.95, 2.45, 3.5))
    xT, st, _ = ora.rk4(f, x0.astype(np.float64), 0.0, 1.0, 1.0, cells=f.locate_seeds(x0))
    assert (st == ora.OK).all()
    np.testing.assert_allclose(xT, x0 + np.array([[1.0], [-1.0], [0.0]]), rtol=0, atol=1e-12)


def test_walk_on_delaunay_pipe_mesh(ora):
    m = inputs.pipe_mesh(h=0.25, L=2.0)
    f = _field(ora, m.xyz, m.tets, m.nbrs)
    rng = np.random.default_rng(32)
    q = rng.uniform([-1, -1, -0.2], [1, 1, 2.2], (150, 3)).astype(np.float32)
    q = np.concatenate([q, m.xyz[rng.choice(len(m.xyz), 30)]])
    for p in q:
        assert f.locate_walk(p, int(rng.integers(len(m.tets)))) == f.locate_brute(p)


def test_p1_interpolation_reproduces_affine_fields(ora):
    pts, tets, nbrs = kuhn_mesh(3)
    A = np.array([[0.5, -1.0, 0.25], [1.0, 0.0, -0.5], [0.125, 0.75, -0.5]])
    b = np.array([0.25, -0.5, 1.0])
    fr = np.stack([pts @ A.T + b, pts @ (2 * A).T + b]).astype(np.float32)
    f = _field(ora, pts, tets, nbrs, fr, (0.0, 2.0))
    rng = np.random.default_rng(33)
    for _ in range(100):
        x = rng.uniform(0, 3, 3)
        t = rng.uniform(0, 2)
        u, c = f.velocity(x, t, cell=int(rng.integers(len(tets))))
        np.testing.assert_allclose(u, (1 + t / 2) * (A @ x) + b, rtol=0, atol=1e-13)
    u, _ = f.velocity([3.5, 1, 1], 0.0)
    assert u is None


def test_rk4_on_tet_affine_field_and_leaving(ora):
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)                       # box [-2, 2]^3
    A = np.array([[0.0, -0.5, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.0]])   # rotation about z
    fr = np.stack([pts @ A.T, pts @ A.T]).astype(np.float32)
    f = _field(ora, pts, tets, nbrs, fr, (0.0, 10.0))
    x0 = np.array([[0.5, -0.25, 1.0], [0.25, 0.5, -0.75], [0.0, 1.0, -1.0]])
    cells = np.array([f.locate_walk(x0[:, i].astype(np.float32)) for i in range(3)], dtype=np.int32)
    xT, st, _ = ora.rk4(f, x0, 0.0, 2.0, 0.1, cells=cells)
    R = np.eye(3) + 0.1 * A + (0.1 * A) @ (0.1 * A) / 2 + np.linalg.matrix_power(0.1 * A, 3) / 6 \
        + np.linalg.matrix_power(0.1 * A, 4) / 24
    np.testing.assert_allclose(xT, np.linalg.matrix_power(R, 20) @ x0, rtol=0, atol=1e-12)
    assert (st == ora.OK).all()
    # uniform upward stream u = (0, 0, 1): from z0 = -1.5 the tracer reaches the top z = 2 at t = 3.5;
    # the step from t_n = 3.5 has its second stage at z = 2.05 (outside), so it freezes at t_e = 3.5
    fr2 = np.zeros((2, len(pts), 3), dtype=np.float32)
    fr2[..., 2] = 1.0
    f2 = _field(ora, pts, tets, nbrs, fr2, (0.0, 10.0))
    x0 = np.array([[0.25], [0.25], [-1.5]])
    c0 = np.array([f2.locate_walk(x0[:, 0].astype(np.float32))], dtype=np.int32)
    xT, st, te = ora.rk4(f2, x0, 0.0, 5.0, 0.1, cells=c0)
    assert st[0] == ora.LEFT and abs(te[0] - 3.5) < 1e-9 and abs(xT[2, 0] - 2.0) < 1e-9
    # a seed given as outside (cell -1) keeps status OUTSIDE
    _, st, _ = ora.rk4(f2, x0, 0.0, 1.0, 0.1, cells=np.array([-1], dtype=np.int32))
    assert st[0] == ora.OUTSIDE
