"""Pins for the oracle's triangle-mesh point location and P1 interpolation (2D unstructured
velocity data such as the stenosis geometries of Sec. 4; the local cell search of Sec. 3.1 one
dimension lower; Sec. 2 "Seed": the cell holding each seed).

* orient2d against exact rational arithmetic (fractions.Fraction) on random, nearly collinear
  and far-from-the-origin FP32 inputs.
* The walk (with the lowest-id tie-break) against brute force over all triangles on a grid
  triangulation with integer nodes and mixed orientations -- queried at vertices and edge points,
  where several triangles hold the point -- and on the jittered stenosis mesh.
* P1 interpolation reproduces affine fields; RK4 on them is R(hA)^N; DP5(4) on them matches the
  analytic affine field's run.
* A uniform stream leaves a box mesh at a time known in closed form.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2209_13775_gb300 import inputs
from meshes import l_tri_grid_mesh, tri_grid_mesh


@pytest.fixture(scope="module")
def ora():
    import oracle

    oracle.build()
    return oracle


def _orient_exact(a, b, c):
    q = [[Fraction(float(v)) for v in p] for p in (a, b, c)]
    det = (q[1][0] - q[0][0]) * (q[2][1] - q[0][1]) - (q[1][1] - q[0][1]) * (q[2][0] - q[0][0])
    return (det > 0) - (det < 0)


def test_orient2d_matches_rational_arithmetic(ora):
    rng = np.random.default_rng(70)
    for _ in range(300):
        P = rng.normal(size=(3, 2)).astype(np.float32)
        assert ora.orient2d(*P) == _orient_exact(*P)
    # nearly collinear: c on the line through a and b (to FP32 rounding), then nudged by one ulp
    for _ in range(300):
        a, b = rng.uniform(-1e3, 1e3, 2), rng.uniform(-1e3, 1e3, 2)
        c = (a + rng.uniform(-2, 2) * (b - a)).astype(np.float32)
        for cc in (c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(-np.inf))):
            P = [a.astype(np.float32), b.astype(np.float32), cc]
            assert ora.orient2d(*P) == _orient_exact(*P)
    # a small triangle far from the origin: the raw products (~2^40) cancel to a few ulps^2
    base = np.float32(2 ** 20)
    signs = set()
    for _ in range(300):
        P = base + np.float32(0.125) * rng.integers(-4, 5, (3, 2)).astype(np.float32)
        o = ora.orient2d(*P)
        assert o == _orient_exact(*P)
        signs.add(o)
    assert signs == {-1, 0, 1}
    # sign convention: c left of a -> b is positive
    assert ora.orient2d([0, 0], [1, 0], [0, 1]) == 1
    assert ora.orient2d([0, 0], [1, 0], [0, -1]) == -1
    assert ora.orient2d([0, 0], [1, 0], [7, 0]) == 0
    t = np.float32(1e-44)
    assert ora.orient2d([0, 0], [t, 0], [0, t]) == 1


def _field(ora, pts, tris, nbrs, frames=None, times=(0.0,)):
    if frames is None:
        frames = np.zeros((1, len(pts), 2), dtype=np.float32)
    return ora.TriField(pts, tris, nbrs, frames, times)


def test_walk_equals_brute_force_with_tie_break(ora):
    pts, tris, nbrs = tri_grid_mesh(5)
    f = _field(ora, pts, tris, nbrs)
    rng = np.random.default_rng(71)
    queries = [pts[i] for i in rng.choice(len(pts), 30, replace=False)]                   # vertices
    queries += [0.5 * (pts[a] + pts[b]) for a, b in rng.choice(tris[:, :2], 40)]           # edge points
    queries += [np.float32([rng.integers(0, 5) + 0.25, rng.integers(0, 5)]) for _ in range(20)]   # on grid lines
    queries += list(rng.uniform(0, 5, (80, 2)).astype(np.float32))                          # generic
    queries += list(rng.uniform(-1, 6, (40, 2)).astype(np.float32))                         # some outside
    n_ties = 0
    for q in queries:
        brute = f.locate_brute(q)
        holders = [t for t in range(len(tris)) if f.contains(t, q)[0]]
        assert brute == (min(holders) if holders else -1)
        n_ties += len(holders) > 1
        for start in rng.choice(len(tris), 3):
            assert f.locate_walk(q, int(start)) == brute
    assert n_ties > 60          # the tie-break path really ran


def test_walk_on_stenosis_mesh(ora):
    m = inputs.stenosis_mesh(h=0.2, L=6.0)
    f = _field(ora, m.xyz, m.tets, m.nbrs)
    rng = np.random.default_rng(72)
    q = rng.uniform([-0.2, -1.1], [6.2, 1.1], (200, 2)).astype(np.float32)
    q = np.concatenate([q, m.xyz[rng.choice(len(m.xyz), 40)]])
    inside = 0
    for p in q:
        b = f.locate_brute(p)
        inside += b >= 0
        assert f.locate_walk(p, int(rng.integers(len(m.tets)))) == b
    assert inside > 150


def test_p1_interpolation_reproduces_affine_fields(ora):
    pts, tris, nbrs = tri_grid_mesh(4)
    A = np.array([[0.5, -1.0], [1.0, -0.25]])
    b = np.array([0.25, -0.5])
    fr = np.stack([pts @ A.T + b, pts @ (2 * A).T + b]).astype(np.float32)
    f = _field(ora, pts, tris, nbrs, fr, (0.0, 2.0))
    rng = np.random.default_rng(73)
    for _ in range(100):
        x = rng.uniform(0, 4, 2)
        t = rng.uniform(0, 2)
        u, c = f.velocity(x, t, cell=int(rng.integers(len(tris))))
        np.testing.assert_allclose(u, (1 + t / 2) * (A @ x) + b, rtol=0, atol=1e-13)
    u, _ = f.velocity([4.5, 1.0], 0.0)
    assert u is None


def _R(Z):
    return np.eye(len(Z)) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def test_rk4_and_dp45_on_tri_affine_field_and_leaving(ora):
    pts, tris, nbrs = tri_grid_mesh(4)
    pts = pts - np.float32(2.0)                       # box [-2, 2]^2
    A = np.array([[0.0, -0.5], [0.5, 0.0]])           # rotation
    fr = np.stack([pts @ A.T, pts @ A.T]).astype(np.float32)
    f = _field(ora, pts, tris, nbrs, fr, (0.0, 10.0))
    x0 = np.array([[0.5, -0.25, 1.0], [0.25, 0.5, -0.75]])
    cells = np.array([f.locate_walk(x0[:, i].astype(np.float32)) for i in range(3)], dtype=np.int32)
    xT, st, _ = ora.rk4(f, x0, 0.0, 2.0, 0.1, cells=cells)
    np.testing.assert_allclose(xT, np.linalg.matrix_power(_R(0.1 * A), 20) @ x0, rtol=0, atol=1e-12)
    assert (st == ora.OK).all()
    # DP5(4) on the mesh equals DP5(4) on the analytic affine field (same velocity to ~1e-15)
    aff = ora.AnalyticField(ora.AN_AFFINE, 2, list(np.pad(A, ((0, 1), (0, 1))).ravel()) + [0.0] * 15)
    xm, stm, tem, nm = ora.dp45(f, x0, 0.0, 2.0, h0=0.05, rtol=1e-8, atol=1e-8, cells=cells)
    xa, sta, tea, na = ora.dp45(aff, x0, 0.0, 2.0, h0=0.05, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(xm, xa, rtol=0, atol=1e-9)
    np.testing.assert_array_equal(nm, na)
    # uniform stream u = (1, 0): from x0 = -1.5 the tracer reaches x = 2 at t = 3.5; the step from
    # t_n = 3.5 has its second stage at x = 2.05 (outside), so it freezes at t_e = 3.5
    fr2 = np.zeros((2, len(pts), 2), dtype=np.float32)
    fr2[..., 0] = 1.0
    f2 = _field(ora, pts, tris, nbrs, fr2, (0.0, 10.0))
    x0 = np.array([[-1.5], [0.3]])
    c0 = np.array([f2.locate_walk(x0[:, 0].astype(np.float32))], dtype=np.int32)
    xT, st, te = ora.rk4(f2, x0, 0.0, 5.0, 0.1, cells=c0)
    assert st[0] == ora.LEFT and abs(te[0] - 3.5) < 1e-9 and abs(xT[0, 0] - 2.0) < 1e-9
    _, st, _ = ora.rk4(f2, x0, 0.0, 1.0, 0.1, cells=np.array([-1], dtype=np.int32))
    assert st[0] == ora.OUTSIDE


def test_rk4_stages_across_the_notch(ora):
    # as on tets: u = (1, -1), one step of h = 1 from the y-arm of an L-shaped mesh; every stage point
    # is inside but the straight line to the later ones crosses the notch
    pts, tris, nbrs = l_tri_grid_mesh(4)
    fr = np.zeros((2, len(pts), 2), np.float32)
    fr[..., 0], fr[..., 1] = 1.0, -1.0
    f = _field(ora, pts, tris, nbrs, fr, (0.0, 10.0))
    x0 = ora.seed_grid(2, (9, 9), (1.55, 2.05), (1.95, 2.45))
    xT, st, _ = ora.rk4(f, x0.astype(np.float64), 0.0, 1.0, 1.0, cells=f.locate_seeds(x0))
    assert (st == ora.OK).all()
    np.testing.assert_allclose(xT, x0 + np.array([[1.0], [-1.0]]), rtol=0, atol=1e-12)
