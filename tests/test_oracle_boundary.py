"""Pins of the oracle's distance from a mesh boundary and of the RK4 margin built on it (the
smallest distance of any stage point from the boundary: where it is large, two computations of
the same trajectory make the same exit decisions, Sec. 3.1's cell search deciding by the sign of
a barycentric coordinate).

Pinned on closed forms: the boundary of a Kuhn-tetrahedralised box and of a triangulated square
are the box's faces and the square's edges, so the distance is min(x, L - x, ...) inside and the
Euclidean distance to the box outside; the grid index returns the brute-force distance below its
cap and the cap above it; a uniform stream parallel to the walls has a margin in closed form,
and an L-shaped (non-convex) mesh has its re-entrant edge in the distance."""
import numpy as np
import pytest

from meshes import kuhn_mesh, l_kuhn_mesh, l_tri_grid_mesh, tri_grid_mesh


@pytest.fixture(scope="module")
def ora():
    import oracle

    oracle.build()
    return oracle


def box_distance(p, lo, hi):
    """Distance from points p [dim][N] to the surface of the box [lo, hi]."""
    lo = np.asarray(lo, float)[:, None]
    hi = np.asarray(hi, float)[:, None]
    inside = np.all((p >= lo) & (p <= hi), axis=0)
    d_in = np.minimum(p - lo, hi - p).min(axis=0)
    excess = np.maximum(np.maximum(lo - p, p - hi), 0.0)
    d_out = np.sqrt((excess ** 2).sum(axis=0))
    return np.where(inside, d_in, d_out)


def tet_field(ora, pts, tets, nbrs):
    return ora.TetField(pts, tets, nbrs, np.zeros((1, len(pts), 3), np.float32), [0.0])


def tri_field(ora, pts, tris, nbrs):
    return ora.TriField(pts, tris, nbrs, np.zeros((1, len(pts), 2), np.float32), [0.0])


def test_box_distance_closed_form(ora):
    rng = np.random.default_rng(3)
    pts, tets, nbrs = kuhn_mesh(3)
    F = tet_field(ora, pts, tets, nbrs)
    p = rng.uniform(-1.0, 4.0, (3, 400))
    p[:, :50] = rng.uniform(0.0, 3.0, (3, 50))                 # well inside
    p[0, 50:100] = rng.choice([0.0, 3.0], 50) + rng.uniform(-1e-6, 1e-6, 50)   # at a face
    want = box_distance(p, (0, 0, 0), (3, 3, 3))
    got = ora.boundary_distance(F, p)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    # the grid index: the brute-force distance below the cap, the cap above it
    for rmax in (0.05, 0.4):
        gi = ora.boundary_distance(F, p, rmax)
        np.testing.assert_allclose(gi, np.minimum(want, rmax), rtol=0, atol=1e-12)

    pts, tris, nbrs = tri_grid_mesh(4)
    T = tri_field(ora, pts, tris, nbrs)
    q = rng.uniform(-1.0, 5.0, (2, 300))
    want = box_distance(q, (0, 0), (4, 4))
    np.testing.assert_allclose(ora.boundary_distance(T, q), want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ora.boundary_distance(T, q, 0.3), np.minimum(want, 0.3), rtol=0, atol=1e-12)


def test_re_entrant_corner_of_an_l_shape(ora):
    # the L-shaped prism [0,4]^2 x [0,4] without [2,4] x [2,4] x [0,4]: near the inner corner (2, 2)
    # the nearest boundary is the re-entrant edge, at distance |(x, y) - (2, 2)|
    pts, tets, nbrs = l_kuhn_mesh(4)
    F = tet_field(ora, pts, tets, nbrs)
    ang = np.linspace(np.pi, 1.5 * np.pi, 7)
    r = 0.3
    p = np.stack([2 + r * np.cos(ang), 2 + r * np.sin(ang), np.full(7, 2.0)])
    np.testing.assert_allclose(ora.boundary_distance(F, p), r, rtol=0, atol=1e-12)
    pts, tris, nbrs = l_tri_grid_mesh(4)
    T = tri_field(ora, pts, tris, nbrs)
    np.testing.assert_allclose(ora.boundary_distance(T, p[:2]), r, rtol=0, atol=1e-12)


def test_rk4_margin_of_a_uniform_stream(ora):
    # u = (1, 0, 0) in the box [0,3]^3: over T = 1 a tracer from (x0, y0, z0) stays at its y and z and
    # reaches x0 + 1, so its stage points' smallest distance from the boundary is
    # min(x0, 3 - (x0 + 1), y0, 3 - y0, z0, 3 - z0), capped at rmax
    pts, tets, nbrs = kuhn_mesh(3)
    fr = np.zeros((2, len(pts), 3), np.float32)
    fr[..., 0] = 1.0
    F = ora.TetField(pts, tets, nbrs, fr, [0.0, 10.0])
    rng = np.random.default_rng(5)
    x0 = np.stack([rng.uniform(0.2, 1.8, 60), rng.uniform(0.05, 2.95, 60), rng.uniform(0.05, 2.95, 60)])
    x0 = x0.astype(np.float32).astype(np.float64)
    cells = F.locate_seeds(x0)
    rmax = 0.5
    xT, st, te, mg = ora.rk4(F, x0, 0.0, 1.0, 0.1, cells=cells, margin=rmax)
    assert (st == ora.OK).all()
    want = np.minimum.reduce([x0[0], 3 - (x0[0] + 1), x0[1], 3 - x0[1], x0[2], 3 - x0[2], np.full(60, rmax)])
    np.testing.assert_allclose(mg, want, rtol=0, atol=1e-9)
    # without the margin the flow map is the same
    xT2, st2, te2 = ora.rk4(F, x0, 0.0, 1.0, 0.1, cells=cells)
    np.testing.assert_array_equal(xT, xT2)
    # a tracer that leaves: its failing stage point is outside, at the distance it overshot
    x1 = np.array([[2.95], [1.5], [1.5]])
    _, s1, t1, m1 = ora.rk4(F, x1, 0.0, 1.0, 0.1, cells=F.locate_seeds(x1), margin=rmax)
    assert s1[0] == ora.LEFT and m1[0] <= 0.05 + 1e-9
