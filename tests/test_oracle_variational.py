"""Pins of the oracle's variational equations (Sec. 1: the linearised flow map grad F obtained by
integrating dM/dt = J(x, t) M, M(t0) = I, instead of differencing the seed grid).

* The interpolant's Jacobian: central differences of the interpolated velocity inside one cell
  (the bilinear / trilinear interpolant is linear along each axis within a cell, so they are exact),
  and a zero column across a clamped (non-periodic, outside-the-box) axis.
* A linear flow u = A x (dyadic A on a dyadic grid, interpolation exact): RK4 advances x and M with
  the same matrix, so M_N = R(hA)^N (R the RK4 stability polynomial) and x_N = M_N x0.
* A linear time-dependent flow u = (A0 + t A1) x: still x_N = M_N x0 (both follow the same product of
  step matrices).
* The double gyre: M agrees with central differences of the flow map over tiny seed offsets.
"""
import numpy as np
import pytest

from paper_2209_13775_gb300 import inputs


@pytest.fixture(scope="module")
def ora():
    import oracle

    oracle.build()
    return oracle


def _R(Z):
    I = np.eye(len(Z))
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_inside_a_cell_and_across_a_clamped_axis(ora, dim):
    g = inputs.abc(n=16, nframes=3, t_end=1.0) if dim == 3 else inputs.double_gyre(nx=33, ny=17, nframes=5)
    from dataclasses import replace
    g = replace(g, periodic=(0,) * dim)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    rng = np.random.default_rng(40 + dim)
    h = np.array(g.spacing)
    for _ in range(20):
        cell = rng.integers(1, np.array(g.n) - 2)
        frac = rng.uniform(0.2, 0.8, dim)
        x = np.array(g.origin) + (cell + frac) * h
        t = rng.uniform(0.0, 0.9)
        u, J = ora.velocity_grad(F, x, t)
        for d in range(dim):
            e = np.zeros(dim)
            e[d] = 0.1 * h[d]
            up, _ = ora.velocity_grad(F, x + e, t)
            um, _ = ora.velocity_grad(F, x - e, t)
            np.testing.assert_allclose(J[:, d], (up - um) / (2 * e[d]), rtol=1e-9, atol=1e-12)
    # outside the box along x: the clamped field does not change with x
    x = np.array(g.origin) + (np.array(g.n) // 2) * h
    x[0] = g.origin[0] - 0.5 * h[0]
    _, J = ora.velocity_grad(F, x, 0.3)
    assert (J[:, 0] == 0).all() and np.abs(J[:, 1]).max() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_flow_closed_form(ora, dim):
    rng = np.random.default_rng(50 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.4 * 16) / 16
    g = inputs.affine_frames(A, np.zeros((dim, dim)), np.zeros(dim), (33,) * dim, (-4.0,) * dim, (0.25,) * dim,
                             [0.0, 5.0])
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    x0 = rng.uniform(-1, 1, (dim, 50))
    dt, T = 0.05, 1.0
    xT, M, st, _ = ora.rk4_var(F, x0, 0.0, T, dt)
    assert (st == ora.OK).all()
    want = np.linalg.matrix_power(_R(dt * A), int(round(T / dt)))
    np.testing.assert_allclose(M, np.broadcast_to(want, M.shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(xT, want @ x0, rtol=0, atol=1e-12)
    # the position part is the plain RK4's
    xr, _, _ = ora.rk4(F, x0, 0.0, T, dt)
    np.testing.assert_allclose(xT, xr, rtol=0, atol=1e-13)


def test_time_dependent_linear_flow(ora):
    A0 = np.array([[0.25, -0.5], [0.5, -0.125]])
    A1 = np.array([[0.0625, 0.0], [0.125, -0.0625]])
    g = inputs.affine_frames(A0, A1, np.zeros(2), (33, 33), (-4.0, -4.0), (0.25, 0.25), np.linspace(0, 4, 9))
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    x0 = np.random.default_rng(5).uniform(-1, 1, (2, 40))
    xT, M, st, _ = ora.rk4_var(F, x0, 0.0, 3.0, 0.05)
    np.testing.assert_allclose(xT, np.einsum("nab,bn->an", M, x0), rtol=0, atol=1e-12)


def test_gyre_against_flow_map_differences(ora):
    g = inputs.double_gyre()
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    x0 = np.random.default_rng(6).uniform([0.1, 0.1], [1.9, 0.9], (200, 2)).T
    T, dt, d = 5.0, 0.05, 1e-7
    _, M, st, _ = ora.rk4_var(F, x0, 0.0, T, dt)
    G = np.empty_like(M)
    for b in range(2):
        e = np.zeros((2, 1))
        e[b] = d
        xp, _, _ = ora.rk4(F, x0 + e, 0.0, T, dt)
        xm, _, _ = ora.rk4(F, x0 - e, 0.0, T, dt)
        G[:, :, b] = ((xp - xm) / (2 * d)).T
    rel = np.abs(M - G).max(axis=(1, 2)) / np.abs(M).max(axis=(1, 2))
    assert np.median(rel) < 1e-6, np.median(rel)


# ------------------------------------------------------------------ meshes (P1: J constant in a cell)

def _tri_field(ora, A, b0=(0.0, 0.0)):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from meshes import tri_grid_mesh
    pts, tris, nbrs = tri_grid_mesh(8)
    pts = (pts - np.float32(4.0)) * np.float32(0.5)        # [-2, 2]^2, dyadic nodes
    fr = np.stack([pts @ np.asarray(A).T + b0, pts @ np.asarray(A).T + b0]).astype(np.float32)
    return ora.TriField(pts, tris, nbrs, fr, [0.0, 10.0])


def _tet_field(ora, A):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from meshes import kuhn_mesh
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)
    fr = np.stack([pts @ np.asarray(A).T, pts @ np.asarray(A).T]).astype(np.float32)
    return ora.TetField(pts, tets, nbrs, fr, [0.0, 10.0])


@pytest.mark.parametrize("dim", [2, 3])
def test_mesh_jacobian_is_the_affine_map_and_cell_differences(ora, dim):
    rng = np.random.default_rng(80 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.5 * 16) / 16
    F = _tri_field(ora, A) if dim == 2 else _tet_field(ora, A)
    for _ in range(30):
        x = rng.uniform(-1.5, 1.5, dim)
        u, J = ora.velocity_grad(F, x, rng.uniform(0, 5))
        np.testing.assert_allclose(J, A, rtol=0, atol=1e-13)
        np.testing.assert_allclose(u, A @ x, rtol=0, atol=1e-13)
    # a non-affine field: J against central differences of u inside the same cell (P1 is affine there)
    from paper_2209_13775_gb300 import inputs
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.25, L=6.0), nframes=8, period=1.0)
    G = ora.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
    if dim == 2:
        for c in rng.choice(len(m.tets), 20):
            v = m.xyz[m.tets[c]].astype(np.float64)
            x = v.T @ np.array([0.4, 0.35, 0.25])               # inside cell c
            u, J = ora.velocity_grad(G, x, 0.3, cell=int(c))
            e = 1e-4 * np.abs(v[1] - v[0]).max()
            for d in range(2):
                dx = np.zeros(2)
                dx[d] = e
                up, _ = ora.velocity_grad(G, x + dx, 0.3, cell=int(c))
                um, _ = ora.velocity_grad(G, x - dx, 0.3, cell=int(c))
                np.testing.assert_allclose(J[:, d], (up - um) / (2 * e), rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_mesh_linear_flow_closed_form(ora, dim):
    rng = np.random.default_rng(90 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.3 * 16) / 16
    F = _tri_field(ora, A) if dim == 2 else _tet_field(ora, A)
    x0 = rng.uniform(-0.6, 0.6, (dim, 40))
    cells = F.locate_seeds(x0.astype(np.float32))
    dt, T = 0.0625, 1.0
    xT, M, st, _ = ora.rk4_var(F, x0, 0.0, T, dt, cells=cells)
    assert (st == ora.OK).all()
    want = np.linalg.matrix_power(_R(dt * A), int(round(T / dt)))
    np.testing.assert_allclose(M, np.broadcast_to(want, M.shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(xT, want @ x0, rtol=0, atol=1e-12)
    xr, _, _ = ora.rk4(F, x0, 0.0, T, dt, cells=cells)
    np.testing.assert_allclose(xT, xr, rtol=0, atol=1e-13)


def test_stenosis_against_flow_map_differences(ora):
    from paper_2209_13775_gb300 import inputs
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.1, L=8.0), nframes=20, period=1.0)
    F = ora.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
    x0 = np.random.default_rng(9).uniform([0.5, -0.4], [6.0, 0.4], (150, 2)).T
    cells = F.locate_seeds(x0.astype(np.float32))
    T, dt, d = 0.5, 0.01, 1e-7
    _, M, st, _ = ora.rk4_var(F, x0, 0.0, T, dt, cells=cells)
    ok = st == ora.OK
    G = np.empty_like(M)
    for b in range(2):
        e = np.zeros((2, 1))
        e[b] = d
        xp, sp, _ = ora.rk4(F, x0 + e, 0.0, T, dt, cells=cells)
        xm, sm, _ = ora.rk4(F, x0 - e, 0.0, T, dt, cells=cells)
        ok &= (sp == ora.OK) & (sm == ora.OK)
        G[:, :, b] = ((xp - xm) / (2 * d)).T
    rel = np.abs(M - G)[ok].max(axis=(1, 2)) / np.abs(M[ok]).max(axis=(1, 2))
    assert ok.sum() > 100 and np.median(rel) < 1e-6, np.median(rel)
