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
