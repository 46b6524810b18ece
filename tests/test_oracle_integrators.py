"""Pins for the oracle's integrators of Eq. 2 (Sec. 2 "Flow Map", Sec. 3.1 RK4).

Closed forms used:
* RK4 on u = A x gives x_N = R(hA)^N x0 exactly, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24.
* DP5 (Dormand-Prince 1980) has stability polynomial 1 + z + ... + z^5/120 + z^6/600.
* Order of convergence (4 and 5) on the analytic double gyre.
* Conservation of the stream function on the steady gyre, time reversal,
  2 pi shift invariance of the periodic ABC flow, det grad F = 1 for
  divergence-free fields.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_2209_13775_gb300 import inputs


def _R4(Z):
    I = np.eye(Z.shape[0])
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def _R5(Z):
    I = np.eye(Z.shape[0])
    P, out = I.copy(), I.copy()
    for j, c in enumerate([1, 1 / 2, 1 / 6, 1 / 24, 1 / 120, 1 / 600], start=1):
        P = P @ Z
        out = out + c * P
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_rk4_linear_flow_is_stability_polynomial(ora, dim):
    rng = np.random.default_rng(10 + dim)
    A = rng.normal(size=(dim, dim)) * 0.7
    field = ora.affine(A)
    x0 = rng.normal(size=(dim, 16))
    T, dt = 1.3, 0.05
    xT, st, _ = ora.rk4(field, x0, 0.0, T, dt)
    N = int(round(T / dt))
    expect = np.linalg.matrix_power(_R4(dt * A), N) @ x0
    np.testing.assert_allclose(xT, expect, rtol=1e-12, atol=1e-12)
    assert (st == ora.OK).all()
    # and converges to exp(A T) x0 at fourth order
    err1 = np.abs(xT - expm(A * T) @ x0).max()
    xT2, _, _ = ora.rk4(field, x0, 0.0, T, dt / 2)
    err2 = np.abs(xT2 - expm(A * T) @ x0).max()
    assert 13.0 < err1 / err2 < 19.0


def test_rk4_on_sampled_affine_grid_is_exact(ora):
    # interpolation of an affine field is exact, so grid data give the same R(hA)^N
    A = np.array([[0.125, -1.0], [1.0, -0.125]])
    g = inputs.affine_frames(A, np.zeros((2, 2)), [0.0, 0.0], (33, 33), (-4.0, -4.0), (0.25, 0.25), [0.0, 5.0])
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing)
    x0 = np.array([[0.5, -1.0, 1.5, 0.0], [0.25, 0.75, -1.0, 2.0]])
    xT, st, _ = ora.rk4(F, x0, 0.0, 2.0, 0.05)
    expect = np.linalg.matrix_power(_R4(0.05 * A), 40) @ x0
    # dyadic nodes and entries: the FP32 samples of A x are exact
    np.testing.assert_allclose(xT, expect, rtol=0, atol=1e-12)


def test_rk4_stage_times(ora):
    # u = b1 t (space-constant, linear in time): RK4 is exact, x(T) = x0 + b1 T^2 / 2 -- a wrong
    # stage time (t instead of t + h/2, or t + h for stage 3) breaks this
    b1 = np.array([0.5, -0.25])
    g = inputs.affine_frames(np.zeros((2, 2)), np.zeros((2, 2)), [0.0, 0.0], (3, 3), (-50, -50), (50, 50),
                             [0.0, 4.0])
    g.frames[1, :, :, :] = (b1 * 4.0).astype(np.float32)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing)
    x0 = np.zeros((2, 3))
    xT, _, _ = ora.rk4(F, x0, 0.5, 3.0, 0.1)
    expect = b1[:, None] * ((3.5 ** 2 - 0.5 ** 2) / 2)
    np.testing.assert_allclose(xT, np.repeat(expect, 3, axis=1), rtol=0, atol=1e-12)
    # backward in time: negative T gives negative steps
    xB, _, _ = ora.rk4(F, x0, 3.5, -3.0, 0.1)
    np.testing.assert_allclose(xB, -np.repeat(expect, 3, axis=1), rtol=0, atol=1e-12)


def _gyre_error(ora, method, dts, T=2.0):
    f = ora.gyre()
    x0 = ora.seed_grid(2, [6, 3], [0.2, 0.2], [1.8, 0.8]).astype(np.float64)
    if method == "rk4":
        ref, _, _ = ora.rk4(f, x0, 0.0, T, dts[-1] / 64)
    else:
        ref, _, _, _ = ora.dp45(f, x0, 0.0, T, h0=dts[-1] / 64, adaptive=False)
    errs = []
    for dt in dts:
        if method == "rk4":
            x, _, _ = ora.rk4(f, x0, 0.0, T, dt)
        else:
            x, _, _, _ = ora.dp45(f, x0, 0.0, T, h0=dt, adaptive=False)
        errs.append(np.abs(x - ref).max())
    return errs


def test_rk4_fourth_order_on_analytic_gyre(ora):
    e = _gyre_error(ora, "rk4", [0.2, 0.1, 0.05])
    assert 13.0 < e[0] / e[1] < 19.0 and 13.0 < e[1] / e[2] < 19.0


def test_dp5_stability_polynomial(ora):
    rng = np.random.default_rng(20)
    A = rng.normal(size=(3, 3)) * 0.5
    x0 = rng.normal(size=(3, 5))
    h = 0.1
    xT, _, _, ns = ora.dp45(ora.affine(A), x0, 0.0, 3 * h, h0=h, adaptive=False)
    assert (ns == 3).all()
    np.testing.assert_allclose(xT, np.linalg.matrix_power(_R5(h * A), 3) @ x0, rtol=1e-13, atol=1e-13)


def test_dp5_fifth_order_on_analytic_gyre(ora):
    e = _gyre_error(ora, "dp45", [0.1, 0.05, 0.025])
    assert 25.0 < e[0] / e[1] < 45.0 and 25.0 < e[1] / e[2] < 40.0


def test_dp45_adaptive_error_tracks_tolerance(ora):
    A = np.array([[0.0, -1.0], [1.0, 0.0]])   # rotation: |x| conserved, exact map is exp(AT)
    x0 = np.array([[1.0, 0.3], [0.0, -0.7]])
    errs = []
    for tol in (1e-5, 1e-7, 1e-9):
        xT, st, _, ns = ora.dp45(ora.affine(A), x0, 0.0, 10.0, h0=0.01, rtol=tol, atol=tol)
        assert (st == ora.OK).all()
        errs.append(np.abs(xT - expm(A * 10.0) @ x0).max())
        assert errs[-1] < 100 * tol
    assert errs[0] > errs[1] > errs[2]


def test_dp45_lands_on_final_time(ora):
    # u = b1 t is integrated exactly by the 5th-order solution; the last step is clipped to t0 + T
    b1 = np.array([0.5, -0.25])
    f = ora.affine(np.zeros((2, 2)), b1=b1)
    xT, st, te, ns = ora.dp45(f, np.zeros((2, 2)), 0.0, 1.234, h0=0.1, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(xT, np.repeat(b1[:, None] * 1.234 ** 2 / 2, 2, axis=1), rtol=0, atol=1e-13)
    assert np.all(te == 1.234)


def test_dp45_leaving_a_rectilinear_box(ora):
    # uniform stream u = (1, 0, 0) sampled on the box [0, 1]^3: every trial has zero error, so
    # steps grow fivefold from h0 (0.01, 0.05, 0.25, 1.25) and the tracer at x = 0.5 ends its
    # fourth step at x = 2.06, more than one cell (0.125) past x = 1: LEFT with t_exit = 1.56
    g = inputs.affine_frames(np.zeros((3, 3)), np.zeros((3, 3)), [1.0, 0.0, 0.0], (9, 9, 9), (0, 0, 0),
                             (0.125, 0.125, 0.125), [0.0, 10.0])
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing)
    x0 = np.array([[0.5, 0.5], [0.5, 0.25], [0.5, 0.75]])
    xT, st, te, ns = ora.dp45(F, x0, 0.0, 10.0, h0=0.01, rtol=1e-6, atol=1e-6)
    assert (st == ora.LEFT).all() and (ns == 4).all()
    np.testing.assert_allclose(te, 1.56, rtol=0, atol=1e-14)
    np.testing.assert_allclose(xT[0], 2.06, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(xT[1:], x0[1:])
    # the same stream backwards from x = 0.5 leaves through x = 0 (past -0.125) at t = -1.56
    _, st, te, _ = ora.dp45(F, x0, 0.0, -10.0, h0=0.01, rtol=1e-6, atol=1e-6)
    assert (st == ora.LEFT).all()
    np.testing.assert_allclose(te, -1.56, rtol=0, atol=1e-14)


def test_dp45_group_mode_equals_per_tracer_when_errors_agree(ora):
    # space-constant field and a pure absolute tolerance: every lane has the same error, so a
    # shared step equals per-tracer stepping bit for bit
    f = ora.affine(np.zeros((2, 2)), b0=[0.3, -0.2], b1=[1.0, 0.5])
    x0 = np.random.default_rng(5).normal(size=(2, 64))
    a = ora.dp45(f, x0, 0.0, 2.0, h0=0.5, rtol=0.0, atol=1e-6, group=1)
    b = ora.dp45(f, x0, 0.0, 2.0, h0=0.5, rtol=0.0, atol=1e-6, group=32)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_dp45_group_mode_shares_the_smallest_step(ora):
    # the gyre gives different errors per lane: the group takes at least as many steps as
    # its hardest lane and every lane of a group takes the same count
    f = ora.gyre()
    x0 = ora.seed_grid(2, [8, 8], [0.1, 0.1], [1.9, 0.9]).astype(np.float64)
    _, _, _, n1 = ora.dp45(f, x0, 0.0, 5.0, h0=0.01, rtol=1e-8, atol=1e-8, group=1)
    _, _, _, n32 = ora.dp45(f, x0, 0.0, 5.0, h0=0.01, rtol=1e-8, atol=1e-8, group=32)
    for g in range(2):
        s = slice(32 * g, 32 * g + 32)
        assert len(set(n32[s].tolist())) == 1
        assert n32[s][0] >= n1[s].max()


def test_dp45_max_steps_status(ora):
    f = ora.gyre()
    x0 = np.array([[0.5], [0.5]])
    _, st, te, ns = ora.dp45(f, x0, 0.0, 10.0, h0=1e-3, rtol=1e-12, atol=1e-12, max_steps=5)
    assert st[0] == ora.MAXSTEPS and ns[0] <= 5


def test_steady_gyre_conserves_stream_function(ora):
    A = 0.1
    f = ora.gyre(A=A, eps=0.0)
    x0 = ora.seed_grid(2, [7, 5], [0.1, 0.1], [1.9, 0.9]).astype(np.float64)
    psi = lambda x: A * np.sin(np.pi * x[0]) * np.sin(np.pi * x[1])
    xT, _, _ = ora.rk4(f, x0, 0.0, 10.0, 0.01)
    assert np.abs(psi(xT) - psi(x0)).max() < 1e-9


def test_time_reversal_returns_seeds(ora):
    f = ora.gyre()
    x0 = ora.seed_grid(2, [9, 5], [0.1, 0.1], [1.9, 0.9]).astype(np.float64)
    xT, _, _ = ora.rk4(f, x0, 0.0, 5.0, 0.01)
    xB, _, _ = ora.rk4(f, xT, 5.0, -5.0, 0.01)
    assert np.abs(xB - x0).max() < 1e-8


def test_periodic_abc_shift_invariance(ora):
    g = inputs.abc(n=16, nframes=5, t_end=1.0)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    L = 2 * np.pi
    x0 = np.random.default_rng(6).uniform(0, L, (3, 8))
    xT, _, _ = ora.rk4(F, x0, 0.0, 1.0, 0.02)
    for j in range(3):
        s = np.zeros((3, 1)); s[j] = L
        xs, _, _ = ora.rk4(F, x0 + s, 0.0, 1.0, 0.02)
        assert np.abs(xs - s - xT).max() < 1e-10


def _det_gradF(ora, field, dim, n, lo, hi, T, dt, periodic=(0, 0, 0), period=(0, 0, 0)):
    x0 = ora.seed_grid(dim, n, lo, hi).astype(np.float64)
    xT, st, _ = ora.rk4(field, x0, 0.0, T, dt)
    h = ora.lattice_spacing(dim, n, lo, hi)
    G = ora.flowmap_gradient(dim, n, h, periodic, period, xT, st)
    return np.linalg.det(G)


def test_incompressible_fields_keep_unit_jacobian(ora):
    d = _det_gradF(ora, ora.gyre(), 2, [5, 5], [0.5, 0.25], [0.5078125, 0.2578125], 2.0, 0.01)
    assert np.abs(d - 1).max() < 1e-4
    d = _det_gradF(ora, ora.abc(), 3, [5, 5, 5], [1.0, 1.0, 1.0], [1.0078125] * 3, 1.0, 0.01)
    assert np.abs(d - 1).max() < 1e-5
    d = _det_gradF(ora, ora.pipe(phases=(0.1, 1.0, 2.0, 3.0)), 3, [5, 5, 5], [0.25, 0.125, 3.0],
                   [0.2578125, 0.1328125, 3.0078125], 1.0, 0.01)
    assert np.abs(d - 1).max() < 1e-5
    # a compressible field fails the same check: u = (x, 0) gives det = e^T
    d = _det_gradF(ora, ora.affine(np.diag([1.0, 0.0])), 2, [5, 5], [0, 0], [1, 1], 1.0, 0.01)
    assert abs(d.mean() - math.e) < 1e-6
