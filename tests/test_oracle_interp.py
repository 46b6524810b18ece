"""Pins for the oracle's space-time interpolation (Sec. 2 "Interpolator").

Each check compares against a closed form that does not come from the oracle:
interpolation reproduces the functions it is exact for (affine in time,
bilinear/trilinear in space) and has the textbook error h^2 f (1 - f) / 2 * u''
on a quadratic, which fixes the cell index and the fraction.
"""
import numpy as np
import pytest

from paper_2209_13775_gb300 import inputs


def test_time_bracket_rules(ora):
    times = [0.0, 1.0, 3.0, 6.0]
    assert ora.time_locate(times, 2.0) == (1, 0.5)
    assert ora.time_locate(times, 1.0) == (1, 0.0)        # largest k with t_k <= t
    assert ora.time_locate(times, 6.0) == (2, 1.0)        # clamped to the last interval
    assert ora.time_locate(times, -1.0) == (0, 0.0)       # before the data: first frame
    assert ora.time_locate(times, 9.0) == (2, 1.0)        # after the data: last frame
    # periodic wrap into [t_0, t_0 + period)
    assert ora.time_locate(times, 7.0, True, 6.0) == (1, 0.0)
    k, a = ora.time_locate(times, -4.5, True, 6.0)        # -4.5 + 6 = 1.5
    assert (k, a) == (1, 0.25)


def _frames_from(fun, n, origin, spacing, times, dim):
    axes = [origin[a] + spacing[a] * np.arange(n[a]) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    fr = np.empty((len(times),) + grids[0].shape + (dim,), dtype=np.float32)
    for k, t in enumerate(times):
        vals = fun(*grids, t)
        for c in range(dim):
            fr[k, ..., c] = vals[c]
    return fr


def test_linear_in_time_is_exact(ora):
    # spatially constant u = c0 + c1 t on uneven frame times: exact up to rounding
    times = np.array([0.0, 0.25, 1.125, 2.0, 3.75])
    fr = _frames_from(lambda x, y, t: (0.5 + 0.25 * t + 0 * x, -1.0 + 0.125 * t + 0 * y),
                      (5, 4), (0, 0), (0.5, 0.5), times, 2)
    F = ora.RectField(fr, times, (0, 0), (0.5, 0.5))
    rng = np.random.default_rng(1)
    for t in rng.uniform(0, 3.75, 50):
        u = F.velocity(rng.uniform(0, 1.5, 2), t)
        np.testing.assert_allclose(u, [0.5 + 0.25 * t, -1.0 + 0.125 * t], rtol=0, atol=1e-14)


def test_bilinear_reproduces_bilinear_functions(ora):
    # u = a + b x + c y + d x y is in the span of the bilinear basis
    f0 = lambda x, y: 0.25 + 0.5 * x - 0.75 * y + 0.125 * x * y
    f1 = lambda x, y: -0.5 * x * y + 0.25 * y
    fr = _frames_from(lambda x, y, t: (f0(x, y), f1(x, y)), (9, 7), (-1.0, 0.5), (0.25, 0.5), [0.0], 2)
    F = ora.RectField(fr, [0.0], (-1.0, 0.5), (0.25, 0.5))
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = np.array([rng.uniform(-1.0, 1.0), rng.uniform(0.5, 3.5)])
        np.testing.assert_allclose(F.velocity(x, 0.0), [f0(*x), f1(*x)], rtol=0, atol=1e-13)


def test_bilinear_error_on_quadratic_fixes_cell_and_fraction(ora):
    # I[x^2] - x^2 = h^2 f (1 - f) with f the fraction inside the cell [x_i, x_i + h]
    h = 0.25
    fr = _frames_from(lambda x, y, t: (x * x, 0 * y), (9, 3), (0.0, 0.0), (h, 1.0), [0.0], 2)
    F = ora.RectField(fr, [0.0], (0.0, 0.0), (h, 1.0))
    for x in [0.1, 0.3, 0.55, 1.0, 1.26, 1.99]:
        i = np.floor(x / h)
        f = x / h - i
        u = F.velocity([x, 0.5], 0.0)[0]
        assert abs(u - (x * x + h * h * f * (1 - f))) < 1e-14


def test_trilinear_reproduces_trilinear_functions(ora):
    f = [lambda x, y, z: 1 + x - 2 * y + 0.5 * z + 0.25 * x * y - 0.5 * y * z + 0.75 * x * z + 0.125 * x * y * z,
         lambda x, y, z: -x * y * z + 0.375 * y,
         lambda x, y, z: 0.25 * x * z - 0.125]
    n, o, h = (5, 6, 7), (0.0, -1.0, 2.0), (0.5, 0.25, 0.125)
    fr = _frames_from(lambda x, y, z, t: (f[0](x, y, z), f[1](x, y, z), f[2](x, y, z)), n, o, h, [0.0], 3)
    F = ora.RectField(fr, [0.0], o, h)
    rng = np.random.default_rng(3)
    for _ in range(200):
        x = np.array([rng.uniform(0, 2), rng.uniform(-1, 0.25), rng.uniform(2, 2.75)])
        np.testing.assert_allclose(F.velocity(x, 0.0), [g(*x) for g in f], rtol=0, atol=1e-12)


def test_trilinear_error_on_quadratic_per_axis(ora):
    # along z only: I[z^2] - z^2 = h^2 f (1 - f)
    h = 0.125
    fr = _frames_from(lambda x, y, z, t: (0 * x, 0 * y, z * z), (3, 3, 17), (0, 0, 0), (1, 1, h), [0.0], 3)
    F = ora.RectField(fr, [0.0], (0, 0, 0), (1, 1, h))
    for z in [0.01, 0.7, 1.3, 1.999]:
        i = np.floor(z / h)
        fz = z / h - i
        assert abs(F.velocity([0.3, 1.7, z], 0.0)[2] - (z * z + h * h * fz * (1 - fz))) < 1e-14


def test_periodic_axis_wraps_cells(ora):
    # periodic nodes at i*h, period n*h: u(x + L) = u(x); cell n-1 joins node n-1 to node 0
    n = 8
    h = 2 * np.pi / n
    fr = _frames_from(lambda x, y, z, t: (np.sin(x), np.cos(y), np.sin(z) * np.cos(x)), (n, n, n),
                      (0, 0, 0), (h, h, h), [0.0], 3)
    F = ora.RectField(fr, [0.0], (0, 0, 0), (h, h, h), periodic=(1, 1, 1))
    rng = np.random.default_rng(4)
    L = 2 * np.pi
    for _ in range(50):
        x = rng.uniform(0, L, 3)
        u = F.velocity(x, 0.0)
        for s in ([L, 0, 0], [0, -L, 0], [0, 0, 3 * L]):
            np.testing.assert_allclose(F.velocity(x + np.array(s), 0.0), u, rtol=0, atol=1e-12)
    # in the last cell, x = L - h/2 interpolates nodes n-1 and 0 with weights 1/2
    u = F.velocity([L - h / 2, 0.0, 0.0], 0.0)
    assert abs(u[0] - 0.5 * (fr[0, 0, 0, n - 1, 0] + fr[0, 0, 0, 0, 0])) < 1e-15


def test_nonperiodic_query_clamped_to_box(ora):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing)
    np.testing.assert_array_equal(F.velocity([-0.3, 0.5], 0.2), F.velocity([0.0, 0.5], 0.2))
    np.testing.assert_array_equal(F.velocity([2.5, 1.7], 0.2), F.velocity([2.0, 1.0], 0.2))


def test_sampled_gyre_matches_analytic_at_nodes(ora):
    # at grid nodes and frame times, interpolation returns the FP32 sample of the analytic field
    g = inputs.double_gyre()
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, time_periodic=True, period=g.period)
    A = ora.gyre()
    for (i, j, k) in [(0, 0, 0), (64, 32, 50), (13, 50, 7), (128, 64, 99)]:
        x = np.array([i * g.spacing[0], j * g.spacing[1]])
        t = g.times[k]
        np.testing.assert_allclose(F.velocity(x, t), A.velocity(x, t), rtol=0, atol=1e-7)
