"""Pins of the oracle's auxiliary-point gradient (Sec. 2 "Seed" and "Cauchy-Green": grad F from points
placed close around each seed).

* Linear flow u = A x with dyadic A on a dyadic grid (node values exact in FP32, interpolation exact): the RK4 flow map is x -> R(hA)^n x, so the
  differences over any auxiliary spacing give R(hA)^n, the RK4 stability polynomial of hA raised to n.
* On a dyadic lattice with delta = the lattice step, the auxiliary points are the lattice neighbours
  exactly, and inside the lattice the gradient equals the lattice central differences bit for bit.
* A point that left makes its seed's gradient NaN.
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
def test_aux_gradient_linear_flow(ora, dim):
    rng = np.random.default_rng(30 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.4 * 16) / 16   # dyadic: A x is exact at the FP32 nodes
    n = (33,) * dim
    g = inputs.affine_frames(A, np.zeros((dim, dim)), np.zeros(dim), n, (-4.0,) * dim, (0.25,) * dim, [0.0, 5.0])
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    lo, hi = (-1.0,) * dim, (1.0,) * dim
    nl = (7, 6, 5)[:dim]
    x0 = ora.seed_grid(dim, nl, lo, hi)
    xa = ora.aux_points(x0, [1e-3 * (b + 1) for b in range(dim)])
    dt, T = 0.05, 1.0
    xT, st, _ = ora.rk4(F, xa.astype(np.float64), 0.0, T, dt)
    G = ora.aux_gradient(xa, xT, st)
    want = np.linalg.matrix_power(_R(dt * A), int(round(T / dt)))
    np.testing.assert_allclose(G, np.broadcast_to(want, G.shape), rtol=0, atol=2e-11)


def test_aux_points_layout(ora):
    x0 = np.array([[0.5, 1.0], [0.25, 0.75]], dtype=np.float32)
    xa = ora.aux_points(x0, [0.125, 0.0625])
    # seed 0: (+x, -x, +y, -y), then seed 1
    np.testing.assert_array_equal(xa[0], [0.625, 0.375, 0.5, 0.5, 1.125, 0.875, 1.0, 1.0])
    np.testing.assert_array_equal(xa[1], [0.25, 0.25, 0.3125, 0.1875, 0.75, 0.75, 0.8125, 0.6875])


def test_aux_with_lattice_step_equals_lattice_differences(ora):
    g = inputs.double_gyre(nx=65, ny=33, nframes=21, t_end=10.0)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    n, lo, hi = (33, 17), (0.0, 0.0), (2.0, 1.0)          # steps 1/16: dyadic
    x0 = ora.seed_grid(2, n, lo, hi)
    h = ora.lattice_spacing(2, n, lo, hi)
    xa = ora.aux_points(x0, h)
    T, dt = 2.0, 0.05
    xTa, sta, _ = ora.rk4(F, xa.astype(np.float64), 0.0, T, dt)
    Ga = ora.aux_gradient(xa, xTa, sta)
    xT, st, _ = ora.rk4(F, x0.astype(np.float64), 0.0, T, dt)
    Gl = ora.flowmap_gradient(2, n, h, (0, 0), (0, 0), xT, st)
    ii, jj = np.meshgrid(np.arange(1, n[0] - 1), np.arange(1, n[1] - 1))
    inner = (jj * n[0] + ii).ravel()
    np.testing.assert_array_equal(Ga[inner], Gl[inner])


def test_aux_point_left_gives_nan(ora):
    xa = np.zeros((2, 8), dtype=np.float32)
    xa[0] = [1, -1, 0, 0, 2, 0, 1, 1]
    xa[1] = [0, 0, 1, -1, 1, 1, 2, 0]
    st = np.zeros(8, dtype=np.uint8)
    st[5] = ora.LEFT
    G = ora.aux_gradient(xa, xa.astype(np.float64), st)
    np.testing.assert_array_equal(G[0], np.eye(2))
    assert np.isnan(G[1]).all()
