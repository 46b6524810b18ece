"""Pins for the oracle's seed lattice, finite-difference grad F, Cauchy-Green
tensor (Eq. 1), eigenvalues and FTLE (Sec. 2 "Seed", "Cauchy-Green").

* Central and second-order one-sided differences are exact on quadratics.
* C = grad F^T grad F is checked on matrices worked out by hand (the
  transposed product grad F grad F^T differs for them).
* Jacobi eigenvalues against the 2x2 quadratic formula and Q diag(L) Q^T with
  known L up to condition 1e14.
* The saddle u = (x, -y) has FTLE ln R(h) / h with R the RK4 polynomial
  (-> 1 as h -> 0), and lambda_min * lambda_max = (R(h) R(-h))^(2N).
"""
import numpy as np
import pytest
from scipy.stats import ortho_group

from paper_2209_13775_gb300 import inputs


def test_seed_lattice_endpoints_order_and_periodic(ora):
    s = ora.seed_grid(2, [5, 3], [0.0, -1.0], [2.0, 1.0])
    assert s.dtype == np.float32 and s.shape == (2, 15)
    np.testing.assert_array_equal(s[0, :5], [0.0, 0.5, 1.0, 1.5, 2.0])   # x fastest
    np.testing.assert_array_equal(s[1, ::5], [-1.0, 0.0, 1.0])
    s3 = ora.seed_grid(3, [4, 2, 2], [0, 0, 0], [2 * np.pi] * 3, endpoint=(0, 1, 1))
    # periodic axis: n points, no duplicate endpoint; x_2 = pi exactly (2 pi / 4 * 2)
    assert s3[0, 2] == np.float32(np.pi) and s3[0, 3] == np.float32(1.5 * np.pi)
    assert s3[2, -1] == np.float32(2 * np.pi)
    # node-inclusive lattice is symmetric about its centre to rounding
    s1 = ora.seed_grid(2, [255, 2], [0.0, 0.0], [2.0, 1.0])
    assert np.abs(s1[0, :255] + s1[0, 254::-1] - 2.0).max() <= 2.5e-7


def _quadratic_map(X, Y):
    F0 = 1.0 + 2.0 * X - 0.5 * Y + 0.25 * X * X - 0.75 * X * Y + 0.5 * Y * Y
    F1 = -X + 3.0 * Y + 0.125 * X * X + Y * Y
    dF = np.array([[2.0 + 0.5 * X - 0.75 * Y, -0.5 - 0.75 * X + Y],
                   [-1.0 + 0.25 * X, 3.0 + 2.0 * Y]])
    return F0, F1, dF


def test_fd_exact_on_quadratic_maps_including_edges(ora):
    n, lo, hi = [9, 6], [0.0, -1.0], [2.0, 1.5]
    s = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    F0, F1, dF = _quadratic_map(s[0], s[1])
    st = np.zeros(s.shape[1], dtype=np.uint8)
    h = ora.lattice_spacing(2, n, lo, hi)
    G = ora.flowmap_gradient(2, n, h, [0, 0], [0, 0], np.stack([F0, F1]), st)
    np.testing.assert_allclose(G, np.moveaxis(dF, -1, 0), rtol=0, atol=1e-12)


def test_fd_skips_invalid_neighbours(ora):
    n, lo, hi = [7, 7], [0.0, 0.0], [1.5, 3.0]
    s = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    F0, F1, dF = _quadratic_map(s[0], s[1])
    st = np.zeros(49, dtype=np.uint8)
    bad = 3 + 7 * 3                       # centre seed has left
    st[bad] = ora.LEFT
    h = ora.lattice_spacing(2, n, lo, hi)
    G = ora.flowmap_gradient(2, n, h, [0, 0], [0, 0], np.stack([F0, F1]), st)
    assert np.isnan(G[bad]).all()
    # its four lattice neighbours fall back to one-sided formulas, still exact on quadratics
    for q in (bad - 1, bad + 1, bad - 7, bad + 7):
        np.testing.assert_allclose(G[q], dF[:, :, q], rtol=0, atol=1e-12)
    # a seed with no valid stencil on an axis gets NaN
    st2 = np.zeros(49, dtype=np.uint8)
    st2[[1, 2, 7 * 1 + 0]] = ora.LEFT     # seed 0: +x and +2x gone, so x has no stencil
    G2 = ora.flowmap_gradient(2, n, h, [0, 0], [0, 0], np.stack([F0, F1]), st2)
    assert np.isnan(G2[0]).any()


def test_fd_periodic_wrap_adds_the_period(ora):
    # translation by c on a periodic lattice: F(x) = x + c, grad F = I everywhere, also across the wrap
    # (integer lattice so that the FP32 seeds are exactly uniform)
    n = [8, 5, 4]
    L = [8.0, 5.0, 4.0]
    s = ora.seed_grid(3, n, [0, 0, 0], L, endpoint=(0, 0, 0)).astype(np.float64)
    xT = s + np.array([[0.25], [-1.125], [7.0]])
    st = np.zeros(s.shape[1], dtype=np.uint8)
    h = ora.lattice_spacing(3, n, [0, 0, 0], L, endpoint=(0, 0, 0))
    np.testing.assert_array_equal(h, [1.0, 1.0, 1.0])
    G = ora.flowmap_gradient(3, n, h, [1, 1, 1], L, xT, st)
    np.testing.assert_allclose(G, np.broadcast_to(np.eye(3), G.shape), rtol=0, atol=1e-12)


def test_cauchy_green_is_gradT_grad(ora):
    G2 = np.array([[[1.0, 2.0], [0.0, 1.0]]])
    np.testing.assert_array_equal(ora.cauchy_green(G2), [[1.0, 2.0, 5.0]])
    G3 = np.array([[[1.0, 2.0, 3.0], [0.0, 1.0, 4.0], [5.0, 6.0, 0.0]]])
    np.testing.assert_array_equal(ora.cauchy_green(G3), [[26.0, 32.0, 3.0, 41.0, 10.0, 25.0]])


def test_eig_2x2_closed_form(ora):
    rng = np.random.default_rng(7)
    for _ in range(100):
        a, b, c = rng.normal(size=3) * [3, 2, 1]
        e = ora.eig_sym([a, b, c], 2)
        m, r = (a + c) / 2, np.hypot((a - c) / 2, b)
        np.testing.assert_allclose(e, [m - r, m + r], rtol=1e-13, atol=1e-13 * (abs(m) + r))


@pytest.mark.parametrize("logk", [0, 4, 8, 14])
def test_eig_3x3_known_spectrum(ora, logk):
    rng = np.random.default_rng(8 + logk)
    for _ in range(20):
        Q = ortho_group.rvs(3, random_state=rng)
        lam = np.sort(np.array([1.0, 10 ** (-logk / 2), 10 ** (-logk)]) * rng.uniform(0.5, 2))
        M = Q @ np.diag(lam) @ Q.T
        e = ora.eig_sym([M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]], 3)
        assert abs(e[2] - lam[2]) <= 1e-14 * lam[2] * 4
        assert np.abs(e - lam).max() <= 1e-15 * lam[2] * 8


def test_ftle_definition(ora):
    C = np.array([[np.e ** 2, 0.0, 0.25], [4.0, 0.0, 1.0], [np.nan, 0.0, 1.0]])
    lam, sig = ora.ftle(C, 2, -2.0)
    assert abs(lam[0] - np.e ** 2) < 1e-14 and abs(sig[0] - 0.5) < 1e-15
    assert abs(sig[1] - np.log(2.0) / 2) < 1e-15
    assert np.isnan(sig[2])


def _R(h):
    return 1 + h + h * h / 2 + h ** 3 / 6 + h ** 4 / 24


@pytest.mark.parametrize("grid", [False, True])
def test_saddle_ftle_closed_form(ora, grid):
    dt, T = 0.1, 2.0
    N = int(round(T / dt))
    if grid:
        g = inputs.affine_frames(np.diag([1.0, -1.0]), np.zeros((2, 2)), [0, 0], (65, 65), (-8, -8),
                                 (0.25, 0.25), [0.0, 5.0])
        f = ora.RectField(g.frames, g.times, g.origin, g.spacing)
    else:
        f = ora.affine(np.diag([1.0, -1.0]))
    n, lo, hi = [9, 5], [-0.5, -0.5], [0.5, 0.5]      # dyadic lattice: exact FP32 seeds
    x0 = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    xT, st, _ = ora.rk4(f, x0, 0.0, T, dt)
    G = ora.flowmap_gradient(2, n, ora.lattice_spacing(2, n, lo, hi), [0, 0], [0, 0], xT, st)
    lam, sig = ora.ftle(ora.cauchy_green(G), 2, T)
    np.testing.assert_allclose(sig, np.log(_R(dt)) / dt, rtol=0, atol=1e-12)
    assert abs(np.log(_R(dt)) / dt - 1.0) < 1e-5        # -> 1 = exact saddle FTLE
    C = ora.cauchy_green(G)
    lmin = C[:, 0] + C[:, 2] - lam
    np.testing.assert_allclose(lmin * lam, (_R(dt) * _R(-dt)) ** (2 * N), rtol=1e-10)


def test_linear_flow_ftle_against_matrix_exponential(ora):
    A = np.array([[0.3, 1.0], [-0.4, -0.3]])
    T = 3.0
    n, lo, hi = [5, 5], [-1, -1], [1, 1]
    x0 = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    xT, st, _ = ora.rk4(ora.affine(A), x0, 0.0, T, 0.001)
    G = ora.flowmap_gradient(2, n, ora.lattice_spacing(2, n, lo, hi), [0, 0], [0, 0], xT, st)
    _, sig = ora.ftle(ora.cauchy_green(G), 2, T)
    from scipy.linalg import expm
    smax = np.linalg.svd(expm(A * T), compute_uv=False)[0]
    np.testing.assert_allclose(sig, np.log(smax) / T, rtol=0, atol=1e-10)


def test_oracle_matches_stored_gyre_fixture(ora):
    # guards the oracle against unintended changes (fixture written by tests/golden/make_golden.py)
    import os
    import importlib.util
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = np.loadtxt(os.path.join(here, "gyre_ftle_32x16.txt"))
    np.testing.assert_allclose(mg.gyre_ftle_32x16(), stored, rtol=1e-12, atol=1e-13)
    # the mesh paths: triangle walk + P1 + RK4 + FD/CG/FTLE, and tets with DP5(4) in 32-lane mode
    st = np.loadtxt(os.path.join(here, "stenosis_ftle_24x8.txt"))
    got = mg.stenosis_ftle_24x8()
    np.testing.assert_array_equal(got[:, 0], st[:, 0])
    np.testing.assert_allclose(got[:, 1], st[:, 1], rtol=1e-12, atol=1e-13)
    kd = np.loadtxt(os.path.join(here, "kuhn_dp45_4x4x4.txt"))
    got = mg.kuhn_dp45_4x4x4()
    np.testing.assert_allclose(got[:, :3], kd[:, :3], rtol=1e-12, atol=1e-13)
    np.testing.assert_array_equal(got[:, 3:], kd[:, 3:])


def _packed(M):
    return [M[0, 0], M[0, 1], M[1, 1]] if M.shape[0] == 2 else [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]]


def test_eigvec_2x2_closed_form(ora):
    # eigenvector of lambda_max of [[a, b], [b, c]] is (b, lambda_max - a) normalised (up to sign)
    rng = np.random.default_rng(9)
    for _ in range(100):
        a, b, c = rng.normal(size=3) * [3, 2, 1]
        e, v = ora.eigvec_sym([a, b, c], 2)
        e0 = ora.eig_sym([a, b, c], 2)
        np.testing.assert_array_equal(e, e0)   # the eigenvalues are the same arithmetic
        u = np.array([b, e[1] - a])
        u /= np.linalg.norm(u)
        assert abs(abs(v[1] @ u) - 1.0) < 1e-12
        assert abs(v[0] @ v[1]) < 1e-13


@pytest.mark.parametrize("logk", [0, 4, 8, 14])
def test_eigvec_3x3_known_basis(ora, logk):
    # Q diag(lam) Q^T with a random orthogonal Q: eigenvector k is column k of Q up to sign, the
    # residual |M v - lam v| is at rounding level of lam_max, and V is orthonormal
    rng = np.random.default_rng(20 + logk)
    for _ in range(20):
        Q = ortho_group.rvs(3, random_state=rng)
        lam = np.sort(np.array([1.0, 10 ** (-logk / 2), 10 ** (-logk)]) * rng.uniform(0.5, 2))
        if logk == 0:
            lam = np.array([0.5, 1.0, 2.0]) * rng.uniform(0.5, 2)   # distinct eigenvalues
        M = Q @ np.diag(lam) @ Q.T
        e, v = ora.eigvec_sym(_packed(M), 3)
        np.testing.assert_allclose(v @ v.T, np.eye(3), atol=1e-14)
        for k in range(3):
            assert np.linalg.norm(M @ v[k] - e[k] * v[k]) <= 1e-14 * lam[2] * 8
        # the top eigenvector is well separated for every logk
        assert abs(abs(v[2] @ Q[:, 2]) - 1.0) < 1e-12


def test_cg_eigen_batch_and_nan(ora):
    rng = np.random.default_rng(11)
    G = rng.normal(size=(5, 3, 3))
    C = ora.cauchy_green(G)
    C[3] = np.nan
    e, v = ora.cg_eigen(C, 3)
    for p in (0, 1, 2, 4):
        e1, v1 = ora.eigvec_sym(C[p], 3)
        np.testing.assert_array_equal(e[p], e1)
        np.testing.assert_array_equal(v[p], v1)
        # eigenvalues of G^T G are the squared singular values of G
        np.testing.assert_allclose(e[p], np.sort(np.linalg.svd(G[p], compute_uv=False) ** 2), rtol=1e-12)
    assert np.isnan(e[3]).all() and np.isnan(v[3]).all()
