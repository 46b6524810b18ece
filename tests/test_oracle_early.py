"""Pins of the oracle's early Cauchy-Green evaluation (Sec. 2 "Flow Map": for trajectories that exit
the data, the CG tensor is formed ahead of the horizon wherever such a trajectory is used).

* A steady shear u = (U + c y, 0) on a box that tracers leave through the x faces: RK4 moves a tracer
  by exactly h (U + c y0) per step (every stage sees the same velocity, and the clamped queries of a
  tracer just outside the box change nothing since u does not depend on x), so each tracer's exit
  step, each seed's early horizon m dt (the fewest in-domain steps over the seed and its lattice
  neighbours, worked out here from the closed form), and the flow map over m steps,
  grad F = [[1, m dt c], [0, 1]], are known: sigma = ln sqrt(lambda_max) / (m dt) with
  lambda_max = 1 + s^2/2 + s sqrt(1 + s^2/4), s = m dt c.
* No tracer leaving: the regular FTLE, unchanged.
"""
import numpy as np
import pytest

from paper_2209_13775_gb300 import inputs


@pytest.fixture(scope="module")
def ora():
    import oracle

    oracle.build()
    return oracle


def shear_case(ora):
    U, c = 0.5 + 2.0 ** -10, 1.0   # dyadic (exact in the FP32 frames) but off the lattice's grid of step sizes
    A0 = np.array([[0.0, c], [0.0, 0.0]])
    g = inputs.affine_frames(A0, np.zeros((2, 2)), [U, 0.0], (33, 9), (0.0, 0.0), (0.125, 0.125), [0.0, 10.0])
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    # dyadic lattice: the FP32 seeds are the lattice points exactly, so the differences are exact too
    n, lo, hi = (33, 8), (0.125, 0.0625), (4.125, 0.9375)
    T, dt = 4.0, 0.1
    return ora, F, n, lo, hi, T, dt, U, c


def test_early_cg_shear_closed_form(ora):
    ora, F, n, lo, hi, T, dt, U, c = shear_case(ora)
    x0 = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    xT, st, te = ora.rk4(F, x0, 0.0, T, dt)
    assert (st == ora.LEFT).any() and (st == ora.OK).any()
    sig, t_eval = ora.ftle_early(F, n, lo, hi, (0, 0), 0.0, T, dt, xT, st, te)
    ns = int(round(T / dt))
    # closed-form exit steps: first k with x0 + k dt u(y0) more than one cell (0.125) beyond x = 4
    u = U + c * x0[1]
    k = np.arange(1, ns + 1)
    d = x0[0][:, None] + k[None, :] * dt * u[:, None] - (4.0 + 0.125)
    ne = np.where((d > 0).any(axis=1), (d > 0).argmax(axis=1), ns)     # steps still in the domain
    tie = (np.abs(d) < 1e-9).any(axis=1)       # lands on the exit threshold: rounding decides
    nx, ny = n
    NE, TIE = ne.reshape(ny, nx), tie.reshape(ny, nx)
    m = NE.copy()
    amb = TIE.copy()
    for j in range(ny):
        for i in range(nx):
            nb = []
            nb += [(j, i + 1), (j, i - 1)] if 0 < i < nx - 1 else ([(j, 1), (j, 2)] if i == 0 else [(j, i - 1), (j, i - 2)])
            nb += [(j + 1, i), (j - 1, i)] if 0 < j < ny - 1 else ([(1, i), (2, i)] if j == 0 else [(j - 1, i), (j - 2, i)])
            m[j, i] = min([NE[j, i]] + [NE[q] for q in nb])
            amb[j, i] = TIE[j, i] or any(TIE[q] for q in nb)
    m, sure = m.ravel(), ~amb.ravel()
    assert sure.sum() > 0.9 * sure.size
    assert (m[sure] < ns).any() and (m[sure] == ns).any() and (m[sure] == 0).any()
    np.testing.assert_array_equal(t_eval[sure], np.where(m == ns, T, m * dt)[sure])
    s = m * dt * c
    lam = 1 + s * s / 2 + s * np.sqrt(1 + s * s / 4)
    with np.errstate(divide="ignore", invalid="ignore"):
        want = np.where(m > 0, np.log(np.sqrt(lam)) / np.where(m == ns, T, m * dt), np.nan)
    np.testing.assert_array_equal(np.isnan(sig[sure]), (m == 0)[sure])
    ok = (m > 0) & sure
    np.testing.assert_allclose(sig[ok], want[ok], rtol=1e-11, atol=1e-13)
    # the ambiguous ones still follow the closed form at the horizon the oracle chose
    fin = np.isfinite(sig) & ~sure
    s2 = np.round(t_eval[fin] / dt) * dt * c
    lam2 = 1 + s2 * s2 / 2 + s2 * np.sqrt(1 + s2 * s2 / 4)
    np.testing.assert_allclose(sig[fin], np.log(np.sqrt(lam2)) / t_eval[fin], rtol=1e-11, atol=1e-13)


def test_early_cg_without_exits_is_regular(ora):
    g = inputs.double_gyre(nx=65, ny=33, nframes=21, t_end=10.0)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    n, lo, hi, T, dt = (48, 24), (0.0, 0.0), (2.0, 1.0), 4.0, 0.05
    x0 = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    xT, st, te = ora.rk4(F, x0, 0.0, T, dt)
    assert (st == ora.OK).all()
    sig, t_eval = ora.ftle_early(F, n, lo, hi, (0, 0), 0.0, T, dt, xT, st, te)
    G = ora.flowmap_gradient(2, n, ora.lattice_spacing(2, n, lo, hi), (0, 0), (0, 0), xT, st)
    _, ref = ora.ftle(ora.cauchy_green(G), 2, T)
    np.testing.assert_array_equal(sig, ref)
    assert (t_eval == T).all()


def test_early_cg_backward(ora):
    # the same shear integrated backward from t0 = 4: tracers leave through x = 0 instead
    ora, F, n, lo, hi, T, dt, U, c = shear_case(ora)
    x0 = ora.seed_grid(2, n, lo, hi).astype(np.float64)
    xT, st, te = ora.rk4(F, x0, 4.0, -T, dt)
    sig, t_eval = ora.ftle_early(F, n, lo, hi, (0, 0), 4.0, -T, dt, xT, st, te)
    ns = int(round(T / dt))
    u = U + c * x0[1]
    k = np.arange(1, ns + 1)
    beyond = x0[0][:, None] - k[None, :] * dt * u[:, None] < -0.125 - 1e-9
    ne = np.where(beyond.any(axis=1), beyond.argmax(axis=1), ns)
    assert (ne < ns).any()
    fin = np.isfinite(sig)
    mdt = np.where(t_eval == T, T, t_eval)
    s = np.round(mdt / dt) * dt * c
    lam = 1 + s * s / 2 + s * np.sqrt(1 + s * s / 4)
    np.testing.assert_allclose(sig[fin], (np.log(np.sqrt(lam)) / mdt)[fin], rtol=1e-11, atol=1e-13)
    # every seed's early horizon is at most its own in-domain time
    assert np.all(np.round(t_eval / dt) <= np.where(ne == ns, ns, ne))


def test_early_on_a_mesh_uniform_stream(ora):
    # u = (1, 0) on a triangulated box [-2, 2]^2: a tracer at x is frozen at the start of the step whose
    # stage point passes x = 2, so it stays floor((2 - x) / dt) steps; a seed's horizon is that of its
    # right-most stencil member (x + h inside, the seed itself at the right edge, whose stencil is
    # backward); the flow map is a translation, so every early FTLE is 0; seeds outside the mesh: NaN
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from meshes import tri_grid_mesh
    pts, tris, nbrs = tri_grid_mesh(4)
    pts = pts - np.float32(2.0)
    fr = np.zeros((2, len(pts), 2), np.float32)
    fr[..., 0] = 1.0
    F = ora.TriField(pts, tris, nbrs, fr, [0.0, 10.0])
    n, lo, hi, dt, T = (23, 9), (-2.55, -1.6), (1.85, 1.6), 0.1, 4.0
    x0 = ora.seed_grid(2, n, lo, hi, [1, 1])
    cells = F.locate_seeds(x0)
    xT, st, te = ora.rk4(F, x0.astype(np.float64), 0.0, T, dt, cells=cells)
    sig, t_eval = ora.ftle_early(F, n, lo, hi, (0, 0), 0.0, T, dt, xT, st, te, cells=cells)
    h = (hi[0] - lo[0]) / (n[0] - 1)
    X = x0[0].astype(np.float64).reshape(n[1], n[0])
    inside = (cells >= 0).reshape(n[1], n[0])
    i = np.arange(n[0])
    v = lambda j, k: 0 <= k < n[0] and inside[j, k]
    checked = 0
    for j in range(1, n[1] - 1):          # rows whose y-stencil is central
        for k in i[inside[j]]:
            if not (v(j - 1, k) and v(j + 1, k)):
                continue
            if v(j, k - 1) and v(j, k + 1):
                right = X[j, k + 1]        # central
            elif v(j, k + 1) and v(j, k + 2):
                right = X[j, k + 2]        # forward
            elif v(j, k - 1) and v(j, k - 2):
                right = X[j, k]            # backward: the seed is the right-most
            else:
                continue
            want = dt * np.floor((2.0 - right) / dt)
            assert abs(t_eval[j * n[0] + k] - min(want, T)) < 1e-9, (j, k, t_eval[j * n[0] + k], want)
            checked += 1
    assert checked > 100
    # a translation: grad F is the identity up to the FP32 rounding of the seeds against the FP64
    # lattice step (~1e-7 relative), so ln sqrt(lambda_max) = sigma * t_eval stays below 1e-6
    ok = np.isfinite(sig)
    assert ok.sum() > 100
    assert np.abs(sig[ok] * t_eval[ok]).max() < 1e-6
    assert np.isnan(sig[~inside.ravel()]).all()
