"""Eigenvalues and eigenvectors of the Cauchy-Green tensor at every seed (Sec. 2 "Cauchy-Green")
through lcs_cg_eigen, against the FP64 oracle's Jacobi eigen-decomposition of the same C.

The oracle's own flow map, rounded to FP32, goes into the library (lcs_flowmap_set); C is then
bit-identical to the oracle's from the same positions (lcs_cauchy_green), so the comparison isolates
the eigen-solver: eigenvalues to 1e-12 of lambda_max (and 1e-10 relative for the
small ones), eigenvectors to 1e-10 in direction wherever the eigenvalue is separated from the others
by more than 1e-6 lambda_max, residuals |C v - lambda v| at rounding level everywhere, and the
library's sign convention (largest-magnitude component positive).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import rect_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


def run(ctx, g, n, lo, hi, periodic, T, dt):
    """The oracle's flow map of the lattice, rounded to FP32, through the library's C, FTLE and eigen
    calls (lcs_flowmap_set); returns the oracle's C (asserted bit-identical to the library's) and the
    library's lambda_max, eigenvalues and eigenvectors."""
    endpoint = [0 if p else 1 for p in periodic]
    x0 = oracle.seed_grid(g.dim, n, lo, hi, endpoint)
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    xT, st, _ = oracle.rk4(F, x0.astype(np.float64), 0.0, T, dt)
    x32 = xT.astype(np.float32)
    h = oracle.lattice_spacing(g.dim, n, lo, hi, endpoint)
    period = [hi[a] - lo[a] if periodic[a] else 0.0 for a in range(g.dim)]
    Co = oracle.cauchy_green(oracle.flowmap_gradient(g.dim, n, h, periodic, period, x32.astype(np.float64), st))
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_flowmap_set(ctx, fm, 0, x32, st, T)
    d, np_ = g.dim, (3 if g.dim == 2 else 6)
    C = np.empty((N, np_))
    lcs.lcs_cauchy_green(ctx, fm, 0, C)
    np.testing.assert_array_equal(C, Co)
    f = np.empty(N, dtype=np.float32)
    lam = np.empty(N)
    lcs.lcs_ftle(ctx, fm, 0, f, lam)
    ev = np.empty((N, d))
    V = np.empty((N, d, d))
    lcs.lcs_cg_eigen(ctx, fm, 0, ev, V)
    # device outputs, and one output alone, give the same values
    evd = torch.empty((N, d), dtype=torch.float64, device="cuda")
    lcs.lcs_cg_eigen(ctx, fm, 0, evd, None)
    lcs.lcs_synchronize(ctx)
    np.testing.assert_array_equal(evd.cpu().numpy(), ev)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    return Co, lam, ev, V


def unpack(C, d):
    if d == 2:
        a, b, c = C.T
        return np.stack([np.stack([a, b], -1), np.stack([b, c], -1)], -2)
    a, b, c, e, f, g = C.T
    return np.stack([np.stack([a, b, c], -1), np.stack([b, e, f], -1), np.stack([c, f, g], -1)], -2)


def check(C, lam, ev, V, d):
    eo, vo = oracle.cg_eigen(C, d)
    bad = np.isnan(C).any(axis=1)
    assert np.isnan(ev[bad]).all() and np.isnan(V[bad]).all()
    ok = ~bad
    C, lam, ev, V, eo, vo = C[ok], lam[ok], ev[ok], V[ok], eo[ok], vo[ok]
    lmax = eo[:, -1]
    assert np.all(np.abs(ev - eo) <= 1e-12 * lmax[:, None] + 1e-10 * np.abs(eo))
    np.testing.assert_allclose(ev[:, -1], lam, rtol=1e-12)       # lcs_ftle's lambda_max
    M = unpack(C, d)
    for k in range(d):
        v = V[:, k, :]
        np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
        r = np.linalg.norm(np.einsum("nij,nj->ni", M, v) - ev[:, k, None] * v, axis=1)
        assert np.all(r <= 1e-12 * lmax), r.max() / lmax[r.argmax()]
        # sign convention
        big = np.take_along_axis(v, np.abs(v).argmax(axis=1)[:, None], 1)[:, 0]
        assert np.all(big > 0)
        gap = np.full(len(ev), np.inf)
        for j in range(d):
            if j != k:
                gap = np.minimum(gap, np.abs(eo[:, j] - eo[:, k]))
        sep = gap > 1e-6 * lmax
        dots = np.abs(np.einsum("ni,ni->n", v[sep], vo[sep, k, :]))
        assert np.all(dots >= 1 - 1e-10), 1 - dots.min()
    return int(ok.sum())


def test_eigen_gyre(ctx):
    g = inputs.double_gyre()
    # a box wider than the gyre's: tracers leave, their stencils give NaN
    C, lam, ev, V = run(ctx, g, (201, 99), (-0.02, -0.02), (2.02, 1.02), (0, 0), 5.0, 0.05)
    assert np.isnan(C).any()
    assert check(C, lam, ev, V, 2) > 15000


def test_eigen_abc(ctx):
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    L = 2 * np.pi
    C, lam, ev, V = run(ctx, g, (37, 30, 29), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1), 2.0, 0.02)
    check(C, lam, ev, V, 3)


def test_eigen_rejects_null_outputs(ctx):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 4), (0.0, 0.0), (2.0, 1.0)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    try:
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_cg_eigen(ctx, fm, 0, None, None)
        assert e.value.status == 1
        with pytest.raises(lcs.LcsError):
            lcs.lcs_cg_eigen(ctx, fm, 3, np.empty((32, 2)), None)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)


def near_double_case(rng, gaps, reps):
    """Positions on a 4M x 3 x 3 lattice (spacing 1) whose central differences give, at the centre
    seeds (1 + 4m, 1, 1), chosen gradients G = diag(s) Q^T with Q a random rotation: C = G^T G =
    Q diag(s^2) Q^T has eigenvalues scale * (1, 1 - gap, mu), the two largest a gap apart.  Each
    difference 2 G[i][j] = A - B is split into FP32 values A = fl(2G) and B = fl(A - 2G), so A - B
    (exact in FP64) carries 2G to about 48 bits and the gap survives down to ~1e-14.  The centres'
    stencils are disjoint; every other position stays 0."""
    cases = [(g, r) for g in gaps for r in range(reps)]
    M = len(cases)
    n = (4 * M, 3, 3)
    N = n[0] * n[1] * n[2]
    x = np.zeros((3, N), dtype=np.float32)
    centres, lams = [], []
    idx = lambda i, j, k: i + n[0] * (j + n[1] * k)
    for m, (gap, _) in enumerate(cases):
        Q, _r = np.linalg.qr(rng.standard_normal((3, 3)))
        scale = [1e-4, 1.0, 3e7][m % 3]
        lam = scale * np.array([1.0, 1.0 - gap, rng.uniform(1e-9, 0.9)])
        G = np.sqrt(lam)[:, None] * Q.T
        c = (1 + 4 * m, 1, 1)
        for j in range(3):
            plus, minus = list(c), list(c)
            plus[j] += 1
            minus[j] -= 1
            D = 2.0 * G[:, j]
            A = D.astype(np.float32)
            B = (A.astype(np.float64) - D).astype(np.float32)
            x[:, idx(*plus)] = A
            x[:, idx(*minus)] = B
        centres.append(idx(*c))
        lams.append(lam)
    return n, x, np.array(centres), np.array(lams)


def test_lambda_max_near_double_root(ctx):
    """lambda_max where the two largest eigenvalues of C coincide or nearly do (gaps from 0 to 1e-1 of
    lambda_max): the characteristic cubic has a double root there, which no cubic-based polish resolves
    in FP64, so the library switches to Jacobi rotations; against the oracle's Jacobi on the
    bit-identical C, relative 1e-12 at every gap, both sides of the switch included."""
    rng = np.random.default_rng(20261204)
    gaps = [0.0, 1e-12, 1e-9, 1e-6, 1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1]
    n, x, centres, lams = near_double_case(rng, gaps, 12)
    N = x.shape[1]
    st = np.zeros(N, dtype=np.uint8)
    h = np.ones(3)
    Co = oracle.cauchy_green(oracle.flowmap_gradient(3, n, h, (0, 0, 0), (0, 0, 0), x.astype(np.float64), st))
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, (0.0, 0.0, 0.0), (n[0] - 1.0, 2.0, 2.0)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    try:
        lcs.lcs_flowmap_set(ctx, fm, 0, x, st, 1.0)
        C = np.empty((N, 6))
        lam = np.empty(N)
        f = np.empty(N, dtype=np.float32)
        lcs.lcs_ftle(ctx, fm, 0, f, lam, C)
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
    np.testing.assert_array_equal(C, Co)
    Cc = Co[centres]
    eo, _ = oracle.cg_eigen(Cc, 3)
    # the construction holds: the oracle's two largest eigenvalues are the designed gap apart
    designed = (lams[:, 0] - lams[:, 1]) / lams[:, 0]
    got_gap = (eo[:, 2] - eo[:, 1]) / eo[:, 2]
    assert np.all(np.abs(got_gap - designed) <= 1e-13 + 1e-6 * designed)
    rel = np.abs(lam[centres] - eo[:, 2]) / eo[:, 2]
    assert np.all(rel <= 1e-12), (rel.max(), designed[rel.argmax()])
    np.testing.assert_allclose(f[centres], np.log(eo[:, 2]) / 2.0, rtol=1e-6, atol=1e-7)
