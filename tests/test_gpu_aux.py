"""Auxiliary-point flow-map gradient (Sec. 2 "Seed" and "Cauchy-Green") through lcs_seed_aux and the
CG calls: the auxiliary points bit-identical to the oracle's, their FTLE against the oracle's within
the fixed-step tolerances, C bit-identical to the oracle's from the same FP32 positions, and, with the
lattice step as spacing on a dyadic lattice, equal to the lattice differences inside the lattice.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import check_ftle, gpu_cg_of, rect_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


def run_aux(ctx, g, n, lo, hi, periodic, delta, T, dt, variant=0):
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    aux = lcs.lcs_seed_aux(ctx, lat, delta)
    N, M = lcs.lcs_seeds_count(lat), lcs.lcs_seeds_count(aux)
    assert M == N * 2 * g.dim
    xa = np.empty((g.dim, M), dtype=np.float32)
    lcs.lcs_seeds_get(ctx, aux, xa)
    fm = lcs.lcs_flowmap_create(ctx, aux, 1)
    lcs.lcs_advect(ctx, field, aux, lcs.advect_opts(lcs.RK4, T=T, dt=dt, variant=variant), fm)
    x = np.empty((g.dim, M), dtype=np.float32)
    st = np.empty(M, dtype=np.uint8)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, st)
    f = np.empty(N, dtype=np.float32)
    C = np.empty((N, 3 if g.dim == 2 else 6))
    lcs.lcs_ftle(ctx, fm, 0, f, None, C)
    ev = np.empty((N, g.dim))
    lcs.lcs_cg_eigen(ctx, fm, 0, ev)
    lcs.lcs_synchronize(ctx)
    out = dict(xa=xa, x=x, st=st, ftle=f, C=C, ev=ev)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(aux)
    lcs.lcs_free_seeds(lat)
    lcs.lcs_free_field(field)
    return out


def oracle_aux(g, n, lo, hi, periodic, delta, T, dt):
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    endpoint = [0 if p else 1 for p in periodic]
    xa = oracle.aux_points(oracle.seed_grid(g.dim, n, lo, hi, endpoint), delta)
    xT, st, _ = oracle.rk4(F, xa.astype(np.float64), 0.0, T, dt)
    G = oracle.aux_gradient(xa, xT, st)
    C = oracle.cauchy_green(G)
    lam, sig = oracle.ftle(C, g.dim, T)
    return xa, st, sig, xT


def cg_on_oracle_flowmap(ctx, g, n, lo, hi, periodic, delta, xa, xT, st, T):
    """The oracle's auxiliary-point flow map, rounded to FP32, through the library's differences and
    Eq. 1 (lcs_flowmap_set on an auxiliary seed set) and through the oracle's: C bit for bit, and the
    largest eigenvalue of both eigen paths within rounding of the oracle's."""
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    aux = lcs.lcs_seed_aux(ctx, lat, delta)
    N = lcs.lcs_seeds_count(lat)
    x32 = xT.astype(np.float32)
    r = gpu_cg_of(ctx, aux, x32, st, T, N, g.dim, want_eig=True)
    lcs.lcs_free_seeds(aux)
    lcs.lcs_free_seeds(lat)
    C = oracle.cauchy_green(oracle.aux_gradient(xa, x32.astype(np.float64), st))
    np.testing.assert_array_equal(r["C"], C)
    lam, _ = oracle.ftle(C, g.dim, T)
    np.testing.assert_allclose(r["lam"], lam, rtol=1e-12)
    np.testing.assert_allclose(r["ev"][:, -1], lam, rtol=1e-12)


def test_aux_gyre(ctx):
    g = inputs.double_gyre()
    n, lo, hi, T, dt = (96, 48), (0.0, 0.0), (2.0, 1.0), 5.0, 0.05
    delta = [2.0 / 95 / 8, 1.0 / 47 / 8]
    r = run_aux(ctx, g, n, lo, hi, (0, 0), delta, T, dt)
    xa, st, sig, xT = oracle_aux(g, n, lo, hi, (0, 0), delta, T, dt)
    np.testing.assert_array_equal(r["xa"], xa)
    np.testing.assert_array_equal(r["st"], st)
    check_ftle(r["ftle"], sig)
    cg_on_oracle_flowmap(ctx, g, n, lo, hi, (0, 0), delta, xa, xT, st, T)


@pytest.mark.parametrize("variant", [1, 3])
def test_aux_abc(ctx, variant):
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    L = 2 * np.pi
    n, lo, hi, T, dt = (20, 18, 16), (0.0, 0.0, 0.0), (L, L, L), 2.0, 0.02
    delta = [L / 20 / 4, L / 18 / 4, L / 16 / 4]
    r = run_aux(ctx, g, n, lo, hi, (1, 1, 1), delta, T, dt, variant=variant)
    xa, st, sig, xT = oracle_aux(g, n, lo, hi, (1, 1, 1), delta, T, dt)
    np.testing.assert_array_equal(r["xa"], xa)
    check_ftle(r["ftle"], sig)
    cg_on_oracle_flowmap(ctx, g, n, lo, hi, (1, 1, 1), delta, xa, xT, st, T)


def test_aux_with_lattice_step_equals_lattice(ctx):
    g = inputs.double_gyre()
    n, lo, hi, T, dt = (65, 33), (0.0, 0.0), (2.0, 1.0), 4.0, 0.05     # steps 1/32: dyadic
    r = run_aux(ctx, g, n, lo, hi, (0, 0), [1.0 / 32, 1.0 / 32], T, dt)
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    N = lcs.lcs_seeds_count(lat)
    fm = lcs.lcs_flowmap_create(ctx, lat, 1)
    lcs.lcs_advect(ctx, field, lat, lcs.advect_opts(lcs.RK4, T=T, dt=dt), fm)
    C = np.empty((N, 3))
    lcs.lcs_cauchy_green(ctx, fm, 0, C)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(lat)
    lcs.lcs_free_field(field)
    ii, jj = np.meshgrid(np.arange(1, n[0] - 1), np.arange(1, n[1] - 1))
    inner = (jj * n[0] + ii).ravel()
    np.testing.assert_array_equal(r["C"][inner], C[inner])


def test_aux_rejects(ctx):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 4), (0.0, 0.0), (2.0, 1.0)))
    try:
        for d in ([0.0, 0.1], [0.1, -1.0], [float("nan"), 0.1]):
            with pytest.raises(lcs.LcsError) as e:
                lcs.lcs_seed_aux(ctx, lat, d)
            assert e.value.status == 1
        aux = lcs.lcs_seed_aux(ctx, lat, [0.01, 0.01])
        with pytest.raises(lcs.LcsError):      # auxiliary points of auxiliary points
            lcs.lcs_seed_aux(ctx, aux, [0.01, 0.01])
        field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
        fm = lcs.lcs_flowmap_create(ctx, aux, 1)
        opts = lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05)
        lcs.lcs_advect(ctx, field, aux, opts, fm)
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_ftle_early(ctx, field, aux, opts, fm, 0, np.empty(32, dtype=np.float32))
        assert e.value.status == 7
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_field(field)
        lcs.lcs_free_seeds(aux)
    finally:
        lcs.lcs_free_seeds(lat)


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_aux_on_meshes(ctx, kind):
    # auxiliary points on a mesh field: located exactly (bit-identical cells), advected with the mesh
    # rules, differenced per seed; FTLE against the oracle's, C bit-identical on the oracle's positions
    from gpu_util import check_exit_statuses
    if kind == "tri":
        m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.05, L=10.0), nframes=40, period=1.0)
        F = oracle.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
        dim, n, lo, hi, lk = 2, (80, 30), (0.05, -0.96), (9.95, 0.96), lcs.TRI
        delta = [0.5 * (hi[0] - lo[0]) / (n[0] - 1), 0.5 * (hi[1] - lo[1]) / (n[1] - 1)]
    else:
        m = inputs.pipe_frames(inputs.pipe_mesh(h=0.1, R=1.0, L=2.0), nframes=50, period=1.0, L=2.0)
        F = oracle.TetField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
        dim, n, lo, hi, lk = 3, (12, 12, 14), (-0.75, -0.75, 0.1), (0.75, 0.75, 1.9), lcs.TET
        delta = [0.5 * (hi[a] - lo[a]) / (n[a] - 1) for a in range(3)]
    t0, T, dt = 0.2, 0.6, 0.01
    desc = lcs.field_desc(dim, times=m.times, time_periodic=True, period=m.period, kind=lk,
                          mesh=(m.xyz, m.tets, m.nbrs))
    field = lcs.lcs_load_field(ctx, desc, m.frames)
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi), field)
    with pytest.raises(lcs.LcsError):            # a mesh lattice needs its field
        lcs.lcs_seed_aux(ctx, lat, delta)
    aux = lcs.lcs_seed_aux(ctx, lat, delta, field)
    N, M = lcs.lcs_seeds_count(lat), lcs.lcs_seeds_count(aux)
    xa = np.empty((dim, M), dtype=np.float32)
    ca = np.empty(M, dtype=np.int32)
    lcs.lcs_seeds_get(ctx, aux, xa, ca)
    fm = lcs.lcs_flowmap_create(ctx, aux, 1)
    lcs.lcs_advect(ctx, field, aux, lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt), fm)
    x = np.empty((dim, M), dtype=np.float32)
    st = np.empty(M, dtype=np.uint8)
    te = np.empty(M, dtype=np.float32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, st, te)
    f = np.empty(N, dtype=np.float32)
    C = np.empty((N, 3 if dim == 2 else 6))
    lcs.lcs_ftle(ctx, fm, 0, f, None, C)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    xo = oracle.aux_points(oracle.seed_grid(dim, n, lo, hi), delta)
    np.testing.assert_array_equal(xa, xo)
    co = F.locate_seeds(xo)
    np.testing.assert_array_equal(ca, co)
    xT, so, teo, mg = oracle.rk4(F, xo.astype(np.float64), t0, T, dt, cells=co, margin=2e-3)
    same = check_exit_statuses(st, te, so, teo, dt, margin=mg)
    assert (so == oracle.OUTSIDE).sum() > 10 and (so == oracle.OK).sum() > 1000
    # the oracle's flow map through the library's differences and Eq. 1: C bit for bit
    x32 = xT.astype(np.float32)
    r = gpu_cg_of(ctx, aux, x32, so, T, N, dim)
    lcs.lcs_free_seeds(aux)
    lcs.lcs_free_seeds(lat)
    lcs.lcs_free_field(field)
    np.testing.assert_array_equal(r["C"], oracle.cauchy_green(oracle.aux_gradient(xo, x32.astype(np.float64), so)))
    Go = oracle.aux_gradient(xo, xT, so)
    _, sig = oracle.ftle(oracle.cauchy_green(Go), dim, T)
    seed_same = same.reshape(N, 2 * dim).all(axis=1)
    check_ftle(np.where(seed_same, f, np.nan), np.where(seed_same, sig, np.nan))
