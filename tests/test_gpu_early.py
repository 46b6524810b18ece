"""Early Cauchy-Green evaluation (Sec. 2 "Flow Map": for trajectories that exit the data, the CG tensor
is formed ahead of the horizon wherever such a trajectory is used) through lcs_ftle_early, against the
oracle's ftle_early on the same seeded inputs, and against separate GPU runs over the early
horizons (the re-integrated stencil is the same arithmetic, so those values are bit-identical).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import check_ftle, rect_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


def gpu_early(ctx, g, n, lo, hi, periodic, t0, T, dt, variant=0):
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    opts = lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt, variant=variant)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    f = np.empty(N, dtype=np.float32)
    te = np.empty(N, dtype=np.float32)
    lcs.lcs_ftle_early(ctx, field, seeds, opts, fm, 0, f, te)
    reg = np.empty(N, dtype=np.float32)
    lcs.lcs_ftle(ctx, fm, 0, reg)
    st = np.empty(N, dtype=np.uint8)
    lcs.lcs_flowmap_get(ctx, fm, 0, None, st)
    # device outputs give the same values
    fd = torch.empty(N, dtype=torch.float32, device="cuda")
    lcs.lcs_ftle_early(ctx, field, seeds, opts, fm, 0, fd)
    lcs.lcs_synchronize(ctx)
    np.testing.assert_array_equal(fd.cpu().numpy(), f)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return f, te, reg, st


def oracle_early(g, n, lo, hi, periodic, t0, T, dt):
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    endpoint = [0 if p else 1 for p in periodic]
    x0 = oracle.seed_grid(g.dim, n, lo, hi, endpoint).astype(np.float64)
    xT, st, te = oracle.rk4(F, x0, t0, T, dt)
    sig, t_eval = oracle.ftle_early(F, n, lo, hi, periodic, t0, T, dt, xT, st, te)
    return sig, t_eval, st


def truncated_gyre():
    # the double gyre on x in [0, 1.5] only: tracers crossing x = 1.5 leave the data
    g = inputs.double_gyre()
    from dataclasses import replace
    return replace(g, frames=np.ascontiguousarray(g.frames[:, :, :97]))


@pytest.mark.parametrize("T", [6.0, -6.0])
def test_early_gyre_against_oracle(ctx, T):
    g = truncated_gyre()
    n, lo, hi, dt = (120, 80), (0.0, 0.0), (1.5, 1.0), 0.05
    t0 = 0.0 if T > 0 else 6.0
    f, te, reg, st = gpu_early(ctx, g, n, lo, hi, (0, 0), t0, T, dt)
    sig, t_eval, sto = oracle_early(g, n, lo, hi, (0, 0), t0, T, dt)
    np.testing.assert_array_equal(st, sto)
    np.testing.assert_array_equal(te, t_eval.astype(np.float32))
    early = te < abs(T)
    assert early.sum() > 500 and (te > 0).any()
    check_ftle(f, sig)
    # seeds whose stencil stayed in: the regular FTLE, bit for bit; the early ones gain a value
    np.testing.assert_array_equal(f[~early], reg[~early])
    assert np.isfinite(f[early & (te > 0)]).all() and (~np.isfinite(reg[early])).sum() > 0


def test_early_equals_runs_over_the_early_horizons(ctx):
    # an early seed's value is the FTLE a run over its own horizon gives (same positions, same formulas)
    g = truncated_gyre()
    n, lo, hi, T, dt = (120, 80), (0.0, 0.0), (1.5, 1.0), 6.0, 0.05
    f, te, reg, st = gpu_early(ctx, g, n, lo, hi, (0, 0), 0.0, T, dt)
    ms = np.rint(te[(te > 0) & (te < T)] / dt).astype(int)
    vals, cnt = np.unique(ms, return_counts=True)
    for m in vals[np.argsort(-cnt)][:3]:
        field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
        seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
        N = lcs.lcs_seeds_count(seeds)
        fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=m * dt, dt=dt), fm)
        fr = np.empty(N, dtype=np.float32)
        lcs.lcs_ftle(ctx, fm, 0, fr)
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)
        at = np.rint(te / dt).astype(int) == m
        np.testing.assert_array_equal(f[at], fr[at])


@pytest.mark.parametrize("variant", [1, 3])
def test_early_3d_against_oracle(ctx, variant):
    from dataclasses import replace
    g = replace(inputs.abc(n=32, nframes=17, t_end=2.0), periodic=(0, 0, 0))
    n, lo, hi, T, dt = (26, 24, 22), (0.3, 0.2, 0.4), (5.5, 5.7, 5.6), 1.5, 0.02
    f, te, reg, st = gpu_early(ctx, g, n, lo, hi, (0, 0, 0), 0.0, T, dt, variant=variant)
    sig, t_eval, sto = oracle_early(g, n, lo, hi, (0, 0, 0), 0.0, T, dt)
    np.testing.assert_array_equal(st, sto)
    np.testing.assert_array_equal(te, t_eval.astype(np.float32))
    assert (te < T).sum() > 1000
    check_ftle(f, sig)


def test_early_rejects(ctx):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 4), (0.0, 0.0), (2.0, 1.0)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    f = np.empty(32, dtype=np.float32)
    try:
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_ftle_early(ctx, field, seeds, lcs.advect_opts(lcs.RK45, T=1.0), fm, 0, f)
        assert e.value.status == 7
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_ftle_early(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05), fm, 1, f)
        assert e.value.status == 1
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)


def mesh_early(ctx, desc, frames, F, dim, n, lo, hi, t0, T, dt):
    field = lcs.lcs_load_field(ctx, desc, frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    cells = np.empty(N, dtype=np.int32)
    lcs.lcs_seeds_get(ctx, seeds, None, cells)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    opts = lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    x = np.empty((dim, N), np.float32)
    st = np.empty(N, np.uint8)
    te = np.empty(N, np.float32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, st, te)
    f = np.empty(N, np.float32)
    tev = np.empty(N, np.float32)
    lcs.lcs_ftle_early(ctx, field, seeds, opts, fm, 0, f, tev)
    # each early value equals the FTLE of a run over its own horizon (same positions, same formulas)
    ms = np.rint(tev[(tev > 0) & (tev < abs(T))] / dt).astype(int)
    vals, cnt = np.unique(ms, return_counts=True)
    one = lcs.lcs_flowmap_create(ctx, seeds, 1)
    for m in vals[np.argsort(-cnt)][:3]:
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=np.sign(T) * m * dt, dt=dt), one)
        fr = np.empty(N, np.float32)
        lcs.lcs_ftle(ctx, one, 0, fr)
        at = np.rint(tev / dt).astype(int) == m
        np.testing.assert_array_equal(f[at], fr[at])
    lcs.lcs_synchronize(ctx)
    for h in (fm, one):
        lcs.lcs_free_flowmap(h)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    # against the oracle, from its own flow map of the same seeds
    x0 = oracle.seed_grid(dim, n, lo, hi)
    ocells = F.locate_seeds(x0)
    np.testing.assert_array_equal(cells, ocells)
    xT, so, teo, mg = oracle.rk4(F, x0.astype(np.float64), t0, T, dt, cells=ocells, margin=2e-3)
    sig, t_eval = oracle.ftle_early(F, n, lo, hi, (0,) * dim, t0, T, dt, xT, so, teo, cells=ocells)
    from gpu_util import check_exit_statuses
    same = check_exit_statuses(st, te, so, teo, dt, margin=mg)
    agree = np.abs(tev - t_eval.astype(np.float32)) == 0
    assert agree.mean() > 0.99, agree.mean()
    early = (t_eval < abs(T)) & (t_eval > 0)
    assert early.sum() > 200
    check_ftle(np.where(agree, f, np.nan), np.where(agree, sig, np.nan))
    return f, tev


@pytest.mark.parametrize("T", [1.0, -1.0])
def test_early_on_triangles(ctx, T):
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.05, L=10.0), nframes=40, period=1.0)
    desc = lcs.field_desc(2, times=m.times, time_periodic=True, period=m.period, kind=lcs.TRI,
                          mesh=(m.xyz, m.tets, m.nbrs))
    F = oracle.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
    mesh_early(ctx, desc, m.frames, F, 2, (100, 33), (0.05, -0.96), (9.95, 0.96), 0.2 if T > 0 else 1.2, T, 0.01)


def test_early_on_tets(ctx):
    p = inputs.pipe_frames(inputs.pipe_mesh(h=0.1, R=1.0, L=2.0), nframes=50, period=1.0, L=2.0)
    desc = lcs.field_desc(3, times=p.times, time_periodic=True, period=p.period, kind=lcs.TET,
                          mesh=(p.xyz, p.tets, p.nbrs))
    F = oracle.TetField(p.xyz, p.tets, p.nbrs, p.frames, p.times, True, p.period)
    mesh_early(ctx, desc, p.frames, F, 3, (14, 14, 18), (-0.9, -0.9, 0.1), (0.9, 0.9, 1.9), 0.3, 0.8, 0.01)
