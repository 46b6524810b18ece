"""grad F by the variational equations (Sec. 1: the linearised flow map as the alternative to
differencing the seed grid) through lcs_advect(variational=True), lcs_flowmap_grad and
lcs_ftle_variational:

* the positions, status and exit times are bit-identical to the plain fixed-step RK4 kernel's (the
  position part of the integration is the same arithmetic);
* grad F against the oracle's FP64 rk4_var within the fixed-step tolerances, and the FTLE formed
  from it against the oracle's;
* C bit-identical to the oracle's Eq. 1 applied to the GPU's own FP32 grad F;
* a linear flow (interpolation exact): grad F = R(hA)^N, R the RK4 stability polynomial;
* invalid combinations are rejected and leave the context usable.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import check_ftle, rect_desc, round_fp16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


def var_run(ctx, g, n, lo, hi, periodic, dt, jobs, storage=lcs.F32, **kw):
    """Variational and plain (variant 1) runs of the same jobs; host arrays per job."""
    dim = g.dim
    field = lcs.lcs_load_field(ctx, rect_desc(g, storage), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    nj = len(jobs[0])
    out = {"N": N, "seeds": np.empty((dim, N), dtype=np.float32)}
    lcs.lcs_seeds_get(ctx, seeds, out["seeds"])
    out["x0_oracle"] = oracle.seed_grid(dim, n, lo, hi, [0 if p else 1 for p in periodic])
    np.testing.assert_array_equal(out["seeds"], out["x0_oracle"])
    for tag, extra in (("var", dict(variational=True, **kw)), ("plain", dict(variant=1))):
        fm = lcs.lcs_flowmap_create(ctx, seeds, nj)
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1], **extra),
                       fm)
        res = []
        for j in range(nj):
            r = {"x": np.empty((dim, N), dtype=np.float32), "st": np.empty(N, dtype=np.uint8),
                 "te": np.empty(N, dtype=np.float32)}
            lcs.lcs_flowmap_get(ctx, fm, j, r["x"], r["st"], r["te"])
            if tag == "var":
                r["M"] = np.empty((N, dim, dim), dtype=np.float32)
                lcs.lcs_flowmap_grad(ctx, fm, j, r["M"])
                r["ftle"] = np.empty(N, dtype=np.float32)
                r["lam"] = np.empty(N)
                r["C"] = np.empty((N, 3 if dim == 2 else 6))
                lcs.lcs_ftle_variational(ctx, fm, j, r["ftle"], r["lam"], r["C"])
                # device outputs give the same values
                fd = torch.empty(N, dtype=torch.float32, device="cuda")
                lcs.lcs_ftle_variational(ctx, fm, j, fd)
                Md = torch.empty((N, dim, dim), dtype=torch.float32, device="cuda")
                lcs.lcs_flowmap_grad(ctx, fm, j, Md)
                lcs.lcs_synchronize(ctx)
                np.testing.assert_array_equal(fd.cpu().numpy(), r["ftle"])
                np.testing.assert_array_equal(Md.cpu().numpy(), r["M"])
            res.append(r)
        lcs.lcs_synchronize(ctx)
        lcs.lcs_free_flowmap(fm)
        out[tag] = res
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


def check_grad(M, Mo, ok):
    """FP32 grad F against the FP64 oracle's, per OK seed, relative to the tensor's size: median
    <= 1e-5, 99th percentile <= 1e-3, all <= 5e-2.  The interpolant's Jacobian jumps across cell
    faces, so a stage that lands on the other side of a face in FP32 than in FP64 takes a different
    J for that stage: an error of order h |dJ| |M| rather than of the rounding, for the few tracers
    (about the position error over the spacing, per stage and axis) that pass that close to a face."""
    rel = np.abs(M[ok] - Mo[ok]).max(axis=(1, 2)) / np.abs(Mo[ok]).max(axis=(1, 2))
    print(f"grad F rel err: median {np.median(rel):.3g} p99 {np.quantile(rel, 0.99):.3g} "
          f"p99.9 {np.quantile(rel, 0.999):.3g} max {rel.max():.3g} n {rel.size}")
    assert np.median(rel) <= 1e-5, np.median(rel)
    assert np.quantile(rel, 0.99) <= 1e-3, np.quantile(rel, 0.99)
    assert rel.max() <= 5e-2, rel.max()


def check_against_oracle(g, r, dt, jobs):
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    x0 = r["x0_oracle"].astype(np.float64)
    for j, (t0, T) in enumerate(zip(*jobs)):
        v, p = r["var"][j], r["plain"][j]
        # the position part: the plain kernel's, bit for bit
        np.testing.assert_array_equal(v["x"], p["x"])
        np.testing.assert_array_equal(v["st"], p["st"])
        np.testing.assert_array_equal(v["te"], p["te"])
        xT, Mo, sto, _ = oracle.rk4_var(F, x0, t0, T, dt)
        np.testing.assert_array_equal(v["st"], sto)
        ok = sto == oracle.OK
        assert ok.sum() > 0
        check_grad(v["M"], Mo, ok)
        lam, sig = oracle.ftle(oracle.cauchy_green(np.where(ok[:, None, None], Mo, np.nan)), g.dim, T)
        check_ftle(v["ftle"], sig)
        assert np.isnan(v["ftle"][~ok]).all()


def test_variational_gyre(ctx):
    g = inputs.double_gyre()
    n, lo, hi, dt = (96, 48), (0.0, 0.0), (2.0, 1.0), 0.05
    jobs = ([0.0, 2.5], [5.0, 4.0])
    r = var_run(ctx, g, n, lo, hi, (0, 0), dt, jobs)
    check_against_oracle(g, r, dt, jobs)


def test_variational_gyre_backward_with_exits(ctx):
    # the double gyre cut at x = 1.5: tracers leave, their grad F and FTLE are NaN
    g = inputs.double_gyre()
    g = replace(g, frames=np.ascontiguousarray(g.frames[:, :, :97]))
    n, lo, hi, dt = (90, 60), (0.0, 0.0), (1.5, 1.0), 0.05
    jobs = ([6.0], [-6.0])
    r = var_run(ctx, g, n, lo, hi, (0, 0), dt, jobs)
    assert (r["var"][0]["st"] != 0).sum() > 100
    check_against_oracle(g, r, dt, jobs)


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16])
def test_variational_abc(ctx, storage):
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    if storage == lcs.F16:
        g = replace(g, frames=round_fp16(g.frames))
    L = 2 * np.pi
    n, lo, hi, dt = (21, 19, 18), (0.0, 0.0, 0.0), (L, L, L), 0.02
    jobs = ([0.0], [2.0])
    r = var_run(ctx, g, n, lo, hi, (1, 1, 1), dt, jobs, storage=storage)
    check_against_oracle(g, r, dt, jobs)


def test_variational_abc_bounded(ctx):
    # non-periodic 3D: tracers leave the box
    g = replace(inputs.abc(n=32, nframes=17, t_end=2.0), periodic=(0, 0, 0))
    n, lo, hi, dt = (20, 18, 17), (0.3, 0.2, 0.4), (5.5, 5.7, 5.6), 0.02
    jobs = ([0.0], [1.5])
    r = var_run(ctx, g, n, lo, hi, (0, 0, 0), dt, jobs)
    assert (r["var"][0]["st"] != 0).sum() > 100
    check_against_oracle(g, r, dt, jobs)


def _R(Z):
    I = np.eye(len(Z))
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


@pytest.mark.parametrize("dim", [2, 3])
def test_variational_linear_flow(ctx, dim):
    rng = np.random.default_rng(60 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.4 * 16) / 16
    nn = (33,) * dim
    g = inputs.affine_frames(A, np.zeros((dim, dim)), np.zeros(dim), nn, (-4.0,) * dim, (0.25,) * dim, [0.0, 5.0])
    n = (24,) * dim
    dt, T = 0.0625, 1.0
    r = var_run(ctx, g, n, (-1.0,) * dim, (1.0,) * dim, (0,) * dim, dt, ([0.0], [T]))
    v = r["var"][0]
    assert (v["st"] == 0).all()
    want = np.linalg.matrix_power(_R(dt * A), int(round(T / dt)))
    err = np.abs(v["M"] - want[None]).max() / np.abs(want).max()
    assert err <= 1e-5, err


def test_variational_rejects(ctx):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 4), (0.0, 0.0), (2.0, 1.0)))
    aux = lcs.lcs_seed_aux(ctx, seeds, [0.01, 0.01])
    fm = lcs.lcs_flowmap_create(ctx, seeds, 2)
    fa = lcs.lcs_flowmap_create(ctx, aux, 1)
    f = np.empty(32, dtype=np.float32)
    M = np.empty((32, 2, 2), dtype=np.float32)
    try:
        for kw in (dict(method=lcs.RK45, T=1.0), dict(method=lcs.RK4, T=1.0, dt=0.05, snap_T=[0.5])):
            with pytest.raises(lcs.LcsError) as e:
                lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(variational=True, **kw), fm)
            assert e.value.status == 7, kw
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_advect(ctx, field, aux, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05, variational=True), fa)
        assert e.value.status == 7
        # a flow map no variational run wrote
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05), fm)
        for call in (lambda: lcs.lcs_flowmap_grad(ctx, fm, 0, M), lambda: lcs.lcs_ftle_variational(ctx, fm, 0, f)):
            with pytest.raises(lcs.LcsError) as e:
                call()
            assert e.value.status == 1
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05, variational=True), fm)
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_flowmap_grad(ctx, fm, 2, M)
        assert e.value.status == 1
        lcs.lcs_flowmap_grad(ctx, fm, 0, M)
        # a later plain run invalidates the gradient
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05), fm)
        with pytest.raises(lcs.LcsError):
            lcs.lcs_ftle_variational(ctx, fm, 0, f)
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_flowmap(fa)
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(aux)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)


def grad_run(ctx, g, n, lo, hi, periodic, dt, t0, T, storage, variant, variational):
    field = lcs.lcs_load_field(ctx, rect_desc(g, storage), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt, variant=variant,
                                                      variational=variational), fm)
    out = {"x": np.empty((g.dim, N), dtype=np.float32), "st": np.empty(N, dtype=np.uint8),
           "te": np.empty(N, dtype=np.float32)}
    lcs.lcs_flowmap_get(ctx, fm, 0, out["x"], out["st"], out["te"])
    if variational:
        out["M"] = np.empty((N, g.dim, g.dim), dtype=np.float32)
        lcs.lcs_flowmap_grad(ctx, fm, 0, out["M"])
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


@pytest.mark.parametrize("storage,bounded", [(lcs.F32, False), (lcs.F16, False), (lcs.F32, True)])
def test_variational_episodes_equal_one_pass(ctx, storage, bounded):
    # the re-bundled episodes (variant 3) carry M with the tracer records through the sort; the
    # Jacobian comes from the same time-slice corners with the one-pass kernel's products, so M, x,
    # status and exit times equal the one-pass variational kernel's bit for bit, and x the plain
    # episode path's
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    if storage == lcs.F16:
        g = replace(g, frames=round_fp16(g.frames))
    L = 2 * np.pi
    if bounded:
        g = replace(g, periodic=(0, 0, 0))
        n, lo, hi, per, T = (20, 18, 17), (0.3, 0.2, 0.4), (5.5, 5.7, 5.6), (0, 0, 0), 1.5
    else:
        n, lo, hi, per, T = (21, 19, 18), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1), 2.0
    ep = grad_run(ctx, g, n, lo, hi, per, 0.02, 0.0, T, storage, 3, True)
    one = grad_run(ctx, g, n, lo, hi, per, 0.02, 0.0, T, storage, 1, True)
    plain = grad_run(ctx, g, n, lo, hi, per, 0.02, 0.0, T, storage, 3, False)
    for k in ("x", "st", "te", "M"):
        np.testing.assert_array_equal(ep[k], one[k])
    for k in ("x", "st", "te"):
        np.testing.assert_array_equal(ep[k], plain[k])
    if bounded:
        assert (ep["st"] != 0).sum() > 100


# ------------------------------------------------------------------ meshes

def mesh_var_run(ctx, desc, frames, dim, n, lo, hi, t0, T, dt):
    field = lcs.lcs_load_field(ctx, desc, frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    out = {"seeds": np.empty((dim, N), dtype=np.float32), "cells": np.empty(N, dtype=np.int32),
           "n": n, "lo": lo, "hi": hi}
    lcs.lcs_seeds_get(ctx, seeds, out["seeds"], out["cells"])
    for tag, var in (("var", True), ("plain", False)):
        fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt, variational=var), fm)
        r = {"x": np.empty((dim, N), dtype=np.float32), "st": np.empty(N, dtype=np.uint8),
             "te": np.empty(N, dtype=np.float32)}
        lcs.lcs_flowmap_get(ctx, fm, 0, r["x"], r["st"], r["te"])
        if var:
            r["M"] = np.empty((N, dim, dim), dtype=np.float32)
            lcs.lcs_flowmap_grad(ctx, fm, 0, r["M"])
            r["ftle"] = np.empty(N, dtype=np.float32)
            lcs.lcs_ftle_variational(ctx, fm, 0, r["ftle"])
        lcs.lcs_synchronize(ctx)
        lcs.lcs_free_flowmap(fm)
        out[tag] = r
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


def check_mesh_against_oracle(F, r, t0, T, dt, dim):
    v, p = r["var"], r["plain"]
    for k in ("x", "st", "te"):
        np.testing.assert_array_equal(v[k], p[k])
    x0 = oracle.seed_grid(dim, r["n"], r["lo"], r["hi"])
    np.testing.assert_array_equal(r["seeds"], x0)
    cells = F.locate_seeds(x0)
    np.testing.assert_array_equal(r["cells"], cells)
    _, Mo, so, teo = oracle.rk4_var(F, x0.astype(np.float64), t0, T, dt, cells=cells)
    _, so2, teo2, mg = oracle.rk4(F, x0.astype(np.float64), t0, T, dt, cells=cells, margin=2e-3)
    np.testing.assert_array_equal(so2, so)
    from gpu_util import check_exit_statuses
    same = check_exit_statuses(v["st"], v["te"], so, teo, dt, margin=mg)
    ok = same & (so == oracle.OK)
    assert ok.sum() > 500
    check_grad(v["M"], Mo, ok)
    _, sig = oracle.ftle(oracle.cauchy_green(np.where(ok[:, None, None], Mo, np.nan)), dim, T)
    both = ok & np.isfinite(v["ftle"])
    check_ftle(np.where(both, v["ftle"], np.nan), np.where(both, sig, np.nan))


def test_variational_triangles(ctx):
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.05, L=10.0), nframes=40, period=1.0)
    desc = lcs.field_desc(2, times=m.times, time_periodic=True, period=m.period, kind=lcs.TRI,
                          mesh=(m.xyz, m.tets, m.nbrs))
    n, lo, hi, t0, T, dt = (100, 33), (0.05, -0.96), (9.95, 0.96), 0.2, 0.6, 0.01
    r = mesh_var_run(ctx, desc, m.frames, 2, n, lo, hi, t0, T, dt)
    F = oracle.TriField(m.xyz, m.tets, m.nbrs, m.frames, m.times, True, m.period)
    check_mesh_against_oracle(F, r, t0, T, dt, 2)


def test_variational_tets(ctx):
    p = inputs.pipe_frames(inputs.pipe_mesh(h=0.1, R=1.0, L=2.0), nframes=50, period=1.0, L=2.0)
    desc = lcs.field_desc(3, times=p.times, time_periodic=True, period=p.period, kind=lcs.TET,
                          mesh=(p.xyz, p.tets, p.nbrs))
    n, lo, hi, t0, T, dt = (16, 16, 20), (-0.6, -0.6, 0.2), (0.6, 0.6, 1.8), 0.3, 0.8, 0.01
    r = mesh_var_run(ctx, desc, p.frames, 3, n, lo, hi, t0, T, dt)
    F = oracle.TetField(p.xyz, p.tets, p.nbrs, p.frames, p.times, True, p.period)
    check_mesh_against_oracle(F, r, t0, T, dt, 3)


@pytest.mark.parametrize("dim", [2, 3])
def test_variational_mesh_linear_flow(ctx, dim):
    from meshes import kuhn_mesh, tri_grid_mesh
    rng = np.random.default_rng(70 + dim)
    A = np.round(rng.normal(size=(dim, dim)) * 0.3 * 16) / 16
    if dim == 2:
        pts, cells, nbrs = tri_grid_mesh(8)
        pts = (pts - np.float32(4.0)) * np.float32(0.5)
        kind = lcs.TRI
    else:
        pts, cells, nbrs = kuhn_mesh(4)
        pts = pts - np.float32(2.0)
        kind = lcs.TET
    fr = np.stack([pts @ A.T, pts @ A.T]).astype(np.float32)
    desc = lcs.field_desc(dim, times=[0.0, 10.0], kind=kind, mesh=(pts, cells, nbrs))
    dt, T = 0.0625, 1.0
    r = mesh_var_run(ctx, desc, fr, dim, (9,) * dim, (-0.6,) * dim, (0.6,) * dim, 0.0, T, dt)
    v = r["var"]
    assert (v["st"] == 0).all()
    want = np.linalg.matrix_power(_R(dt * A), int(round(T / dt)))
    err = np.abs(v["M"] - want[None]).max() / np.abs(want).max()
    assert err <= 1e-5, err
