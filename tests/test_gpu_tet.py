"""GPU parity of the tetrahedral path and of the adaptive integrator through the C ABI
against the FP64 oracle.

* Seed cells (Sec. 2 "Seed" on unstructured data, Sec. 3.1 local cell search): the
  lowest-id closed tet holding each FP32 seed, -1 outside.  Both sides decide with
  exact orientation predicates, so the comparison is bit-exact -- on a Kuhn mesh whose
  seeds sit on vertices, edges and faces (the tie-break runs) and on a Delaunay pipe.
* Fixed-step RK4 on tets (P1 interpolation, Sec. 3.1 walk per stage): closed form on
  affine fields; the pipe flow against the oracle with the rectilinear tolerances.
  A stage point outside the mesh freezes the tracer at the start of that step; near the
  outlet plane the FP32 and FP64 decisions can fall on either side of a stage point that
  lies within rounding of the plane, so statuses may differ there, and then only by one
  step of exit time.
* DP5(4) with one step size per warp (Sec. 2 "Flow Map", Runge-Kutta family): against
  the closed-form flow of affine fields and against the oracle's 32-lane shared-step
  mode, whose step sequence the kernel follows up to FP32 rounding of the error norms.
"""
import numpy as np
import pytest
import torch
from scipy.linalg import expm

import oracle
from meshes import kuhn_mesh, l_kuhn_mesh
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import MARGIN, check_exit_statuses, mesh_snapshots_equal_separate_runs, round_bf16, round_fp16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


@pytest.fixture(scope="module")
def pipe():
    m = inputs.pipe_mesh(h=0.1, R=1.0, L=2.0)
    return inputs.pipe_frames(m, nframes=50, period=1.0, L=2.0)


def tet_desc(xyz, tets, nbrs, times, storage=lcs.F32, time_periodic=False, period=0.0):
    return lcs.field_desc(3, times=times, time_periodic=time_periodic, period=period, storage=storage,
                          kind=lcs.TET, mesh=(xyz, tets, nbrs))


def gpu_tet(ctx, desc, frames, n, lo, hi, opts, want_steps=False):
    """Load a tet field, seed a lattice on it, advect; host arrays of job 0 (or every job)."""
    field = lcs.lcs_load_field(ctx, desc, frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    out = {"seeds": np.empty((3, N), dtype=np.float32), "cells": np.empty(N, dtype=np.int32)}
    lcs.lcs_seeds_get(ctx, seeds, out["seeds"], out["cells"])
    if opts is not None:
        njobs = max(1, opts.njobs)
        fm = lcs.lcs_flowmap_create(ctx, seeds, njobs)
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        out["xyz"], out["status"], out["t_exit"], out["steps"] = [], [], [], []
        for j in range(njobs):
            x = np.empty((3, N), dtype=np.float32)
            s = np.empty(N, dtype=np.uint8)
            te = np.empty(N, dtype=np.float32)
            lcs.lcs_flowmap_get(ctx, fm, j, x, s, te)
            out["xyz"].append(x)
            out["status"].append(s)
            out["t_exit"].append(te)
            if want_steps:
                ns = np.empty(N, dtype=np.int32)
                lcs.lcs_flowmap_steps(ctx, fm, j, ns)
                out["steps"].append(ns)
        lcs.lcs_free_flowmap(fm)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


def ora_seeds(n, lo, hi):
    return oracle.seed_grid(3, n, lo, hi)


# ------------------------------------------------------------------ seed cells

def test_seed_cells_on_kuhn_mesh_with_ties(ctx):
    # lattice step 1/2 on integer nodes: most seeds lie on a vertex, edge or face shared by several
    # tets; the lattice also reaches one cell outside the mesh on every side
    pts, tets, nbrs = kuhn_mesh(4)
    F = oracle.TetField(pts, tets, nbrs, np.zeros((1, len(pts), 3), np.float32), [0.0])
    n, lo, hi = (13, 13, 13), (-1.0, -1.0, -1.0), (5.0, 5.0, 5.0)
    fr = np.zeros((1, len(pts), 3), np.float32)
    g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0]), fr, n, lo, hi, None)
    x0 = ora_seeds(n, lo, hi)
    np.testing.assert_array_equal(g["seeds"], x0)
    want = F.locate_seeds(x0)
    np.testing.assert_array_equal(g["cells"], want)
    ties = sum(len([t for t in range(len(tets)) if F.contains(t, x0[:, i])[0]]) > 1
               for i in range(0, x0.shape[1], 3) if want[i] >= 0)
    assert ties > 150 and (want < 0).sum() > 500 and (want >= 0).sum() > 500


def test_seed_cells_on_delaunay_pipe(ctx, pipe):
    n, lo, hi = (23, 23, 31), (-1.1, -1.1, -0.1), (1.1, 1.1, 2.1)
    F = oracle.TetField(pipe.xyz, pipe.tets, pipe.nbrs, pipe.frames[:1], [0.0])
    x0 = ora_seeds(n, lo, hi)
    want = F.locate_seeds(x0)
    for nbrs in (pipe.nbrs, None):   # None: the library builds the face neighbours itself
        g = gpu_tet(ctx, tet_desc(pipe.xyz, pipe.tets, nbrs, [0.0]), pipe.frames[:1], n, lo, hi, None)
        np.testing.assert_array_equal(g["cells"], want)
    assert (want < 0).sum() > 1000 and (want >= 0).sum() > 5000


def test_seed_cells_and_stages_on_non_convex_mesh(ctx):
    # an L-shaped prism: seed cells bit-exact (ties included); u = (1, -1, 0) with one step of h = 1
    # from the y-arm puts every stage point inside but across the notch from the previous cell, so the
    # walk meets a boundary face and the bin lists must settle it: x0 + (1, -1, 0), all OK
    pts, tets, nbrs = l_kuhn_mesh(4)
    F = oracle.TetField(pts, tets, nbrs, np.zeros((1, len(pts), 3), np.float32), [0.0])
    n, lo, hi = (13, 13, 9), (-1.0, -1.0, 0.0), (5.0, 5.0, 4.0)
    g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0]), np.zeros((1, len(pts), 3), np.float32), n, lo, hi, None)
    want = F.locate_seeds(ora_seeds(n, lo, hi))
    np.testing.assert_array_equal(g["cells"], want)
    assert (want < 0).sum() > 300 and (want >= 0).sum() > 300
    fr = np.zeros((2, len(pts), 3), np.float32)
    fr[..., 0], fr[..., 1] = 1.0, -1.0
    # DP5(4) samples the line at c = 0.2, 0.3, 0.8, 8/9, 1: seeds less than 0.2 above y = 2 keep every
    # stage point out of the notch
    for method in (lcs.RK4, lcs.RK45):
        n, lo, hi = ((5, 5, 4), (1.55, 2.05, 0.5), (1.95, 2.45, 3.5)) if method == lcs.RK4 else ((5, 5, 4), (1.55, 2.02, 0.5), (1.95, 2.18, 3.5))
        opts = (lcs.advect_opts(lcs.RK4, t0=0.0, T=1.0, dt=1.0) if method == lcs.RK4 else
                lcs.advect_opts(lcs.RK45, t0=0.0, T=1.0, h0=1.0, rtol=1e-3, atol=1e-3))
        g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0, 10.0]), fr, n, lo, hi, opts)
        x0 = ora_seeds(n, lo, hi).astype(np.float64)
        assert (g["status"][0] == lcs.TRACER_OK).all()
        np.testing.assert_allclose(g["xyz"][0], x0 + np.array([[1.0], [-1.0], [0.0]]), rtol=0, atol=4e-6)


# ------------------------------------------------------------------ RK4 on tets

def test_rk4_tet_affine_rotation_closed_form(ctx):
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)                       # box [-2, 2]^3
    A = np.array([[0.0, -0.5, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.0]])   # rotation about z
    fr = np.stack([pts @ A.T, pts @ A.T]).astype(np.float32)
    n, lo, hi = (9, 9, 7), (-1.0, -1.0, -1.5), (1.0, 1.0, 1.5)
    opts = lcs.advect_opts(lcs.RK4, t0=0.0, T=2.0, dt=0.1)
    g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0, 10.0]), fr, n, lo, hi, opts)
    x0 = ora_seeds(n, lo, hi).astype(np.float64)
    Z = 0.1 * A
    R = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    want = np.linalg.matrix_power(R, 20) @ x0
    assert (g["status"][0] == lcs.TRACER_OK).all()
    err = np.abs(g["xyz"][0] - want).max()
    assert err <= 4e-6, err


def test_rk4_tet_uniform_stream_leaves_at_the_top(ctx):
    # u = (0, 0, 1) on [-2, 2]^3: a tracer at z0 is frozen at the start of the first step with a
    # stage point above z = 2; the last stage is the highest, so t_e = dt floor((2 - z0) / dt) when
    # (2 - z0) / dt is not an integer (the lattice keeps it 0.3 away from one)
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)
    fr = np.zeros((2, len(pts), 3), np.float32)
    fr[..., 2] = 1.0
    n, lo, hi = (4, 4, 9), (-1.5, -1.5, -1.73), (1.5, 1.5, 1.47)
    opts = lcs.advect_opts(lcs.RK4, t0=0.0, T=5.0, dt=0.1)
    g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0, 10.0]), fr, n, lo, hi, opts)
    x0 = ora_seeds(n, lo, hi).astype(np.float64)
    te_want = 0.1 * np.floor((2.0 - x0[2]) / 0.1)
    assert (g["status"][0] == lcs.TRACER_LEFT).all()
    np.testing.assert_allclose(g["t_exit"][0], te_want, rtol=0, atol=2e-6)
    np.testing.assert_allclose(g["xyz"][0][2], x0[2] + te_want, rtol=0, atol=4e-6)
    np.testing.assert_array_equal(g["xyz"][0][:2], x0[:2].astype(np.float32))


def _pipe_oracle(pipe, frames, n, lo, hi, t0, T, dt):
    F = oracle.TetField(pipe.xyz, pipe.tets, pipe.nbrs, frames, pipe.times, True, pipe.period)
    x0 = ora_seeds(n, lo, hi)
    cells = F.locate_seeds(x0)
    xT, st, te, mg = oracle.rk4(F, x0.astype(np.float64), t0, T, dt, cells=cells, margin=2 * MARGIN)
    return F, x0, cells, (xT, st, te), mg


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16, lcs.BF16])
def test_rk4_tet_pipe_matches_oracle(ctx, pipe, storage):
    # seeds inside the pipe; the pulsatile centreline carries many of them out through z = L
    n, lo, hi = (24, 24, 40), (-0.69, -0.69, 0.05), (0.69, 0.69, 1.95)
    frames = pipe.frames
    if storage == lcs.F16:
        frames = round_fp16(frames)
    elif storage == lcs.BF16:
        frames = round_bf16(frames)
    t0, T, dt = 0.3, 1.0, 0.01
    opts = lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt)
    g = gpu_tet(ctx, tet_desc(pipe.xyz, pipe.tets, pipe.nbrs, pipe.times, storage, True, pipe.period),
                pipe.frames, n, lo, hi, opts)
    F, x0, cells, (xT, st, te), mg = _pipe_oracle(pipe, frames, n, lo, hi, t0, T, dt)
    np.testing.assert_array_equal(g["cells"], cells)
    assert (st == oracle.LEFT).sum() > 1000 and (st == oracle.OK).sum() > 5000
    same = check_exit_statuses(g["status"][0], g["t_exit"][0], st, te, dt, margin=mg)
    err = np.abs(g["xyz"][0][:, same].astype(np.float64) - xT[:, same]).max()
    assert err <= 2e-5, err


def test_rk4_tet_backward_and_batched_jobs(ctx, pipe):
    # two jobs (one backward) in one launch equal two single-job launches bit for bit
    n, lo, hi = (16, 16, 20), (-0.6, -0.6, 0.2), (0.6, 0.6, 1.8)
    desc = tet_desc(pipe.xyz, pipe.tets, pipe.nbrs, pipe.times, lcs.F32, True, pipe.period)
    both = gpu_tet(ctx, desc, pipe.frames, n, lo, hi,
                   lcs.advect_opts(lcs.RK4, dt=0.02, job_t0=[0.1, 0.9], job_T=[0.6, -0.8]))
    one = gpu_tet(ctx, desc, pipe.frames, n, lo, hi, lcs.advect_opts(lcs.RK4, t0=0.9, T=-0.8, dt=0.02))
    np.testing.assert_array_equal(both["xyz"][1], one["xyz"][0])
    np.testing.assert_array_equal(both["status"][1], one["status"][0])
    _, _, _, (xT, st, te), mg = _pipe_oracle(pipe, pipe.frames, n, lo, hi, 0.9, -0.8, 0.02)
    same = check_exit_statuses(one["status"][0], one["t_exit"][0], st, te, 0.02, margin=mg)
    assert np.abs(one["xyz"][0][:, same] - xT[:, same]).max() <= 2e-5
    assert (st == oracle.LEFT).sum() > 50     # backwards through the inlet z = 0


def test_snapshots_on_tets(ctx, pipe):
    desc = tet_desc(pipe.xyz, pipe.tets, pipe.nbrs, pipe.times, lcs.F32, True, pipe.period)
    left = mesh_snapshots_equal_separate_runs(ctx, desc, pipe.frames, 3, (12, 12, 16), (-0.6, -0.6, 0.2),
                                              (0.6, 0.6, 1.8), ([0.1, 0.9], [0.6, -0.8]), [0.2, 0.4], 0.02)
    assert left > 50


# ------------------------------------------------------------------ DP5(4)

def rect_affine(A, b, n=(17, 17, 17), origin=(-2.0, -2.0, -2.0), spacing=(0.25, 0.25, 0.25)):
    return inputs.affine_frames(A, np.zeros((3, 3)), b, n, origin, spacing, [0.0, 100.0])


def gpu_rect_rk45(ctx, g, n, lo, hi, opts):
    desc = lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times)
    field = lcs.lcs_load_field(ctx, desc, g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, lo, hi))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    x = np.empty((3, N), dtype=np.float32)
    s = np.empty(N, dtype=np.uint8)
    te = np.empty(N, dtype=np.float32)
    ns = np.empty(N, dtype=np.int32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, s, te)
    lcs.lcs_flowmap_steps(ctx, fm, 0, ns)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return x, s, te, ns


def test_rk45_rect_affine_matches_expm_and_oracle(ctx):
    # a stable spiral with strain; trilinear interpolation of an affine field is exact, so the exact
    # flow map is expm(T A) x0 and the DP5(4) error is set by the tolerance (and FP32 rounding)
    A = np.array([[-0.25, -1.0, 0.0], [1.0, -0.25, 0.5], [0.0, -0.5, -0.125]])
    g = rect_affine(A, [0.0, 0.0, 0.0])
    n, lo, hi = (10, 9, 7), (-1.2, -1.1, -1.0), (1.2, 1.1, 1.0)
    T = 3.0
    x, s, te, ns = gpu_rect_rk45(ctx, g, n, lo, hi, lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-5,
                                                                     atol=1e-5, h0=0.01))
    x0 = ora_seeds(n, lo, hi).astype(np.float64)
    exact = expm(T * A) @ x0
    assert (s == lcs.TRACER_OK).all() and np.all(te == np.float32(T))
    assert np.abs(x - exact).max() <= 2e-4
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing)
    xo, so, teo, nso = oracle.dp45(F, x0, 0.0, T, h0=0.01, rtol=1e-5, atol=1e-5, group=32)
    assert np.abs(x - xo).max() <= 1e-4
    # every lane of a 32-seed group reports the group's count; counts track the oracle's
    N = x0.shape[1]
    for q in range(0, N, 32):
        assert len(set(ns[q:q + 32].tolist())) == 1
    assert np.abs(ns.astype(np.int64) - nso).max() <= 3


def gpu_rect2_rk45(ctx, g, n, lo, hi, opts):
    desc = lcs.field_desc(2, g.n, g.origin, g.spacing, g.periodic, g.times, g.time_periodic, g.period)
    field = lcs.lcs_load_field(ctx, desc, g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    x = np.empty((2, N), dtype=np.float32)
    s = np.empty(N, dtype=np.uint8)
    ns = np.empty(N, dtype=np.int32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, s)
    lcs.lcs_flowmap_steps(ctx, fm, 0, ns)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return x, s, ns


def test_rk45_rect2d_affine_and_gyre(ctx):
    # 2D rectilinear DP5(4): the closed form on an affine spiral (bilinear interpolation is exact), and the
    # double gyre against a converged oracle run, held to twice the oracle's own error at the same
    # tolerance (bilinear kinks at cell edges escape the embedded estimate, as P1 kinks do on meshes)
    A = np.array([[-0.25, -1.0], [1.0, -0.25]])
    g = inputs.affine_frames(A, np.zeros((2, 2)), np.zeros(2), (17, 17), (-2.0, -2.0), (0.25, 0.25), [0.0, 100.0])
    n, lo, hi, T = (12, 10), (-1.2, -1.1), (1.2, 1.1), 3.0
    x, s, ns = gpu_rect2_rk45(ctx, g, n, lo, hi, lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-5, atol=1e-5,
                                                                 h0=0.01))
    x0 = oracle.seed_grid(2, n, lo, hi).astype(np.float64)
    assert (s == lcs.TRACER_OK).all()
    assert np.abs(x - expm(T * A) @ x0).max() <= 2e-4
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing)
    xo, _, _, nso = oracle.dp45(F, x0, 0.0, T, h0=0.01, rtol=1e-5, atol=1e-5, group=32)
    assert np.abs(x - xo).max() <= 1e-4 and np.abs(ns.astype(np.int64) - nso).max() <= 3
    gy = inputs.double_gyre()
    n, lo, hi, T = (64, 32), (0.0, 0.0), (2.0, 1.0), 5.0
    x, s, ns = gpu_rect2_rk45(ctx, gy, n, lo, hi, lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-6, atol=1e-6,
                                                                  h0=0.01))
    F = oracle.RectField(gy.frames, gy.times, gy.origin, gy.spacing, gy.periodic, gy.time_periodic, gy.period)
    x0 = oracle.seed_grid(2, n, lo, hi).astype(np.float64)
    xo, so, _, nso = oracle.dp45(F, x0, 0.0, T, h0=0.01, rtol=1e-6, atol=1e-6, group=32)
    xr, sr, _, _ = oracle.dp45(F, x0, 0.0, T, h0=0.01, rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(s, so)
    ok = (so == oracle.OK) & (sr == oracle.OK)
    e_ora = np.abs(xo[:, ok] - xr[:, ok]).max(axis=0)
    e_gpu = np.abs(x[:, ok] - xr[:, ok]).max(axis=0)
    assert np.median(e_gpu) <= 2 * np.median(e_ora) + 1e-6, (np.median(e_gpu), np.median(e_ora))
    assert e_gpu.max() <= 2 * e_ora.max() + 1e-5, (e_gpu.max(), e_ora.max())
    steps = np.abs(ns.astype(np.int64) - nso)
    assert np.median(steps) <= 1 and steps.max() <= 10


def test_rk45_rect_uniform_stream_leaves(ctx):
    # a uniform stream has a zero error estimate up to FP32 rounding of the interpolation weights
    # (about 1e-3 of a 1e-6 tolerance, 1e-6 of a 1e-3 one): at tolerance 1e-3 every step grows
    # fivefold (0.01, 0.05, 0.25, 1.25) and a seed at x = 0.5 on the box [0, 1]^3 ends its fourth
    # step at x = 2.06, past x = 1.125: LEFT at t = 1.56
    g = inputs.affine_frames(np.zeros((3, 3)), np.zeros((3, 3)), [1.0, 0.0, 0.0], (9, 9, 9), (0, 0, 0),
                             (0.125, 0.125, 0.125), [0.0, 10.0])
    n, lo, hi = (1, 5, 5), (0.5, 0.0, 0.0), (0.5, 1.0, 1.0)
    x, s, te, ns = gpu_rect_rk45(ctx, g, n, lo, hi, lcs.advect_opts(lcs.RK45, T=10.0, h0=0.01, rtol=1e-3,
                                                                     atol=1e-3))
    assert (s == lcs.TRACER_LEFT).all() and (ns == 4).all()
    np.testing.assert_allclose(te, 1.56, rtol=0, atol=2e-6)
    np.testing.assert_allclose(x[0], 2.06, rtol=0, atol=4e-6)
    # at tolerance 1e-6 the steps grow more slowly; the frozen position still equals the elapsed time
    x, s, te, ns = gpu_rect_rk45(ctx, g, n, lo, hi, lcs.advect_opts(lcs.RK45, T=-10.0, h0=0.01))
    assert (s == lcs.TRACER_LEFT).all() and (ns >= 4).all()
    np.testing.assert_allclose(x[0] - 0.5, te, rtol=0, atol=2e-6)
    assert (x[0] < -0.125).all()


def test_rk45_tet_affine_closed_form(ctx):
    pts, tets, nbrs = kuhn_mesh(4)
    pts = pts - np.float32(2.0)
    A = np.array([[-0.125, -0.5, 0.0], [0.5, -0.125, 0.0], [0.0, 0.0, -0.25]])
    fr = np.stack([pts @ A.T, pts @ A.T]).astype(np.float32)
    n, lo, hi = (8, 8, 8), (-1.5, -1.5, -1.5), (1.5, 1.5, 1.5)
    T = 4.0
    opts = lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-5, atol=1e-5, h0=0.05)
    g = gpu_tet(ctx, tet_desc(pts, tets, nbrs, [0.0, 10.0]), fr, n, lo, hi, opts, want_steps=True)
    x0 = ora_seeds(n, lo, hi).astype(np.float64)
    assert (g["status"][0] == lcs.TRACER_OK).all()
    assert np.abs(g["xyz"][0] - expm(T * A) @ x0).max() <= 2e-4
    F = oracle.TetField(pts, tets, nbrs, fr, [0.0, 10.0])
    xo, so, _, nso = oracle.dp45(F, x0, 0.0, T, h0=0.05, rtol=1e-5, atol=1e-5, group=32,
                                 cells=F.locate_seeds(x0))
    assert np.abs(g["xyz"][0] - xo).max() <= 1e-4
    assert np.abs(g["steps"][0].astype(np.int64) - nso).max() <= 3


def test_rk45_tet_pipe_matches_oracle(ctx, pipe):
    n, lo, hi = (16, 16, 24), (-0.65, -0.65, 0.1), (0.65, 0.65, 1.9)
    t0, T = 0.2, 1.0
    opts = lcs.advect_opts(lcs.RK45, t0=t0, T=T, rtol=1e-6, atol=1e-6, h0=0.01)
    g = gpu_tet(ctx, tet_desc(pipe.xyz, pipe.tets, pipe.nbrs, pipe.times, lcs.F32, True, pipe.period),
                pipe.frames, n, lo, hi, opts, want_steps=True)
    F = oracle.TetField(pipe.xyz, pipe.tets, pipe.nbrs, pipe.frames, pipe.times, True, pipe.period)
    x0 = ora_seeds(n, lo, hi)
    cells = F.locate_seeds(x0)
    xo, so, teo, nso = oracle.dp45(F, x0.astype(np.float64), t0, T, h0=0.01, rtol=1e-6, atol=1e-6,
                                   group=32, cells=cells)
    st = g["status"][0]
    assert (so == oracle.LEFT).sum() > 300 and (so == oracle.OK).sum() > 2000
    diff = st != so
    assert diff.mean() <= 5e-3, diff.sum()
    ok = (st == so) & (so == oracle.OK)
    assert np.abs(g["xyz"][0][:, ok] - xo[:, ok]).max() <= 2e-4
    steps_ok = np.abs(g["steps"][0].astype(np.int64) - nso)
    assert np.median(steps_ok) <= 1 and steps_ok.max() <= 10


def test_full_size_pipe_rk45_sampled(ctx):
    """The benchmark's tetrahedral workload at full size -- the 2.36M-tet pipe, 64x64x512 seeds,
    DP5(4) rtol = atol = 1e-6, T = 1, the same launch options -- against the oracle at sampled seeds.
    The kernel shares one step size per warp of 32 consecutive seeds, so the oracle integrates, in
    its 32-lane mode, every whole group holding one of 120 sampled seeds or a member of their
    stencils: at least 1000 groups (about 34K tracers)."""
    mesh = inputs.pipe_frames(inputs.pipe_mesh(), nframes=50, period=1.0)
    n, lo, hi, T = (64, 64, 512), (-1.0, -1.0, 0.0), (1.0, 1.0, 10.0), 1.0
    field = lcs.lcs_load_field(ctx, tet_desc(mesh.xyz, mesh.tets, mesh.nbrs, mesh.times, lcs.F32, True,
                                             mesh.period), mesh.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-6, atol=1e-6, h0=0.01), fm)
    cells = np.empty(N, dtype=np.int32)
    lcs.lcs_seeds_get(ctx, seeds, None, cells)
    x = np.empty((3, N), dtype=np.float32)
    st = np.empty(N, dtype=np.uint8)
    te = np.empty(N, dtype=np.float32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x, st, te)
    ftle = np.empty(N, dtype=np.float32)
    lcs.lcs_ftle(ctx, fm, 0, ftle)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    assert N == 64 * 64 * 512 and (st == lcs.TRACER_WALKFAIL).sum() == 0
    # samples: seeds whose six neighbours exist on the lattice, spread over the pipe's length
    rng = np.random.default_rng(44)
    cand = np.flatnonzero(np.isfinite(ftle))
    ix, iy, iz = cand % 64, (cand // 64) % 64, cand // 4096
    cand = cand[(ix > 1) & (ix < 62) & (iy > 1) & (iy < 62) & (iz > 1) & (iz < 510)]
    sample = np.sort(rng.choice(cand, 120, replace=False))
    # +-1 and +-2 along each axis: near the wall a one-sided difference needs the second neighbour
    stencil = np.concatenate([sample + s * o for o in (1, 64, 4096) for s in (-2, -1, 0, 1, 2)])
    groups = np.unique(stencil // 32)
    assert len(groups) >= 1000
    ids = (groups[:, None] * 32 + np.arange(32)[None, :]).ravel()
    x0 = oracle.seed_grid(3, n, lo, hi)[:, ids]
    F = oracle.TetField(mesh.xyz, mesh.tets, mesh.nbrs, mesh.frames, mesh.times, True, mesh.period)
    oc = F.locate_seeds(x0)
    np.testing.assert_array_equal(oc, cells[ids])          # seed cells bit-exact
    xo, so, teo, _ = oracle.dp45(F, x0.astype(np.float64), 0.0, T, h0=0.01, rtol=1e-6, atol=1e-6,
                                 group=32, cells=oc)
    diff = st[ids] != so                                   # exits decided a step apart, near the outlet
    assert diff.mean() <= 2e-2, diff.sum()
    # P1 velocity has kinks across every face, which the embedded error estimate does not see, so
    # the oracle itself is off the converged flow by up to a few 1e-4 at rtol 1e-6; the kernel (FP32
    # error norms, so its own accept/reject sequence) is held to the oracle's accuracy against a
    # converged run (rtol 1e-10), as on the small pipe and the stenosis
    # (the converged run, the costly part, on every eighth integrated group)
    sub = (np.arange(len(ids)) // 32) % 8 == 0
    xr, sr, _, _ = oracle.dp45(F, x0[:, sub].astype(np.float64), 0.0, T, h0=0.01, rtol=1e-10, atol=1e-10,
                               cells=oc[sub])
    ok = (st[ids][sub] == so[sub]) & (so[sub] == oracle.OK) & (sr == oracle.OK)
    assert ok.sum() > 2000
    e_ora = np.abs(xo[:, sub][:, ok] - xr[:, ok]).max(axis=0)
    e_gpu = np.abs(x[:, ids][:, sub][:, ok] - xr[:, ok]).max(axis=0)
    assert np.median(e_gpu) <= 2 * np.median(e_ora) + 1e-6, (np.median(e_gpu), np.median(e_ora))
    assert e_gpu.max() <= 2 * e_ora.max() + 1e-5, (e_gpu.max(), e_ora.max())
    # FTLE at the samples from the oracle's own flow map of the integrated groups.  Weyl's inequality
    # bounds the change of grad F's largest singular value s_max by the norm of the change of grad F;
    # each column of that change is a combination of position differences over 2h (central: weights
    # 1, 1; one-sided: 3, 4, 1), so with E the largest position difference over a sample's stencil,
    # |d sigma| <= ln(1 + 4 sqrt(3) E / h_min) / T, as s_max >= 1 for this volume-preserving flow
    h = oracle.lattice_spacing(3, n, lo, hi)
    xT = np.zeros((3, N))
    sT = np.full(N, oracle.LEFT, dtype=np.uint8)
    xT[:, ids] = xo
    sT[ids] = so
    G = oracle.flowmap_gradient(3, n, h, (0, 0, 0), (0, 0, 0), xT, sT)[sample]
    _, sig = oracle.ftle(oracle.cauchy_green(G), 3, T)
    members = stencil.reshape(15, len(sample))
    agree = (st[members] == sT[members]).all(axis=0)
    use = agree & np.isfinite(sig)
    assert use.sum() >= 90
    E = np.abs(x[:, members].astype(np.float64) - xT[:, members]).max(axis=(0, 1))
    bound = np.log1p(4 * np.sqrt(3) * E / min(h)) / T + 1e-6
    d = np.abs(ftle[sample].astype(np.float64) - sig)
    print("\nC4 full size, %d sampled seeds: FTLE |d| median %.2e max %.2e (bound median %.2e)"
          % (use.sum(), np.median(d[use]), d[use].max(), np.median(bound[use])))
    assert (d[use] <= bound[use]).all(), (d[use] - bound[use]).max()


# ------------------------------------------------------------------ errors

def test_rk45_and_tet_argument_errors(ctx, pipe):
    g2 = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g2.n, g2.origin, g2.spacing, times=g2.times), g2.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 8), (0, 0), (2, 1)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    with pytest.raises(lcs.LcsError) as e:
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK45, T=1.0, snap_T=[0.5]), fm)
    assert e.value.status == 7                      # LCS_EUNSUPPORTED: no adaptive snapshots
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.1), fm)
    with pytest.raises(lcs.LcsError) as e:          # no adaptive integration wrote step counts
        lcs.lcs_flowmap_steps(ctx, fm, 0, np.empty(64, dtype=np.int32))
    assert e.value.status == 1
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    # tet fields: seeds must be located on that field; bad node ids are rejected at load
    desc = tet_desc(pipe.xyz, pipe.tets, pipe.nbrs, pipe.times, lcs.F32, True, pipe.period)
    tf = lcs.lcs_load_field(ctx, desc, pipe.frames)
    plain = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, (4, 4, 4), (-0.5, -0.5, 0.5), (0.5, 0.5, 1.5)))
    fm = lcs.lcs_flowmap_create(ctx, plain, 1)
    with pytest.raises(lcs.LcsError) as e:
        lcs.lcs_advect(ctx, tf, plain, lcs.advect_opts(lcs.RK4, T=0.1, dt=0.01), fm)
    assert e.value.status == 1
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(plain)
    lcs.lcs_free_field(tf)
    bad = pipe.tets.copy()
    bad[5, 2] = len(pipe.xyz)
    with pytest.raises(lcs.LcsError) as e:
        lcs.lcs_load_field(ctx, tet_desc(pipe.xyz, bad, None, pipe.times), pipe.frames)
    assert e.value.status == 1
