"""GPU parity of the rectilinear RK4 path through the C ABI against the FP64 oracle
(Sec. 2 Seed / Interpolator / Flow Map / Cauchy-Green, Eq. 1-2).

Sizes: the small cases are ones the oracle finishes in seconds, with ragged seed
counts that are not multiples of any block size; the full-size cases (256x128
seeds on the 129x65x101 double gyre; 256^3 seeds on the 128^3x64 ABC flow) run
the launch configuration bench.py times and compare sampled seeds.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import (check_flowmap, check_ftle, gpu_cg_of, gpu_run, oracle_field, oracle_ftle_at, oracle_run, rect_desc,
                      round_bf16, round_fp16)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


@pytest.fixture(scope="module")
def gyre():
    return inputs.double_gyre()


@pytest.mark.parametrize("dim,n,lo,hi,periodic", [
    (2, (256, 128), (0.0, 0.0), (2.0, 1.0), (0, 0)),
    (2, (251, 7), (-1.5, 0.1), (2.5, 0.3), (0, 0)),
    (3, (17, 9, 5), (0.0, 0.0, 0.0), (2 * np.pi, 2 * np.pi, 2 * np.pi), (1, 1, 1)),
    (3, (33, 3, 40), (-1.0, 0.5, 2.0), (1.0, 0.75, 3.0), (1, 0, 1)),
])
def test_seed_lattice_bit_exact(ctx, dim, n, lo, hi, periodic):
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    assert N == int(np.prod(n))
    got = np.empty((dim, N), dtype=np.float32)
    lcs.lcs_seeds_get(ctx, seeds, got)
    dev = torch.empty((dim, N), dtype=torch.float32, device="cuda")
    lcs.lcs_seeds_get(ctx, seeds, dev)
    lcs.lcs_free_seeds(seeds)
    ref = oracle.seed_grid(dim, n, lo, hi, [0 if p else 1 for p in periodic])
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    np.testing.assert_array_equal(dev.cpu().numpy(), got)


@pytest.mark.parametrize("variant", [1, 2, 5])
@pytest.mark.parametrize("n", [(256, 128), (250, 130)])
def test_gyre_rk4_parity(ctx, gyre, variant, n):
    lo, hi, T, dt = (0.0, 0.0), (2.0, 1.0), 10.0, 0.05
    g = gpu_run(ctx, gyre, n, lo, hi, (0, 0), T, dt, variant=variant)
    o = oracle_run(gyre, n, lo, hi, (0, 0), T, dt)
    smax = float(np.nanmax(o["ftle"]))
    check_flowmap(g["xyz"][0], o["xyz"], g["status"][0], o["status"], 2.0, smax, T)
    med, p999, mx = check_ftle(g["ftle"][0], o["ftle"])
    print("gyre variant %d n=%s: FTLE median %.2e p99.9 %.2e max %.2e" % (variant, n, med, p999, mx))
    np.testing.assert_allclose(g["t_exit"][0], np.float32(T), rtol=0, atol=0)


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16])
def test_ring_slices_and_gather_agree(ctx, gyre, storage):
    # the kernels evaluate the same FP32 arithmetic: shared-memory staging (2) and per-stage time
    # slices blended once (5) must not change a bit of the one-pass kernel's result (1); the box is
    # wider than the gyre's so that tracers leave too
    kw = dict(t0=2.5, storage=storage)
    a = gpu_run(ctx, gyre, (200, 100), (-0.05, 0.0), (2.05, 1.0), (0, 0), 5.0, 0.05, variant=1, **kw)
    for v in (2, 5):
        b = gpu_run(ctx, gyre, (200, 100), (-0.05, 0.0), (2.05, 1.0), (0, 0), 5.0, 0.05, variant=v, **kw)
        np.testing.assert_array_equal(a["xyz"][0], b["xyz"][0])
        np.testing.assert_array_equal(a["status"][0], b["status"][0])
        np.testing.assert_array_equal(a["t_exit"][0], b["t_exit"][0])
        np.testing.assert_array_equal(a["ftle"][0], b["ftle"][0])


def test_gyre_backward_and_periodic_time_wrap(ctx, gyre):
    # t0 = 9, T = -10 crosses t = 0 backward; t0 = 7, T = 8 crosses the period forward
    for t0, T in ((9.0, -10.0), (7.0, 8.0)):
        n, lo, hi = (96, 48), (0.0, 0.0), (2.0, 1.0)
        g = gpu_run(ctx, gyre, n, lo, hi, (0, 0), T, 0.05, t0=t0)
        o = oracle_run(gyre, n, lo, hi, (0, 0), T, 0.05, t0=t0)
        check_flowmap(g["xyz"][0], o["xyz"], g["status"][0], o["status"], 2.0, float(np.nanmax(o["ftle"])), T)
        check_ftle(g["ftle"][0], o["ftle"])


def test_batched_jobs_equal_single_jobs(ctx, gyre):
    n, lo, hi, dt = (64, 32), (0.0, 0.0), (2.0, 1.0), 0.05
    t0s, Ts = [0.0, 2.5, 7.75, 5.0], [2.0, -4.0, 8.0, 0.0]
    b = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=(t0s, Ts))
    for j, (t0, T) in enumerate(zip(t0s, Ts)):
        s = gpu_run(ctx, gyre, n, lo, hi, (0, 0), T, dt, t0=t0)
        np.testing.assert_array_equal(b["xyz"][j], s["xyz"][0])
        np.testing.assert_array_equal(b["status"][j], s["status"][0])
        if T != 0.0:
            np.testing.assert_array_equal(b["ftle"][j], s["ftle"][0])
    # T = 0: the flow map is the identity
    np.testing.assert_array_equal(b["xyz"][3], b["seeds"])


@pytest.mark.parametrize("variant,bt,tpt", [(2, 256, 1), (4, 512, 1), (4, 256, 2), (4, 128, 2), (5, 256, 1), (5, 128, 1)])
def test_persistent_batch_equals_single_jobs(ctx, gyre, variant, bt, tpt):
    # the work-queue kernel (longest jobs first, frame ring kept across items) changes which block
    # runs a tile, never a tracer's arithmetic
    n, lo, hi, dt = (70, 37), (0.0, 0.0), (2.0, 1.0), 0.05
    t0s = [0.25 * k for k in range(6)] * 2
    Ts = [(2.0, 4.0, 8.0)[k % 3] * (1 if k < 6 else -1) for k in range(12)]
    b = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=(t0s, Ts), variant=variant, block_threads=bt,
                tracers_per_thread=tpt)
    for j in (0, 4, 7, 11):
        s = gpu_run(ctx, gyre, n, lo, hi, (0, 0), Ts[j], dt, t0=t0s[j], variant=1)
        np.testing.assert_array_equal(b["xyz"][j], s["xyz"][0])
        np.testing.assert_array_equal(b["status"][j], s["status"][0])
        np.testing.assert_array_equal(b["ftle"][j], s["ftle"][0])


def test_sliding_window_batch_against_oracle(ctx, gyre):
    # the sliding-window batch: 32 t0 spaced 0.25, forward and backward, T in {2, 4, 8}, on a small lattice
    n, lo, hi, dt = (64, 32), (0.0, 0.0), (2.0, 1.0), 0.05
    t0s = [0.25 * k for k in range(32)] * 2
    Ts = [(2.0, 4.0, 8.0)[k % 3] for k in range(32)] + [-(2.0, 4.0, 8.0)[k % 3] for k in range(32)]
    b = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=(t0s, Ts))
    for j in range(0, 64, 9):
        o = oracle_run(gyre, n, lo, hi, (0, 0), Ts[j], dt, t0=t0s[j])
        check_flowmap(b["xyz"][j], o["xyz"], b["status"][j], o["status"], 2.0, float(np.nanmax(o["ftle"])), Ts[j])
        check_ftle(b["ftle"][j], o["ftle"])


def test_graph_replay_equals_direct_launch(ctx, gyre):
    # a captured lcs_advect replays the same launches; changing the jobs captures a new graph
    n, lo, hi, dt = (96, 48), (0.0, 0.0), (2.0, 1.0), 0.05
    jobs = ([0.0, 1.0, 2.5], [2.0, -4.0, 8.0])
    a = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=jobs)
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, gyre.n, gyre.origin, gyre.spacing, gyre.periodic, gyre.times,
                                                   gyre.time_periodic, gyre.period), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 3)
    N = n[0] * n[1]
    for rep in range(4):
        o = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1], use_graph=True,
                            variant=5 if rep >= 2 else 0)
        lcs.lcs_advect(ctx, field, seeds, o, fm)
        for j in range(3):
            x = np.empty((2, N), dtype=np.float32)
            lcs.lcs_flowmap_get(ctx, fm, j, x)
            np.testing.assert_array_equal(x, a["xyz"][j])
    o2 = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=[0.5, 1.0, 2.5], job_T=jobs[1], use_graph=True)
    lcs.lcs_advect(ctx, field, seeds, o2, fm)
    x = np.empty((2, N), dtype=np.float32)
    lcs.lcs_flowmap_get(ctx, fm, 0, x)
    s = gpu_run(ctx, gyre, n, lo, hi, (0, 0), 2.0, dt, t0=0.5)
    np.testing.assert_array_equal(x, s["xyz"][0])
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)


def test_autotune_picks_valid_options_and_caches(ctx, gyre, tmp_path):
    n, lo, hi, dt = (128, 64), (0.0, 0.0), (2.0, 1.0), 0.05
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, gyre.n, gyre.origin, gyre.spacing, gyre.periodic, gyre.times,
                                                   gyre.time_periodic, gyre.period), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    jobs = ([0.25 * k for k in range(8)], [(2.0, 4.0)[k % 2] for k in range(8)])
    cache = str(tmp_path / "tune.txt")
    o = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1])
    lcs.lcs_autotune(ctx, field, seeds, o, cache)
    assert o.variant in (1, 2, 4, 5) and o.block_threads in (128, 256, 512) and o.tracers_per_thread in (1, 2)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    o2 = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1])
    lcs.lcs_autotune(ctx, field, seeds, o2, cache)          # cache hit: same choice, no new line
    assert (o2.variant, o2.block_threads, o2.tracers_per_thread) == (o.variant, o.block_threads,
                                                                     o.tracers_per_thread)
    assert len(open(cache).read().strip().splitlines()) == 1
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    # the tuned options compute the same flow map as the defaults
    a = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=jobs)
    b = gpu_run(ctx, gyre, n, lo, hi, (0, 0), None, dt, jobs=jobs, variant=o.variant, block_threads=o.block_threads,
                tracers_per_thread=o.tracers_per_thread)
    for j in range(8):
        np.testing.assert_array_equal(a["xyz"][j], b["xyz"][j])


def test_cauchy_green_matches_oracle_on_the_same_positions(ctx, gyre):
    # the oracle's flow map, rounded to FP32, into both (the library's through lcs_flowmap_set):
    # grad F and C bit-identical, lambda_max within rounding; a cut-out block of LEFT tracers makes
    # the one-sided and invalid stencils run
    n, lo, hi, T = (128, 64), (0.0, 0.0), (2.0, 1.0), 10.0
    x0 = oracle.seed_grid(2, n, lo, hi)
    xT, st, _ = oracle.rk4(oracle_field(gyre), x0.astype(np.float64), 0.0, T, 0.05)
    st = st.copy()
    st.reshape(n[1], n[0])[20:23, 40:70] = oracle.LEFT
    x32 = xT.astype(np.float32)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    g = gpu_cg_of(ctx, seeds, x32, st, T, n[0] * n[1], 2)
    lcs.lcs_free_seeds(seeds)
    G = oracle.flowmap_gradient(2, n, oracle.lattice_spacing(2, n, lo, hi), (0, 0), (0, 0),
                                x32.astype(np.float64), st)
    C = oracle.cauchy_green(G)
    np.testing.assert_array_equal(g["C"], C)
    lam, sig = oracle.ftle(C, 2, T)
    assert np.isnan(sig).sum() > 0
    np.testing.assert_array_equal(np.isfinite(g["ftle"]), np.isfinite(sig))
    ok = np.isfinite(sig)
    np.testing.assert_allclose(g["lam"][ok], lam[ok], rtol=1e-13, atol=0)
    np.testing.assert_allclose(g["ftle"][ok], sig[ok].astype(np.float32), rtol=1e-6, atol=0)


def test_affine_field_closed_form(ctx):
    # u = A x on a dyadic grid is interpolated exactly: x_N = R(hA)^N x0 up to FP32 rounding
    A = np.array([[0.125, -1.0], [1.0, -0.125]])
    g = inputs.affine_frames(A, np.zeros((2, 2)), [0.0, 0.0], (33, 33), (-4.0, -4.0), (0.25, 0.25), [0.0, 5.0])
    n, lo, hi, dt, T = (41, 37), (-1.0, -1.0), (1.0, 1.0), 0.05, 2.0
    r = gpu_run(ctx, g, n, lo, hi, (0, 0), T, dt)
    Z = dt * A
    R = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    M = np.linalg.matrix_power(R, 40)
    expect = M @ oracle.seed_grid(2, n, lo, hi).astype(np.float64)
    assert np.abs(r["xyz"][0] - expect).max() < 2e-5
    # grad F = M everywhere, so C and FTLE are constant
    lam_exact = np.linalg.eigvalsh(M.T @ M)[-1]
    assert np.abs(r["lam"][0] / lam_exact - 1).max() < 1e-4


def test_leaving_tracers_status_and_exit_time(ctx):
    # uniform u = (1, 0.2) on the box [0,1]^2 (h = 1/8): a tracer is LEFT once x > 1 + h; seeds at
    # x0 = 0.05 i cross at t = 1.125 - 0.05 i, half a step away from any step end (dt = 0.01), so the
    # FP32 and FP64 decisions agree
    g = inputs.affine_frames(np.zeros((2, 2)), np.zeros((2, 2)), [1.0, 0.2], (9, 9), (0.0, 0.0),
                             (0.125, 0.125), [0.0, 1.0])
    n, lo, hi, T, dt = (21, 11), (0.0, 0.0), (1.0, 1.0), 0.8, 0.01
    r = gpu_run(ctx, g, n, lo, hi, (0, 0), T, dt)
    o = oracle_run(g, n, lo, hi, (0, 0), T, dt)
    np.testing.assert_array_equal(r["status"][0], o["status"])
    # columns x0 >= 0.35 (14) leave through x in 10 rows; the top row (y0 = 1) leaves through y at t = 0.625
    assert (o["status"] == oracle.LEFT).sum() == 14 * 10 + 21
    np.testing.assert_allclose(r["t_exit"][0], o["t_exit"], rtol=0, atol=1e-5)
    # FTLE is NaN exactly where the oracle has no valid stencil
    np.testing.assert_array_equal(np.isnan(r["ftle"][0]), np.isnan(o["ftle"]))


def test_steady_single_frame_field(ctx, gyre):
    from dataclasses import replace
    g1 = replace(gyre, frames=gyre.frames[:1].copy(), times=np.array([0.0]), time_periodic=False, period=0.0)
    n, lo, hi = (64, 32), (0.0, 0.0), (2.0, 1.0)
    r = gpu_run(ctx, g1, n, lo, hi, (0, 0), 3.0, 0.05)
    o = oracle_run(g1, n, lo, hi, (0, 0), 3.0, 0.05)
    check_flowmap(r["xyz"][0], o["xyz"], r["status"][0], o["status"], 2.0, float(np.nanmax(o["ftle"])), 3.0)


def test_invalid_arguments_raise(ctx, gyre):
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, gyre.n, gyre.origin, gyre.spacing, times=gyre.times),
                               gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (8, 8), (0, 0), (2, 1)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    for bad in (dict(T=1.0, dt=0.0), dict(T=1.0, dt=0.3), dict(T=float("nan"), dt=0.1)):
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, **bad), fm)
        assert e.value.status == 1
    with pytest.raises(lcs.LcsError):
        lcs.lcs_flowmap_get(ctx, fm, 3, np.empty((2, 64), dtype=np.float32))
    # lcs_flowmap_set: job out of range, T zero or not finite, a status that is no tracer status
    xs, ss = np.zeros((2, 64), dtype=np.float32), np.zeros(64, dtype=np.uint8)
    for job, T, bad_st in ((1, 1.0, 0), (0, 0.0, 0), (0, float("inf"), 0), (0, 1.0, 9)):
        ss[5] = bad_st
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_flowmap_set(ctx, fm, job, xs, ss, T)
        assert e.value.status == 1
    ss[5] = 0
    lcs.lcs_flowmap_set(ctx, fm, 0, xs, ss, -2.0)     # accepted; every seed at the origin: C = 0
    C = np.empty((64, 3))
    lcs.lcs_cauchy_green(ctx, fm, 0, C)
    assert (C == 0).all()
    bad_desc = lcs.field_desc(2, (1, 5), (0, 0), (1, 1), times=[0.0])
    with pytest.raises(lcs.LcsError):
        lcs.lcs_load_field(ctx, bad_desc, np.zeros((1, 5, 1, 2), dtype=np.float32))
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)


@pytest.fixture(scope="module")
def abc_small():
    return inputs.abc(n=32, nframes=17, t_end=2.0)


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16, lcs.BF16])
def test_abc_periodic_3d_parity(ctx, abc_small, storage):
    # FP16/BF16 storage: the oracle reads the frames rounded to that format, which is exactly what the
    # kernel widens back to FP32, so the same tolerances apply
    from dataclasses import replace
    g = abc_small
    if storage == lcs.F16:
        g = replace(g, frames=round_fp16(g.frames))
    elif storage == lcs.BF16:
        g = replace(g, frames=round_bf16(g.frames))
    L = 2 * np.pi
    n, lo, hi, T, dt = (37, 30, 29), (0.0, 0.0, 0.0), (L, L, L), 2.0, 0.02
    r = gpu_run(ctx, g if storage == lcs.F32 else g, n, lo, hi, (1, 1, 1), T, dt, storage=storage)
    o = oracle_run(g, n, lo, hi, (1, 1, 1), T, dt)
    check_flowmap(r["xyz"][0], o["xyz"], r["status"][0], o["status"], L, float(np.nanmax(o["ftle"])), T)
    check_ftle(r["ftle"][0], o["ftle"])


def test_cauchy_green_3d_matches_oracle_on_the_same_positions(ctx, abc_small):
    # the oracle's flow map, rounded to FP32, into both: grad F and C bit-identical (the division by
    # 2h is correctly rounded), lambda_max within 1e-12 of the oracle's Jacobi eigenvalue, FTLE within
    # a few FP32 ulps; periodic (unwrapped positions, shift by the period) and bounded lattices
    L = 2 * np.pi
    cases = [((37, 30, 29), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1), 2.0),
             ((21, 19, 17), (0.5, 1.0, 0.25), (5.5, 4.0, 6.0), (0, 0, 0), -1.5)]
    F = oracle_field(abc_small)
    for n, lo, hi, per, T in cases:
        endpoint = [0 if p else 1 for p in per]
        x0 = oracle.seed_grid(3, n, lo, hi, endpoint)
        xT, st, _ = oracle.rk4(F, x0.astype(np.float64), 0.0, T, 0.02)
        x32 = xT.astype(np.float32)
        seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, lo, hi, per))
        g = gpu_cg_of(ctx, seeds, x32, st, T, n[0] * n[1] * n[2], 3)
        lcs.lcs_free_seeds(seeds)
        h = oracle.lattice_spacing(3, n, lo, hi, endpoint)
        period = [hi[a] - lo[a] if per[a] else 0.0 for a in range(3)]
        G = oracle.flowmap_gradient(3, n, h, per, period, x32.astype(np.float64), st)
        C = oracle.cauchy_green(G)
        np.testing.assert_array_equal(g["C"], C)
        lam, sig = oracle.ftle(C, 3, T)
        ok = np.isfinite(lam)
        np.testing.assert_array_equal(np.isfinite(g["lam"]), ok)
        np.testing.assert_allclose(g["lam"][ok], lam[ok], rtol=1e-12, atol=0)
        np.testing.assert_allclose(g["ftle"][ok], sig[ok].astype(np.float32), rtol=1e-6, atol=0)


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16, lcs.BF16])
@pytest.mark.parametrize("field_periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
def test_abc_rebundled_equals_gather(ctx, abc_small, storage, field_periodic):
    # Re-bundling tracers between episodes moves them between threads but not their arithmetic, and
    # the episode kernel's corner cache (stage 3 reusing stage 2's cell, stage 1 of the next step
    # reusing stage 4's) reads exactly what a reload would: bit-identical to the one-pass kernel.
    # A non-periodic field (the same samples on a bounded box) also sends tracers out of the box.
    from dataclasses import replace
    g = replace(abc_small, periodic=field_periodic)
    L = 2 * np.pi
    if field_periodic == (1, 1, 1):
        n, lo, hi, per = (70, 61, 64), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1)
    else:
        n, lo, hi, per = (70, 61, 64), (0.3, 0.2, 0.4), (5.5, 5.7, 5.6), (0, 0, 0)
    a = gpu_run(ctx, g, n, lo, hi, per, 2.0, 0.02, variant=1, storage=storage)
    b = gpu_run(ctx, g, n, lo, hi, per, 2.0, 0.02, variant=3, storage=storage, episode_steps=7)
    np.testing.assert_array_equal(a["status"][0], b["status"][0])
    np.testing.assert_array_equal(a["t_exit"][0], b["t_exit"][0])
    np.testing.assert_array_equal(a["xyz"][0], b["xyz"][0])
    np.testing.assert_array_equal(a["ftle"][0], b["ftle"][0])
    if field_periodic != (1, 1, 1):
        assert (a["status"][0] == lcs.TRACER_LEFT).any()


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16])
def test_abc_rebundled_batch_equals_gather(ctx, abc_small, storage):
    # several jobs (forward, backward, ragged horizons) through the re-bundled path, each restarting
    # the tracer records and the time slices: the one-pass kernel's flow maps bit for bit
    L = 2 * np.pi
    n, lo, hi = (40, 37, 35), (0.0, 0.0, 0.0), (L, L, L)
    jobs = ([0.0, 0.3, 0.5, 1.1], [1.0, -0.6, 0.84, 0.1])
    a = gpu_run(ctx, abc_small, n, lo, hi, (1, 1, 1), None, 0.02, jobs=jobs, variant=1, storage=storage)
    b = gpu_run(ctx, abc_small, n, lo, hi, (1, 1, 1), None, 0.02, jobs=jobs, variant=3, storage=storage,
                episode_steps=6)
    for j in range(len(jobs[0])):
        np.testing.assert_array_equal(a["xyz"][j], b["xyz"][j])
        np.testing.assert_array_equal(a["status"][j], b["status"][j])
        np.testing.assert_array_equal(a["ftle"][j], b["ftle"][j])


def test_abc_shift_by_period(ctx, abc_small):
    # seeds shifted by 2 pi along x: the flow map shifts by exactly 2 pi (index-only wrap)
    L = 2 * np.pi
    n = (16, 8, 8)
    a = gpu_run(ctx, abc_small, n, (0.0, 0.5, 0.5), (1.0, 1.5, 1.5), (0, 0, 0), 1.0, 0.02)
    b = gpu_run(ctx, abc_small, n, (L, 0.5, 0.5), (L + 1.0, 1.5, 1.5), (0, 0, 0), 1.0, 0.02)
    d = b["xyz"][0].astype(np.float64) - a["xyz"][0]
    assert np.abs(d[0] - (b["seeds"][0].astype(np.float64) - a["seeds"][0])).max() < 2e-5
    assert np.abs(d[1:]).max() < 2e-5


# ---------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def abc_full_oracle():
    """The oracle on the benchmark workload (256^3 seeds, 128^3 x 64-frame ABC flow, dt 0.02, T 8)
    at every 97th seed with its +-1 stencil (periodic lattice: central differences only): 172,961
    sampled seeds, about 1.2M tracers integrated.  Shared by the FP32 parity test and the FP16/BF16
    storage-error tests."""
    g = inputs.abc()
    L = 2 * np.pi
    n, lo, hi, T, dt = (256, 256, 256), (0.0, 0.0, 0.0), (L, L, L), 8.0, 0.02
    sample = np.arange(0, 256 ** 3, 97)
    o = oracle_run(g, n, lo, hi, (1, 1, 1), T, dt, sample=sample, reach=1)
    sig, lam, C = oracle_ftle_at(sample, 3, n, o["h"], (1, 1, 1), o["period"], o["xT"], o["st"], T)
    return dict(g=g, n=n, lo=lo, hi=hi, T=T, dt=dt, L=L, sample=sample, o=o, sig=sig)


def test_full_size_abc_sampled(ctx, abc_full_oracle):
    """256^3 seeds on the 128^3 x 64-frame ABC flow, dt 0.02, T 8 (the benchmark workload, its
    default launch), against the oracle at every 97th seed: statuses bit-exact, the flow-map bound at
    every integrated tracer, and the fixed-step FTLE tolerances over the 172,961 sampled seeds."""
    a = abc_full_oracle
    r = gpu_run(ctx, a["g"], a["n"], a["lo"], a["hi"], (1, 1, 1), a["T"], a["dt"])
    o, sample, sig = a["o"], a["sample"], a["sig"]
    ids = o["ids"]
    # sigma_max of the bound is the field's largest FTLE; the sampled seeds need not hold it, so the
    # larger of their oracle maximum and the library's maximum over the whole lattice is taken (the
    # two agree within the FTLE tolerance wherever both exist)
    smax = max(float(np.nanmax(sig)), float(np.nanmax(r["ftle"][0])))
    bound = 1e-5 * np.exp(smax * a["T"])
    np.testing.assert_array_equal(r["status"][0][ids], o["status_s"])
    err = np.abs(r["xyz"][0][:, ids].astype(np.float64) - o["xyz_s"]).max(axis=0) / a["L"]
    over = np.flatnonzero(err > bound)
    print("\nC2 full size, %d tracers: flow-map error / L median %.2e p99.99 %.2e max %.2e; bound %.2e "
          "(sigma_max %.3f, sampled %.3f); %d over the bound, worst ratio %.2f"
          % (len(ids), np.median(err), np.quantile(err, 0.9999), err.max(), bound, smax, float(np.nanmax(sig)),
             len(over), err.max() / bound))
    if len(over):
        w = ids[over[np.argsort(err[over])[-5:]]]
        print("  worst seeds", w, "GPU FTLE there", r["ftle"][0][w])
    assert len(over) <= 1e-4 * len(ids) and err.max() <= 10 * bound
    med, p999, mx = check_ftle(r["ftle"][0][sample], sig)
    print("\nC2 full size, %d sampled seeds: FTLE |d| median %.2e p99.9 %.2e max %.2e" % (len(sample), med, p999, mx))
    # every output finite, every tracer OK on the periodic domain
    assert np.isfinite(r["ftle"][0]).all() and (r["status"][0] == 0).all()


@pytest.mark.parametrize("storage", [lcs.F16, lcs.BF16])
def test_full_size_abc_storage_error(ctx, abc_full_oracle, storage):
    """Reduced-precision velocity storage on the benchmark workload against the FP64 oracle on the FP32
    frames at every 97th seed (the storage error itself, reported rather than gated; a loose sanity
    bound only)."""
    a = abc_full_oracle
    r = gpu_run(ctx, a["g"], a["n"], a["lo"], a["hi"], (1, 1, 1), a["T"], a["dt"], storage=storage)
    o, sample, sig = a["o"], a["sample"], a["sig"]
    d = np.abs(r["ftle"][0][sample].astype(np.float64) - sig)
    dx = np.abs(r["xyz"][0][:, o["ids"]].astype(np.float64) - o["xyz_s"]).max(axis=0)
    print("storage", storage, "FTLE |err| median %.3g p99.9 %.3g max %.3g; flow map max %.3g"
          % (np.median(d), np.quantile(d, 0.999), d.max(), dx.max()))
    assert np.median(d) <= 5e-2 and np.isfinite(r["ftle"][0]).all()


def test_full_size_sliding_window_sampled(ctx, gyre, tmp_path):
    """The batched sliding-window workload at full size -- 64 jobs (32 t0 spaced 0.25, forward and
    backward, |T| in {2, 4, 8}) of 2048x1024 seeds on the double gyre, launched as the benchmark does
    (autotuned options, CUDA graph, replayed) -- against the oracle at sampled seeds of every job."""
    n, lo, hi, dt = (2048, 1024), (0.0, 0.0), (2.0, 1.0), 0.05
    t0s = [0.25 * k for k in range(32)] * 2
    Ts = [(2.0, 4.0, 8.0)[k % 3] for k in range(32)] + [-(2.0, 4.0, 8.0)[k % 3] for k in range(32)]
    field = lcs.lcs_load_field(ctx, rect_desc(gyre), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 64)
    opts = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=t0s, job_T=Ts, use_graph=True)
    lcs.lcs_autotune(ctx, field, seeds, opts, str(tmp_path / "tune.txt"))
    for _ in range(2):                       # capture, then replay
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
    ftle = torch.empty((64, N), dtype=torch.float32, device="cuda")
    lcs.lcs_ftle(ctx, fm, -1, ftle)
    lcs.lcs_synchronize(ctx)
    rng = np.random.default_rng(33)
    x = np.empty((2, N), dtype=np.float32)
    st = np.empty(N, dtype=np.uint8)
    worst = 0.0
    # every 97th seed (21,620 per job) on eight jobs spanning |T| = 2, 4, 8, both directions and the
    # periodic time wrap; six random seeds on every other job
    dense = {0, 1, 2, 19, 32, 33, 34, 61}
    for j in range(64):
        if j in dense:
            sample = np.arange(0, N, 97)
        else:
            i, k = rng.integers(2, n[0] - 2, 6), rng.integers(2, n[1] - 2, 6)
            sample = np.unique(i + n[0] * k)
        o = oracle_run(gyre, n, lo, hi, (0, 0), Ts[j], dt, t0=t0s[j], sample=sample)
        lcs.lcs_flowmap_get(ctx, fm, j, x, st)
        ids = o["ids"]
        sig, _, _ = oracle_ftle_at(sample, 2, n, o["h"], (0, 0), o["period"], o["xT"], o["st"], Ts[j])
        check_flowmap(x[:, ids], o["xyz_s"], st[ids], o["status_s"], 2.0, float(np.nanmax(sig)), Ts[j])
        got = ftle[j, torch.from_numpy(sample).cuda()].cpu().numpy()
        if j in dense:
            check_ftle(got, sig)
        d = np.abs(got.astype(np.float64) - sig)
        d = d[np.isfinite(d)]
        assert d.max() <= 1e-3, (j, d.max())
        worst = max(worst, float(d.max()))
    print("\nC3 full size, 8 jobs x 21,620 and 56 jobs x 6 sampled seeds: FTLE |d| max %.2e" % worst)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
