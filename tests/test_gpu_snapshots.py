"""Multi-horizon snapshots (the flow map at several horizons from one integration; Sec. 3.1 and
Sec. 4 read the flow map of an interval off the steps of a longer one): snapshot s of job j must
equal, bit for bit, a separate run with horizon min(|T_s|, |T_j|) -- the schedule of step n does
not depend on the horizon -- for every kernel variant, and match the FP64 oracle within the
fixed-step tolerances.
"""
import numpy as np
import pytest
import torch

from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import check_flowmap, check_ftle, gpu_run, oracle_run, rect_desc

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


@pytest.fixture(scope="module")
def abc_small():
    return inputs.abc(n=32, nframes=17, t_end=2.0)


def snap_run(ctx, g, n, lo, hi, periodic, jobs, snap_T, dt, **kw):
    """One lcs_advect with snapshots; returns per slot (xyz, status, t_exit, ftle), slots ordered
    as the library stores them: the jobs, then job j's snapshot s at njobs + j * nsnap + s."""
    field = lcs.lcs_load_field(ctx, rect_desc(g, kw.pop("storage", lcs.F32)), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(g.dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    nj, ns = len(jobs[0]), len(snap_T)
    fm = lcs.lcs_flowmap_create(ctx, seeds, nj * (1 + ns))
    opts = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1], snap_T=snap_T, **kw)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    out = []
    for slot in range(nj * (1 + ns)):
        x = np.empty((g.dim, N), dtype=np.float32)
        s = np.empty(N, dtype=np.uint8)
        te = np.empty(N, dtype=np.float32)
        lcs.lcs_flowmap_get(ctx, fm, slot, x, s, te)
        f = np.empty(N, dtype=np.float32)
        lcs.lcs_ftle(ctx, fm, slot, f)
        out.append((x, s, te, f))
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


def check_against_separate(ctx, g, n, lo, hi, periodic, jobs, snap_T, dt, **kw):
    got = snap_run(ctx, g, n, lo, hi, periodic, jobs, snap_T, dt, **dict(kw))
    nj, ns = len(jobs[0]), len(snap_T)
    kw.pop("use_graph", None)
    for j in range(nj):
        t0, T = jobs[0][j], jobs[1][j]
        horizons = [(j, T)] + [(nj + j * ns + s, np.sign(T) * min(snap_T[s], abs(T))) for s in range(ns)]
        for slot, Th in horizons:
            r = gpu_run(ctx, g, n, lo, hi, periodic, Th, dt, t0=t0, **kw)
            x, s, te, f = got[slot]
            np.testing.assert_array_equal(x, r["xyz"][0], err_msg="slot %d" % slot)
            np.testing.assert_array_equal(s, r["status"][0])
            np.testing.assert_array_equal(te, r["t_exit"][0])
            np.testing.assert_array_equal(f, r["ftle"][0])
    return got


@pytest.mark.parametrize("variant,bt,tpt", [(1, 256, 1), (2, 256, 1), (4, 256, 2), (5, 256, 1)])
def test_snapshots_2d_equal_separate_runs(ctx, gyre, variant, bt, tpt):
    # forward and backward jobs; the last snapshot lies beyond the short job's horizon (it holds
    # that job's final state); seeds on a box larger than the gyre's so that some tracers leave
    jobs = ([0.0, 2.5, 7.0], [3.0, -2.0, 1.0])
    check_against_separate(ctx, gyre, (67, 35), (-0.05, -0.05), (2.05, 1.05), (0, 0), jobs, [0.5, 1.25, 2.5],
                           0.05, variant=variant, block_threads=bt, tracers_per_thread=tpt)


def test_snapshots_2d_in_a_graph(ctx, gyre):
    # the snapshot slots are written by the captured launches too (capture, then replay)
    jobs = ([0.0, 1.0], [2.0, -2.0])
    ref = snap_run(ctx, gyre, (64, 32), (0.0, 0.0), (2.0, 1.0), (0, 0), jobs, [0.5, 1.0], 0.05, variant=1)
    field = lcs.lcs_load_field(ctx, rect_desc(gyre), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (64, 32), (0.0, 0.0), (2.0, 1.0)))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 6)
    opts = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=jobs[0], job_T=jobs[1], snap_T=[0.5, 1.0], variant=1,
                           use_graph=True)
    try:
        for _ in range(2):
            lcs.lcs_advect(ctx, field, seeds, opts, fm)
            for slot in range(6):
                x = np.empty((2, N), dtype=np.float32)
                lcs.lcs_flowmap_get(ctx, fm, slot, x)
                f = np.empty(N, dtype=np.float32)
                lcs.lcs_ftle(ctx, fm, slot, f)
                np.testing.assert_array_equal(x, ref[slot][0])
                np.testing.assert_array_equal(f, ref[slot][3])
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)


@pytest.mark.parametrize("storage", [lcs.F32, lcs.F16])
@pytest.mark.parametrize("field_periodic", [(1, 1, 1), (0, 0, 0)])
@pytest.mark.parametrize("variant", [1, 3])
def test_snapshots_3d_equal_separate_runs(ctx, abc_small, storage, field_periodic, variant):
    # the re-bundled path ends an episode at every snapshot step; a bounded box sends tracers out
    from dataclasses import replace
    g = replace(abc_small, periodic=field_periodic)
    L = 2 * np.pi
    if field_periodic == (1, 1, 1):
        n, lo, hi, per = (30, 27, 25), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1)
    else:
        n, lo, hi, per = (30, 27, 25), (0.3, 0.2, 0.4), (5.5, 5.7, 5.6), (0, 0, 0)
    jobs = ([0.0, 0.5], [1.0, -0.6])
    got = check_against_separate(ctx, g, n, lo, hi, per, jobs, [0.14, 0.3, 0.62], 0.02, variant=variant,
                                 storage=storage, episode_steps=5)
    if field_periodic != (1, 1, 1):
        assert (got[0][1] == lcs.TRACER_LEFT).any()


def test_snapshot_matches_oracle(ctx, gyre):
    n, lo, hi, dt = (128, 64), (0.0, 0.0), (2.0, 1.0), 0.05
    got = snap_run(ctx, gyre, n, lo, hi, (0, 0), ([0.0], [10.0]), [2.5, 5.0], dt)
    for slot, T in ((1, 2.5), (2, 5.0), (0, 10.0)):
        o = oracle_run(gyre, n, lo, hi, (0, 0), T, dt)
        x, s, te, f = got[slot]
        check_flowmap(x, o["xyz"], s, o["status"], 2.0, float(np.nanmax(o["ftle"])), T)
        check_ftle(f, o["ftle"])


def test_snapshot_options_rejected(ctx, gyre):
    field = lcs.lcs_load_field(ctx, rect_desc(gyre), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (16, 8), (0.0, 0.0), (2.0, 1.0)))
    fm = lcs.lcs_flowmap_create(ctx, seeds, 3)
    try:
        bad = [
            dict(T=2.0, dt=0.05, snap_T=[1.0, 0.5]),            # not increasing
            dict(T=2.0, dt=0.05, snap_T=[0.0125]),              # not a whole number of steps
            dict(T=2.0, dt=0.05, snap_T=[-0.5]),                # not > 0
            dict(T=2.0, dt=0.05, snap_T=[0.5, 1.0, 1.5]),       # 4 slots needed, 3 in the flow map
            dict(T=2.0, dt=0.05, snap_T=[0.05 * k for k in range(1, 10)]),   # more than MAX_SNAP
        ]
        for kw in bad:
            with pytest.raises(lcs.LcsError) as e:
                lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, **kw), fm)
            assert e.value.status == 1, kw
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK45, T=1.0, snap_T=[0.5]), fm)
        assert e.value.status == 7
        # the context stays usable
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, T=1.0, dt=0.05, snap_T=[0.5, 0.75]), fm)
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)
