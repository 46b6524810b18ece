"""Failure detection without faulting the GPU: bad inputs are refused on the host or by a
device-side check before any integration, and the capped device loops (cell walk, adaptive
step count) end with a per-tracer status and an error code that lcs_synchronize reports.
Nothing here hangs, traps or faults a GPU."""
import numpy as np
import pytest
import torch

from paper_2209_13775_gb300 import inputs, lcs

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


def tet_desc(p):
    return lcs.field_desc(3, times=p.times, time_periodic=True, period=p.period, kind=lcs.TET,
                          mesh=(p.xyz, p.tets, p.nbrs))


def test_non_finite_frames_are_refused(ctx, pipe):
    g = inputs.double_gyre(nx=17, ny=9, nframes=5, t_end=1.0)
    for bad in (np.nan, np.inf):
        fr = g.frames.copy()
        fr[3, 4, 5, 1] = bad
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, times=g.times), fr)
        assert e.value.status == 1
        # device-resident frames are checked the same way
        with pytest.raises(lcs.LcsError):
            lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, times=g.times),
                               torch.from_numpy(fr).cuda())
    fr = pipe.frames.copy()
    fr[7, 100, 2] = np.nan
    with pytest.raises(lcs.LcsError) as e:
        lcs.lcs_load_field(ctx, tet_desc(pipe), fr)
    assert e.value.status == 1
    # a field whose update brings a NaN is refused, and the context stays usable
    f = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, times=g.times), g.frames)
    fr = g.frames.copy()
    fr[0, 0, 0, 0] = np.nan
    with pytest.raises(lcs.LcsError):
        lcs.lcs_update_frames(ctx, f, fr)
    lcs.lcs_update_frames(ctx, f, g.frames)
    lcs.lcs_free_field(f)
    lcs.lcs_synchronize(ctx)


def run_tet(ctx, pipe, opts, n=(12, 12, 16), lo=(-0.6, -0.6, 0.2), hi=(0.6, 0.6, 1.8)):
    field = lcs.lcs_load_field(ctx, tet_desc(pipe), pipe.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    err = None
    try:
        lcs.lcs_synchronize(ctx)
    except lcs.LcsError as e:
        err = e.status
    st = np.empty(N, dtype=np.uint8)
    lcs.lcs_flowmap_get(ctx, fm, 0, None, st)
    lcs.lcs_synchronize(ctx)   # the error word was cleared by the first read
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return err, st


def test_walk_limit_reports_walkfail(ctx, pipe):
    err, st = run_tet(ctx, pipe, lcs.advect_opts(lcs.RK4, t0=0.0, T=0.5, dt=0.05, walk_limit=1))
    assert err == 5                                             # LCS_EWALK
    assert (st == lcs.TRACER_WALKFAIL).sum() > 0
    err, st = run_tet(ctx, pipe, lcs.advect_opts(lcs.RK4, t0=0.0, T=0.5, dt=0.05))
    assert err is None and (st != lcs.TRACER_WALKFAIL).all()


def test_step_cap_reports_maxsteps(ctx, pipe):
    err, st = run_tet(ctx, pipe, lcs.advect_opts(lcs.RK45, t0=0.0, T=1.0, rtol=1e-8, atol=1e-8, h0=1e-3,
                                                 max_steps=3))
    assert err == 6                                             # LCS_EMAXSTEPS
    assert (st == lcs.TRACER_MAXSTEPS).sum() > 0
    assert set(np.unique(st)) <= {lcs.TRACER_OK, lcs.TRACER_LEFT, lcs.TRACER_MAXSTEPS}


def test_frame_copy_wait_limit_reports_timeout(ctx):
    """A bounded device wait that gives up (Sec. 3: the frames of the current interval staged into
    on-chip memory; here the shared-memory frame ring).  With wait_limit under a microsecond a block
    tests each frame copy once when it first needs it; a copy still in flight then counts as late:
    the block stops, sets the error word and drains its copies before it exits (those waits keep the
    full 1 s bound), and lcs_synchronize reports LCS_ETIMEOUT.  Whether some copy is still in flight
    depends on timing, so the workload makes many fresh copies (64 one-step jobs whose start times
    need other frames, each block loading its own) and the call is repeated up to five times; on
    GB300 the first call already reported the timeout.  The same context then integrates normally
    and matches the oracle.  Nothing traps or spins without bound."""
    from gpu_util import check_flowmap, check_ftle, oracle_run, rect_desc

    g = inputs.double_gyre()    # 129 x 65 FP32 frames: 67 KB copies, three ring slots
    n, lo, hi, T, dt = (128, 64), (0.0, 0.0), (2.0, 1.0), 2.0, 0.05
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
    N = lcs.lcs_seeds_count(seeds)
    t0s = [0.15 * k for k in range(64)]
    fm = lcs.lcs_flowmap_create(ctx, seeds, len(t0s))
    try:
        for variant in (2, 4):
            opts = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=t0s, job_T=[dt] * len(t0s), variant=variant,
                                   wait_limit=1e-9)
            seen = []
            for attempt in range(5):
                lcs.lcs_advect(ctx, field, seeds, opts, fm)
                try:
                    lcs.lcs_synchronize(ctx)
                    seen.append(0)
                except lcs.LcsError as e:
                    seen.append(e.status)
                    break
            assert seen[-1] == 4, (variant, seen)                 # LCS_ETIMEOUT
            assert set(seen) <= {0, 4}
            lcs.lcs_synchronize(ctx)                              # the error word was cleared
        with pytest.raises(lcs.LcsError) as e:
            lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=0.0, T=T, dt=dt, wait_limit=-1.0), fm)
        assert e.value.status == 1
        # the same context, the default limit: a normal integration that matches the oracle
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=0.0, T=T, dt=dt, variant=2), fm)
        x = np.empty((2, N), np.float32)
        st = np.empty(N, np.uint8)
        f = np.empty(N, np.float32)
        lcs.lcs_flowmap_get(ctx, fm, 0, x, st)
        lcs.lcs_ftle(ctx, fm, 0, f)
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)
    o = oracle_run(g, n, lo, hi, (0, 0), T, dt)
    check_flowmap(x, o["xyz"], st, o["status"], 2.0, float(np.nanmax(o["ftle"])), T)
    check_ftle(f, o["ftle"])
