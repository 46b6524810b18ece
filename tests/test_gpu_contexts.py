"""Handles used from two contexts on one device: a loader context on its own stream refreshes
one field of a double buffer (lcs_update_frames) while another context advects with the other
field, and results are read back on the loader stream once their lcs_ftle is done -- the
pipelined serving loop the bench's end-to-end leg runs.  Every step's FTLE and Cauchy-Green
tensor must equal, bit for bit, a plain serial run on a freshly loaded field with the same frames."""
import math

import numpy as np
import pytest
import torch

from paper_2209_13775_gb300 import inputs, lcs

pytestmark = pytest.mark.gpu


def _serial(desc, frames, sd, opts):
    ctx = lcs.lcs_create(0, torch.cuda.current_stream())
    f = lcs.lcs_load_field(ctx, desc, frames)
    s = lcs.lcs_seed_grid(ctx, sd)
    N = lcs.lcs_seeds_count(s)
    fm = lcs.lcs_flowmap_create(ctx, s, 1)
    lcs.lcs_advect(ctx, f, s, opts, fm)
    ftle = np.empty(N, dtype=np.float32)
    C = np.empty((N, 6), dtype=np.float64)
    lcs.lcs_ftle(ctx, fm, 0, ftle, None, C)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(s)
    lcs.lcs_free_field(f)
    lcs.lcs_destroy(ctx)
    return ftle, C


def test_double_buffered_fields_across_two_contexts():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    g = inputs.abc(n=32, nframes=8, t_end=1.0)
    L = 2 * math.pi
    desc = lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times)
    # three steps with different frames: the field, the field at half strength, the field reversed
    step_frames = [g.frames, (0.5 * g.frames).astype(np.float32), (-g.frames).astype(np.float32)]
    sd = lcs.seed_desc(3, (40, 40, 40), (0.0,) * 3, (L,) * 3, (1, 1, 1))
    opts = lcs.advect_opts(lcs.RK4, t0=0.0, T=0.8, dt=0.02)
    want = [_serial(desc, fr, sd, opts) for fr in step_frames]

    stream = torch.cuda.current_stream()
    load_stream = torch.cuda.Stream()
    ctx = lcs.lcs_create(0, stream)
    ctx_load = lcs.lcs_create(0, load_stream)
    pinned = [torch.from_numpy(fr).pin_memory() for fr in step_frames]
    fbuf = [lcs.lcs_load_field(ctx_load, desc, pinned[0]) for _ in range(2)]
    s = lcs.lcs_seed_grid(ctx, sd)
    N = lcs.lcs_seeds_count(s)
    fm = lcs.lcs_flowmap_create(ctx, s, 1)
    ftle_d = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(2)]
    C_d = [torch.empty((N, 6), dtype=torch.float64, device="cuda") for _ in range(2)]
    got = []
    try:
        lcs.lcs_update_frames(ctx_load, fbuf[0], pinned[0])
        for k in range(len(step_frames)):
            b = k % 2
            lcs.lcs_advect(ctx, fbuf[b], s, opts, fm)
            lcs.lcs_ftle(ctx, fm, 0, ftle_d[b], None, C_d[b])
            done = torch.cuda.Event()
            done.record(stream)
            if k + 1 < len(step_frames):
                lcs.lcs_update_frames(ctx_load, fbuf[1 - b], pinned[k + 1])
            ftle_h = torch.empty(N, dtype=torch.float32).pin_memory()
            C_h = torch.empty((N, 6), dtype=torch.float64).pin_memory()
            with torch.cuda.stream(load_stream):
                load_stream.wait_event(done)
                ftle_h.copy_(ftle_d[b], non_blocking=True)
                C_h.copy_(C_d[b], non_blocking=True)
            got.append((ftle_h, C_h))
        torch.cuda.synchronize()
        for k, ((ftle_h, C_h), (wf, wC)) in enumerate(zip(got, want)):
            np.testing.assert_array_equal(ftle_h.numpy(), wf, err_msg="step %d FTLE" % k)
            np.testing.assert_array_equal(C_h.numpy(), wC, err_msg="step %d C" % k)
        # the three steps differ, so equality is not the same answer three times
        assert not np.array_equal(want[0][0], want[1][0])
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(s)
        for f in fbuf:
            lcs.lcs_free_field(f)
        lcs.lcs_destroy(ctx_load)
        lcs.lcs_destroy(ctx)
