"""lcs_advect_rk4_noalloc: the RK4 flow map for callers that cannot allocate device memory.

Such callers (a plugin inside another runtime that owns the device memory, a process whose
memory sits in a pool reserved up front, a loop that cannot afford an allocation) pass every
buffer themselves; the entry point takes its working memory from a fixed array in the library.
This test checks, through the C ABI, that two calls in a row give the same flow map as
lcs_advect on the same inputs (within the flow-map tolerance the other parity tests use), and
that a request larger than the fixed array is refused.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
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


def _case(ctx, g, dim, n, lo, hi, periodic, t0, T, dt, L):
    field = lcs.lcs_load_field(ctx, lcs.field_desc(dim, g.n, g.origin, g.spacing, g.periodic, g.times,
                                                   g.time_periodic, g.period), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    # reference: the allocating entry point
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt), fm)
    ref_x = torch.empty((dim, N), dtype=torch.float32, device="cuda")
    ref_s = torch.empty(N, dtype=torch.uint8, device="cuda")
    ref_t = torch.empty(N, dtype=torch.float32, device="cuda")
    lcs.lcs_flowmap_get(ctx, fm, 0, ref_x, ref_s, ref_t)
    # the caller's own buffers for the no-allocation entry point
    x0 = torch.empty((dim, N), dtype=torch.float32, device="cuda")
    lcs.lcs_seeds_get(ctx, seeds, x0)
    for call in range(2):
        x = torch.full((dim, N), float("nan"), dtype=torch.float32, device="cuda")
        s = torch.full((N,), 255, dtype=torch.uint8, device="cuda")
        te = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        lcs.lcs_advect_rk4_noalloc(ctx, field, x0, t0, T, dt, x, s, te)
        lcs.lcs_synchronize(ctx)
        np.testing.assert_array_equal(s.cpu().numpy(), ref_s.cpu().numpy())
        ok = (ref_s == 0).cpu().numpy()
        err = (x.double() - ref_x.double()).abs().amax(dim=0).cpu().numpy()[ok] / L
        assert np.isfinite(err).all() and err.max() <= 1e-5, (call, err.max())
        np.testing.assert_allclose(te.cpu().numpy(), ref_t.cpu().numpy(), rtol=0, atol=1e-5)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    return field


def test_noalloc_matches_lcs_advect_2d(ctx):
    g = inputs.double_gyre()
    field = _case(ctx, g, 2, (250, 130), (0.0, 0.0), (2.0, 1.0), (0, 0), 0.0, 10.0, 0.05, 2.0)
    lcs.lcs_free_field(field)


def test_noalloc_matches_lcs_advect_3d_backward(ctx):
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    L = 2 * np.pi
    field = _case(ctx, g, 3, (40, 33, 31), (0.0, 0.0, 0.0), (L, L, L), (1, 1, 1), 2.0, -2.0, 0.02, L)
    lcs.lcs_free_field(field)


def test_noalloc_rejects_requests_beyond_its_scratch(ctx):
    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, times=g.times), g.frames)
    x0 = torch.zeros((2, 8), dtype=torch.float32, device="cuda")
    out = [torch.empty((2, 8), device="cuda"), torch.empty(8, dtype=torch.uint8, device="cuda"),
           torch.empty(8, device="cuda")]
    dt = 1e-3
    with pytest.raises(lcs.LcsError) as e:
        lcs.lcs_advect_rk4_noalloc(ctx, field, x0, 0.0, (lcs.NOALLOC_MAX_STEPS + 1) * dt, dt, *out)
    assert e.value.status == 1 and "LCS_NOALLOC_MAX_STEPS" in str(e.value)
    # the largest accepted request runs
    lcs.lcs_advect_rk4_noalloc(ctx, field, x0, 0.0, lcs.NOALLOC_MAX_STEPS * dt, dt, *out)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_field(field)
