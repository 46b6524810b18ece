"""lcs_advect_rk4_noalloc: the RK4 flow map for callers that cannot allocate device memory.

Such callers (a plugin inside another runtime that owns the device memory, a process whose
memory sits in a pool reserved up front, a loop that cannot afford an allocation) pass every
buffer themselves; the entry point takes its working memory from a fixed array in the library.
This test checks, through the C ABI, that two calls in a row give the same flow map as
lcs_advect on the same inputs, bit for bit (every RK4 variant of the library does the same
arithmetic), that the second call leaves the device's free memory unchanged, that a request
larger than the fixed array is refused, and that buffers of the wrong shape, type or kind are
refused before any launch.  The file sorts last so that a run that stops at the first failure
has already run every other test.
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
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        lcs.lcs_advect_rk4_noalloc(ctx, field, x0, t0, T, dt, x, s, te)
        lcs.lcs_synchronize(ctx)
        if call == 1:   # the first call may load the library's module (and its fixed array)
            assert torch.cuda.mem_get_info()[0] == free0
        np.testing.assert_array_equal(s.cpu().numpy(), ref_s.cpu().numpy())
        np.testing.assert_array_equal(x.cpu().numpy(), ref_x.cpu().numpy())
        np.testing.assert_array_equal(te.cpu().numpy(), ref_t.cpu().numpy())
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


def test_noalloc_refuses_mismatched_buffers(ctx):
    """Wrong shapes, types or devices never reach a kernel: the binding refuses them (ValueError),
    and the C entry point refuses host memory (LCS_EINVAL) before any launch."""
    import ctypes

    g = inputs.double_gyre(nx=17, ny=9, nframes=3, t_end=1.0)
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, times=g.times), g.frames)
    n = 64
    ok = dict(seeds=torch.zeros((2, n), device="cuda"), xyz=torch.empty((2, n), device="cuda"),
              status=torch.empty(n, dtype=torch.uint8, device="cuda"), t_exit=torch.empty(n, device="cuda"))
    bad = [dict(seeds=torch.zeros((3, n), device="cuda")),                 # 3D seeds on a 2D field
           dict(seeds=torch.zeros(2 * n, device="cuda")),
           dict(seeds=torch.zeros((2, n), dtype=torch.float64, device="cuda")),
           dict(xyz=torch.empty((2, n - 1), device="cuda")),              # short output
           dict(status=torch.empty(n, dtype=torch.int32, device="cuda")),
           dict(t_exit=torch.empty(n - 1, device="cuda")),
           dict(xyz=torch.empty((2, n))),                                  # host tensor
           dict(status=np.empty(n, dtype=np.uint8))]
    try:
        for b in bad:
            a = dict(ok, **b)
            with pytest.raises(ValueError):
                lcs.lcs_advect_rk4_noalloc(ctx, field, a["seeds"], 0.0, 0.5, 0.05, a["xyz"], a["status"], a["t_exit"])
        # straight through the C ABI with a host output buffer: refused, nothing launched
        host = np.empty((2, n), dtype=np.float32)
        st = lcs.load().lcs_advect_rk4_noalloc(ctx, field, ctypes.c_void_p(ok["seeds"].data_ptr()), n, 0.0, 0.5,
                                               0.05, ctypes.c_void_p(host.ctypes.data),
                                               ctypes.c_void_p(ok["status"].data_ptr()),
                                               ctypes.c_void_p(ok["t_exit"].data_ptr()))
        assert st == 1 and "device memory" in lcs.lcs_last_error(ctx)
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_field(field)
