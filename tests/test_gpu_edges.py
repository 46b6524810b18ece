"""Edge cases of the path through the C ABI against the FP64 oracle: lattices with a single seed or a
single row (the finite differences then have no stencil on some axes), ragged seed counts that fill
no block or warp evenly, the re-bundled 3D path forced onto a lattice smaller than one block,
integrations of zero steps, a DP5(4) warp group with fewer than 32 live lanes, and the surrogate
path on a seed count that is not a multiple of its 128-tracer tiles (Sec. 2 "Seed", "Flow Map",
"Cauchy-Green")."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import check_flowmap, gpu_run, oracle_run, rect_desc

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


def compare(r, o, L, T):
    """Positions within the flow-map bound, statuses bit-exact, the same seeds with a finite FTLE, and
    the finite values within the fixed-step p99.9 bound (too few seeds for a median)."""
    f_o = o["ftle"]
    smax = float(np.nanmax(f_o)) if np.isfinite(f_o).any() else 0.0
    check_flowmap(r["xyz"][0], o["xyz"], r["status"][0], o["status"], L, smax, T)
    f_g = r["ftle"][0]
    np.testing.assert_array_equal(np.isfinite(f_g), np.isfinite(f_o))
    fin = np.isfinite(f_o)
    if fin.any():
        assert np.abs(f_g[fin].astype(np.float64) - f_o[fin]).max() <= 1e-3
    return int(fin.sum())


def advect_only(ctx, g, n, lo, hi, periodic, T, dt, variant):
    """Flow map of a lattice through lcs_advect, and whether lcs_ftle refused the lattice."""
    dim = g.dim
    field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    try:
        lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=0.0, T=T, dt=dt, variant=variant), fm)
        x = np.empty((dim, N), np.float32)
        s = np.empty(N, np.uint8)
        lcs.lcs_flowmap_get(ctx, fm, 0, x, s)
        lcs.lcs_synchronize(ctx)
        refused = None
        try:
            lcs.lcs_ftle(ctx, fm, 0, np.empty(N, np.float32))
        except lcs.LcsError as e:
            refused = e.status
        lcs.lcs_synchronize(ctx)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)
    return x, s, refused


@pytest.mark.parametrize("n", [(1, 1), (2, 1), (1, 3), (2, 2), (3, 2), (33, 1)])
@pytest.mark.parametrize("variant", [1, 2, 5])
def test_lattices_below_the_difference_stencil_2d(ctx, gyre, n, variant):
    # a single seed, a single row, two seeds along an axis: the flow map is the oracle's (every 2D
    # kernel, each with a last warp and block mostly empty), and the FD/CG/FTLE calls refuse the
    # lattice (LCS_EINVAL): no difference rule has three points along that axis
    lo, hi, T, dt = (0.1, 0.05), (1.9, 0.95), 2.0, 0.05
    x, s, refused = advect_only(ctx, gyre, n, lo, hi, (0, 0), T, dt, variant)
    o = oracle_run(gyre, n, lo, hi, (0, 0), T, dt)
    check_flowmap(x, o["xyz"], s, o["status"], 2.0, 0.5, T)
    assert refused == 1


@pytest.mark.parametrize("n", [(3, 3), (5, 3), (257, 3), (250, 130)])
@pytest.mark.parametrize("variant", [1, 2, 5])
def test_small_and_ragged_lattices_2d(ctx, gyre, n, variant):
    # the smallest lattices the differences accept (three seeds: forward, central, backward) and
    # ragged counts, every 2D kernel
    lo, hi, T, dt = (0.1, 0.05), (1.9, 0.95), 2.0, 0.05
    r = gpu_run(ctx, gyre, n, lo, hi, (0, 0), T, dt, variant=variant)
    o = oracle_run(gyre, n, lo, hi, (0, 0), T, dt)
    np.testing.assert_array_equal(r["seeds"], o["seeds"])
    assert compare(r, o, 2.0, T) == n[0] * n[1]


@pytest.mark.parametrize("n,periodic", [((3, 3, 3), (1, 1, 1)), ((7, 5, 3), (1, 1, 1)), ((7, 5, 3), (0, 0, 0)),
                                        ((37, 3, 4), (1, 0, 1))])
def test_tiny_lattices_3d_every_variant(ctx, abc_small, n, periodic):
    # the one-pass gather kernel and the re-bundled episodes (forced on a lattice smaller than one
    # block; one block, partly empty) give the same flow map bit for bit, and both match the oracle
    L = 2 * np.pi
    hi = tuple(L if p else 2.0 for p in periodic)
    lo = (0.0, 0.0, 0.0) if periodic != (0, 0, 0) else (0.5, 0.5, 0.5)
    T, dt = 1.0, 0.02
    a = gpu_run(ctx, abc_small, n, lo, hi, periodic, T, dt, variant=1)
    b = gpu_run(ctx, abc_small, n, lo, hi, periodic, T, dt, variant=3, episode_steps=16)
    for k in ("xyz", "status", "t_exit"):
        np.testing.assert_array_equal(a[k][0], b[k][0])
    np.testing.assert_array_equal(a["ftle"][0], b["ftle"][0])
    o = oracle_run(abc_small, n, lo, hi, periodic, T, dt)
    compare(a, o, L, T)


def test_single_seed_3d(ctx, abc_small):
    # one seed through both 3D paths: the flow map is the oracle's, the differences refuse the lattice
    L = 2 * np.pi
    for variant in (1, 3):
        x, s, refused = advect_only(ctx, abc_small, (1, 1, 1), (0.3, 0.2, 0.1), (0.3, 0.2, 0.1), (0, 0, 0), 1.0,
                                    0.02, variant)
        o = oracle_run(abc_small, (1, 1, 1), (0.3, 0.2, 0.1), (0.3, 0.2, 0.1), (0, 0, 0), 1.0, 0.02)
        check_flowmap(x, o["xyz"], s, o["status"], L, 1.0, 1.0)
        assert refused == 1


def test_zero_step_integration(ctx, gyre, abc_small):
    # T = 0: the flow map is the seed lattice bit for bit, every tracer OK with exit time t0; the FTLE
    # divides by |T| = 0 and is not finite on either side
    for g, dim, n, lo, hi, per in ((gyre, 2, (9, 5), (0.0, 0.0), (2.0, 1.0), (0, 0)),
                                   (abc_small, 3, (6, 5, 4), (0.0, 0.0, 0.0), (2 * np.pi,) * 3, (1, 1, 1))):
        for variant in ((1, 5) if dim == 2 else (1, 3)):
            r = gpu_run(ctx, g, n, lo, hi, per, 0.0, 0.05, t0=1.25, variant=variant)
            np.testing.assert_array_equal(r["xyz"][0], r["seeds"])
            assert (r["status"][0] == lcs.TRACER_OK).all()
            assert (r["t_exit"][0] == np.float32(1.25)).all()
            assert not np.isfinite(r["ftle"][0]).any()
        o = oracle_run(g, n, lo, hi, per, 0.0, 0.05, t0=1.25)
        np.testing.assert_array_equal(o["xyz"], o["seeds"].astype(np.float64))
        assert not np.isfinite(o["ftle"]).any()


def test_rk45_partial_warp_group(ctx):
    # DP5(4) shares one step size per 32 consecutive seeds; 15 and 47 seeds leave a group with fewer
    # live lanes, which must step as the oracle's 32-lane mode does with the same partial group
    from scipy.linalg import expm

    A = np.array([[-0.25, -1.0], [1.0, -0.25]])
    g = inputs.affine_frames(A, np.zeros((2, 2)), np.zeros(2), (17, 17), (-2.0, -2.0), (0.25, 0.25), [0.0, 100.0])
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing)
    for n in ((5, 3), (47, 1)):
        lo, hi, T = (-1.2, -0.9), (1.2, 0.9), 3.0
        field = lcs.lcs_load_field(ctx, rect_desc(g), g.frames)
        seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n, lo, hi))
        N = lcs.lcs_seeds_count(seeds)
        fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
        try:
            lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK45, t0=0.0, T=T, rtol=1e-5, atol=1e-5, h0=0.01),
                           fm)
            x = np.empty((2, N), np.float32)
            s = np.empty(N, np.uint8)
            ns = np.empty(N, np.int32)
            lcs.lcs_flowmap_get(ctx, fm, 0, x, s)
            lcs.lcs_flowmap_steps(ctx, fm, 0, ns)
            lcs.lcs_synchronize(ctx)
        finally:
            lcs.lcs_free_flowmap(fm)
            lcs.lcs_free_seeds(seeds)
            lcs.lcs_free_field(field)
        x0 = oracle.seed_grid(2, n, lo, hi).astype(np.float64)
        xo, so, _, nso = oracle.dp45(F, x0, 0.0, T, h0=0.01, rtol=1e-5, atol=1e-5, group=32)
        assert (s == lcs.TRACER_OK).all() and (so == oracle.OK).all()
        assert np.abs(x - xo).max() <= 1e-4 and np.abs(x - expm(T * A) @ x0).max() <= 2e-4
        assert np.abs(ns.astype(np.int64) - nso).max() <= 3
        for q in range(0, N, 32):
            assert len(set(ns[q:q + 32].tolist())) == 1


def test_surrogate_on_a_ragged_seed_count(ctx, gyre):
    # 300 seeds: the network's 128-tracer tiles and the audit's 32-seed groups end part-full; gate 0
    # integrates every sub-interval by RK4 and equals LCS_RK4 bit for bit, gate infinity never falls back
    d = lcs.mlp_desc((1.0, 0.5), np.pi, np.pi, 2 * np.pi / 10, 0.5, 0.1)
    m = lcs.lcs_mlp_create(ctx, d, inputs.mlp_init(seed=95))
    field = lcs.lcs_load_field(ctx, rect_desc(gyre), gyre.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (20, 15), (0.1, 0.1), (1.9, 0.9)))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    out = {}
    try:
        for name, o in (("rk4", lcs.advect_opts(lcs.RK4, t0=0.0, T=2.0, dt=0.05)),
                        ("gate0", lcs.advect_opts(lcs.SURROGATE, t0=0.0, T=2.0, dt=0.05, surrogate=m, gate_tol=0.0)),
                        ("gateinf", lcs.advect_opts(lcs.SURROGATE, t0=0.0, T=2.0, dt=0.05, surrogate=m,
                                                    gate_tol=float("inf")))):
            lcs.lcs_advect(ctx, field, seeds, o, fm)
            x = np.empty((2, N), np.float32)
            s = np.empty(N, np.uint8)
            lcs.lcs_flowmap_get(ctx, fm, 0, x, s)
            steps = np.zeros(N, np.int32)
            if o.method == lcs.SURROGATE:
                lcs.lcs_flowmap_steps(ctx, fm, 0, steps)
            lcs.lcs_synchronize(ctx)
            out[name] = (x, s, steps)
    finally:
        lcs.lcs_free_flowmap(fm)
        lcs.lcs_free_seeds(seeds)
        lcs.lcs_free_field(field)
        lcs.lcs_mlp_free(m)
    np.testing.assert_array_equal(out["gate0"][0], out["rk4"][0])
    np.testing.assert_array_equal(out["gate0"][1], out["rk4"][1])
    assert (out["gate0"][2] == 4).all() and (out["gateinf"][2] == 0).all()
    assert np.isfinite(out["gateinf"][0]).all()
