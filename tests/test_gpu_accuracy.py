"""The paper's trajectory-accuracy measure (Sec. 3.3 "Verification"): e_S(t), the mean over several
thousand tracers of the distance between the single-precision GPU trajectory and the double-precision
CPU one, against integration time normalised by the nominal LCS horizon.  Here the GPU side is the
library (FP32 arithmetic, snapshots of one integration give every horizon) and the CPU side the FP64
oracle.  Cases: the double gyre (2D Cartesian), the ABC flow (3D Cartesian) and the pipe on tets (3D
unstructured, the stand-in for the aneurysm).  Each e_S(t) stays within the flow-map tolerance
(1e-5 L exp(sigma_max t), L the domain extent); run with -s to print the curves.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_13775_gb300 import inputs, lcs
from gpu_util import rect_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


def gpu_curve(ctx, desc, frames, dim, n, lo, hi, periodic, t0, T, dt, fracs, mesh=False):
    field = lcs.lcs_load_field(ctx, desc, frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic), field if mesh else None)
    N = lcs.lcs_seeds_count(seeds)
    snaps = [f * T for f in fracs[:-1]]
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1 + len(snaps))
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt, snap_T=snaps), fm)
    xs, sts = [], []
    for slot in list(range(1, 1 + len(snaps))) + [0]:
        x = np.empty((dim, N), np.float32)
        st = np.empty(N, np.uint8)
        lcs.lcs_flowmap_get(ctx, fm, slot, x, st)
        xs.append(x)
        sts.append(st)
    x0 = np.empty((dim, N), np.float32)
    cells = np.empty(N, np.int32) if mesh else None
    lcs.lcs_seeds_get(ctx, seeds, x0, cells)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    endpoint = [0 if p else 1 for p in periodic]
    np.testing.assert_array_equal(x0, oracle.seed_grid(dim, n, lo, hi, endpoint))
    return x0, cells, xs, sts


def e_s_curve(F, n, lo, hi, gpu_cells, xs, sts, t0, T, dt, fracs, L, periodic):
    """e_S from the oracle's own seeds (and, on meshes, its own seed cells, which the library's equal)."""
    x0 = oracle.seed_grid(len(n), n, lo, hi, [0 if p else 1 for p in periodic])
    cells = None
    if gpu_cells is not None:
        cells = F.locate_seeds(x0)
        np.testing.assert_array_equal(gpu_cells, cells)
    out = []
    for f, xg, sg in zip(fracs, xs, sts):
        xo, so, _ = oracle.rk4(F, x0.astype(np.float64), t0, f * T, dt, cells=cells)
        ok = (sg == lcs.TRACER_OK) & (so == oracle.OK)
        d = xg[:, ok].astype(np.float64) - xo[:, ok]
        for a in range(len(periodic)):   # unwrapped on both sides; periodic images agree
            if periodic[a]:
                d[a] -= np.round(d[a] / L[a]) * L[a]
        out.append((f, float(np.linalg.norm(d, axis=0).mean()), int(ok.sum())))
    return out


def report(name, curve):
    print("\n" + name + ": e_S(t) at t/T = " + ", ".join("%.2g: %.2e" % (f, e) for f, e, _ in curve))


def sigma_max(F, dim, n, lo, hi, periodic, t0, T, dt):
    endpoint = [0 if p else 1 for p in periodic]
    x0 = oracle.seed_grid(dim, n, lo, hi, endpoint)
    xT, st, _ = oracle.rk4(F, x0.astype(np.float64), t0, T, dt)
    h = oracle.lattice_spacing(dim, n, lo, hi, endpoint)
    period = [hi[a] - lo[a] if periodic[a] else 0.0 for a in range(dim)]
    G = oracle.flowmap_gradient(dim, n, h, periodic, period, xT, st)
    _, sig = oracle.ftle(oracle.cauchy_green(G), dim, T)
    return float(np.nanmax(sig))


FRACS = [0.1, 0.25, 0.5, 0.75, 1.0]


def test_e_s_double_gyre(ctx):
    g = inputs.double_gyre()
    n, lo, hi, T, dt = (64, 64), (0.0, 0.0), (2.0, 1.0), 10.0, 0.05
    x0, _, xs, sts = gpu_curve(ctx, rect_desc(g), g.frames, 2, n, lo, hi, (0, 0), 0.0, T, dt, FRACS)
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    curve = e_s_curve(F, n, lo, hi, None, xs, sts, 0.0, T, dt, FRACS, (2.0, 1.0), (0, 0))
    report("double gyre (4096 tracers)", curve)
    smax = sigma_max(F, 2, n, lo, hi, (0, 0), 0.0, T, dt)
    for f, e, nok in curve:
        assert nok > 4000 and e <= 1e-5 * 2.0 * np.exp(smax * f * T), (f, e)


def test_e_s_abc(ctx):
    g = inputs.abc(n=32, nframes=17, t_end=2.0)
    L = 2 * np.pi
    n, lo, hi, T, dt = (16, 16, 16), (0.0, 0.0, 0.0), (L, L, L), 2.0, 0.02
    x0, _, xs, sts = gpu_curve(ctx, rect_desc(g), g.frames, 3, n, lo, hi, (1, 1, 1), 0.0, T, dt, FRACS)
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    curve = e_s_curve(F, n, lo, hi, None, xs, sts, 0.0, T, dt, FRACS, (L, L, L), (1, 1, 1))
    report("ABC (4096 tracers)", curve)
    smax = sigma_max(F, 3, n, lo, hi, (1, 1, 1), 0.0, T, dt)
    for f, e, nok in curve:
        assert nok == 4096 and e <= 1e-5 * L * np.exp(smax * f * T), (f, e)


def test_e_s_pipe_on_tets(ctx):
    p = inputs.pipe_frames(inputs.pipe_mesh(h=0.1, R=1.0, L=2.0), nframes=50, period=1.0, L=2.0)
    desc = lcs.field_desc(3, times=p.times, time_periodic=True, period=p.period, kind=lcs.TET,
                          mesh=(p.xyz, p.tets, p.nbrs))
    n, lo, hi, T, dt = (16, 16, 16), (-0.6, -0.6, 0.1), (0.6, 0.6, 1.3), 1.0, 0.01
    x0, cells, xs, sts = gpu_curve(ctx, desc, p.frames, 3, n, lo, hi, (0, 0, 0), 0.0, T, dt, FRACS, mesh=True)
    F = oracle.TetField(p.xyz, p.tets, p.nbrs, p.frames, p.times, True, p.period)
    curve = e_s_curve(F, n, lo, hi, cells, xs, sts, 0.0, T, dt, FRACS, (2.0, 2.0, 2.0), (0, 0, 0))
    report("pipe on tets (4096 tracers)", curve)
    for f, e, nok in curve:
        assert nok > 2000 and e <= 2e-5, (f, e)     # the tet path's flow-map tolerance
