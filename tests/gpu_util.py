"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare with the stated
tolerances.

Tolerances (fixed-step FP32 path against the FP64 oracle):
  * seed lattice, status: bit-exact;
  * flow map: ||x_gpu - x_oracle||_inf / L <= 1e-5 * exp(sigma_max * |T|) per OK seed,
    L the domain extent, sigma_max the oracle's largest FTLE;
  * FTLE: median |d sigma| <= 1e-5 and 99.9th percentile <= 1e-3 over seeds valid
    in both.
"""
import numpy as np
import torch

import oracle
from paper_2209_13775_gb300 import lcs


def rect_desc(g, storage=lcs.F32):
    return lcs.field_desc(g.dim, g.n, g.origin, g.spacing, g.periodic, g.times, g.time_periodic, g.period,
                          storage=storage)


def gpu_run(ctx, g, n, lo, hi, periodic, T, dt, t0=0.0, storage=lcs.F32, variant=0, block_threads=0,
            jobs=None, want_C=False, tracers_per_thread=0, episode_steps=0, use_graph=False):
    """Load, seed, advect, FTLE through the C ABI.  Returns dict of host arrays (job 0 unless jobs)."""
    dim = g.dim
    field = lcs.lcs_load_field(ctx, rect_desc(g, storage), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi, periodic))
    N = lcs.lcs_seeds_count(seeds)
    njobs = 1 if jobs is None else len(jobs[0])
    fm = lcs.lcs_flowmap_create(ctx, seeds, njobs)
    kw = dict(variant=variant, block_threads=block_threads, tracers_per_thread=tracers_per_thread,
              episode_steps=episode_steps, use_graph=use_graph)
    if jobs is None:
        opts = lcs.advect_opts(lcs.RK4, t0=t0, T=T, dt=dt, **kw)
    else:
        opts = lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1], **kw)
    lcs.lcs_advect(ctx, field, seeds, opts, fm)
    out = {"N": N, "seeds": np.empty((dim, N), dtype=np.float32)}
    lcs.lcs_seeds_get(ctx, seeds, out["seeds"])
    out["xyz"], out["status"], out["t_exit"], out["ftle"], out["lam"], out["C"] = [], [], [], [], [], []
    np_ = 3 if dim == 2 else 6
    for j in range(njobs):
        x = np.empty((dim, N), dtype=np.float32)
        s = np.empty(N, dtype=np.uint8)
        te = np.empty(N, dtype=np.float32)
        lcs.lcs_flowmap_get(ctx, fm, j, x, s, te)
        f = np.empty(N, dtype=np.float32)
        lam = np.empty(N, dtype=np.float64)
        C = np.empty((N, np_), dtype=np.float64) if want_C else None
        lcs.lcs_ftle(ctx, fm, j, f, lam, C)
        for k, v in (("xyz", x), ("status", s), ("t_exit", te), ("ftle", f), ("lam", lam), ("C", C)):
            out[k].append(v)
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return out


def gpu_cg_of(ctx, seeds, xT, st, T, nout, dim, want_eig=False):
    """The library's grad F / Eq. 1 / FTLE (and eigenpairs) on a flow map made elsewhere: xT [dim][M]
    (rounded to FP32) and st [M] go in through lcs_flowmap_set over `seeds`; nout values per output
    (the lattice seeds).  Lets a test feed the oracle's own flow map to the library's FD/CG/FTLE."""
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_flowmap_set(ctx, fm, 0, np.ascontiguousarray(xT, dtype=np.float32),
                        np.ascontiguousarray(st, dtype=np.uint8), T)
    out = {"ftle": np.empty(nout, dtype=np.float32), "lam": np.empty(nout),
           "C": np.empty((nout, 3 if dim == 2 else 6))}
    lcs.lcs_ftle(ctx, fm, 0, out["ftle"], out["lam"], out["C"])
    if want_eig:
        out["ev"] = np.empty((nout, dim))
        lcs.lcs_cg_eigen(ctx, fm, 0, out["ev"])
    lcs.lcs_synchronize(ctx)
    lcs.lcs_free_flowmap(fm)
    return out


def oracle_field(g):
    return oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)


def stencil_ids(sample, n, periodic, reach=2):
    """The sampled seed ids with their lattice neighbours up to `reach` along each axis (a one-sided
    difference at a non-periodic edge needs the second neighbour; periodic lattices need only 1)."""
    dim = len(periodic)
    sample = np.asarray(sample, dtype=np.int64)
    strides = [1, n[0], n[0] * n[1]][:dim]
    idx = [(sample // strides[a]) % n[a] for a in range(dim)]
    out = [sample]
    for a in range(dim):
        for off in range(-reach, reach + 1):
            if off == 0:
                continue
            q = idx[a] + off
            keep = np.ones(len(sample), dtype=bool)
            if periodic[a]:
                q = q % n[a]
            else:
                keep = (q >= 0) & (q < n[a])
            out.append((sample + (q - idx[a]) * strides[a])[keep])
    return np.unique(np.concatenate(out))


def oracle_run(g, n, lo, hi, periodic, T, dt, t0=0.0, sample=None, reach=2):
    """Oracle flow map and FTLE; `sample` restricts the FTLE to those seed ids (advecting them and
    their lattice neighbours up to `reach` only)."""
    dim = g.dim
    endpoint = [0 if p else 1 for p in periodic]
    x0 = oracle.seed_grid(dim, n, lo, hi, endpoint)
    F = oracle_field(g)
    h = oracle.lattice_spacing(dim, n, lo, hi, endpoint)
    period = [hi[a] - lo[a] if periodic[a] else 0.0 for a in range(dim)]
    if sample is None:
        xT, st, te = oracle.rk4(F, x0.astype(np.float64), t0, T, dt)
        G = oracle.flowmap_gradient(dim, n, h, periodic, period, xT, st)
        C = oracle.cauchy_green(G)
        lam, sig = oracle.ftle(C, dim, T)
        return {"seeds": x0, "xyz": xT, "status": st, "t_exit": te, "ftle": sig, "lam": lam, "C": C}
    # stencils of the sampled seeds: +-1, +-2 along each axis (one-sided fallbacks need 2)
    ids = stencil_ids(sample, n, periodic[:dim], reach)
    xT_s, st_s, te_s = oracle.rk4(F, x0[:, ids].astype(np.float64), t0, T, dt)
    N = x0.shape[1]
    # scatter into full-size arrays; seeds not integrated are marked LEFT so no stencil uses them
    xT = np.zeros((dim, N))
    st = np.full(N, oracle.LEFT, dtype=np.uint8)
    xT[:, ids] = xT_s
    st[ids] = st_s
    return {"seeds": x0, "ids": ids, "xyz_s": xT_s, "status_s": st_s, "t_exit_s": te_s, "xT": xT, "st": st,
            "h": h, "period": period}


def oracle_ftle_at(sample, dim, n, h, periodic, period, xT, st, T):
    """Oracle FTLE at `sample` from (partial) full-size flow-map arrays."""
    G = oracle.flowmap_gradient(dim, n, h, periodic, period, xT, st)[sample]
    C = oracle.cauchy_green(G)
    lam, sig = oracle.ftle(C, dim, T)
    return sig, lam, C


def check_flowmap(x_gpu, x_ora, st_gpu, st_ora, L, sigma_max, T):
    np.testing.assert_array_equal(st_gpu, st_ora)
    ok = st_ora == oracle.OK
    err = np.abs(x_gpu[:, ok].astype(np.float64) - x_ora[:, ok]).max(axis=0) / L
    bound = 1e-5 * np.exp(sigma_max * abs(T))
    assert err.max() <= bound, (err.max(), bound)
    return err


def check_ftle(f_gpu, f_ora):
    both = np.isfinite(f_gpu) & np.isfinite(f_ora)
    np.testing.assert_array_equal(np.isfinite(f_gpu), np.isfinite(f_ora))
    d = np.abs(f_gpu[both].astype(np.float64) - f_ora[both])
    med, p999 = float(np.median(d)), float(np.quantile(d, 0.999))
    assert med <= 1e-5 and p999 <= 1e-3, (med, p999)
    return med, p999, float(d.max())


def round_bf16(a):
    """FP32 -> nearest-even BF16 -> FP32 (what BF16 storage holds)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def round_fp16(a):
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float32)


MARGIN = 1e-3   # a stage point this far from a mesh boundary is on the same side of it in FP32 and FP64


def check_exit_statuses(st_g, te_g, st_o, te_o, dt, frac=2e-3, margin=None, delta=MARGIN):
    """Mesh fields: statuses agree except where an exit was decided one step apart (stage points
    within rounding of a boundary face or edge); returns the seeds where both are OK or both left
    at the same step.  With margin (the oracle's smallest distance of each tracer's stage points
    from the mesh boundary, oracle.rk4(..., margin=rmax)), every tracer whose stage points all kept
    farther than delta from the boundary -- far beyond the positions' difference -- must have the
    oracle's status bit for bit and its exit time to FP32 rounding; only the others may differ."""
    if margin is not None:
        far = margin > delta
        np.testing.assert_array_equal(st_g[far], st_o[far])
        dtf = np.abs(te_g[far].astype(np.float64) - te_o[far])
        assert (dtf <= 1e-4 * dt + 1e-6 * np.abs(te_o[far])).all(), dtf.max()
        assert far.mean() > 0.5, far.mean()
    diff = st_g != st_o
    assert diff.mean() <= frac, diff.sum()
    assert set(np.unique(st_g[diff])) <= {lcs.TRACER_OK, lcs.TRACER_LEFT}
    dte = np.abs(te_g.astype(np.float64) - te_o)
    assert (dte[diff] <= dt * (1 + 1e-4)).all(), dte[diff].max()
    same = ~diff & (dte <= 1e-4 * dt)
    assert ((~diff) & ~same).sum() <= frac * len(st_g)
    return same


def mesh_snapshots_equal_separate_runs(ctx, desc, frames, dim, n, lo, hi, jobs, snap_T, dt):
    """A run with snapshots against separate runs over each snapshot horizon: bit for bit."""
    field = lcs.lcs_load_field(ctx, desc, frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(dim, n, lo, hi), field)
    N = lcs.lcs_seeds_count(seeds)
    nj, ns = len(jobs[0]), len(snap_T)
    fm = lcs.lcs_flowmap_create(ctx, seeds, nj * (1 + ns))
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, dt=dt, job_t0=jobs[0], job_T=jobs[1], snap_T=snap_T), fm)
    one = lcs.lcs_flowmap_create(ctx, seeds, 1)
    left = 0
    for j, (t0, T) in enumerate(zip(*jobs)):
        for q, a in enumerate(list(snap_T) + [abs(T)]):
            slot = j if q == ns else nj + j * ns + q
            h = min(a, abs(T))
            lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=t0, T=h if T > 0 else -h, dt=dt), one)
            got = [np.empty((dim, N), np.float32), np.empty(N, np.uint8), np.empty(N, np.float32)]
            want = [np.empty((dim, N), np.float32), np.empty(N, np.uint8), np.empty(N, np.float32)]
            lcs.lcs_flowmap_get(ctx, fm, slot, *got)
            lcs.lcs_flowmap_get(ctx, one, 0, *want)
            for a_, b_ in zip(got, want):
                np.testing.assert_array_equal(a_, b_)
            left += int((want[1] == lcs.TRACER_LEFT).sum())
    lcs.lcs_synchronize(ctx)
    for fmx in (fm, one):
        lcs.lcs_free_flowmap(fmx)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    return left
