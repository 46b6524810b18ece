"""Thin ctypes binding of liblcs (include/lcs.h), one Python function per C entry point.

Argument marshalling only: numpy arrays are host buffers, torch tensors on a
CUDA device are device buffers, and every step of the path runs in the CUDA
library.  A non-OK status raises ``LcsError`` carrying ``lcs_last_error``.
There is no fallback: importing this module on a machine where liblcs.so cannot
be loaded raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RECTILINEAR, TET, TRI = 0, 1, 2
F32, F16, BF16 = 0, 1, 2
RK4, RK45, SURROGATE = 0, 1, 2
TRACER_OK, TRACER_LEFT, TRACER_OUTSIDE, TRACER_MAXSTEPS, TRACER_WALKFAIL = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "LCS_OK", 1: "LCS_EINVAL", 2: "LCS_ENOMEM", 3: "LCS_ECUDA", 4: "LCS_ETIMEOUT",
                5: "LCS_EWALK", 6: "LCS_EMAXSTEPS", 7: "LCS_EUNSUPPORTED"}

EXPORTS = ["lcs_create", "lcs_destroy", "lcs_last_error", "lcs_set_stream", "lcs_synchronize",
           "lcs_load_field", "lcs_update_frames", "lcs_free_field", "lcs_seed_grid", "lcs_seed_aux", "lcs_seed_aux_field",
           "lcs_seeds_count",
           "lcs_seeds_get", "lcs_free_seeds", "lcs_flowmap_create", "lcs_advect", "lcs_flowmap_get",
           "lcs_flowmap_set", "lcs_flowmap_steps",
           "lcs_free_flowmap", "lcs_autotune", "lcs_cauchy_green", "lcs_ftle", "lcs_cg_eigen", "lcs_ftle_early", "lcs_ftle_variational",
           "lcs_flowmap_grad",
           "lcs_timing_enable",
           "lcs_timing_read",
           "lcs_advect_rk4_noalloc", "lcs_gemm_bf16", "lcs_mlp_create", "lcs_mlp_set_params",
           "lcs_mlp_get_params", "lcs_mlp_free", "lcs_mlp_forward", "lcs_mlp_loss_grad", "lcs_mlp_adam",
           "lcs_surrogate_train", "lcs_context_device", "lcs_field_dim"]
PHASE_ADVECT, PHASE_REBUNDLE, PHASE_SLICES, PHASE_CG = 0, 1, 2, 3
NOALLOC_MAX_STEPS = 43680
MAX_SNAP = 8
MLP_NPARAMS = 50947


class LcsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class FieldDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kind", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("nframes", ctypes.c_int),
                ("frame_times", ctypes.c_void_p), ("time_periodic", ctypes.c_int),
                ("period", ctypes.c_double), ("storage", ctypes.c_int),
                ("nnodes", ctypes.c_longlong), ("ncells", ctypes.c_longlong),
                ("node_xyz", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("nbrs", ctypes.c_void_p)]


class SeedDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3)]


class AdvectOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("t0", ctypes.c_double), ("T", ctypes.c_double),
                ("njobs", ctypes.c_int), ("job_t0", ctypes.c_void_p), ("job_T", ctypes.c_void_p),
                ("dt", ctypes.c_double), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("h0", ctypes.c_double), ("max_steps", ctypes.c_longlong), ("walk_limit", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("variant", ctypes.c_int), ("surrogate", ctypes.c_void_p),
                ("episode_steps", ctypes.c_int), ("tracers_per_thread", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("gate_tol", ctypes.c_double), ("nsnap", ctypes.c_int), ("snap_T", ctypes.c_void_p),
                ("variational", ctypes.c_int), ("wait_limit", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblcs.so (building it first when missing); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) and build_if_missing:
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    P, I, LL, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int
    sig = {
        "lcs_create": ([P, I, P], S), "lcs_destroy": ([P], None), "lcs_last_error": ([P], ctypes.c_char_p),
        "lcs_set_stream": ([P, P], S), "lcs_synchronize": ([P], S),
        "lcs_context_device": ([P], I), "lcs_field_dim": ([P], I),
        "lcs_load_field": ([P, P, P, I, P], S), "lcs_update_frames": ([P, P, P, I], S),
        "lcs_free_field": ([P], None), "lcs_seed_grid": ([P, P, P, P], S), "lcs_seeds_count": ([P], LL),
        "lcs_seed_aux": ([P, P, P, P], S), "lcs_seed_aux_field": ([P, P, P, P, P], S),
        "lcs_seeds_get": ([P, P, P, P, I], S), "lcs_free_seeds": ([P], None),
        "lcs_flowmap_create": ([P, P, I, P], S), "lcs_advect": ([P, P, P, P, P], S),
        "lcs_flowmap_get": ([P, P, I, P, P, P, I], S), "lcs_free_flowmap": ([P], None),
        "lcs_flowmap_set": ([P, P, I, P, P, P, ctypes.c_double, I], S),
        "lcs_cauchy_green": ([P, P, I, P, I], S), "lcs_ftle": ([P, P, I, P, P, P, I], S),
        "lcs_cg_eigen": ([P, P, I, P, P, I], S), "lcs_ftle_early": ([P, P, P, P, P, I, P, P, I], S),
        "lcs_ftle_variational": ([P, P, I, P, P, P, I], S), "lcs_flowmap_grad": ([P, P, I, P, I], S),
        "lcs_advect_rk4_noalloc": ([P, P, P, LL, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P], S),
        "lcs_timing_enable": ([P, I], S), "lcs_timing_read": ([P, I, P, P], S),
        "lcs_autotune": ([P, P, P, P, ctypes.c_char_p], S),
        "lcs_flowmap_steps": ([P, P, I, P, I], S),
        "lcs_gemm_bf16": ([P, LL, I, LL, P, LL, P, LL, P, LL, I, I], S),
        "lcs_mlp_create": ([P, P, P, I, P], S), "lcs_mlp_set_params": ([P, P, P, I], S),
        "lcs_mlp_get_params": ([P, P, P, I], S), "lcs_mlp_free": ([P], None),
        "lcs_mlp_forward": ([P, P, LL, P, P, I], S),
        "lcs_mlp_loss_grad": ([P, P, LL, P, P, ctypes.c_double, P, P, I], S),
        "lcs_mlp_adam": ([P, P, P, I, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double], S),
        "lcs_surrogate_train": ([P, P, P, P, LL, P, I, P], S),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor; (None, 0) for None."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _check(ctx, st):
    if st != 0:
        msg = load().lcs_last_error(ctx)
        raise LcsError(st, msg.decode() if msg else "")


# ---------------------------------------------------------------- context

def lcs_create(device: int = 0, stream=None):
    """Context on `device` queuing work on `stream` (a torch.cuda.Stream, an int handle or None)."""
    L = load()
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    out = ctypes.c_void_p()
    st = L.lcs_create(ctypes.byref(out), int(device), ctypes.c_void_p(stream or 0))
    if st != 0:
        raise LcsError(st, "lcs_create(device=%d)" % device)
    return out.value


def lcs_destroy(ctx):
    load().lcs_destroy(ctx)


def lcs_last_error(ctx) -> str:
    m = load().lcs_last_error(ctx)
    return m.decode() if m else ""


def lcs_set_stream(ctx, stream):
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(ctx, load().lcs_set_stream(ctx, ctypes.c_void_p(stream or 0)))


def lcs_synchronize(ctx):
    _check(ctx, load().lcs_synchronize(ctx))


def lcs_context_device(ctx) -> int:
    return int(load().lcs_context_device(ctx))


def lcs_field_dim(field) -> int:
    return int(load().lcs_field_dim(field))


# ----------------------------------------------------------------- field

def field_desc(dim, n=(1, 1, 1), origin=(0, 0, 0), spacing=(1, 1, 1), periodic=(0, 0, 0), times=(0.0,),
               time_periodic=False, period=0.0, storage=F32, kind=RECTILINEAR, mesh=None):
    """Build an lcs_field_desc; the returned object keeps its arrays alive."""
    d = FieldDesc()
    d.dim, d.kind, d.storage = int(dim), int(kind), int(storage)
    for a in range(3):
        d.n[a] = int(n[a]) if a < len(n) else 1
        d.origin[a] = float(origin[a]) if a < len(origin) else 0.0
        d.spacing[a] = float(spacing[a]) if a < len(spacing) else 1.0
        d.periodic[a] = int(periodic[a]) if a < len(periodic) else 0
    t = np.ascontiguousarray(times, dtype=np.float64)
    d.nframes = len(t)
    d.frame_times = t.ctypes.data
    d.time_periodic = int(bool(time_periodic))
    d.period = float(period)
    keep = [t]
    if mesh is not None:
        xyz = np.ascontiguousarray(mesh[0], dtype=np.float32)
        tets = np.ascontiguousarray(mesh[1], dtype=np.int32)
        nbrs = None if mesh[2] is None else np.ascontiguousarray(mesh[2], dtype=np.int32)
        d.nnodes, d.ncells = xyz.shape[0], tets.shape[0]
        d.node_xyz, d.tets = xyz.ctypes.data, tets.ctypes.data
        d.nbrs = None if nbrs is None else nbrs.ctypes.data
        keep += [xyz, tets, nbrs]
    d._keep = keep
    return d


def lcs_load_field(ctx, desc: FieldDesc, frames):
    p, dev = _ptr(frames)
    out = ctypes.c_void_p()
    _check(ctx, load().lcs_load_field(ctx, ctypes.byref(desc), ctypes.c_void_p(p), dev, ctypes.byref(out)))
    return out.value


def lcs_update_frames(ctx, field, frames):
    p, dev = _ptr(frames)
    _check(ctx, load().lcs_update_frames(ctx, field, ctypes.c_void_p(p), dev))


def lcs_free_field(field):
    load().lcs_free_field(field)


# ------------------------------------------------------------- seed grid

def seed_desc(dim, n, lo, hi, periodic=(0, 0, 0)):
    d = SeedDesc()
    d.dim = int(dim)
    for a in range(3):
        d.n[a] = int(n[a]) if a < dim else 1
        d.lo[a] = float(lo[a]) if a < dim else 0.0
        d.hi[a] = float(hi[a]) if a < dim else 0.0
        d.periodic[a] = int(periodic[a]) if a < len(periodic) and a < dim else 0
    return d


def lcs_seed_grid(ctx, desc: SeedDesc, field=None):
    out = ctypes.c_void_p()
    _check(ctx, load().lcs_seed_grid(ctx, ctypes.byref(desc), field, ctypes.byref(out)))
    return out.value


def lcs_seed_aux_field(ctx, lattice, field, delta):
    """lcs_seed_aux for a lattice made on `field` (mesh fields: the points get their exact cells)."""
    return lcs_seed_aux(ctx, lattice, delta, field)


def lcs_seed_aux(ctx, lattice, delta, field=None):
    """The 2 dim auxiliary points around every seed of a lattice, at +-delta[b] along each axis b
    (located on `field` when the lattice was made on a mesh field)."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    out = ctypes.c_void_p()
    if field is None:
        _check(ctx, load().lcs_seed_aux(ctx, lattice, d.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)))
    else:
        _check(ctx, load().lcs_seed_aux_field(ctx, lattice, field, d.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(out)))
    return out.value


def lcs_seeds_count(seeds) -> int:
    return int(load().lcs_seeds_count(seeds))


def lcs_seeds_get(ctx, seeds, xyz=None, cells=None):
    px, dx = _ptr(xyz)
    pc, dc = _ptr(cells)
    on_dev = dx if xyz is not None else dc
    if xyz is not None and cells is not None and dx != dc:
        raise ValueError("xyz and cells must both be host or both be device buffers")
    _check(ctx, load().lcs_seeds_get(ctx, seeds, ctypes.c_void_p(px), ctypes.c_void_p(pc), on_dev))


def lcs_free_seeds(seeds):
    load().lcs_free_seeds(seeds)


# -------------------------------------------------------------- flow map

def advect_opts(method=RK4, t0=0.0, T=0.0, dt=0.0, job_t0=None, job_T=None, rtol=1e-6, atol=1e-6, h0=0.01,
                max_steps=0, walk_limit=0, block_threads=0, variant=0, episode_steps=0, tracers_per_thread=0,
                use_graph=False, surrogate=None, gate_tol=1e-3, snap_T=None, variational=False, wait_limit=0.0):
    o = AdvectOpts()
    o.method, o.t0, o.T, o.dt = int(method), float(t0), float(T), float(dt)
    o.rtol, o.atol, o.h0, o.max_steps = float(rtol), float(atol), float(h0), int(max_steps)
    o.walk_limit, o.block_threads, o.variant = int(walk_limit), int(block_threads), int(variant)
    o.episode_steps = int(episode_steps)
    o.tracers_per_thread = int(tracers_per_thread)
    o.use_graph = int(bool(use_graph))
    o.surrogate = surrogate
    o.gate_tol = float(gate_tol)
    o.variational = int(bool(variational))
    o.wait_limit = float(wait_limit)
    keep = []
    if snap_T is not None and len(snap_T) > 0:
        sn = np.ascontiguousarray(snap_T, dtype=np.float64)
        o.nsnap, o.snap_T = len(sn), sn.ctypes.data
        keep.append(sn)
    if job_t0 is not None:
        a = np.ascontiguousarray(job_t0, dtype=np.float64)
        b = np.ascontiguousarray(job_T, dtype=np.float64)
        o.njobs = len(a)
        o.job_t0, o.job_T = a.ctypes.data, b.ctypes.data
        keep += [a, b]
        if len(a) == 1:   # the library reads a single job from t0 and T
            o.t0, o.T = float(a[0]), float(b[0])
    else:
        o.njobs = 1
    o._keep = tuple(keep)
    return o


def lcs_flowmap_create(ctx, seeds, njobs=1):
    out = ctypes.c_void_p()
    _check(ctx, load().lcs_flowmap_create(ctx, seeds, int(njobs), ctypes.byref(out)))
    return out.value


def lcs_advect(ctx, field, seeds, opts: AdvectOpts, fm):
    _check(ctx, load().lcs_advect(ctx, field, seeds, ctypes.byref(opts), fm))


def lcs_flowmap_get(ctx, fm, job=0, xyz=None, status=None, t_exit=None):
    ptrs = [_ptr(a) for a in (xyz, status, t_exit)]
    devs = {d for (p, d), a in zip(ptrs, (xyz, status, t_exit)) if a is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device buffers")
    _check(ctx, load().lcs_flowmap_get(ctx, fm, int(job), *[ctypes.c_void_p(p) for p, _ in ptrs],
                                       devs.pop() if devs else 0))


def lcs_flowmap_set(ctx, fm, job, xyz, status, T, t_exit=None):
    """Overwrite job `job` with end states computed elsewhere: xyz [dim][N] float32, status [N] uint8,
    t_exit [N] float32 or None, T the job's integration time."""
    arrs = (xyz, status, t_exit)
    ptrs = [_ptr(a) for a in arrs]
    devs = {d for (p, d), a in zip(ptrs, arrs) if a is not None}
    if len(devs) > 1:
        raise ValueError("inputs must all be host or all be device buffers")
    _check(ctx, load().lcs_flowmap_set(ctx, fm, int(job), *[ctypes.c_void_p(p) for p, _ in ptrs], float(T),
                                       devs.pop() if devs else 0))


def lcs_flowmap_steps(ctx, fm, job, steps):
    p, dev = _ptr(steps)
    _check(ctx, load().lcs_flowmap_steps(ctx, fm, int(job), ctypes.c_void_p(p), dev))


def lcs_free_flowmap(fm):
    load().lcs_free_flowmap(fm)


def lcs_autotune(ctx, field, seeds, opts: AdvectOpts, cache_path=None):
    """Tune opts in place (variant, block_threads, tracers_per_thread, episode_steps); returns opts."""
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(ctx, load().lcs_autotune(ctx, field, seeds, ctypes.byref(opts), path))
    return opts


# ----------------------------------------------------- grad F, C, FTLE

def lcs_cauchy_green(ctx, fm, job, C):
    p, dev = _ptr(C)
    _check(ctx, load().lcs_cauchy_green(ctx, fm, int(job), ctypes.c_void_p(p), dev))


def lcs_ftle(ctx, fm, job, ftle, lambda_max=None, C=None):
    ptrs = [_ptr(a) for a in (ftle, lambda_max, C)]
    devs = {d for (p, d), a in zip(ptrs, (ftle, lambda_max, C)) if a is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device buffers")
    _check(ctx, load().lcs_ftle(ctx, fm, int(job), *[ctypes.c_void_p(p) for p, _ in ptrs], devs.pop()))


def lcs_ftle_early(ctx, field, seeds, opts: AdvectOpts, fm, job, ftle, t_eval=None):
    """FTLE with early Cauchy-Green evaluation where a seed's stencil leaves the domain; t_eval gets the
    horizon of each value."""
    ptrs = [_ptr(a) for a in (ftle, t_eval)]
    devs = {d for (p, d), a in zip(ptrs, (ftle, t_eval)) if a is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device buffers")
    _check(ctx, load().lcs_ftle_early(ctx, field, seeds, ctypes.byref(opts), fm, int(job),
                                      *[ctypes.c_void_p(p) for p, _ in ptrs], devs.pop()))


def lcs_ftle_variational(ctx, fm, job, ftle, lambda_max=None, C=None):
    """FTLE from the variational grad F (after lcs_advect with variational=True)."""
    ptrs = [_ptr(a) for a in (ftle, lambda_max, C)]
    devs = {d for (p, d), a in zip(ptrs, (ftle, lambda_max, C)) if a is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device buffers")
    _check(ctx, load().lcs_ftle_variational(ctx, fm, int(job), *[ctypes.c_void_p(p) for p, _ in ptrs], devs.pop()))


def lcs_flowmap_grad(ctx, fm, job, grad):
    """Variational grad F [N][dim][dim] of job `job`."""
    p, d = _ptr(grad)
    _check(ctx, load().lcs_flowmap_grad(ctx, fm, int(job), ctypes.c_void_p(p), d))


def lcs_cg_eigen(ctx, fm, job, eigval=None, eigvec=None):
    """Eigenvalues [N][dim] (ascending) and unit eigenvectors [N][dim][dim] of C (either may be None)."""
    ptrs = [_ptr(a) for a in (eigval, eigvec)]
    devs = {d for (p, d), a in zip(ptrs, (eigval, eigvec)) if a is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device buffers")
    _check(ctx, load().lcs_cg_eigen(ctx, fm, int(job), *[ctypes.c_void_p(p) for p, _ in ptrs],
                                    devs.pop() if devs else 0))


# ------------------------------------------------------------ kernel timing

def lcs_timing_enable(ctx, on=True):
    _check(ctx, load().lcs_timing_enable(ctx, int(bool(on))))


def lcs_timing_read(ctx, phase):
    """(total milliseconds, launches) of the phase's kernels since the last read."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(ctx, load().lcs_timing_read(ctx, int(phase), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ---------------------------------------------- advection without allocation

def lcs_advect_rk4_noalloc(ctx, field, seeds, t0, T, dt, xyz, status, t_exit):
    """RK4 flow map of one job into caller-provided DEVICE tensors; the library allocates nothing.

    For callers that cannot allocate device memory (see include/lcs.h).  `seeds` is a [dim][n] FP32
    device tensor; `xyz` [dim][n] FP32, `status` [n] uint8 and `t_exit` [n] FP32 are device outputs.
    """
    import torch

    L = load()
    dim, dev = L.lcs_field_dim(field), L.lcs_context_device(ctx)
    if dim not in (2, 3) or dev < 0:
        raise ValueError("lcs_advect_rk4_noalloc: null field or context")
    # the C entry point cannot see buffer sizes: every shape, type and device is checked here
    for name, a in (("seeds", seeds), ("xyz", xyz), ("status", status), ("t_exit", t_exit)):
        if not (hasattr(a, "is_cuda") and a.is_cuda and a.device.index == dev):
            raise ValueError("lcs_advect_rk4_noalloc: %s must be a tensor on the context's device cuda:%d" % (name, dev))
    if seeds.dim() != 2 or seeds.shape[0] != dim or seeds.dtype != torch.float32:
        raise ValueError("lcs_advect_rk4_noalloc: seeds must be [%d][n] float32" % dim)
    n = int(seeds.shape[1])
    if tuple(xyz.shape) != (dim, n) or xyz.dtype != torch.float32:
        raise ValueError("lcs_advect_rk4_noalloc: xyz must be [%d][%d] float32" % (dim, n))
    if tuple(status.shape) != (n,) or status.dtype != torch.uint8:
        raise ValueError("lcs_advect_rk4_noalloc: status must be [%d] uint8" % n)
    if tuple(t_exit.shape) != (n,) or t_exit.dtype != torch.float32:
        raise ValueError("lcs_advect_rk4_noalloc: t_exit must be [%d] float32" % n)
    ptrs = [_ptr(a) for a in (seeds, xyz, status, t_exit)]
    _check(ctx, load().lcs_advect_rk4_noalloc(ctx, field, ctypes.c_void_p(ptrs[0][0]), n, float(t0), float(T),
                                              float(dt), *[ctypes.c_void_p(p) for p, _ in ptrs[1:]]))


# ------------------------------------------------------------ tensor-core GEMM

def lcs_gemm_bf16(ctx, A, B, C, splits=1, accumulate=False):
    """C[M x N] (+)= A[M x K] @ B[N x K]^T; A, B bf16 CUDA tensors, C float32 CUDA tensor."""
    M, K = A.shape
    N = B.shape[0]
    _check(ctx, load().lcs_gemm_bf16(ctx, M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                     ctypes.c_void_p(B.data_ptr()), B.stride(0), ctypes.c_void_p(C.data_ptr()),
                                     C.stride(0), int(splits), int(bool(accumulate))))


# ------------------------------------------------------------ learned surrogate

class MlpDesc(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 2), ("kx", ctypes.c_double), ("ky", ctypes.c_double),
                ("omega", ctypes.c_double), ("tau", ctypes.c_double), ("out_scale", ctypes.c_double)]


def mlp_desc(center, kx, ky, omega, tau, out_scale):
    d = MlpDesc()
    d.center[0], d.center[1] = float(center[0]), float(center[1])
    d.kx, d.ky, d.omega, d.tau, d.out_scale = float(kx), float(ky), float(omega), float(tau), float(out_scale)
    return d


def lcs_mlp_create(ctx, desc, params):
    p, dev = _ptr(params)
    out = ctypes.c_void_p()
    _check(ctx, load().lcs_mlp_create(ctx, ctypes.byref(desc), ctypes.c_void_p(p), dev, ctypes.byref(out)))
    return out.value


def lcs_mlp_set_params(ctx, mlp, params):
    p, dev = _ptr(params)
    _check(ctx, load().lcs_mlp_set_params(ctx, mlp, ctypes.c_void_p(p), dev))


def lcs_mlp_get_params(ctx, mlp, params):
    p, dev = _ptr(params)
    _check(ctx, load().lcs_mlp_get_params(ctx, mlp, ctypes.c_void_p(p), dev))


def lcs_mlp_free(mlp):
    load().lcs_mlp_free(mlp)


def lcs_mlp_forward(ctx, mlp, xyt, out):
    """out [3][n] = network outputs at xyt [3][n] (x, y, t rows)."""
    p, dev = _ptr(xyt)
    q, dev2 = _ptr(out)
    if dev != dev2:
        raise ValueError("xyt and out must both be host or both be device buffers")
    n = xyt.shape[1]
    _check(ctx, load().lcs_mlp_forward(ctx, mlp, n, ctypes.c_void_p(p), ctypes.c_void_p(q), dev))


def lcs_mlp_loss_grad(ctx, mlp, xyt, disp, rho_weight, grads=None):
    """Mean loss (returned) and its gradient (into grads, if given) over the points xyt [3][n]."""
    p, dev = _ptr(xyt)
    q, dev2 = _ptr(disp)
    g, dev3 = _ptr(grads)
    if dev != dev2 or (grads is not None and dev3 != dev):
        raise ValueError("xyt, disp and grads must all be host or all be device buffers")
    loss = ctypes.c_double(0.0)
    _check(ctx, load().lcs_mlp_loss_grad(ctx, mlp, xyt.shape[1], ctypes.c_void_p(p), ctypes.c_void_p(q),
                                         float(rho_weight), ctypes.c_void_p(g), ctypes.byref(loss), dev))
    return loss.value


def lcs_mlp_adam(ctx, mlp, grads=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    g, dev = _ptr(grads)
    _check(ctx, load().lcs_mlp_adam(ctx, mlp, ctypes.c_void_p(g), dev, float(lr), float(beta1), float(beta2),
                                    float(eps)))


class TrainDesc(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_longlong), ("epochs", ctypes.c_int), ("lr", ctypes.c_double),
                ("lr_min", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("rho_weight", ctypes.c_double), ("dt", ctypes.c_double)]


def train_desc(batch=65536, epochs=10, lr=1e-3, lr_min=1e-5, beta1=0.9, beta2=0.999, eps=1e-8, rho_weight=0.01,
               dt=0.05):
    d = TrainDesc()
    d.batch, d.epochs, d.lr, d.lr_min = int(batch), int(epochs), float(lr), float(lr_min)
    d.beta1, d.beta2, d.eps, d.rho_weight, d.dt = float(beta1), float(beta2), float(eps), float(rho_weight), float(dt)
    return d


def lcs_surrogate_train(ctx, field, mlp, desc, samples):
    """Train on samples [3][ns] (x0, y0, t0); returns the mean loss of each epoch."""
    p, dev = _ptr(samples)
    out = np.empty(desc.epochs, dtype=np.float64)
    _check(ctx, load().lcs_surrogate_train(ctx, field, mlp, ctypes.byref(desc), samples.shape[1], ctypes.c_void_p(p),
                                           dev, out.ctypes.data))
    return out

