"""Plain FP64 CPU oracle for the LCS flow-map / FTLE hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_2209_13775_gb300`` never imports it, and it never imports the library:
the two share no code.  Inputs reach both sides from
``paper_2209_13775_gb300.inputs`` (seeded generators, none of the method's
arithmetic).

The C part (``lcs_oracle.c``) is the literal FP64 definition of each step of the
paper's path (arXiv 2209.13775): the linear-in-time, (bi/tri)linear-in-space
Interpolator and the Seed, Flow Map and Cauchy-Green filters of Sec. 2, Eq. 1 and
Eq. 2, and the local cell search of Sec. 3.1 on tetrahedra and triangles.  This module only
marshals numpy arrays into it.  ``oracle.mlp`` holds the FP64 network oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_HDR = os.path.join(_HERE, "lcs_oracle.h")
_SO = os.path.join(_HERE, "liblcs_oracle.so")
_lock = threading.Lock()
_lib = None

OK, LEFT, OUTSIDE, MAXSTEPS = 0, 1, 2, 3
AN_GYRE, AN_ABC, AN_AFFINE, AN_PIPE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``lcs_oracle.c`` into ``liblcs_oracle.so`` (gcc, FP64, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Rect(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("nframes", ctypes.c_int),
                ("times", ctypes.c_void_p), ("time_periodic", ctypes.c_int),
                ("period", ctypes.c_double), ("frames", ctypes.c_void_p)]


class _Tet(ctypes.Structure):
    _fields_ = [("nnodes", ctypes.c_longlong), ("ncells", ctypes.c_longlong),
                ("xyz", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("nbrs", ctypes.c_void_p),
                ("nframes", ctypes.c_int), ("times", ctypes.c_void_p),
                ("time_periodic", ctypes.c_int), ("period", ctypes.c_double),
                ("frames", ctypes.c_void_p), ("walk_limit", ctypes.c_int)]


class _Tri(ctypes.Structure):
    _fields_ = [("nnodes", ctypes.c_longlong), ("ncells", ctypes.c_longlong),
                ("xy", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("nbrs", ctypes.c_void_p),
                ("nframes", ctypes.c_int), ("times", ctypes.c_void_p),
                ("time_periodic", ctypes.c_int), ("period", ctypes.c_double),
                ("frames", ctypes.c_void_p), ("walk_limit", ctypes.c_int)]


class _Analytic(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("p", ctypes.c_double * 24)]


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, I, LL, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
            L.ora_time_locate.argtypes = [P, I, I, D, D, P, P]
            L.ora_rect_velocity.argtypes = [P, P, D, P]
            L.ora_analytic_velocity.argtypes = [P, P, D, P]
            L.ora_tet_velocity.argtypes = [P, P, D, P, P]
            L.ora_seed_grid.argtypes = [I, P, P, P, P, P]
            L.ora_rk4.argtypes = [I, P, I, LL, P, P, D, D, D, P, P, P]
            L.ora_rk4_var.argtypes = [P, LL, P, D, D, D, P, P, P, P]
            L.ora_rk4_var.restype = LL
            L.ora_rk4_var_kind.argtypes = [I, P, I, LL, P, P, D, D, D, P, P, P, P]
            L.ora_rk4_var_kind.restype = LL
            L.ora_tet_velocity_grad.argtypes = [P, P, D, P, P, P]
            L.ora_tri_velocity_grad.argtypes = [P, P, D, P, P, P]
            L.ora_rect_velocity_grad.argtypes = [P, P, D, P, P]
            L.ora_rk4.restype = LL
            L.ora_dp45.argtypes = [I, P, I, LL, P, P, D, D, D, D, D, LL, I, I, P, P, P, P]
            L.ora_dp45.restype = LL
            L.ora_flowmap_gradient.argtypes = [I, P, P, P, P, P, P, P]
            L.ora_cauchy_green.argtypes = [I, LL, P, P]
            L.ora_eig_sym.argtypes = [I, P, P]
            L.ora_eigvec_sym.argtypes = [I, P, P, P]
            L.ora_cg_eigen.argtypes = [I, LL, P, P, P]
            L.ora_ftle.argtypes = [I, LL, P, D, P, P]
            L.ora_orient3d_exact.argtypes = [P, P, P, P]
            L.ora_tet_contains.argtypes = [P, LL, P, P]
            L.ora_tet_locate_brute.argtypes = [P, P]
            L.ora_tet_locate_brute.restype = LL
            L.ora_tet_locate_walk.argtypes = [P, LL, P]
            L.ora_tet_locate_walk.restype = LL
            L.ora_tri_velocity.argtypes = [P, P, D, P, P]
            L.ora_orient2d_exact.argtypes = [P, P, P]
            L.ora_tri_contains.argtypes = [P, LL, P, P]
            L.ora_tri_locate_brute.argtypes = [P, P]
            L.ora_tri_locate_brute.restype = LL
            L.ora_tri_locate_walk.argtypes = [P, LL, P]
            L.ora_tri_locate_walk.restype = LL
            L.ora_set_threads.argtypes = [I]
            L.ora_boundary_build.argtypes = [I, P, D]
            L.ora_boundary_build.restype = P
            L.ora_boundary_free.argtypes = [P]
            L.ora_boundary_distance.argtypes = [P, P, D]
            L.ora_boundary_distance.restype = D
            L.ora_boundary_distance_brute.argtypes = [P, P]
            L.ora_boundary_distance_brute.restype = D
            L.ora_rk4_margin.argtypes = [I, P, I, LL, P, P, D, D, D, P, P, P, P, D, P]
            L.ora_rk4_margin.restype = LL
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    """OpenMP threads used over seeds (<=0 keeps the default); returns the count in effect."""
    return int(lib().ora_set_threads(int(n)))


# ----------------------------------------------------------------- fields

class RectField:
    """Rectilinear frames [nframes][nz][ny][nx][dim] FP32 (Sec. 2 Interpolator)."""

    kind = 0

    def __init__(self, frames, times, origin, spacing, periodic=(0, 0, 0),
                 time_periodic=False, period=0.0):
        self.frames = np.ascontiguousarray(frames, dtype=np.float32)
        self.dim = int(self.frames.shape[-1])
        grid = self.frames.shape[1:-1][::-1]          # (nx, ny[, nz])
        self.n = list(grid) + [1] * (3 - len(grid))
        self.times = np.ascontiguousarray(times, dtype=np.float64)
        s = _Rect()
        s.dim = self.dim
        for a in range(3):
            s.n[a] = int(self.n[a])
            s.origin[a] = float(origin[a]) if a < len(origin) else 0.0
            s.spacing[a] = float(spacing[a]) if a < len(spacing) else 1.0
            s.periodic[a] = int(periodic[a]) if a < len(periodic) else 0
        s.nframes = int(self.frames.shape[0])
        s.times = self.times.ctypes.data
        s.time_periodic = int(bool(time_periodic))
        s.period = float(period)
        s.frames = self.frames.ctypes.data
        self.struct = s

    def velocity(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.zeros(self.dim)
        lib().ora_rect_velocity(ctypes.byref(self.struct), _p(x), float(t), _p(u))
        return u


class AnalyticField:
    """Analytic velocity (pins only): gyre, ABC, affine, pipe."""

    kind = 1

    def __init__(self, kind: int, dim: int, params):
        s = _Analytic()
        s.kind, s.dim = int(kind), int(dim)
        for i, v in enumerate(params):
            s.p[i] = float(v)
        self.dim = dim
        self.struct = s

    def velocity(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.zeros(self.dim)
        lib().ora_analytic_velocity(ctypes.byref(self.struct), _p(x), float(t), _p(u))
        return u


def gyre(A=0.1, eps=0.25, omega=2 * np.pi / 10):
    return AnalyticField(AN_GYRE, 2, [A, eps, omega])


def abc(A=np.sqrt(3.0), B=np.sqrt(2.0), C=1.0, mod=0.5):
    return AnalyticField(AN_ABC, 3, [A, B, C, mod])


def affine(A0, A1=None, b0=None, b1=None):
    A0 = np.asarray(A0, dtype=np.float64)
    d = A0.shape[0]
    p = np.zeros(24)
    M0 = np.zeros((3, 3)); M0[:d, :d] = A0
    M1 = np.zeros((3, 3))
    if A1 is not None:
        M1[:d, :d] = np.asarray(A1, dtype=np.float64)
    p[0:9] = M0.ravel(); p[9:18] = M1.ravel()
    if b0 is not None:
        p[18:18 + d] = b0
    if b1 is not None:
        p[21:21 + d] = b1
    return AnalyticField(AN_AFFINE, d, p)


def pipe(R=1.0, L=10.0, amp=0.05, phases=(0.0, 0.0, 0.0, 0.0)):
    return AnalyticField(AN_PIPE, 3, [R, L, amp] + list(phases))


class TetField:
    """Tetrahedral mesh with nodal frames [nframes][nnodes][3] FP32 (Sec. 3.1)."""

    kind = 2
    dim = 3

    def __init__(self, xyz, tets, nbrs, frames, times, time_periodic=False, period=0.0,
                 walk_limit=100000):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.nbrs = np.ascontiguousarray(nbrs, dtype=np.int32)
        self.frames = np.ascontiguousarray(frames, dtype=np.float32)
        self.times = np.ascontiguousarray(times, dtype=np.float64)
        s = _Tet()
        s.nnodes = self.xyz.shape[0]
        s.ncells = self.tets.shape[0]
        s.xyz = self.xyz.ctypes.data
        s.tets = self.tets.ctypes.data
        s.nbrs = self.nbrs.ctypes.data
        s.nframes = int(self.frames.shape[0])
        s.times = self.times.ctypes.data
        s.time_periodic = int(bool(time_periodic))
        s.period = float(period)
        s.frames = self.frames.ctypes.data
        s.walk_limit = int(walk_limit)
        self.struct = s

    def velocity(self, x, t, cell=0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.zeros(3)
        c = ctypes.c_int(int(cell))
        out = lib().ora_tet_velocity(ctypes.byref(self.struct), _p(x), float(t), ctypes.byref(c), _p(u))
        return (None if out else u), c.value

    def contains(self, t, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        onb = ctypes.c_int(0)
        r = lib().ora_tet_contains(ctypes.byref(self.struct), int(t), _p(p), ctypes.byref(onb))
        return bool(r), bool(onb.value)

    def locate_brute(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        return int(lib().ora_tet_locate_brute(ctypes.byref(self.struct), _p(p)))

    def locate_walk(self, p, start=0):
        p = np.ascontiguousarray(p, dtype=np.float32)
        return int(lib().ora_tet_locate_walk(ctypes.byref(self.struct), int(start), _p(p)))

    def locate_seeds(self, seeds_soa):
        """Exact cell of every FP32 seed (-1 outside), walking from the previous seed's cell."""
        s = np.ascontiguousarray(np.asarray(seeds_soa, dtype=np.float32).T)
        out = np.empty(s.shape[0], dtype=np.int32)
        start = 0
        for i in range(s.shape[0]):
            c = self.locate_walk(s[i], start)
            out[i] = c
            if c >= 0:
                start = c
        return out


class TriField:
    """Triangle mesh with nodal frames [nframes][nnodes][2] FP32 (2D unstructured data, Sec. 4)."""

    kind = 3
    dim = 2

    def __init__(self, xy, tris, nbrs, frames, times, time_periodic=False, period=0.0,
                 walk_limit=100000):
        self.xy = np.ascontiguousarray(xy, dtype=np.float32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.nbrs = np.ascontiguousarray(nbrs, dtype=np.int32)
        self.frames = np.ascontiguousarray(frames, dtype=np.float32)
        self.times = np.ascontiguousarray(times, dtype=np.float64)
        s = _Tri()
        s.nnodes = self.xy.shape[0]
        s.ncells = self.tris.shape[0]
        s.xy = self.xy.ctypes.data
        s.tris = self.tris.ctypes.data
        s.nbrs = self.nbrs.ctypes.data
        s.nframes = int(self.frames.shape[0])
        s.times = self.times.ctypes.data
        s.time_periodic = int(bool(time_periodic))
        s.period = float(period)
        s.frames = self.frames.ctypes.data
        s.walk_limit = int(walk_limit)
        self.struct = s

    def velocity(self, x, t, cell=0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.zeros(2)
        c = ctypes.c_int(int(cell))
        out = lib().ora_tri_velocity(ctypes.byref(self.struct), _p(x), float(t), ctypes.byref(c), _p(u))
        return (None if out else u), c.value

    def contains(self, t, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        onb = ctypes.c_int(0)
        r = lib().ora_tri_contains(ctypes.byref(self.struct), int(t), _p(p), ctypes.byref(onb))
        return bool(r), bool(onb.value)

    def locate_brute(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        return int(lib().ora_tri_locate_brute(ctypes.byref(self.struct), _p(p)))

    def locate_walk(self, p, start=0):
        p = np.ascontiguousarray(p, dtype=np.float32)
        return int(lib().ora_tri_locate_walk(ctypes.byref(self.struct), int(start), _p(p)))

    def locate_seeds(self, seeds_soa):
        """Exact cell of every FP32 seed (-1 outside), walking from the previous seed's cell."""
        s = np.ascontiguousarray(np.asarray(seeds_soa, dtype=np.float32).T)
        out = np.empty(s.shape[0], dtype=np.int32)
        start = 0
        for i in range(s.shape[0]):
            c = self.locate_walk(s[i], start)
            out[i] = c
            if c >= 0:
                start = c
        return out


def orient2d(a, b, c):
    """Exact sign of (b - a) x (c - a) for FP32 points."""
    a, b, c = (np.ascontiguousarray(v, dtype=np.float32) for v in (a, b, c))
    return int(lib().ora_orient2d_exact(_p(a), _p(b), _p(c)))


def time_locate(times, t, time_periodic=False, period=0.0):
    times = np.ascontiguousarray(times, dtype=np.float64)
    k = ctypes.c_int(0)
    a = ctypes.c_double(0.0)
    lib().ora_time_locate(_p(times), len(times), int(bool(time_periodic)), float(period), float(t),
                          ctypes.byref(k), ctypes.byref(a))
    return k.value, a.value


def orient3d(a, b, c, d) -> int:
    arr = [np.ascontiguousarray(v, dtype=np.float32) for v in (a, b, c, d)]
    return int(lib().ora_orient3d_exact(*[_p(v) for v in arr]))


# ------------------------------------------------------------ path steps

def seed_grid(dim, n, lo, hi, endpoint=(1, 1, 1)):
    """FP32 seed lattice [dim][N] (Sec. 2 Seed)."""
    nn = np.zeros(3, dtype=np.int32); nn[:dim] = n[:dim]
    if dim == 2:
        nn[2] = 1
    l3 = np.zeros(3); l3[:dim] = lo[:dim]
    h3 = np.zeros(3); h3[:dim] = hi[:dim]
    e3 = np.ones(3, dtype=np.int32); e3[:dim] = endpoint[:dim]
    N = int(np.prod(nn[:dim]))
    out = np.empty((dim, N), dtype=np.float32)
    lib().ora_seed_grid(dim, _p(nn), _p(l3), _p(h3), _p(e3), _p(out))
    return out


def lattice_spacing(dim, n, lo, hi, endpoint=(1, 1, 1)):
    """Lattice step per axis; an axis of one node has no step (1.0 stands in: no difference uses it)."""
    return np.array([(hi[a] - lo[a]) / ((n[a] - 1) if endpoint[a] else n[a]) if (n[a] > 1 or not endpoint[a])
                     else 1.0 for a in range(dim)])


def rk4_var(field, x0, t0, T, dt, cells=None):
    """RK4 with the variational equations dM/dt = J M (any field kind; cells as for rk4).
    x0 [dim][N] -> (xT, M [N][dim][dim], status, t_exit)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    dim, n = x0.shape
    xT = np.empty_like(x0)
    M = np.empty((n, dim, dim))
    st = np.empty(n, dtype=np.uint8)
    te = np.empty(n, dtype=np.float64)
    c = None if cells is None else np.ascontiguousarray(cells, dtype=np.int32)
    lib().ora_rk4_var_kind(field.kind, ctypes.byref(field.struct), dim, n, _p(x0), None if c is None else _p(c),
                           float(t0), float(T), float(dt), _p(xT), _p(M), _p(st), _p(te))
    return xT, M, st, te


def velocity_grad(field, x, t, cell=0):
    """u(x, t) and its spatial Jacobian (rectilinear fields; on meshes also the cell, None outside)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.empty(field.dim)
    J = np.empty((field.dim, field.dim))
    if field.kind == 0:
        lib().ora_rect_velocity_grad(ctypes.byref(field.struct), _p(x), float(t), _p(u), _p(J))
        return u, J
    c = ctypes.c_int(int(cell))
    fn = lib().ora_tri_velocity_grad if field.kind == 3 else lib().ora_tet_velocity_grad
    out = fn(ctypes.byref(field.struct), _p(x), float(t), ctypes.byref(c), _p(u), _p(J))
    return (None, None) if out else (u, J)


def rk4(field, x0, t0, T, dt, cells=None, margin=None):
    """Fixed-step RK4 flow map (Sec. 2 Flow Map, Sec. 3.1).  x0 [dim][N] -> (xT, status, t_exit).
    margin = rmax (mesh fields): also each tracer's smallest distance from the mesh boundary over the
    stage points it evaluated, capped at rmax -> (xT, status, t_exit, margin)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    dim, n = x0.shape
    xT = np.empty_like(x0)
    st = np.empty(n, dtype=np.uint8)
    te = np.empty(n, dtype=np.float64)
    c = None if cells is None else np.ascontiguousarray(cells, dtype=np.int32)
    if margin is None:
        lib().ora_rk4(field.kind, ctypes.byref(field.struct), dim, n, _p(x0),
                      None if c is None else _p(c), float(t0), float(T), float(dt),
                      _p(xT), _p(st), _p(te))
        return xT, st, te
    mg = np.empty(n)
    bi = lib().ora_boundary_build(field.kind, ctypes.byref(field.struct), float(margin))
    try:
        lib().ora_rk4_margin(field.kind, ctypes.byref(field.struct), dim, n, _p(x0),
                             None if c is None else _p(c), float(t0), float(T), float(dt),
                             _p(xT), _p(st), _p(te), bi, float(margin), _p(mg))
    finally:
        lib().ora_boundary_free(bi)
    return xT, st, te, mg


def boundary_distance(field, pts, rmax=None):
    """Distance of each point pts [dim][N] from the boundary of a mesh field: every boundary face
    tested (rmax None), or through the grid index with the cap rmax."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    dim, n = pts.shape
    bi = lib().ora_boundary_build(field.kind, ctypes.byref(field.struct), float(rmax or 1e-3))
    out = np.empty(n)
    try:
        for i in range(n):
            p = np.ascontiguousarray(pts[:, i])
            out[i] = (lib().ora_boundary_distance_brute(bi, _p(p)) if rmax is None
                      else lib().ora_boundary_distance(bi, _p(p), float(rmax)))
    finally:
        lib().ora_boundary_free(bi)
    return out


def dp45(field, x0, t0, T, h0=0.01, rtol=1e-6, atol=1e-6, max_steps=1000000, group=1,
         adaptive=True, cells=None):
    """Dormand-Prince 5(4), per-tracer (group=1) or 32-lane shared step (group=32)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    dim, n = x0.shape
    xT = np.empty_like(x0)
    st = np.empty(n, dtype=np.uint8)
    te = np.empty(n, dtype=np.float64)
    ns = np.empty(n, dtype=np.int64)
    c = None if cells is None else np.ascontiguousarray(cells, dtype=np.int32)
    lib().ora_dp45(field.kind, ctypes.byref(field.struct), dim, n, _p(x0),
                   None if c is None else _p(c), float(t0), float(T), float(h0), float(rtol),
                   float(atol), int(max_steps), int(group), int(bool(adaptive)),
                   _p(xT), _p(st), _p(te), _p(ns))
    return xT, st, te, ns


def flowmap_gradient(dim, n, h, periodic, period, xT, status):
    """grad F [N][dim][dim] by lattice finite differences (Sec. 2 Cauchy-Green)."""
    xT = np.ascontiguousarray(xT, dtype=np.float64)
    N = xT.shape[1]
    nn = np.ones(3, dtype=np.int32); nn[:dim] = n[:dim]
    h3 = np.ones(3); h3[:dim] = h[:dim]
    p3 = np.zeros(3, dtype=np.int32); p3[:dim] = periodic[:dim]
    L3 = np.zeros(3); L3[:dim] = period[:dim]
    st = np.ascontiguousarray(status, dtype=np.uint8)
    grad = np.empty((N, dim, dim))
    lib().ora_flowmap_gradient(dim, _p(nn), _p(h3), _p(p3), _p(L3), _p(xT), _p(st), _p(grad))
    return grad


def cauchy_green(grad):
    """Eq. 1 packed: 2D (C00, C01, C11), 3D (C00, C01, C02, C11, C12, C22)."""
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    N, dim, _ = grad.shape
    C = np.empty((N, 3 if dim == 2 else 6))
    lib().ora_cauchy_green(dim, N, _p(grad), _p(C))
    return C


def eig_sym(Cp, dim):
    Cp = np.ascontiguousarray(Cp, dtype=np.float64)
    e = np.empty(dim)
    lib().ora_eig_sym(dim, _p(Cp), _p(e))
    return e


def eigvec_sym(Cp, dim):
    """Eigenvalues (ascending) and unit eigenvectors (rows) of one packed symmetric matrix."""
    Cp = np.ascontiguousarray(Cp, dtype=np.float64)
    e = np.empty(dim)
    v = np.empty((dim, dim))
    lib().ora_eigvec_sym(dim, _p(Cp), _p(e), _p(v))
    return e, v


def cg_eigen(C, dim):
    """Eigenvalues [N][dim] (ascending) and eigenvectors [N][dim][dim] (row k: that of eigenvalue k)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = C.shape[0]
    e = np.empty((N, dim))
    v = np.empty((N, dim, dim))
    lib().ora_cg_eigen(dim, N, _p(C), _p(e), _p(v))
    return e, v


def fd_stencil_members(dim, n, periodic, valid0=None):
    """Lattice neighbours the finite differences of a seed use (Sec. 2 "Cauchy-Green"), chosen as the
    difference rule chooses them from the seeds valid at the start (valid0; all of them when None):
    per axis the two central neighbours when both are valid, else the two on a side whose two
    neighbours are valid (forward first), else none (-1).  On a lattice whose seeds are all valid
    that is: central, or the two inner neighbours at a non-periodic edge.  Returns [N][2 dim] ids."""
    N = int(np.prod(n[:dim]))
    p = np.arange(N)
    idx = [(p // int(np.prod(n[:a]))) % n[a] for a in range(dim)]
    strides = [int(np.prod(n[:a])) for a in range(dim)]
    valid = np.ones(N, dtype=bool) if valid0 is None else np.asarray(valid0, dtype=bool)
    out = np.empty((N, 2 * dim), dtype=np.int64)
    for a in range(dim):
        i = idx[a]

        def nbr(o):
            j = i + o
            if periodic[a]:
                return p + ((j % n[a]) - i) * strides[a]
            inside = (j >= 0) & (j < n[a])
            return np.where(inside, p + o * strides[a], -1)

        q = {o: nbr(o) for o in (1, -1, 2, -2)}
        ok = {o: (q[o] >= 0) & valid[np.maximum(q[o], 0)] for o in q}
        central = ok[1] & ok[-1]
        fwd = ~central & ok[1] & ok[2]
        bwd = ~central & ~fwd & ok[-1] & ok[-2]
        out[:, 2 * a] = np.where(central, q[1], np.where(fwd, q[1], np.where(bwd, q[-1], -1)))
        out[:, 2 * a + 1] = np.where(central, q[-1], np.where(fwd, q[2], np.where(bwd, q[-2], -1)))
    return out


def ftle_early(field, n, lo, hi, periodic, t0, T, dt, xT, status, t_exit, endpoint=None, cells=None):
    """Early Cauchy-Green evaluation (Sec. 2 "Flow Map": for trajectories that exit the data, the CG tensor
    is formed ahead of the horizon wherever such a trajectory is used) for fixed-step RK4, from a full
    run's (xT, status, t_exit) over (t0, t0 + T).

    Per seed: m = the fewest steps that the seed or any lattice neighbour its finite differences use
    (fd_stencil_members) stayed in the domain -- all steps for a tracer still OK at the end, one less
    than the step it left in otherwise.  m = all steps: the regular FTLE over |T|.  0 < m: grad F
    from those tracers re-integrated over m steps, C (Eq. 1), lambda_max and
    sigma = ln sqrt(lambda_max) / (m dt).  m = 0: NaN.  Returns (ftle, t_eval).

    Mesh fields (cells: each seed's start cell, -1 outside): a tracer that leaves is frozen at the
    start of the step it failed in, so its in-domain steps are |t_exit - t0| / dt; the stencil is the
    one the differences choose from the seeds inside the mesh at the start."""
    mesh = cells is not None
    dim = len(n)
    N = int(np.prod(n[:dim]))
    endpoint = endpoint if endpoint is not None else [0 if q else 1 for q in periodic]
    h = lattice_spacing(dim, n, lo, hi, endpoint)
    period = [hi[a] - lo[a] if periodic[a] else 0.0 for a in range(dim)]
    adt = abs(dt)
    ns = int(round(abs(T) / adt))
    ne = np.where(status == OK, ns, np.rint(np.abs(t_exit - t0) / adt).astype(np.int64) - (0 if mesh else 1))
    ne = np.where((status == OK) | (status == LEFT), np.maximum(ne, 0), 0)
    mem = fd_stencil_members(dim, n, periodic, None if not mesh else np.asarray(cells) >= 0)
    m = np.where((mem < 0).any(axis=1), 0, np.minimum(ne, ne[np.maximum(mem, 0)].min(axis=1)))
    G = flowmap_gradient(dim, n, h, periodic, period, xT, status)
    lam, sig = ftle(cauchy_green(G), dim, T)
    t_eval = np.full(N, abs(T))
    x0 = seed_grid(dim, n, lo, hi, endpoint).astype(np.float64)
    sgn = -1.0 if T < 0 else 1.0
    for mm in np.unique(m[m < ns]):
        seeds = np.nonzero(m == mm)[0]
        t_eval[seeds] = mm * adt
        if mm == 0:
            sig[seeds] = np.nan
            continue
        ids = np.unique(np.concatenate([seeds, mem[seeds].ravel()]))
        xm, stm, _ = rk4(field, x0[:, ids], t0, sgn * mm * adt, dt, cells=None if not mesh else np.asarray(cells)[ids])
        assert (stm == OK).all()
        xf = np.zeros((dim, N))
        sf = np.full(N, LEFT, dtype=np.uint8)
        xf[:, ids] = xm
        sf[ids] = OK
        Gm = flowmap_gradient(dim, n, h, periodic, period, xf, sf)[seeds]
        _, sg = ftle(cauchy_green(Gm), dim, mm * adt)
        sig[seeds] = sg
    return sig, t_eval


def aux_points(x0, delta):
    """Auxiliary points around each seed of x0 [dim][N] FP32 (Sec. 2 "Seed"): point (p dim + b) 2 + s is
    seed p moved by +delta[b] (s = 0) or -delta[b] (s = 1) along axis b, in FP64, rounded to FP32."""
    x0 = np.asarray(x0, dtype=np.float32)
    dim, N = x0.shape
    out = np.repeat(x0[:, :, None, None], dim, axis=2).repeat(2, axis=3)      # [dim][N][dim][2]
    for b in range(dim):
        base = x0[b].astype(np.float64)
        out[b, :, b, 0] = (base + float(delta[b])).astype(np.float32)
        out[b, :, b, 1] = (base - float(delta[b])).astype(np.float32)
    return out.reshape(dim, N * 2 * dim)


def aux_gradient(x0aux, xT, status):
    """grad F per lattice seed from its auxiliary points (Sec. 2 "Cauchy-Green", the auxiliary-point
    variant): grad F[a][b] = (F_a(+) - F_a(-)) / (x0_b(+) - x0_b(-)) with the FP32 starting points; NaN
    unless all 2 dim points are OK.  Returns [N][dim][dim]."""
    dim, M = np.shape(xT)
    N = M // (2 * dim)
    X = np.asarray(xT, dtype=np.float64).reshape(dim, N, dim, 2)
    X0 = np.asarray(x0aux, dtype=np.float32).astype(np.float64).reshape(dim, N, dim, 2)
    G = np.empty((N, dim, dim))
    for b in range(dim):
        den = X0[b, :, b, 0] - X0[b, :, b, 1]
        for a in range(dim):
            G[:, a, b] = (X[a, :, b, 0] - X[a, :, b, 1]) / den
    ok = (np.asarray(status).reshape(N, 2 * dim) == OK).all(axis=1)
    G[~ok] = np.nan
    return G


def ftle(C, dim, T):
    """lambda_max of C and sigma = ln(sqrt(lambda_max)) / |T|."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = C.shape[0]
    lam = np.empty(N)
    sig = np.empty(N)
    lib().ora_ftle(dim, N, _p(C), float(T), _p(lam), _p(sig))
    return lam, sig
