"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no step of the method: it only samples analytic velocity
fields at grid nodes (FP64, rounded to FP32 for storage) and builds meshes.
Both the CUDA library and the CPU oracle consume what it returns; neither
contributes to it.

The fields stand in for the paper's four applications (Sec. 3.2: double gyre,
3D Cartesian convection, 2D stenosis, 3D aneurysm on 1.01M tets), whose data
are not available:

* ``double_gyre``: the 2D Cartesian case itself (Shadden, Lekien, Marsden 2005),
  A = 0.1, eps = 0.25, omega = 2 pi / 10 on [0,2]x[0,1], 129x65 nodes, 101 frames.
* ``abc``: a time-modulated Arnold-Beltrami-Childress flow, 128^3 periodic nodes,
  64 frames on [0, 8]; stands in for the 3D Cartesian data.
* ``pipe_mesh`` / ``pipe_frames``: a Delaunay tetrahedralisation of a jittered
  lattice in a cylinder (R = 1, L = 10) carrying pulsatile Poiseuille flow plus
  a random-phase swirl; stands in for the 3D unstructured aneurysm data.
* ``stenosis_mesh`` / ``stenosis_frames``: a body-fitted triangulation of a 2D
  channel with a Gaussian constriction carrying pulsatile, flux-conserving
  Poiseuille flow plus a travelling wall-bounded wave; stands in for the 2D
  unstructured stenosis data.
* ``affine_frames``: u = (A0 + t A1) x + b, which bilinear/trilinear/P1
  interpolation reproduces exactly (used by parity tests with closed forms).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 1234


@dataclass
class RectInput:
    """Nodal frames on a rectilinear grid: frames[nframes][nz][ny][nx][dim] FP32."""

    frames: np.ndarray
    times: np.ndarray
    origin: tuple
    spacing: tuple
    periodic: tuple
    time_periodic: bool = False
    period: float = 0.0

    @property
    def dim(self) -> int:
        return int(self.frames.shape[-1])

    @property
    def n(self) -> tuple:
        return tuple(int(v) for v in self.frames.shape[1:-1][::-1])


@dataclass
class TetInput:
    """Tetrahedral mesh: xyz[nnodes][3] FP32, tets/nbrs[ncells][4] int32, frames[nf][nnodes][3]."""

    xyz: np.ndarray
    tets: np.ndarray
    nbrs: np.ndarray
    frames: np.ndarray = None
    times: np.ndarray = None
    time_periodic: bool = True
    period: float = 1.0
    extra: dict = field(default_factory=dict)


def double_gyre(nx=129, ny=65, nframes=101, t_end=10.0, A=0.1, eps=0.25,
                omega=2 * np.pi / 10) -> RectInput:
    """Double gyre sampled at nodes (FP64 -> FP32); time-periodic with period 2 pi / omega."""
    x = np.linspace(0.0, 2.0, nx)
    y = np.linspace(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)                   # [ny][nx]
    times = np.array([t_end * k / (nframes - 1) for k in range(nframes)], dtype=np.float64)
    frames = np.empty((nframes, ny, nx, 2), dtype=np.float32)
    for k, t in enumerate(times):
        a = eps * np.sin(omega * t)
        b = 1.0 - 2.0 * eps * np.sin(omega * t)
        f = a * X * X + b * X
        dfdx = 2.0 * a * X + b
        frames[k, :, :, 0] = -np.pi * A * np.sin(np.pi * f) * np.cos(np.pi * Y)
        frames[k, :, :, 1] = np.pi * A * np.cos(np.pi * f) * np.sin(np.pi * Y) * dfdx
    return RectInput(frames, times, (0.0, 0.0), (2.0 / (nx - 1), 1.0 / (ny - 1)), (0, 0),
                     time_periodic=True, period=2 * np.pi / omega)


def abc(n=128, nframes=64, t_end=8.0, A=np.sqrt(3.0), B=np.sqrt(2.0), C=1.0, mod=0.5,
        dtype=np.float32) -> RectInput:
    """ABC flow with A(t) = A + mod * t * sin(pi t), n^3 periodic nodes at i * 2 pi / n."""
    h = 2 * np.pi / n
    g = np.arange(n, dtype=np.float64) * h
    times = np.array([t_end * k / (nframes - 1) for k in range(nframes)], dtype=np.float64)
    frames = np.empty((nframes, n, n, n, 3), dtype=dtype)
    sx, cx = np.sin(g), np.cos(g)
    # broadcast shapes: z -> [n,1,1], y -> [1,n,1], x -> [1,1,n]
    sz, cz = sx[:, None, None], cx[:, None, None]
    sy, cy = sx[None, :, None], cx[None, :, None]
    sxx, cxx = sx[None, None, :], cx[None, None, :]
    for k, t in enumerate(times):
        At = A + mod * t * np.sin(np.pi * t)
        frames[k, ..., 0] = At * sz + C * cy
        frames[k, ..., 1] = B * sxx + At * cz
        frames[k, ..., 2] = C * sy + B * cxx
    return RectInput(frames, times, (0.0, 0.0, 0.0), (h, h, h), (1, 1, 1))


def affine_frames(A0, A1, b0, n, origin, spacing, times, periodic=None) -> RectInput:
    """u(x, t) = (A0 + t A1) x + b0 sampled on a rectilinear grid (exact under interpolation)."""
    A0 = np.asarray(A0, dtype=np.float64)
    A1 = np.asarray(A1, dtype=np.float64)
    b0 = np.asarray(b0, dtype=np.float64)
    dim = A0.shape[0]
    axes = [origin[a] + spacing[a] * np.arange(n[a]) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # each [nz][ny][nx] (or [ny][nx])
    X = np.stack(grids, axis=-1)
    times = np.asarray(times, dtype=np.float64)
    frames = np.empty((len(times),) + X.shape[:-1] + (dim,), dtype=np.float32)
    for k, t in enumerate(times):
        M = A0 + t * A1
        frames[k] = X @ M.T + b0
    return RectInput(frames, times, tuple(origin), tuple(spacing),
                     tuple(periodic) if periodic is not None else (0,) * dim)


def pipe_mesh(h=0.0466, R=1.0, L=10.0, jitter=0.2, seed=SEED) -> TetInput:
    """Delaunay tets of a jittered lattice inside a cylinder plus boundary rings.

    Points: lattice nodes with r < R - h/2 jittered by +-jitter*h (interior
    slices only, so the end caps stay planar), and rings of points on r = R at
    every lattice slice.  scipy's Qhull gives the tets and the face neighbours
    (neighbour j is across the face opposite vertex j, -1 on the boundary).
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    nz = int(round(L / h))
    zs = np.linspace(0.0, L, nz + 1)
    m = int(np.ceil(R / h))
    xy = np.arange(-m, m + 1, dtype=np.float64) * h
    XX, YY = np.meshgrid(xy, xy)
    inner = (XX * XX + YY * YY) < (R - 0.5 * h) ** 2
    px, py = XX[inner], YY[inner]
    nring = int(round(2 * np.pi * R / h))
    th = 2 * np.pi * np.arange(nring) / nring
    pts = []
    for k, z in enumerate(zs):
        jx = rng.uniform(-jitter, jitter, px.size) * h
        jy = rng.uniform(-jitter, jitter, px.size) * h
        if 0 < k < nz:
            jz = rng.uniform(-jitter, jitter, px.size) * h
        else:
            jz = np.zeros(px.size)
        pts.append(np.stack([px + jx, py + jy, z + jz], axis=1))
        rot = rng.uniform(0, 2 * np.pi / nring)
        pts.append(np.stack([R * np.cos(th + rot), R * np.sin(th + rot), np.full(nring, z)], axis=1))
    P = np.concatenate(pts).astype(np.float32)
    tri = Delaunay(P.astype(np.float64))
    tets = tri.simplices.astype(np.int32)
    nbrs = tri.neighbors.astype(np.int32)
    return TetInput(P, tets, nbrs, extra={"R": R, "L": L, "h": h})


def pipe_swirl_amp(mesh: TetInput, times, phases, R=1.0, L=10.0, frac=0.05) -> float:
    """Swirl scale so that max |u_swirl| over nodes and frames is frac * centreline peak (1.5)."""
    x = mesh.xyz.astype(np.float64)
    r2 = (x[:, 0] ** 2 + x[:, 1] ** 2) / (R * R)
    r = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    best = 0.0
    for t in times:
        sw = sum(np.sin(2 * np.pi * m * x[:, 2] / L + phases[m - 1] + 2 * np.pi * t) / m
                 for m in range(1, 5))
        best = max(best, float(np.max(np.abs((1.0 - r2) * sw * r))))
    return frac * 1.5 / best if best > 0 else 0.0


def pipe_frames(mesh: TetInput, nframes=50, period=1.0, R=1.0, L=10.0, seed=SEED) -> TetInput:
    """Pulsatile Poiseuille u_z = (1 - r^2/R^2)(1 + 0.5 sin 2 pi t) plus swirl s(r,z,t)(-y, x, 0).

    s = amp (1 - r^2/R^2) sum_{m=1..4} sin(2 pi m z / L + phi_m + 2 pi t) / m with
    phi_m ~ U[0, 2 pi) from the seed; nframes frames per period at t_k = k * period / nframes,
    plus the closing frame t = period (equal to the first), time-periodic.  The field is
    divergence-free.
    """
    rng = np.random.default_rng(seed)
    phases = rng.uniform(0.0, 2 * np.pi, 4)
    times = np.array([period * k / nframes for k in range(nframes + 1)], dtype=np.float64)
    amp = pipe_swirl_amp(mesh, times, phases, R, L)
    x = mesh.xyz.astype(np.float64)
    r2 = (x[:, 0] ** 2 + x[:, 1] ** 2) / (R * R)
    prof = 1.0 - r2
    frames = np.empty((nframes + 1, x.shape[0], 3), dtype=np.float32)
    for k, t in enumerate(times):
        sw = sum(np.sin(2 * np.pi * m * x[:, 2] / L + phases[m - 1] + 2 * np.pi * t) / m
                 for m in range(1, 5))
        s = amp * prof * sw
        frames[k, :, 0] = -s * x[:, 1]
        frames[k, :, 1] = s * x[:, 0]
        frames[k, :, 2] = prof * (1.0 + 0.5 * np.sin(2 * np.pi * t))
    mesh.frames = frames
    mesh.times = times
    mesh.time_periodic = True
    mesh.period = period
    mesh.extra.update({"phases": phases, "amp": amp})
    return mesh


def tri_neighbours(tris):
    """Triangle across the edge opposite vertex j of each triangle (-1 on the boundary)."""
    tris = np.asarray(tris, dtype=np.int64)
    nc = tris.shape[0]
    u = np.stack([tris[:, 1], tris[:, 2], tris[:, 0]], axis=1).ravel()   # edge j: vertices j+1, j+2
    v = np.stack([tris[:, 2], tris[:, 0], tris[:, 1]], axis=1).ravel()
    key = np.minimum(u, v) * (int(tris.max()) + 1) + np.maximum(u, v)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    nbrs = np.full(nc * 3, -1, dtype=np.int64)
    pair = np.nonzero(ks[1:] == ks[:-1])[0]          # an interior edge appears exactly twice
    a, b = order[pair], order[pair + 1]
    nbrs[a] = b // 3
    nbrs[b] = a // 3
    return nbrs.reshape(nc, 3).astype(np.int32)


def stenosis_halfwidth(x, H=1.0, depth=0.5, xc=3.0, w=0.75):
    """Channel half-width H (1 - depth exp(-((x - xc) / w)^2)) and its x-derivative."""
    e = np.exp(-((x - xc) / w) ** 2)
    return H * (1.0 - depth * e), 2.0 * H * depth * e * (x - xc) / (w * w)


def stenosis_mesh(h=0.05, L=10.0, H=1.0, depth=0.5, xc=3.0, w=0.75, jitter=0.2, seed=SEED,
                  with_neighbours=True) -> TetInput:
    """Body-fitted triangles of the channel 0 <= x <= L, |y| <= hw(x) (stenosis_halfwidth).

    Columns x_i = i L / nx (nx = round(L / h)); on column i, nodes at y = hw(x_i) s_j with
    s_j = -1 + 2 j / ny (ny = 2 round(H / h)), so every column has the same node count and the
    walls are node rows.  Interior nodes move by +-jitter (x and s, in units of the column and
    row spacing; x fixed on the inlet and outlet columns, s fixed on the walls).  Each quad splits
    along a diagonal chosen per quad from the seeded generator; triangles are counter-clockwise.
    Returned as TetInput with xyz = xy [nnodes][2], tets = triangles [ncells][3] and, when
    with_neighbours, nbrs [ncells][3] (across the edge opposite vertex j), else None.
    """
    rng = np.random.default_rng(seed)
    nx = int(round(L / h))
    ny = 2 * int(round(H / h))
    i = np.arange(nx + 1, dtype=np.float64)
    j = np.arange(ny + 1, dtype=np.float64)
    I, Jg = np.meshgrid(i, j, indexing="xy")          # [ny+1][nx+1]
    jx = rng.uniform(-jitter, jitter, I.shape)
    js = rng.uniform(-jitter, jitter, I.shape)
    jx[:, 0] = jx[:, -1] = 0.0
    js[0, :] = js[-1, :] = 0.0
    X = (I + jx) * (L / nx)
    S = -1.0 + (Jg + js) * (2.0 / ny)
    hw, _ = stenosis_halfwidth(X, H, depth, xc, w)
    xy = np.stack([X.ravel(), (hw * S).ravel()], axis=1).astype(np.float32)
    node = lambda a, b: b * (nx + 1) + a
    a, b = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    a, b = a.ravel(), b.ravel()
    v00, v10, v01, v11 = node(a, b), node(a + 1, b), node(a, b + 1), node(a + 1, b + 1)
    diag = rng.integers(0, 2, a.size).astype(bool)
    t1 = np.where(diag[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(diag[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    tris = np.empty((2 * a.size, 3), dtype=np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    nbrs = tri_neighbours(tris) if with_neighbours else None
    return TetInput(xy, tris, nbrs, extra={"L": L, "H": H, "depth": depth, "xc": xc, "w": w, "h": h})


def stenosis_frames(mesh: TetInput, nframes=40, period=1.0, eps=0.05, wavelength=2.0, speed=2.0) -> TetInput:
    """Stream function psi = Q(t) f(s) + eps g(s) sin(k (x - c t)), s = y / hw(x):
    f(s) = (3 s - s^3) / 2 carries the flux Q(t) = 1 + 0.5 sin(2 pi t / period) through every
    section, g(s) = (1 - s^2)^2 a wave travelling downstream; u = d psi / dy, v = -d psi / dx,
    so the field is divergence-free and vanishes on the walls.  nframes frames per period plus the
    closing frame (equal to the first), time-periodic."""
    x = mesh.xyz[:, 0].astype(np.float64)
    y = mesh.xyz[:, 1].astype(np.float64)
    ex = mesh.extra
    hw, dhw = stenosis_halfwidth(x, ex["H"], ex["depth"], ex["xc"], ex["w"])
    s = y / hw
    ds_dx = -s * dhw / hw
    fp = 1.5 * (1.0 - s * s)
    g = (1.0 - s * s) ** 2
    gp = -4.0 * s * (1.0 - s * s)
    k = 2 * np.pi / wavelength
    times = np.array([period * q / nframes for q in range(nframes + 1)], dtype=np.float64)
    frames = np.empty((nframes + 1, x.size, 2), dtype=np.float32)
    for q, t in enumerate(times):
        Q = 1.0 + 0.5 * np.sin(2 * np.pi * t / period)
        ph = k * (x - speed * t)
        u = Q * fp / hw + eps * gp * np.sin(ph) / hw
        v = -(Q * fp * ds_dx + eps * (gp * ds_dx * np.sin(ph) + g * k * np.cos(ph)))
        frames[q, :, 0] = u
        frames[q, :, 1] = v
    mesh.frames = frames
    mesh.times = times
    mesh.time_periodic = True
    mesh.period = period
    return mesh


def random_points(n, lo, hi, seed=SEED):
    """Uniform points [dim][n] FP32 in the box [lo, hi] (seeded)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (lo[:, None] + (hi - lo)[:, None] * rng.random((len(lo), n))).astype(np.float32)


# ------------------------------------------------------------ surrogate network

MLP_SHAPES = [(128, 7), (128,), (128, 128), (128,), (128, 128), (128,), (128, 128), (128,), (3, 128), (3,)]


def mlp_init(seed=SEED, gain=1.0):
    """Packed FP32 parameters of the 7-128x4-3 network (W0 b0 ... W4 b4, row-major W[out][in]):
    weights uniform in +-gain*sqrt(6/fan_in) (He-uniform for SiLU), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            lim = gain * np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, s))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def surrogate_samples(n, t_period=10.0, lo=(0.0, 0.0), hi=(2.0, 1.0), seed=SEED):
    """Training points (x0, y0, t0) [3][n] FP32, uniform in the box and over one period."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(lo[0], hi[0], n), rng.uniform(lo[1], hi[1], n),
                     rng.uniform(0.0, t_period, n)]).astype(np.float32)
