"""Small test meshes shared by the oracle pins and the GPU parity tests."""
import itertools

import numpy as np


def kuhn_mesh(n):
    """n^3 unit cubes, each split into 6 tets along its main diagonal; neighbours by face matching."""
    idx = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    pts = np.array([[i, j, k] for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)],
                   dtype=np.float32)
    tets = []
    E = np.eye(3, dtype=int)
    for k, j, i in itertools.product(range(n), range(n), range(n)):
        for perm in itertools.permutations(range(3)):
            v = np.array([i, j, k])
            vs = [idx(*v)]
            for ax in perm:
                v = v + E[ax]
                vs.append(idx(*v))
            tets.append(vs)
    tets = np.array(tets, dtype=np.int32)
    faces = {}
    nbrs = -np.ones_like(tets)
    for t, vs in enumerate(tets):
        for j in range(4):
            key = tuple(sorted(np.delete(vs, j)))
            if key in faces:
                s, sj = faces[key]
                nbrs[t, j], nbrs[s, sj] = s, t
            else:
                faces[key] = (t, j)
    return pts, tets, nbrs


def l_kuhn_mesh(n):
    """kuhn_mesh(n) without the cubes with i >= n/2 and j >= n/2 (an L-shaped prism: non-convex),
    ids renumbered; neighbours by face matching."""
    pts, tets, _ = kuhn_mesh(n)
    c = pts[tets].mean(axis=1)
    keep = ~((c[:, 0] > n / 2) & (c[:, 1] > n / 2))
    tets = tets[keep]
    used = np.unique(tets)
    remap = -np.ones(len(pts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    pts = pts[used]
    tets = remap[tets].astype(np.int32)
    faces = {}
    nbrs = -np.ones_like(tets)
    for t, vs in enumerate(tets):
        for j in range(4):
            key = tuple(sorted(np.delete(vs, j)))
            if key in faces:
                s, sj = faces[key]
                nbrs[t, j], nbrs[s, sj] = s, t
            else:
                faces[key] = (t, j)
    return pts, tets, nbrs


def tri_grid_mesh(n, seed=7):
    """n^2 unit squares with integer nodes, each split into 2 triangles along a diagonal chosen
    per square; the vertex order of about half the triangles is reversed (clockwise), so location
    and interpolation are exercised on both orientations.  Neighbours by edge matching."""
    from paper_2209_13775_gb300.inputs import tri_neighbours

    rng = np.random.default_rng(seed)
    idx = lambda i, j: i + (n + 1) * j
    pts = np.array([[i, j] for j in range(n + 1) for i in range(n + 1)], dtype=np.float32)
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i, j + 1), idx(i + 1, j + 1)
            pair = [[a, b, d], [a, d, c]] if rng.integers(2) else [[a, b, c], [b, d, c]]
            for t in pair:
                tris.append(t[::-1] if rng.integers(2) else t)
    tris = np.array(tris, dtype=np.int32)
    return pts, tris, tri_neighbours(tris)


def l_tri_grid_mesh(n, seed=7):
    """tri_grid_mesh(n) without the squares with i >= n/2 and j >= n/2 (L-shaped: non-convex)."""
    from paper_2209_13775_gb300.inputs import tri_neighbours

    pts, tris, _ = tri_grid_mesh(n, seed)
    c = pts[tris].mean(axis=1)
    tris = tris[~((c[:, 0] > n / 2) & (c[:, 1] > n / 2))]
    used = np.unique(tris)
    remap = -np.ones(len(pts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    tris = remap[tris].astype(np.int32)
    return pts[used], tris, tri_neighbours(tris)
