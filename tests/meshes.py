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
