"""The synthetic mesh generators (stand-ins for the paper's unstructured stenosis and aneurysm data,
Sec. 4): triangles and tets are non-degenerate, neighbours are symmetric and share the named face or
edge, the boundary is closed, and the stenosis flow is divergence-free with no slip on the walls."""
import numpy as np

from paper_2209_13775_gb300 import inputs


def _check_tri_mesh(xy, tris, nbrs):
    a, b, c = (xy[tris[:, k]].astype(np.float64) for k in range(3))
    area = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert (area > 0).all()                       # counter-clockwise, non-degenerate
    for t in range(len(tris)):
        for j in range(3):
            n = nbrs[t, j]
            if n < 0:
                continue
            edge = {tris[t, (j + 1) % 3], tris[t, (j + 2) % 3]}
            assert edge <= set(tris[n]) and t in nbrs[n]


def test_stenosis_mesh_is_a_valid_triangulation():
    m = inputs.stenosis_mesh(h=0.1, L=4.0)
    _check_tri_mesh(m.xyz, m.tets, m.nbrs)
    # boundary edges: two walls of nx edges each, inlet and outlet of ny edges each
    nx, ny = int(round(4.0 / 0.1)), 2 * int(round(1.0 / 0.1))
    assert (m.nbrs < 0).sum() == 2 * nx + 2 * ny
    np.testing.assert_array_equal(inputs.tri_neighbours(m.tets), m.nbrs)


def test_stenosis_flow_no_slip_and_flux():
    m = inputs.stenosis_frames(inputs.stenosis_mesh(h=0.05, L=10.0), nframes=8, period=1.0)
    hw, _ = inputs.stenosis_halfwidth(m.xyz[:, 0].astype(np.float64))
    wall = np.isclose(np.abs(m.xyz[:, 1]), hw, rtol=0, atol=1e-6)
    assert wall.sum() > 100
    assert np.abs(m.frames[:, wall]).max() < 1e-5   # no slip
    # flux through the inlet column equals Q(t) = 1 + 0.5 sin(2 pi t) (trapezoid rule on the nodes)
    inlet = np.isclose(m.xyz[:, 0], 0.0)
    y = m.xyz[inlet, 1].astype(np.float64)
    order = np.argsort(y)
    for q, t in enumerate(m.times):
        u = m.frames[q, inlet, 0].astype(np.float64)[order]
        flux = np.trapezoid(u, y[order]) / 2.0        # the stream function difference is 2 Q
        assert abs(flux - (1.0 + 0.5 * np.sin(2 * np.pi * t))) < 2e-3


def test_pipe_mesh_neighbours():
    m = inputs.pipe_mesh(h=0.25, L=2.0)
    for t in range(0, len(m.tets), 7):
        for j in range(4):
            n = m.nbrs[t, j]
            if n >= 0:
                face = set(np.delete(m.tets[t], j))
                assert face <= set(m.tets[n]) and t in m.nbrs[n]
