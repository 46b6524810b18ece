"""Pins for the FP64 surrogate oracle (oracle/mlp.py): features, SiLU, the network's
forward pass on hand-built weights, gradients against central finite differences,
Adam's first steps in closed form, the cosine schedule, the audit hash, and the
gated advection at its two limits (always audited out -> RK4; never -> the network).
"""
import math

import numpy as np
import pytest

from oracle import mlp

GYRE = dict(center=(1.0, 0.5), kx=math.pi, ky=math.pi, omega=2 * math.pi / 10)


def rand_params(rng, scale=1.0):
    out = []
    for s in mlp.SHAPES:
        fan_in = s[1] if len(s) == 2 else 128
        out.append(rng.normal(size=s) * scale / math.sqrt(fan_in))
    return mlp.pack(out)


def test_features_closed_form():
    phi = mlp.features([0.25, 2.0], [0.75, 0.0], 2.5, **GYRE)
    want = np.array([[-0.75, 1.0], [0.25, -0.5], [1.0, 1.0], [0.0, 0.0],
                     [math.sqrt(0.5), 0.0], [math.sqrt(0.5), 1.0], [math.sqrt(0.5), 0.0]])
    np.testing.assert_allclose(phi, want, atol=1e-15)


def test_silu_and_its_derivative():
    z = np.linspace(-30, 30, 601)
    np.testing.assert_allclose(mlp.silu(z), z * 0.5 * (1 + np.tanh(z / 2)), rtol=1e-13, atol=1e-14)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu(40.0) - 40.0) < 1e-12
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=1e-7, atol=1e-9)
    assert mlp.silu_grad(0.0) == 0.5


def test_forward_on_hand_built_weights():
    # zero hidden weights: every hidden unit is SiLU(bias), the output is W4 SiLU(...) + b4
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[1][:] = 1.0
    W[3][:] = 2.0
    W[5][:] = -1.0
    W[7][:] = 0.5
    W[8][0, :] = 1.0
    W[9][:] = [0.0, 3.0, -2.0]
    o, _ = mlp.forward(mlp.pack(W), np.ones((7, 4)))
    np.testing.assert_allclose(o[0], 128 * mlp.silu(0.5), rtol=1e-15)
    np.testing.assert_allclose(o[1:], [[3.0] * 4, [-2.0] * 4])
    # a single path: o0 = SiLU^4 applied to phi_2 through unit weights
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[0][0, 2] = 1.0
    for l in (2, 4, 6):
        W[l][0, 0] = 1.0
    W[8][0, 0] = 1.0
    phi = np.zeros((7, 3))
    phi[2] = [-1.0, 0.5, 2.0]
    o, _ = mlp.forward(mlp.pack(W), phi)
    np.testing.assert_allclose(o[0], mlp.silu(mlp.silu(mlp.silu(mlp.silu(phi[2])))), rtol=1e-15)
    assert mlp.NPARAMS == 50947


def test_gradients_match_central_differences():
    rng = np.random.default_rng(40)
    p = rand_params(rng)
    phi = mlp.features(rng.uniform(0, 2, 9), rng.uniform(0, 1, 9), rng.uniform(0, 10, 9), **GYRE)
    disp = rng.normal(scale=0.05, size=(2, 9))
    rt = mlp.rho_target(p, phi, disp, 0.1)        # held constant, as in the gradient
    loss, g = mlp.loss_and_grad(p, phi, disp, 0.1, 0.25)
    idx = np.concatenate([rng.choice(n, min(n, 12), replace=False) + o for n, o in
                          zip([int(np.prod(s)) for s in mlp.SHAPES],
                              np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])[:-1])])
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, phi, disp, 0.1, 0.25, rt)[0] - mlp.loss_and_grad(pm, phi, disp, 0.1, 0.25, rt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_loss_definition_at_a_perfect_fit():
    # o0, o1 equal to the scaled targets: only the rho term remains, with target log10(1e-7) = -7
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[9][:] = [0.25, -0.5, -5.0]
    disp = np.array([[0.03125] * 5, [-0.0625] * 5])
    loss, g = mlp.loss_and_grad(mlp.pack(W), np.zeros((7, 5)), disp, 0.125, 0.5)
    assert abs(loss - 0.5 * 4.0) < 1e-12
    gb4 = mlp.unpack(g)[9]
    np.testing.assert_allclose(gb4, [0.0, 0.0, 2 * 0.5 * 2.0], atol=1e-12)


def test_adam_first_steps_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    p1, m, v = mlp.adam(p, g, m, v, 1, 1e-2)
    # step 1: m_hat = g, v_hat = g^2 -> update lr g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    p2, m, v = mlp.adam(p1, g, m, v, 2, 1e-2)
    np.testing.assert_allclose(p2, p1 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert p2[2] == p[2]


def test_cosine_schedule():
    assert mlp.cosine_lr(0, 100, 1e-3, 1e-5) == 1e-3
    assert abs(mlp.cosine_lr(100, 100, 1e-3, 1e-5) - 1e-5) < 1e-18
    assert abs(mlp.cosine_lr(50, 100, 1e-3, 1e-5) - (1e-3 + 1e-5) / 2) < 1e-15


def test_audit_hash():
    assert mlp.lowbias32(0) == 0
    vals = [mlp.lowbias32(i) for i in range(1 << 14)]
    assert len(set(vals)) == 1 << 14                       # a bijection of 32-bit words
    lanes = np.array([mlp.audit_lane(s, w) for s in range(16) for w in range(512)])
    counts = np.bincount(lanes, minlength=32)
    assert counts.min() > 150 and counts.max() < 370       # about 256 each
    assert all(0 <= mlp.audit_lane(3, w, 7) < 7 for w in range(100))


def test_gated_advection_limits(ora):
    from paper_2209_13775_gb300 import inputs
    g = inputs.double_gyre(nx=33, ny=17, nframes=21, t_end=10.0)
    F = ora.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic, g.time_periodic, g.period)
    rng = np.random.default_rng(41)
    p = rand_params(rng, 0.5)
    x0 = np.stack([rng.uniform(0.2, 1.8, 70), rng.uniform(0.1, 0.9, 70)])
    # tol 0: every group falls back at every step -> plain RK4 over the whole interval
    x, fb, per = mlp.surrogate_advect(p, F, x0, 0.0, 4, 0.5, 0.05, 0.0, **GYRE, out_scale=0.1)
    xr, _, _ = ora.rk4(F, x0, 0.0, 2.0, 0.05)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-13)
    assert (fb == 4).all() and (per == 3).all()
    # tol inf: never -> the composition of network steps
    x, fb, per = mlp.surrogate_advect(p, F, x0, 0.0, 4, 0.5, 0.05, math.inf, **GYRE, out_scale=0.1)
    y = x0.copy()
    for k in range(4):
        o, _ = mlp.forward(p, mlp.features(y[0], y[1], 0.5 * k, **GYRE))
        y = y + 0.1 * o[:2]
    np.testing.assert_allclose(x, y, rtol=0, atol=1e-14)
    assert (fb == 0).all()
