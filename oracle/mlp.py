"""FP64 oracle of the learned surrogate: features, the 7 -> 128 x 4 -> 3 SiLU network,
its loss and gradients, Adam, the cosine learning-rate schedule, and the gated
surrogate advection.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy in FP64; the
gradients are written out layer by layer (reverse-mode chain rule), and the
integrator targets come from the oracle's own RK4 (``oracle.rk4``).

The surrogate is not in the paper.  Its role is the one of the local flow-map
approximations mentioned among the related work (Sec. 4, Discussion): a cheap map
x(t) -> x(t + tau) that replaces integration over one sub-interval, checked by an
audit against the integrator (Eq. 2) and replaced by it where the check fails.

Definitions (shared with the CUDA library by specification, not by code):
  phi(x, y, t) = (x - cx, y - cy, sin(omega t), cos(omega t), sin(kx x), cos(kx x), sin(ky y))
  h_0 = phi;  h_{l+1} = SiLU(W_l h_l + b_l), l = 0..3;  o = W_4 h_4 + b_4
  displacement = out_scale * (o_0, o_1);  rho = o_2 (log10 of the predicted error)
  SiLU(z) = z / (1 + exp(-z))
  loss = mean over samples of (o_0 - d_x / s)^2 + (o_1 - d_y / s)^2
         + w_rho (o_2 - log10(|out_scale (o_0, o_1) - d| + 1e-7))^2
  with the log10 target held constant (no gradient through it).
Parameters are packed as W0[128][7] b0[128] W1[128][128] b1 W2 b2 W3 b3 W4[3][128] b4[3]
(row-major W[out][in]).
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 7, 128, 3
SHAPES = [(HID, IN), (HID,), (HID, HID), (HID,), (HID, HID), (HID,), (HID, HID), (HID,), (OUT, HID), (OUT,)]
NPARAMS = sum(int(np.prod(s)) for s in SHAPES)
RHO_EPS = 1e-7


def unpack(params):
    """Flat FP64 vector -> [W0, b0, ..., W4, b4] (views)."""
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    return out


def pack(tensors):
    return np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in tensors])


def features(x, y, t, center, kx, ky, omega):
    """phi [7][n] of positions x, y and times t (broadcast)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape)
    return np.stack([x - center[0], y - center[1], np.sin(omega * t), np.cos(omega * t),
                     np.sin(kx * x), np.cos(kx * x), np.sin(ky * y)])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, phi):
    """o [3][n] and the cache of pre-activations z_l and activations h_l."""
    W = unpack(params)
    h = [np.asarray(phi, dtype=np.float64)]
    z = []
    for l in range(4):
        z.append(W[2 * l] @ h[-1] + W[2 * l + 1][:, None])
        h.append(silu(z[-1]))
    o = W[8] @ h[-1] + W[9][:, None]
    return o, (h, z)


def rho_target(params, phi, disp, out_scale):
    """log10 of the network's own displacement error per sample (the rho head's target)."""
    o, _ = forward(params, phi)
    d = np.asarray(disp, dtype=np.float64)
    return np.log10(np.sqrt(((out_scale * o[:2] - d) ** 2).sum(axis=0)) + RHO_EPS)


def loss_and_grad(params, phi, disp, out_scale, rho_weight, rho_t=None):
    """Mean loss over the n samples and its gradient (flat, FP64).  disp [2][n].

    The rho target is computed from these parameters unless given; either way it is a
    constant of the gradient."""
    W = unpack(params)
    o, (h, z) = forward(params, phi)
    n = phi.shape[1]
    d = np.asarray(disp, dtype=np.float64)
    e = o[:2] - d / out_scale
    if rho_t is None:
        rho_t = rho_target(params, phi, disp, out_scale)
    er = o[2] - rho_t
    loss = float(((e ** 2).sum(axis=0) + rho_weight * er ** 2).mean())
    do = np.concatenate([2.0 * e, (2.0 * rho_weight * er)[None]], axis=0) / n
    grads = [None] * 10
    grads[8] = do @ h[4].T
    grads[9] = do.sum(axis=1)
    dh = W[8].T @ do
    for l in range(3, -1, -1):
        dz = dh * silu_grad(z[l])
        grads[2 * l] = dz @ h[l].T
        grads[2 * l + 1] = dz.sum(axis=1)
        dh = W[2 * l].T @ dz
    return loss, pack(grads)


def adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) at step >= 1; returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_lr(step, total, lr0, lr_min):
    """Cosine decay from lr0 at step 0 to lr_min at step total."""
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * min(step, total) / total))


def lowbias32(x):
    """32-bit integer hash (Wellons' lowbias32): xor-shift / multiply rounds."""
    x = int(x) & 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def audit_lane(step, warp, m=32):
    """Lane of a group of m <= 32 tracers whose displacement is audited at surrogate step
    `step` (m = 32 for every full group; the last group of a ragged count is smaller)."""
    return lowbias32(lowbias32(step) ^ (int(warp) & 0xFFFFFFFF)) % m


def surrogate_advect(params, field, x0, t0, K, tau, dt, tol, center, kx, ky, omega, out_scale):
    """Gated surrogate flow map over (t0, t0 + K tau), 2D.

    Per sub-interval k, every group of 32 consecutive tracers proposes x + displacement;
    the audit lane of the group integrates RK4 (step dt) over the sub-interval, and the
    whole group integrates RK4 instead when the audit residual |displacement - RK4| or
    any lane's 10^rho exceeds tol.  Returns (x [2][n], fallbacks per tracer [n],
    fallback groups per sub-interval [K]).
    """
    import oracle

    x = np.array(x0, dtype=np.float64)
    n = x.shape[1]
    nwarps = (n + 31) // 32
    fb = np.zeros(n, dtype=np.int64)
    per_step = np.zeros(K, dtype=np.int64)
    log_tol = math.log10(tol) if tol > 0 else -math.inf
    for k in range(K):
        tk = t0 + k * tau
        phi = features(x[0], x[1], tk, center, kx, ky, omega)
        o, _ = forward(params, phi)
        prop = x + out_scale * o[:2]
        for w in range(nwarps):
            s = slice(32 * w, min(32 * w + 32, n))
            a = 32 * w + audit_lane(k, w, s.stop - s.start)
            ra, _, _ = oracle.rk4(field, x[:, a:a + 1], tk, tau, dt)
            r = float(np.sqrt(((prop[:, a] - ra[:, 0]) ** 2).sum()))
            if r > tol or (o[2, s] > log_tol).any():
                xr, _, _ = oracle.rk4(field, x[:, s], tk, tau, dt)
                x[:, s] = xr
                fb[s] += 1
                per_step[k] += 1
            else:
                x[:, s] = prop[:, s]
    return x, fb, per_step
