"""CPU oracle for the learned surrogate -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
use it.  Plain numpy FP64, written from the network's definition, sharing
no code with the CUDA kernels (paper_2009_06635_gb300/csrc/surrogate.cu).

The surrogate (no counterpart in the paper; the growth axis that replaces
the interpolator where a network is accurate enough) maps a query point to
all flavours:
  z   = (2 (ln x - lx_lo)/(lx_hi - lx_lo) - 1, 2 (ln Q^2 - lq_lo)/(lq_hi - lq_lo) - 1)
  a_j = pi (F[j,0] z_0 + F[j,1] z_1),  phi = [sin a_0..15, cos a_0..15]   (32 features)
  h1  = silu(W1 phi + b1), h2..h4 = silu(W h + b)   (width 128)
  y   = W5 h4 + b5                                    (one output per flavour)
  xf_f = c_f sinh(y_f)     (inverse of the training target y_f = asinh(xf_f / c_f)),
  or, with the envelope target, xf_f = E_f(x) y_f (target xf_f / E_f(x)), where
  E_f(x_i) = max over the Q knots of |xf_f(x_i, Q)| (at least c_f) and ln E_f is
  linear in ln x between knots, tabulated at ENV_N + 1 equal steps of ln x;
  or, with the residual target, xf_f = B_f(z) + RES_EPS E_f(x) y_f (target
  (xf_f - B_f) / (RES_EPS E_f) clipped to [-RES_CLIP, RES_CLIP]), B_f bilinear
  in (z0, z1) between the nodes of a uniform (BASE_N + 1)^2 table of the
  interpolator's values rounded to float.
silu(v) = v sigmoid(v) = v (1 + tanh(v/2)) / 2.
Training loss: mean over batch and flavours of (y - target)^2.

With bf16=True the oracle rounds to bfloat16 exactly where the GPU keeps
bfloat16 values (weights, features, activations, and the backward signals
that feed matrix products), so the comparison isolates accumulation order.
"""
from __future__ import annotations

import numpy as np

WIDTH = 128
NFEAT = 16  # frequencies; features = 2 * NFEAT
ENV_N = 1024  # envelope table intervals
BASE_N = 256  # base table intervals per axis (residual target)
RES_EPS = 2.0**-10  # residual target scale
RES_CLIP = 32.0  # residual targets clipped to [-RES_CLIP, RES_CLIP]


def bf16(a):
    """Round to bfloat16 (round to nearest even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(v):
    return 0.5 * v * (1.0 + np.tanh(0.5 * v))


def dsilu(v):
    s = 0.5 * (1.0 + np.tanh(0.5 * v))
    return s + v * s * (1.0 - s)


def unpack(params, nflav):
    """Flat parameter vector -> [(W, b)] for the five layers, W as [out][in]."""
    shapes = [(WIDTH, 2 * NFEAT), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (nflav, WIDTH)]
    out, k = [], 0
    p = np.asarray(params, dtype=np.float64)
    for (o, i) in shapes:
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    assert k == p.size, (k, p.size)
    return out


def features(x, q2, freq, bounds, bf=False):
    lx_lo, lx_hi, lq_lo, lq_hi = bounds
    z0 = 2.0 * (np.log(x) - lx_lo) / (lx_hi - lx_lo) - 1.0
    z1 = 2.0 * (np.log(q2) - lq_lo) / (lq_hi - lq_lo) - 1.0
    a = np.pi * (np.outer(z0, freq[:, 0]) + np.outer(z1, freq[:, 1]))
    phi = np.concatenate([np.sin(a), np.cos(a)], axis=1)
    return bf16(phi) if bf else phi


def forward(params, x, q2, freq, bounds, nflav, bf=False):
    """-> (y [n][nflav], cache for backward)."""
    layers = unpack(params, nflav)
    r = bf16 if bf else (lambda t: t)
    h = features(x, q2, freq, bounds, bf)
    cache = {"h": [h], "z": []}
    for li, (W, b) in enumerate(layers):
        z = h @ r(W).T + b
        if li < 4:
            cache["z"].append(z)
            h = r(silu(z))
            cache["h"].append(h)
        else:
            y = z
    return y, cache


def target(xf, scale, env=None, base_vals=None):
    if base_vals is not None:
        return np.clip((np.asarray(xf) - base_vals) / (RES_EPS * env), -RES_CLIP, RES_CLIP)
    return np.asarray(xf) / env if env is not None else np.arcsinh(np.asarray(xf) / scale)


def envelope_table(x_knots, values, bounds):
    """ln E_f at ENV_N + 1 equal steps of ln x over [bounds[0], bounds[1]]: [nflav][ENV_N + 1]."""
    v = np.abs(np.asarray(values, dtype=np.float64))  # [rows][nx][nflav]
    m = v.reshape(-1, v.shape[2]).max(axis=0)
    floor = 1e-5 * np.where(m > 0, m, 1.0)
    E = np.maximum(v.max(axis=0), floor)  # [nx][nflav]
    lxt = bounds[0] + (bounds[1] - bounds[0]) * np.arange(ENV_N + 1) / ENV_N
    lx = np.log(np.asarray(x_knots, dtype=np.float64))
    return np.stack([np.interp(lxt, lx, np.log(E[:, f])) for f in range(E.shape[1])])


def envelope(table, x, bounds):
    """E_f(x) for every point and flavour: [n][nflav]."""
    z0 = 2.0 * (np.log(x) - bounds[0]) / (bounds[1] - bounds[0]) - 1.0
    u = np.clip((z0 + 1.0) * 0.5 * ENV_N, 0.0, ENV_N)
    k = np.minimum(np.floor(u).astype(int), ENV_N - 1)
    a, b = table[:, k], table[:, k + 1]
    return np.exp(a + (u - k) * (b - a)).T


def loss_grad(params, x, q2, xf, scale, freq, bounds, nflav, bf=False, env=None, base_vals=None):
    """Mean-square loss on the targets (asinh; xf / E with env = E [n][nflav];
    or (xf - B) / (RES_EPS E) with base_vals = B as well) and its gradient
    (flat, FP64)."""
    layers = unpack(params, nflav)
    r = bf16 if bf else (lambda t: t)
    y, c = forward(params, x, q2, freq, bounds, nflav, bf)
    t = target(xf, scale, env, base_vals)
    n = y.shape[0]
    diff = y - t
    loss = float(np.mean(diff * diff))
    g = r(2.0 * diff / (n * nflav))  # dL/dy
    grads = [None] * 5
    for li in range(4, -1, -1):
        W, b = layers[li]
        h_in = c["h"][li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        if li > 0:
            dh = g @ r(W)
            g = r(dh * dsilu(c["z"][li - 1]))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat


def predict(params, x, q2, scale, freq, bounds, nflav, bf=False, env=None, base_vals=None):
    y, _ = forward(params, x, q2, freq, bounds, nflav, bf)
    if base_vals is not None:
        return base_vals + RES_EPS * env * y
    return env * y if env is not None else scale * np.sinh(y)


def base_nodes(bounds):
    """(x, Q^2) of the base table's nodes, [BASE_N + 1][BASE_N + 1] (z0 outer)."""
    i = np.arange(BASE_N + 1)
    lx = bounds[0] + (bounds[1] - bounds[0]) * i / BASE_N
    lq = bounds[2] + (bounds[3] - bounds[2]) * i / BASE_N
    X, Q = np.meshgrid(np.exp(lx), np.exp(lq), indexing="ij")
    return X, Q


def base_table(values_at_nodes):
    """The table from the interpolator's values at base_nodes ([nodes][nflav]
    FP64): rounded to float, [BASE_N + 1][BASE_N + 1][nflav]."""
    v = np.asarray(values_at_nodes, dtype=np.float64).astype(np.float32).astype(np.float64)
    return v.reshape(BASE_N + 1, BASE_N + 1, -1)


def base(table, x, q2, bounds):
    """B_f for every point: bilinear between the table's nodes in (z0, z1), [n][nflav]."""
    z0 = 2.0 * (np.log(x) - bounds[0]) / (bounds[1] - bounds[0]) - 1.0
    z1 = 2.0 * (np.log(q2) - bounds[2]) / (bounds[3] - bounds[2]) - 1.0
    u0 = np.clip((z0 + 1.0) * 0.5 * BASE_N, 0.0, BASE_N)
    u1 = np.clip((z1 + 1.0) * 0.5 * BASE_N, 0.0, BASE_N)
    i = np.minimum(np.floor(u0).astype(int), BASE_N - 1)
    j = np.minimum(np.floor(u1).astype(int), BASE_N - 1)
    a, b = (u0 - i)[:, None], (u1 - j)[:, None]
    v00, v01 = table[i, j], table[i, j + 1]
    v10, v11 = table[i + 1, j], table[i + 1, j + 1]
    return (1 - a) * ((1 - b) * v00 + b * v01) + a * ((1 - b) * v10 + b * v11)
