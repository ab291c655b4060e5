"""The element-wise surrogate checks (tests/surrogate_bounds.py) on the CPU:
a float32 numpy model of the GPU's arithmetic (bfloat16 at the same points,
float32 sums in another order, a tanh with an error near the hardware
approximation's bound, float32 coordinates, envelope and base) passes every
stage and the inference check for all three targets, the bounds are tight
enough to mean something, and planted mistakes of the kinds a kernel can make
(a dropped bias, a wrong SiLU argument, a transposed gradient, a missing
base, a signal through the wrong derivative) each fail."""
import math

import numpy as np
import pytest

import surrogate_bounds as sb
from oracle import mlp

F32 = np.float32


def bf(a):
    return mlp.bf16(a).astype(F32)


class SimSurrogate:
    """Float32 model of one loss_grad pass and of inference; plant names a mistake."""

    def __init__(self, params, freq, bounds, nflav, kind, scale, env_table, base_table, seed, plant=None):
        self.layers = mlp.unpack(np.asarray(params, dtype=np.float64), nflav)
        self.freq, self.bounds, self.nflav, self.kind = freq, bounds, nflav, kind
        self.scale, self.env_table, self.base_table = scale, env_table, base_table
        self.rng = np.random.default_rng(seed)
        self.plant = plant
        self.tr = {}

    def _z(self, x, q2):
        b = self.bounds
        z = []
        for v, lo, hi in ((x, b[0], b[1]), (q2, b[2], b[3])):
            lv = np.log(v.astype(F32))
            z.append(F32(2) * (lv - F32(lo)) * F32(1.0 / (hi - lo)) - F32(1))
        return z

    def _tanh(self, v):
        return (np.tanh(v.astype(np.float64)) + self.rng.uniform(-0.9, 0.9, v.shape) * sb.TANH_ERR).astype(F32)

    def _silu(self, z):
        if self.plant == "silu_argument":
            return F32(0.5) * z * (F32(1) + self._tanh(z))
        return F32(0.5) * z * (F32(1) + self._tanh(F32(0.5) * z))

    def _forward(self, x, q2):
        z0, z1 = self._z(x, q2)
        f = self.freq.astype(F32)
        a = F32(np.pi) * (np.outer(z0, f[:, 0]) + np.outer(z1, f[:, 1]))
        h = [bf(np.concatenate([np.sin(a), np.cos(a)], axis=1))]
        zs = []
        for l, (W, b) in enumerate(self.layers):
            bb = b.astype(F32)
            if self.plant == "drop_bias" and l == 2:
                bb = np.zeros_like(bb)
            z = h[l] @ bf(W).T + bb
            if l < 4:
                zs.append(z)
                h.append(bf(self._silu(z)))
            else:
                y = z
        return h, zs, y

    def _env(self, x):
        b = self.bounds
        z0, _ = self._z(x, x)
        N = mlp.ENV_N
        u = np.clip((z0 + F32(1)) * F32(0.5 * N), F32(0), F32(N))
        k = np.minimum(u.astype(int), N - 1)
        T = self.env_table.astype(F32)
        a, c = T[:, k].T, T[:, k + 1].T
        return np.exp(a + (u - k.astype(F32))[:, None] * (c - a))

    def _base(self, x, q2):
        z0, z1 = self._z(x, q2)
        N = mlp.BASE_N
        u0 = np.clip((z0 + F32(1)) * F32(0.5 * N), F32(0), F32(N))
        u1 = np.clip((z1 + F32(1)) * F32(0.5 * N), F32(0), F32(N))
        i, j = np.minimum(u0.astype(int), N - 1), np.minimum(u1.astype(int), N - 1)
        a, c = (u0 - i.astype(F32))[:, None], (u1 - j.astype(F32))[:, None]
        T = self.base_table.astype(F32)
        lo = c * (T[i, j + 1] - T[i, j]) + T[i, j]
        hi = c * (T[i + 1, j + 1] - T[i + 1, j]) + T[i + 1, j]
        return a * (hi - lo) + lo

    def loss_grad(self, x, q2, xf):
        n, nf = len(x), self.nflav
        h, zs, y = self._forward(x, q2)
        if self.kind == "asinh":
            t = np.arcsinh(xf / self.scale.astype(F32).astype(np.float64)).astype(F32)
        elif self.kind == "envelope":
            t = (xf / self._env(x).astype(np.float64)).astype(F32)
        else:
            base = self._base(x, q2).astype(np.float64)
            if self.plant == "no_base":
                base = 0.0 * base
            t = np.clip((xf - base) / (mlp.RES_EPS * self._env(x).astype(np.float64)), -32.0, 32.0).astype(F32)
        g = [None] * 5
        g[4] = bf(F32(2) * (y - t) / F32(n * nf))
        for l in range(4, 0, -1):
            dh = g[l] @ bf(self.layers[l][0])
            zz = zs[l - 1]
            if self.plant == "dsilu_of_h":
                zz = h[l]
            s = F32(0.5) * (F32(1) + self._tanh(F32(0.5) * zz))
            g[l - 1] = bf(dh * (s + zz * s * (F32(1) - s)))
        grads = []
        for l in range(5):
            gw = g[l].T @ h[l]
            if self.plant == "transposed_gradient" and l == 2:
                gw = gw.T
            grads.append(np.concatenate([gw.ravel(), g[l].sum(axis=0)]))
        pad = lambda a: np.concatenate([a, np.zeros((n, 16 - nf), F32)], axis=1)
        self.tr = {"h": h, "z": zs, "y": [pad(y)], "t": [pad(t)], "g": g[:4] + [pad(g[4])]}
        return float(np.mean((y - t).astype(np.float64) ** 2)), np.concatenate(grads).astype(F32)

    def trace(self, what, layer=0, n=None):
        return self.tr[what][layer][:n]

    def eval(self, x, q2):
        _, _, y = self._forward(x, q2)
        if self.kind == "asinh":
            return self.scale.astype(F32) * np.sinh(y)
        eps = F32(mlp.RES_EPS) if self.kind == "residual" else F32(1)
        out = eps * self._env(x) * y
        return out + self._base(x, q2) if self.kind == "residual" else out


@pytest.fixture(scope="module")
def net(synth, oracle_mod):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    params, freq = synth.surrogate_init(g.nflav, 9)
    # biases away from zero, as after training
    rng = np.random.default_rng(5)
    p = params.astype(np.float64)
    k = 0
    for (o, i) in [(128, 32), (128, 128), (128, 128), (128, 128), (g.nflav, 128)]:
        k += o * i
        p[k:k + o] = rng.normal(0.0, 0.3, o)
        k += o
    scale = 1e-5 * np.abs(g.values).reshape(-1, g.nflav).max(axis=0)
    bounds = (math.log(g.x_knots[0]), math.log(g.x_knots[-1]), math.log(g.q2_knots[0]), math.log(g.q2_knots[-1]))
    env_table = mlp.envelope_table(g.x_knots, g.values, bounds)
    X, Q = mlp.base_nodes(bounds)
    X[0, :], X[-1, :], Q[:, 0], Q[:, -1] = g.x_knots[0], g.x_knots[-1], g.q2_knots[0], g.q2_knots[-1]
    base_table = mlp.base_table(og.xfxq2(X.ravel(), Q.ravel())[0])
    x, q2 = synth.ingrid_samples(g, 600, 41)
    xf = og.xfxq2(x, q2)[0]
    return g, p, freq.astype(np.float64), scale, bounds, env_table, base_table, x, q2, xf


def _run(net, kind, plant=None, seed=3):
    g, p, freq, scale, bounds, env_table, base_table, x, q2, xf = net
    s = SimSurrogate(p, freq, bounds, g.nflav, kind, scale, env_table, base_table, seed, plant)
    _, grad = s.loss_grad(x, q2, xf)
    return sb.check_training_pass(s, p, x, q2, xf, scale, freq, bounds, g.nflav, grad, kind, env_table, base_table)


@pytest.mark.parametrize("kind", ["asinh", "envelope", "residual"])
def test_float32_model_passes_every_stage(net, kind):
    worst = _run(net, kind)
    print(kind, {k: round(v, 3) for k, v in worst.items()})
    assert max(worst.values()) <= 1.0


@pytest.mark.parametrize("kind", ["asinh", "envelope", "residual"])
def test_float32_model_passes_the_inference_check(net, kind):
    g, p, freq, scale, bounds, env_table, base_table, x, q2, xf = net
    s = SimSurrogate(p, freq, bounds, g.nflav, kind, scale, env_table, base_table, 4)
    w = sb.check_inference(s.eval(x, q2), p, x, q2, scale, freq, bounds, g.nflav, kind, env_table, base_table)
    print(kind, "inference: worst element at", round(w, 3), "of its bound")
    assert w < 0.3


def test_inference_bound_is_informative(net):
    """The first-order bound allows every bfloat16 rounding in the network to
    go the other way, so it sits well above the typical difference (the
    float32 model above uses under a tenth of it), but it stays below half
    the output's mean size everywhere: an output off by that much (a dropped
    bias, a wrong layer) fails."""
    g, p, freq, scale, bounds, env_table, base_table, x, q2, xf = net
    y, dy = sb.forward_bound(p, x, q2, freq, bounds, g.nflav)
    rel = dy / np.abs(y).mean()
    print("bound / mean |y|: median", np.median(rel), "max", rel.max())
    assert np.median(rel) < 0.35 and rel.max() < 0.75


@pytest.mark.parametrize("kind,plant", [("asinh", "drop_bias"), ("asinh", "silu_argument"),
                                        ("envelope", "dsilu_of_h"), ("asinh", "transposed_gradient"),
                                        ("residual", "no_base")])
def test_planted_mistakes_fail(net, kind, plant):
    with pytest.raises(AssertionError):
        _run(net, kind, plant)


def test_planted_mistake_in_inference_fails(net):
    g, p, freq, scale, bounds, env_table, base_table, x, q2, xf = net
    s = SimSurrogate(p, freq, bounds, g.nflav, "envelope", scale, env_table, base_table, 4, "drop_bias")
    with pytest.raises(AssertionError):
        sb.check_inference(s.eval(x, q2), p, x, q2, scale, freq, bounds, g.nflav, "envelope", env_table, base_table)
