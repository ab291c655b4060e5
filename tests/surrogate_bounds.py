"""Element-wise checks of the GPU surrogate against the numpy oracle of the
same network (oracle/mlp.py), every element within a bound derived from the
arithmetic each side does.

The GPU rounds to bfloat16 at the points where the oracle with bf=True does;
what is left between them (u = 2^-24):
  - FP32 accumulation of bfloat16 products on the tensor core, in the GPU's
    order: (K + 1) 2u (sum |W h| + |b|) for K terms (2u per addition covers
    an accumulation that truncates when it aligns the addends);
  - SiLU through the hardware tanh approximation (absolute error 2^-10.99 in
    the PTX description; 2^-10 taken), at half argument: 0.5 |z| 2^-10;
  - one bfloat16 rounding that may go the other way when the values before
    it differ: one bfloat16 ulp;
  - FP32 coordinates (logf of the float-rounded input), sinf/cosf or
    sincospif (two float ulps), the envelope's expf and the base table's FP32
    bilinear arithmetic.

Propagated through four layers of width 128 by absolute values these bounds
grow by the sum of |W| per layer and say nothing.  So:
  - the training pass is checked stage by stage on the GPU's own
    intermediates (pdf_surrogate_trace): each pre-activation, activation,
    backward signal and gradient against the oracle's formula applied to the
    GPU's inputs of that stage, where only the local terms above remain;
  - the fused inference output is checked against the oracle's forward pass
    with each local term carried to the output by the oracle's own signed
    Jacobian (first order; the second-order remainder is below 2^-4 of the
    first-order bound for perturbations of a bfloat16 ulp, and the factor
    (1 + 2^-4) covers it).
"""
import numpy as np

U = 2.0**-24
TC_U = 2 * U
TANH_ERR = 2.0**-10
SECOND_ORDER = 1.0 + 2.0**-4


def ulp_bf16(v):
    """One bfloat16 ulp of |v| (8 significant bits); 2^-133 for 0."""
    a = np.abs(np.asarray(v, dtype=np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 2.0**-126)))
    return 2.0 ** (e - 7)


def assert_within(got, want, bound, what=""):
    """Every element |got - want| <= bound; returns the largest ratio."""
    got, want, bound = (np.asarray(a, dtype=np.float64) for a in (got, want, bound))
    assert got.shape == want.shape == bound.shape, (what, got.shape, want.shape, bound.shape)
    assert np.all(np.isfinite(got)), what
    diff = np.abs(got - want)
    ratio = np.where(diff > 0, diff / np.maximum(bound, 1e-300), 0.0)
    k = int(np.argmax(ratio))
    assert ratio.flat[k] <= 1.0, (f"{what}: element {np.unravel_index(k, ratio.shape)} differs by "
                                  f"{diff.flat[k]:.3e} (got {got.flat[k]:.6e}, want {want.flat[k]:.6e}), "
                                  f"bound {bound.flat[k]:.3e}")
    return float(ratio.max())


# ---------------------------------------------------------------------------
# coordinates and features
# ---------------------------------------------------------------------------

def coords(x, q2, bounds):
    """(z0, z1, dz0, dz1): the scaled coordinates in FP64 and bounds on the
    GPU's FP32 values' errors: x rounded to float and logf within an ulp
    (u (1 + 2 |ln x|)), the float constants lx_lo and 1/(lx_hi - lx_lo),
    three roundings of the affine map; times 1.5 as margin."""
    out = []
    for l, lo, hi in ((np.log(x), bounds[0], bounds[1]), (np.log(q2), bounds[2], bounds[3])):
        inv = 1.0 / (hi - lo)
        z = 2.0 * (l - lo) * inv - 1.0
        dl = U * (1.0 + 2.0 * np.abs(l))
        dz = 2.0 * inv * (dl + U * abs(lo) + 2.0 * U * np.abs(l - lo)) + U * (3.0 * np.abs(z + 1.0) + np.abs(z))
        out.append((z, 1.5 * dz))
    (z0, dz0), (z1, dz1) = out
    return z0, z1, dz0, dz1


def feature_diff(x, q2, freq, bounds):
    """Bound on |GPU feature - exact feature| before the bfloat16 rounding,
    [n][32]: the coordinates' errors through pi F, the FP32 angle (three
    roundings of F0 z0 + F1 z1, the float pi) and two float ulps of the sine
    or cosine (sinf / cosf in training, sincospif in inference)."""
    z0, z1, dz0, dz1 = coords(x, q2, bounds)
    f0, f1 = np.abs(freq[:, 0]), np.abs(freq[:, 1])
    a0, a1 = np.outer(np.abs(z0), f0), np.outer(np.abs(z1), f1)
    d = np.pi * (np.outer(dz0, f0) + np.outer(dz1, f1) + 3.0 * U * (a0 + a1) + 2.0 * U * (a0 + a1)) + 4.0 * U
    return np.concatenate([d, d], axis=1)


def _acc(h, Wb, b):
    """FP32 tensor-core accumulation bound of h Wb^T + b, [n][out]."""
    K = Wb.shape[1]
    return (K + 1) * TC_U * (np.abs(h) @ np.abs(Wb).T + np.abs(b))


def _silu_local(z):
    """|GPU silu(z) - silu(z)| at the same FP32 argument, before rounding."""
    from oracle import mlp

    return 0.5 * np.abs(z) * TANH_ERR + 3.0 * U * (np.abs(mlp.silu(z)) + np.abs(z))


def _round_pair(d, v):
    """|bf16(a) - bf16(b)| for |a - b| <= d, b = v: d plus one bfloat16 ulp."""
    return d + ulp_bf16(np.abs(v) + d)


# ---------------------------------------------------------------------------
# the output transforms: envelope, base and targets
# ---------------------------------------------------------------------------

def envelope_rel(env_table, x, bounds):
    """Bound on |E_gpu / E - 1| per point and flavour: the float ln E table
    (u |ln E| each end), the float position in it (the coordinate's error and
    its rounding, times the table's slope), the float interpolation and expf
    (two ulps)."""
    from oracle import mlp

    z0, _, dz0, _ = coords(x, np.ones_like(x), (bounds[0], bounds[1], 0.0, 1.0))
    N = mlp.ENV_N
    u = np.clip((z0 + 1.0) * 0.5 * N, 0.0, N)
    k = np.minimum(np.floor(u).astype(int), N - 1)
    a, b = env_table[:, k].T, env_table[:, k + 1].T  # [n][nflav]
    lo, hi = env_table[:, np.maximum(k - 1, 0)].T, env_table[:, np.minimum(k + 2, N)].T
    slope = np.maximum.reduce([np.abs(b - a), np.abs(a - lo), np.abs(hi - b)])
    du = 0.5 * N * (dz0 + 2.0 * U * 2.0)[:, None] + 2.0 * U * N
    dln = 4.0 * U * np.maximum(np.abs(a), np.abs(b)) + slope * du + 4.0 * U
    return np.expm1(dln)


def base_diff(base_table, x, q2, bounds):
    """Bound on |B_gpu - B| per point and flavour: the two tables' nodes may
    round to float differently (2u |v|), the coordinates' errors times the
    largest slope of the neighbouring cells, and the FP32 bilinear arithmetic
    (8u of the largest corner)."""
    from oracle import mlp

    z0, z1, dz0, dz1 = coords(x, q2, bounds)
    N = mlp.BASE_N
    u0 = np.clip((z0 + 1.0) * 0.5 * N, 0.0, N)
    u1 = np.clip((z1 + 1.0) * 0.5 * N, 0.0, N)
    i = np.minimum(np.floor(u0).astype(int), N - 1)
    j = np.minimum(np.floor(u1).astype(int), N - 1)
    T = base_table
    corner = np.maximum.reduce([np.abs(T[i, j]), np.abs(T[i + 1, j]), np.abs(T[i, j + 1]), np.abs(T[i + 1, j + 1])])
    s0 = np.zeros_like(corner)
    s1 = np.zeros_like(corner)
    for di in (-1, 0, 1):
        ii = np.clip(i + di, 0, N - 1)
        for dj in (-1, 0, 1, 2):
            jj = np.clip(j + dj, 0, N)
            s0 = np.maximum(s0, np.abs(T[ii + 1, jj] - T[ii, jj]))
    for dj in (-1, 0, 1):
        jj = np.clip(j + dj, 0, N - 1)
        for di in (-1, 0, 1, 2):
            ii = np.clip(i + di, 0, N)
            s1 = np.maximum(s1, np.abs(T[ii, jj + 1] - T[ii, jj]))
    du0 = 0.5 * N * (dz0 + 4.0 * U)[:, None] + 2.0 * U * N
    du1 = 0.5 * N * (dz1 + 4.0 * U)[:, None] + 2.0 * U * N
    return 2.0 * U * corner + s0 * du0 + s1 * du1 + 8.0 * U * corner


def transforms(kind, x, q2, scale, bounds, env_table=None, base_table=None):
    """The oracle's E and B for the points (None where the target has none)
    and the bounds on the GPU's differences from them."""
    from oracle import mlp

    env = mlp.envelope(env_table, x, bounds) if kind != "asinh" else None
    base = mlp.base(base_table, x, q2, bounds) if kind == "residual" else None
    denv = envelope_rel(env_table, x, bounds) if env is not None else None
    dbase = base_diff(base_table, x, q2, bounds) if base is not None else None
    return env, base, denv, dbase


def target_bound(kind, xf, scale, env, base, denv, dbase):
    """(t, |t_gpu - t|): the oracle's FP64 training targets and the bound on
    the GPU's FP32 targets (computed in FP64 from the GPU's float E and B,
    then rounded)."""
    from oracle import mlp

    t = mlp.target(xf, scale, env, base)
    if kind == "asinh":
        return t, 3.0 * U * (np.abs(t) + 1.0)
    if kind == "envelope":
        return t, np.abs(t) * denv * (1.0 + denv) + 2.0 * U * np.abs(t)
    return t, (dbase / (mlp.RES_EPS * env) + np.abs(t) * denv) * (1.0 + denv) + 2.0 * U * np.abs(t) + 1e-300


# ---------------------------------------------------------------------------
# the training pass, stage by stage
# ---------------------------------------------------------------------------

def check_training_pass(s, params, x, q2, xf, scale, freq, bounds, nflav, grad, kind="asinh", env_table=None,
                        base_table=None):
    """Every stage of surrogate s's last loss_grad pass (on x, q2 with
    interpolator values xf, returning grad) against the oracle's formulas on
    the GPU's inputs of that stage.  Returns {stage: largest ratio to bound}."""
    from oracle import mlp

    n = len(x)
    layers = mlp.unpack(np.asarray(params, dtype=np.float64), nflav)
    Wb = [mlp.bf16(W) for W, _ in layers]
    h = [s.trace("h", l, n).astype(np.float64) for l in range(5)]
    z = [s.trace("z", l, n).astype(np.float64) for l in range(4)]
    y = s.trace("y", 0, n).astype(np.float64)
    t = s.trace("t", 0, n).astype(np.float64)
    gs = [s.trace("g", l, n).astype(np.float64) for l in range(5)]
    worst = {}
    # padded output columns: no output, no target, no signal
    assert np.all(y[:, nflav:] == 0) and np.all(t[:, nflav:] == 0) and np.all(gs[4][:, nflav:] == 0)
    y, t, g4 = y[:, :nflav], t[:, :nflav], gs[4][:, :nflav]
    # features
    phi = mlp.features(x, q2, freq, bounds)
    worst["features"] = assert_within(h[0], mlp.bf16(phi), _round_pair(feature_diff(x, q2, freq, bounds), phi),
                                      "features")
    # forward: z_l = h_l W_l^T + b_l (FP32), h_{l+1} = bf16(silu(z_l)), y = h_4 W_4^T + b_4
    for l in range(5):
        want = h[l] @ Wb[l].T + layers[l][1]
        bound = _acc(h[l], Wb[l], layers[l][1])
        if l < 4:
            worst[f"z{l}"] = assert_within(z[l], want, bound + U * np.abs(want), f"pre-activation {l}")
            sv = mlp.silu(z[l])
            worst[f"h{l + 1}"] = assert_within(h[l + 1], mlp.bf16(sv), _round_pair(_silu_local(z[l]), sv),
                                               f"activation {l + 1}")
        else:
            worst["y"] = assert_within(y, want, bound + U * np.abs(want), "output")
    # targets
    env, base, denv, dbase = transforms(kind, x, q2, scale, bounds, env_table, base_table)
    tw, tb = target_bound(kind, xf, scale, env, base, denv, dbase)
    worst["t"] = assert_within(t, tw, tb, "targets")
    # backward: g_4 = bf16(2 (y - t) / (n nflav)), g_{l-1} = bf16((g_l W_l) silu'(z_{l-1}))
    gw = 2.0 * (y - t) / (n * nflav)
    worst["g4"] = assert_within(g4, mlp.bf16(gw), _round_pair(4.0 * U * np.abs(gw), gw), "output signal")
    for l in range(4, 0, -1):
        gl = gs[l][:, :nflav] if l == 4 else gs[l]
        W = Wb[l][:nflav] if l == 4 else Wb[l]
        dh = gl @ W
        ddh = (W.shape[0] + 1) * TC_U * (np.abs(gl) @ np.abs(W))
        zz = z[l - 1]
        ds = mlp.dsilu(zz)
        dds = (1.0 + np.abs(zz)) * (0.5 * TANH_ERR + 4.0 * U)
        want = dh * ds
        worst[f"g{l - 1}"] = assert_within(gs[l - 1], mlp.bf16(want),
                                           _round_pair(np.abs(ds) * ddh + np.abs(dh) * dds + 2.0 * U * np.abs(want),
                                                       want), f"signal {l - 1}")
    # gradients: dW_l = g_l^T h_l, db_l = sum over the batch of g_l (FP32 sums
    # of n terms: the tensor core per chunk, atomics across chunks)
    parts = mlp.unpack(np.asarray(grad, dtype=np.float64), nflav)
    for l in range(5):
        gl = g4 if l == 4 else gs[l]
        gwl, gbl = parts[l]
        worst[f"dW{l}"] = assert_within(gwl, gl.T @ h[l], (n + 1) * TC_U * (np.abs(gl).T @ np.abs(h[l])),
                                        f"weight gradient {l}")
        worst[f"db{l}"] = assert_within(gbl, gl.sum(axis=0), (n + 1) * TC_U * np.abs(gl).sum(axis=0),
                                        f"bias gradient {l}")
    return worst


# ---------------------------------------------------------------------------
# the fused inference output
# ---------------------------------------------------------------------------

def forward_bound(params, x, q2, freq, bounds, nflav):
    """(y, dy): the oracle's network output (bf=True) and the first-order
    bound on |y_gpu - y| per element: every local term (features, each
    product's accumulation, each SiLU and each bfloat16 rounding) times the
    absolute value of the oracle's Jacobian of y with respect to the quantity
    it perturbs, summed, times (1 + 2^-4)."""
    from oracle import mlp

    layers = mlp.unpack(np.asarray(params, dtype=np.float64), nflav)
    Wb = [mlp.bf16(W) for W, _ in layers]
    y, cache = mlp.forward(params, x, q2, freq, bounds, nflav, bf=True)
    h, z = cache["h"], cache["z"]
    n = len(x)
    dy = _acc(h[4], Wb[4], layers[4][1]) + U * np.abs(y)
    J = np.broadcast_to(Wb[4], (n,) + Wb[4].shape)  # dy/dh_4 [n][nflav][128]
    for l in range(3, -1, -1):
        # h_{l+1} = bf16(silu(z_l)): the SiLU and the rounding
        sv = mlp.silu(z[l])
        dy += np.einsum("njk,nk->nj", np.abs(J), _round_pair(_silu_local(z[l]), sv))
        Jz = J * mlp.dsilu(z[l])[:, None, :]
        dy += np.einsum("njk,nk->nj", np.abs(Jz), _acc(h[l], Wb[l], layers[l][1]))
        J = Jz @ Wb[l]  # dy/dh_l
    phi = mlp.features(x, q2, freq, bounds)
    dy += np.einsum("njk,nk->nj", np.abs(J), _round_pair(feature_diff(x, q2, freq, bounds), phi))
    return y, SECOND_ORDER * dy


def check_inference(out, params, x, q2, scale, freq, bounds, nflav, kind="asinh", env_table=None, base_table=None):
    """The GPU's inference output xf [n][nflav] against the oracle's
    prediction (bf=True), every element within the network's first-order
    bound carried through the output transform plus the transform's own
    terms (float sinhf, expf envelope, FP32 base).  Returns the largest
    ratio to the bound."""
    from oracle import mlp

    y, dy = forward_bound(params, x, q2, freq, bounds, nflav)
    out = np.asarray(out, dtype=np.float64)
    if kind == "asinh":
        want = scale * np.sinh(y)
        bound = scale * np.cosh(np.abs(y) + dy) * dy + 6.0 * U * np.abs(want) + 1e-300
    else:
        env, base, denv, dbase = transforms(kind, x, q2, scale, bounds, env_table, base_table)
        eps = mlp.RES_EPS if kind == "residual" else 1.0
        want = eps * env * y + (base if base is not None else 0.0)
        bound = eps * env * ((1.0 + denv) * dy + np.abs(y) * denv) + 4.0 * U * eps * env * np.abs(y)
        if base is not None:
            bound = bound + dbase + 2.0 * U * (np.abs(base) + np.abs(want))
    return assert_within(out, want, bound, f"inference ({kind})")
