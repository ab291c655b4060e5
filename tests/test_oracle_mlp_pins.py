"""Pins of the surrogate's CPU oracle (oracle/mlp.py) against things it does
not compute itself: central finite differences of its loss, the sigmoid
form of SiLU, bfloat16 rounding as torch performs it and on hand-checked bit
patterns, the identities of the Fourier features, and the target/prediction
pair being inverse maps."""
import numpy as np
import pytest

mlp = pytest.importorskip("oracle.mlp")

NF = 5


def small_problem(seed=3, n=7):
    r = np.random.default_rng(seed)
    shapes = [(mlp.WIDTH, 2 * mlp.NFEAT), (mlp.WIDTH, mlp.WIDTH), (mlp.WIDTH, mlp.WIDTH), (mlp.WIDTH, mlp.WIDTH),
              (NF, mlp.WIDTH)]
    parts = []
    for (o, i) in shapes:
        parts.append(r.uniform(-1, 1, o * i) * np.sqrt(6.0 / i))
        parts.append(r.normal(0, 0.1, o))
    params = np.concatenate(parts)
    freq = r.normal(0, 2.0, (mlp.NFEAT, 2))
    bounds = (np.log(1e-9), 0.0, 0.0, np.log(1e10))
    x = np.exp(r.uniform(np.log(1e-9), 0.0, n))
    q2 = np.exp(r.uniform(0.0, np.log(1e10), n))
    xf = r.normal(0, 1.0, (n, NF))
    scale = np.abs(r.normal(1.0, 0.2, NF)) + 0.1
    return params, freq, bounds, x, q2, xf, scale


def test_silu_matches_the_sigmoid_form():
    v = np.linspace(-30, 30, 2001)
    # equal to rounding of the larger of v and 1 (the tanh form's tail below
    # v ~ -30 carries an absolute, not a relative, error of that size)
    assert np.all(np.abs(mlp.silu(v) - v / (1.0 + np.exp(-v))) <= 1e-15 * np.maximum(np.abs(v), 1.0))
    h = 1e-6
    fd = (mlp.silu(v + h) - mlp.silu(v - h)) / (2 * h)
    assert np.allclose(mlp.dsilu(v), fd, rtol=1e-7, atol=1e-9)


def test_loss_gradient_matches_central_differences():
    params, freq, bounds, x, q2, xf, scale = small_problem()
    loss, grad = mlp.loss_grad(params, x, q2, xf, scale, freq, bounds, NF)
    r = np.random.default_rng(4)
    # every layer's weights and biases are probed
    sizes = [mlp.WIDTH * 2 * mlp.NFEAT, mlp.WIDTH] + [mlp.WIDTH * mlp.WIDTH, mlp.WIDTH] * 3 + [NF * mlp.WIDTH, NF]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    idx = np.concatenate([s + r.integers(0, z, 4) for s, z in zip(starts, sizes)])
    for i in idx:
        h = 1e-6 * max(1.0, abs(params[i]))
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, x, q2, xf, scale, freq, bounds, NF)[0] -
              mlp.loss_grad(pm, x, q2, xf, scale, freq, bounds, NF)[0]) / (2 * h)
        # truncation O(h^2) is negligible; rounding of the difference ~1e-16 * loss / h
        assert abs(fd - grad[i]) <= 1e-6 * abs(fd) + 1e-9, (i, fd, grad[i])
    # the loss is the mean square distance to the asinh targets
    y, _ = mlp.forward(params, x, q2, freq, bounds, NF)
    assert np.isclose(loss, np.mean((y - np.arcsinh(xf / scale)) ** 2), rtol=1e-15)


def test_bf16_rounding_matches_torch_and_bit_patterns():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(5)
    a = np.concatenate([r.normal(0, 1, 10000) * 10.0 ** r.integers(-20, 20, 10000), [0.0, -0.0, 1.0, -2.5]])
    a32 = a.astype(np.float32)
    want = torch.from_numpy(a32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a32), want)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1;
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6 -> 1 + 2^-6
    assert mlp.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    assert mlp.bf16(np.array([1 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1 + 2.0 ** -7


def test_features_span_the_box_and_lie_on_circles():
    params, freq, bounds, x, q2, xf, scale = small_problem()
    lx_lo, lx_hi, lq_lo, lq_hi = bounds
    xe = np.array([np.exp(lx_lo), np.exp(lx_hi)])
    qe = np.array([np.exp(lq_lo), np.exp(lq_hi)])
    phi = mlp.features(xe, qe, freq, bounds)
    # corners (-1, -1) and (1, 1): the angle is pi (+-f0 +- f1)
    a_lo = np.pi * (-freq[:, 0] - freq[:, 1])
    a_hi = np.pi * (freq[:, 0] + freq[:, 1])
    assert np.allclose(phi[0, :mlp.NFEAT], np.sin(a_lo), atol=1e-12)
    assert np.allclose(phi[1, mlp.NFEAT:], np.cos(a_hi), atol=1e-12)
    phi = mlp.features(x, q2, freq, bounds)
    assert np.allclose(phi[:, :mlp.NFEAT] ** 2 + phi[:, mlp.NFEAT:] ** 2, 1.0, atol=1e-14)


def test_prediction_inverts_the_target_map():
    params, freq, bounds, x, q2, xf, scale = small_problem()
    y, _ = mlp.forward(params, x, q2, freq, bounds, NF)
    pred = mlp.predict(params, x, q2, scale, freq, bounds, NF)
    assert np.allclose(mlp.target(pred, scale), y, rtol=1e-12, atol=1e-12)
    # a network whose last layer is zero predicts zero for every flavour
    p0 = params.copy()
    p0[-(NF * mlp.WIDTH + NF):] = 0.0
    assert np.array_equal(mlp.predict(p0, x, q2, scale, freq, bounds, NF), np.zeros((len(x), NF)))


def test_envelope_reproduces_power_laws_and_the_floor():
    # |xf| maximal over Q = 2 x^-0.3 (1 + 0.1 * row): a power law in x, so
    # ln E is linear in ln x and the tabulated envelope is exact everywhere
    xk = np.geomspace(1e-6, 1.0, 37)
    rows = 5
    vals = np.zeros((rows, len(xk), 3))
    for j in range(rows):
        vals[j, :, 0] = 2.0 * xk ** -0.3 * (1 + 0.1 * j) / 1.4  # largest at the top row: 2 x^-0.3
        vals[j, :, 1] = -(0.5 + j) * xk ** 0.7                    # sign does not matter: 4.5 x^0.7
    bounds = (np.log(1e-6), 0.0, 0.0, 1.0)
    T = mlp.envelope_table(xk, vals, bounds)
    x = np.exp(np.random.default_rng(8).uniform(np.log(1e-6), 0.0, 1000))
    E = mlp.envelope(T, x, bounds)
    assert np.allclose(E[:, 0], 2.0 * x ** -0.3, rtol=1e-12)
    assert np.allclose(E[:, 1], 4.5 * x ** 0.7, rtol=1e-12)
    assert np.allclose(E[:, 2], 1e-5, rtol=1e-12)  # an all-zero flavour sits on the floor

