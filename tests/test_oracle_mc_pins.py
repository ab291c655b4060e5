"""Pins of the Monte Carlo oracle (oracle/mc.py): the 64-bit wrap-around
arithmetic of its SplitMix64 against Python's unbounded integers, the
uniformity of the draws, and the estimator against the integral computed by
quadrature on a grid whose values are constant (so the integrand has a
closed form: every term of the weight, the Jacobian, the cut and the flavour
pairing enter it)."""
import numpy as np
import pytest

mc = pytest.importorskip("oracle.mc")

G, M1, M2, MASK = 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9, 0x94D049BB133111EB, (1 << 64) - 1


def splitmix64_int(seed, k):
    z = (seed + (k + 1) * G) & MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def test_wraparound_arithmetic_matches_unbounded_integers():
    r = np.random.default_rng(1)
    seeds = [0, 1, 2024, MASK, int(r.integers(0, 2**63)) * 2 + 1]
    ks = [0, 1, 2, 10**6, 2**40 + 3, 2**62]
    for s in seeds:
        got = mc.splitmix64(s, np.array(ks, dtype=np.uint64))
        assert [int(v) for v in got] == [splitmix64_int(s, k) for k in ks]


def test_draws_are_uniform_and_uncorrelated():
    n = 1_000_000
    u = mc.uniform(mc.splitmix64(77, np.arange(n, dtype=np.uint64)))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    counts = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 63 + 5 * np.sqrt(2 * 63)
    rho = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(rho) < 5 / np.sqrt(n)
    # the two coordinates of an event are independent streams of the counter
    x1, x2 = mc.events(5, 0, n, 1e-6, 1.0)
    assert abs(np.corrcoef(np.log(x1), np.log(x2))[0, 1]) < 5 / np.sqrt(n)
    assert x1.min() >= 1e-6 and x1.max() <= 1.0


def test_estimator_matches_quadrature_on_a_constant_grid(oracle_mod):
    integrate = pytest.importorskip("scipy.integrate")
    pids = [-5, -4, -3, -2, -1, 21, 1, 2, 3, 4, 5]
    const = {-5: 0.3, -4: 0.7, -3: 1.1, -2: 0.4, -1: 0.9, 21: 2.5, 1: 1.3, 2: 0.6, 3: 0.8, 4: 1.7, 5: 0.2}
    xk = np.geomspace(1e-3, 1.0, 20)
    qk = np.geomspace(1.0, 1e8, 15)
    vals = np.empty((len(qk), len(xk), len(pids)))
    for k, p in enumerate(pids):
        vals[:, :, k] = const[p]
    alpha = 0.2
    og = oracle_mod.OracleGrid(x_knots=xk, nq=[len(qk)], q2_knots=qk, values=vals, as_q2=qk,
                               as_vals=np.full(len(qk), alpha))
    sqrt_s, x_min, shat_min = 1e4, 1e-3, 1e3
    s = sqrt_s ** 2
    n = 400_000
    w = mc.weights(og, pids, sqrt_s, x_min, shat_min, 11, 0, n, 1.0)
    est = w.mean()
    err = w.std(ddof=1) / np.sqrt(n)
    # E[w] = int int dx1 dx2 K / (x1 x2)^2 / s over x1 x2 s >= shat_min, with
    # K = 2 sum_q e_q^2 a_q a_-q + alpha^2 a_g^2 (xf constant, f = xf / x)
    charge = {1: -1 / 3, 2: 2 / 3, 3: -1 / 3, 4: 2 / 3, 5: -1 / 3}  # d, u, s, c, b
    K = sum(charge[q] ** 2 * 2 * const[q] * const[-q] for q in range(1, 6)) + alpha ** 2 * const[21] ** 2
    a, c = np.log(x_min), np.log(shat_min / s)
    # in y = ln x: dx / x^2 = e^-y dy
    J, _ = integrate.dblquad(lambda y2, y1: np.exp(-y1 - y2), a, 0.0, lambda y1: max(a, c - y1), lambda y1: 0.0,
                             epsabs=0, epsrel=1e-12)
    exact = K * J / s
    assert abs(est - exact) < 5 * err, (est, exact, err)
    assert err < 0.02 * exact  # the test resolves the integral to ~2%
    # without the cut the same integral factorises
    w0 = mc.weights(og, pids, sqrt_s, x_min, 0.0, 12, 0, n, 1.0)
    exact0 = K * (1 / x_min - 1) ** 2 / s
    assert abs(w0.mean() - exact0) < 5 * w0.std(ddof=1) / np.sqrt(n)
