"""CPU oracle for the Monte Carlo integration -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
use it.  Plain numpy, written from the definitions (no code shared with the
CUDA path, paper_2009_06635_gb300/csrc/mc.cu and mc.cuh):

  splitmix64(seed, k)  the k-th output of SplitMix64 (G. L. Steele, D. Lea,
                       C. H. Flood, OOPSLA 2014): state seed + (k+1) * gamma,
                       gamma = 0x9E3779B97F4A7C15, through the generator's
                       published 64-bit finaliser.  A counter-based generator
                       drawn on both sides from its definition, because the
                       device draws the events itself.
  events               event i: u_j = (z >> 11) 2^-53 with z = splitmix64(seed,
                       2i + j); ln x_j = ln x_max + u_j (ln x_min - ln x_max),
                       capped at x_max; s-hat = x1 x2 s.
  weights              the toy leading-order observable standing in for the
                       paper's processes (Sec. 5 integrates single-top and VBF
                       Higgs matrix elements with VegasFlow; those are not part
                       of this library): with L = ln x_max - ln x_min,
                       w = L^2 / s-hat [sum_q e_q^2 (xf_q(x1) xf_-q(x2) +
                       xf_-q(x1) xf_q(x2)) + alpha_s(s-hat)^2 xf_g(x1) xf_g(x2)]
                       for s-hat >= s-hat_min, else 0; e_q = -1/3, 2/3, -1/3,
                       2/3, -1/3 for d, u, s, c, b.  The PDF load (all flavours
                       at x1 and x2, alpha_s at Q^2 = s-hat) is PDFFlow Sec. 4.1's.
  sums                 (sum w, sum w^2, sum |w|) over a range of events.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
CHARGE2 = {1: 1.0 / 9.0, 2: 4.0 / 9.0, 3: 1.0 / 9.0, 4: 4.0 / 9.0, 5: 1.0 / 9.0}


def splitmix64(seed, k):
    """k-th output (k >= 0, array) of SplitMix64 seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
    return z ^ (z >> np.uint64(31))


def uniform(z):
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def events(seed, first, n, x_min, x_max):
    i = np.arange(first, first + n, dtype=np.uint64)
    u1 = uniform(splitmix64(seed, 2 * i))
    u2 = uniform(splitmix64(seed, 2 * i + 1))
    lmin, lmax = np.log(x_min), np.log(x_max)
    x1 = np.minimum(np.exp(lmax + u1 * (lmin - lmax)), x_max)
    x2 = np.minimum(np.exp(lmax + u2 * (lmin - lmax)), x_max)
    return x1, x2


def weights(og, pids, sqrt_s, x_min, shat_min, seed, first, n, x_max):
    """Per-event weights; og is an OracleGrid, pids its flavour codes."""
    x1, x2 = events(seed, first, n, x_min, x_max)
    s = sqrt_s * sqrt_s
    shat = x1 * x2 * s
    f1, _, _ = og.xfxq2(x1, shat)
    f2, _, _ = og.xfxq2(x2, shat)
    a, _ = og.alphas(shat)
    col = {p: k for k, p in enumerate(pids)}
    acc = np.zeros(n)
    for q in range(1, 6):
        cq, cb = col[q], col[-q]
        acc += CHARGE2[q] * (f1[:, cq] * f2[:, cb] + f1[:, cb] * f2[:, cq])
    acc += a * a * (f1[:, col[21]] * f2[:, col[21]])
    L = np.log(x_max) - np.log(x_min)
    w = L * L * acc / shat
    return np.where(shat >= shat_min, w, 0.0)


def sums(w):
    w = np.asarray(w, dtype=np.float64)
    return float(w.sum()), float((w * w).sum()), float(np.abs(w).sum())
