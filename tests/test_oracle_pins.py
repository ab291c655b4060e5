"""Pins for the CPU oracle: each test checks the oracle against something
other than itself -- the defining properties of the Hermite segment and of
the finite-difference tangents, polynomial classes the scheme reproduces
exactly, an exact-rational implementation written in the other (Q-first)
order, extrapolation identities, and the linearity of the interpolant in the
knot values.  PDFFlow Sec. 2.2 (log-bicubic, subgrids, edges), Sec. 2.3
(alpha_s), Fig. 1 (EXTRAPOLATE).

Note on cubic exactness: finite-difference tangents make the full scheme
exact for functions linear in ln x and ln Q^2 (any spacing) and for
quadratics in interior cells of uniformly log-spaced knots, not for general
cubics.  The cubic class is pinned on the Hermite segment itself, given exact
tangents (test_hermite_segment_reproduces_cubics)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import rng

U = 2.0**-53


def mk(synth, x_knots, q2_subs, fn, nflav, alphas_fn=None):
    return synth.make_grid(x_knots, q2_subs, list(range(nflav)), values_fn=fn, alphas_fn=alphas_fn)


def scale_ok(got, want, s, rtol):
    got, want, s = map(np.asarray, (got, want, s))
    return np.abs(got - want) <= rtol * np.maximum(np.abs(want), s)


def rand_knots(r, lo, hi, n):
    """n strictly increasing log-spaced-ish knots with exact endpoints."""
    inner = np.sort(r.uniform(np.log(lo), np.log(hi), n - 2))
    k = np.exp(np.concatenate([[np.log(lo)], inner, [np.log(hi)]]))
    k[0], k[-1] = lo, hi
    return k


def rand_subgrids(r, bounds, counts):
    subs = []
    for s in range(len(counts)):
        subs.append(rand_knots(r, bounds[s], bounds[s + 1], counts[s]))
    return subs


# ---------------------------------------------------------------------------
# knots, ties, thresholds
# ---------------------------------------------------------------------------

def test_knots_reproduced_exactly(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    X, Q = np.meshgrid(g.x_knots, g.q2_knots)
    v, s, fl = og.xfxq2(X.ravel(), Q.ravel())
    want = g.values.reshape(-1, g.nflav)
    assert np.array_equal(v, want)
    assert not fl.any()


def test_threshold_point_belongs_to_upper_subgrid(oracle_mod, synth):
    x = synth.geom_knots(1e-4, 1.0, 8)
    subs = [np.array([1.0, 2.0, 3.0, 4.0]), np.array([4.0, 6.0, 9.0])]

    def fn(xk, q2):
        v = np.zeros((q2.shape[0], xk.shape[0], 1))
        v[:4, :, 0] = 1.0 + np.log(xk)[None, :] * 0.1 + np.log(q2[:4])[:, None]
        v[4:, :, 0] = 10.0 + np.log(xk)[None, :] * 0.2 + np.log(q2[4:])[:, None]
        return v

    g = mk(synth, x, subs, fn, 1)
    og = oracle_mod.OracleGrid(g)
    v, _, _ = og.xfxq2(x, np.full(x.shape, 4.0))
    assert np.array_equal(v[:, 0], g.values[4, :, 0])  # upper subgrid's first row
    v, _, _ = og.xfxq2(x, np.full(x.shape, 4.0 * (1 - 1e-12)))
    assert np.allclose(v[:, 0], g.values[3, :, 0], rtol=1e-9)  # lower subgrid's last row


def test_invalid_points_are_nan(oracle_mod, synth):
    g = synth.grid_single_subgrid()
    og = oracle_mod.OracleGrid(g)
    bad_x = [0.0, -1e-3, 1.0 + 1e-12, np.nan, np.inf, 0.5, 0.5, 0.5, 0.5]
    bad_q = [10.0, 10.0, 10.0, 10.0, 10.0, 0.0, -1.0, np.nan, np.inf]
    v, _, _ = og.xfxq2(bad_x, bad_q)
    assert np.isnan(v).all()
    # a grid whose last x knot is below 1: x above it is outside the domain
    g2 = synth.make_grid(synth.geom_knots(1e-3, 0.5, 6), [synth.geom_knots(2.0, 50.0, 5)], [0],
                         values_fn=lambda xk, q2: np.ones((q2.shape[0], xk.shape[0], 1)))
    v, _, _ = oracle_mod.OracleGrid(g2).xfxq2([0.5, 0.6], [10.0, 10.0])
    assert v[0, 0] == 1.0 and np.isnan(v[1, 0])


def test_rejects_malformed_grids(oracle_mod, synth):
    base = dict(x_knots=[1e-3, 1e-2, 1e-1, 1.0], nq=[3], q2_knots=[2.0, 4.0, 8.0],
                values=np.ones((3, 4, 1)), as_q2=[2.0, 8.0], as_vals=[0.3, 0.2])
    oracle_mod.OracleGrid(**base)
    for key, bad in [("x_knots", [1e-3, 1e-3, 1e-1, 1.0]), ("x_knots", [0.0, 1e-2, 1e-1, 1.0]),
                     ("x_knots", [1e-3, 1e-2, 1e-1, 1.5]), ("q2_knots", [2.0, 1.0, 8.0]),
                     ("as_q2", [2.0, 2.0])]:
        kw = dict(base)
        kw[key] = bad
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.OracleGrid(**kw)
    kw = dict(base, nq=[2, 2], q2_knots=[2.0, 4.0, 5.0, 8.0], values=np.ones((4, 4, 1)))
    with pytest.raises(oracle_mod.OracleError):  # boundary knots not duplicated
        oracle_mod.OracleGrid(**kw)
    kw = dict(base, values=np.full((3, 4, 1), np.nan))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.OracleGrid(**kw)


# ---------------------------------------------------------------------------
# the Hermite segment and the finite-difference tangents
# ---------------------------------------------------------------------------

def test_hermite_segment_reproduces_cubics(oracle_mod):
    r = rng(11)
    for _ in range(20):
        c = r.standard_normal(4)
        P = np.polynomial.Polynomial(c)
        dP = P.deriv()
        for t in np.linspace(0.0, 1.0, 13):
            got = oracle_mod.hermite(t, P(0.0), P(1.0), dP(0.0), dP(1.0))
            assert abs(got - P(t)) <= 1e-14 * np.abs(c).sum()


def _expected_slopes(l, f):
    """R-slope: mean of adjacent secants inside, one-sided secant at the ends."""
    n = len(l)
    sec = [(f[k + 1] - f[k]) / (l[k + 1] - l[k]) for k in range(n - 1)]
    return [sec[0]] + [0.5 * (sec[k - 1] + sec[k]) for k in range(1, n - 1)] + [sec[-1]]


def _fit_cubic(ts, vals):
    return np.polynomial.Polynomial.fit(ts, vals, 3, domain=[0, 1], window=[0, 1])


def test_x_cells_meet_hermite_conditions(oracle_mod, synth):
    """In every x cell (edges included), along a knot row, the interpolant is a
    cubic in t whose end values are the knot values and whose end derivatives
    are the R-slope tangents times the cell width."""
    r = rng(12)
    x = rand_knots(r, 1e-5, 1.0, 7)
    vals = r.standard_normal((3, 7, 1))
    g = mk(synth, x, [np.array([2.0, 5.0, 11.0])], lambda xk, q2: vals, 1)
    og = oracle_mod.OracleGrid(g)
    lx = np.log(x)
    for row in range(3):
        f = vals[row, :, 0]
        sl = _expected_slopes(lx, f)
        for i in range(6):
            d = lx[i + 1] - lx[i]
            ts = np.linspace(0.0, 1.0, 9)
            xs = np.exp(lx[i] + ts * d)
            xs[0], xs[-1] = x[i], x[i + 1]
            v, _, _ = og.xfxq2(xs, np.full(9, g.q2_knots[row]))
            p = _fit_cubic(ts, v[:, 0])
            dp = p.deriv()
            sc = np.abs(f).max()
            assert abs(p(0) - f[i]) < 1e-9 * sc and abs(p(1) - f[i + 1]) < 1e-9 * sc
            assert abs(dp(0) - d * sl[i]) < 1e-7 * sc, (row, i)
            assert abs(dp(1) - d * sl[i + 1]) < 1e-7 * sc, (row, i)


def test_q_cells_meet_hermite_conditions_within_subgrids(oracle_mod, synth):
    """Same in the Q direction; tangents never reach across a subgrid boundary,
    and a two-knot subgrid is linear in ln Q^2."""
    r = rng(13)
    x = rand_knots(r, 1e-4, 1.0, 5)
    subs = rand_subgrids(r, [1.0, 3.0, 7.0, 400.0], [4, 2, 5])
    q2 = np.concatenate(subs)
    vals = r.standard_normal((q2.shape[0], 5, 1))
    vals[4, :, :] = vals[3, :, :]  # continuous at the thresholds
    vals[6, :, :] = vals[5, :, :]
    g = mk(synth, x, subs, lambda xk, q: vals, 1)
    og = oracle_mod.OracleGrid(g)
    lq = np.log(q2)
    starts = [0, 4, 6]
    for col in range(5):
        for s, j0 in enumerate(starts):
            n = len(subs[s])
            ls, fs = lq[j0:j0 + n], vals[j0:j0 + n, col, 0]
            sl = _expected_slopes(ls, fs)
            for j in range(n - 1):
                d = ls[j + 1] - ls[j]
                ts = np.linspace(0.0, 1.0, 9)
                qs = np.exp(ls[j] + ts * d)
                qs[0], qs[-1] = q2[j0 + j], q2[j0 + j + 1]
                # the upper end of a lower subgrid is evaluated just below it
                if j == n - 2 and s < 2:
                    qs[-1] = np.nextafter(q2[j0 + j + 1], 0)
                v, _, _ = og.xfxq2(np.full(9, x[col]), qs)
                p = _fit_cubic(ts, v[:, 0])
                dp = p.deriv()
                sc = np.abs(fs).max()
                assert abs(dp(0) - d * sl[j]) < 1e-6 * sc, (col, s, j)
                assert abs(dp(1) - d * sl[j + 1]) < 1e-6 * sc, (col, s, j)
                if n == 2:
                    assert abs(p.coef[2]) < 1e-7 * sc and abs(p.coef[3]) < 1e-7 * sc


# ---------------------------------------------------------------------------
# polynomial classes reproduced exactly
# ---------------------------------------------------------------------------

def test_bilinear_in_logs_is_exact(oracle_mod, synth):
    r = rng(14)
    x = rand_knots(r, 1e-6, 1.0, 9)
    subs = rand_subgrids(r, [1.5, 4.0, 30.0, 1e4], [3, 2, 6])
    coef = r.uniform(-2, 2, (4, 3))

    def fn(xk, q2):
        lx, lq = np.log(xk)[None, :, None], np.log(q2)[:, None, None]
        return (coef[0] + coef[1] * lx) * (coef[2] + coef[3] * lq)

    g = mk(synth, x, subs, fn, 3)
    og = oracle_mod.OracleGrid(g)
    xs, qs = synth.ingrid_samples(g, 3000, 15)
    v, s, _ = og.xfxq2(xs, qs)
    want = fn(xs, qs)  # shape (n, n, 3) would be wrong: evaluate pointwise
    lx, lq = np.log(xs)[:, None], np.log(qs)[:, None]
    want = (coef[0] + coef[1] * lx) * (coef[2] + coef[3] * lq)
    assert scale_ok(v, want, s, 1e-13).all()


def test_quadratics_exact_in_interior_cells_of_uniform_grids(oracle_mod, synth):
    L = np.linspace(np.log(1e-4), 0.0, 9)
    x = np.exp(L)
    x[-1] = 1.0
    LQ = [np.linspace(0.0, 2.0, 6), np.linspace(2.0, 5.0, 7)]
    subs = [np.exp(l) for l in LQ]
    subs[1][0] = subs[0][-1]
    a, b, c = 0.7, -0.3, 0.11

    g = mk(synth, x, subs, lambda xk, q2: (a + b * np.log(xk) + c * np.log(xk) ** 2)[None, :, None]
           * np.ones((q2.shape[0], 1, 1)), 1)
    og = oracle_mod.OracleGrid(g)
    lx = np.log(x)
    for i in range(8):
        ts = np.array([0.13, 0.5, 0.77])
        xs = np.exp(lx[i] + ts * (lx[i + 1] - lx[i]))
        v, s, _ = og.xfxq2(xs, np.full(3, 3.0))
        want = a + b * np.log(xs) + c * np.log(xs) ** 2
        err = np.abs(v[:, 0] - want).max()
        if 1 <= i <= 6:
            assert err < 1e-12, i
        else:  # one-sided tangent at the grid edge: not exact for a quadratic
            assert err > 1e-4, i

    g = mk(synth, x, subs, lambda xk, q2: (a + b * np.log(q2) + c * np.log(q2) ** 2)[:, None, None]
           * np.ones((1, xk.shape[0], 1)), 1)
    og = oracle_mod.OracleGrid(g)
    for s_, l in enumerate(LQ):
        for j in range(len(l) - 1):
            us = np.array([0.21, 0.6, 0.9])
            qs = np.exp(l[j] + us * (l[j + 1] - l[j]))
            v, _, _ = og.xfxq2(np.full(3, 0.01), qs)
            want = a + b * np.log(qs) + c * np.log(qs) ** 2
            err = np.abs(v[:, 0] - want).max()
            if 1 <= j <= len(l) - 3:
                assert err < 1e-12, (s_, j)
            else:
                assert err > 1e-4, (s_, j)


# ---------------------------------------------------------------------------
# exact-rational brute force, Q direction first
# ---------------------------------------------------------------------------

def _frac_hermite(t, f0, f1, m0, m1):
    h00 = 2 * t**3 - 3 * t**2 + 1
    h01 = -2 * t**3 + 3 * t**2
    h10 = t**3 - 2 * t**2 + t
    h11 = t**3 - t**2
    return h00 * f0 + h01 * f1 + h10 * m0 + h11 * m1


def _frac_1d(l, f, k, t):
    """Hermite on cell k of the sequence (l, f) with R-slope tangents, exact."""
    n = len(l)

    def slope(m):
        if m == 0:
            return (f[1] - f[0]) / (l[1] - l[0])
        if m == n - 1:
            return (f[n - 1] - f[n - 2]) / (l[n - 1] - l[n - 2])
        return ((f[m + 1] - f[m]) / (l[m + 1] - l[m]) + (f[m] - f[m - 1]) / (l[m] - l[m - 1])) / 2

    d = l[k + 1] - l[k]
    return _frac_hermite(t, f[k], f[k + 1], d * slope(k), d * slope(k + 1))


def _frac_eval(g, x, q2, col):
    """Exact-rational log-bicubic value: interpolate every x column in Q
    (within the subgrid that holds Q^2), then interpolate those in x."""
    xk, q2k = list(g.x_knots), list(g.q2_knots)
    lxk = [Fraction(math.log(v)) for v in xk]
    lqk = [Fraction(math.log(v)) for v in q2k]
    i = max(k for k in range(len(xk) - 1) if xk[k] <= x)
    starts = np.cumsum([0] + list(g.nq))[:-1]
    s = max(k for k in range(len(starts)) if q2k[starts[k]] <= q2)
    j0, n = int(starts[s]), g.nq[s]
    ls = lqk[j0:j0 + n]
    jl = max(k for k in range(n - 1) if q2k[j0 + k] <= q2)
    u = (Fraction(math.log(q2)) - ls[jl]) / (ls[jl + 1] - ls[jl])
    cols = [_frac_1d(ls, [Fraction(float(g.values[j0 + k, a, col])) for k in range(n)], jl, u)
            for a in range(len(xk))]
    t = (Fraction(math.log(x)) - lxk[i]) / (lxk[i + 1] - lxk[i])
    return _frac_1d(lxk, cols, i, t)


@pytest.mark.parametrize("shape", [(4, [4]), (5, [3, 4]), (2, [2]), (3, [2, 3, 2]), (6, [5, 2])])
def test_matches_exact_rational_q_first(oracle_mod, synth, shape):
    nx, nq = shape
    r = rng(100 + nx * 7 + len(nq))
    x = rand_knots(r, 1e-3, 1.0, nx)
    bounds = np.exp(np.sort(r.uniform(0.0, 6.0, len(nq) + 1)))
    subs = rand_subgrids(r, bounds, nq)
    rows = sum(nq)
    vals = r.standard_normal((rows, nx, 2))
    g = mk(synth, x, subs, lambda xk, q: vals, 2)
    og = oracle_mod.OracleGrid(g)
    xs, qs = synth.ingrid_samples(g, 60, 16 + nx)
    xs = np.concatenate([xs, x, np.full(len(g.q2_knots), x[0])])
    qs = np.concatenate([qs, np.full(nx, g.q2_knots[0]), g.q2_knots])
    v, s, _ = og.xfxq2(xs, qs)
    for p in range(len(xs)):
        for col in range(2):
            want = float(_frac_eval(g, xs[p], qs[p], col))
            assert abs(v[p, col] - want) <= 1e-13 * max(abs(want), s[p, col]), (p, col)


# ---------------------------------------------------------------------------
# continuity and smoothness
# ---------------------------------------------------------------------------

def test_continuous_across_subgrid_boundaries(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    xs = np.exp(rng(17).uniform(np.log(1e-9), 0.0, 16))
    for b in (synth.Q_THRESHOLDS[0] ** 2, synth.Q_THRESHOLDS[1] ** 2):
        diffs = []
        for d in (1e-3, 1e-5, 1e-7):
            hi, s, _ = og.xfxq2(xs, np.full(16, b * (1 + d)))
            lo, _, _ = og.xfxq2(xs, np.full(16, b * (1 - d)))
            diffs.append(np.abs(hi - lo) / s)
        assert (diffs[2] < 1e-4).all()
        assert (diffs[2] <= 1e-2 * diffs[0] + 1e-12).all()  # shrinks ~linearly


def test_c1_at_interior_knots(oracle_mod, synth):
    g = synth.grid_single_subgrid()
    og = oracle_mod.OracleGrid(g)
    lx, lq = np.log(g.x_knots), np.log(g.q2_knots)
    h = 1e-5
    for i in (3, 17, 30):
        for j in (5, 20):
            q = np.full(3, g.q2_knots[j] * 1.37)
            xs = np.exp(lx[i] + np.array([-h, 0.0, h]))
            v, s, _ = og.xfxq2(xs, q)
            dl, dr = (v[1] - v[0]) / h, (v[2] - v[1]) / h
            assert (np.abs(dr - dl) < 1e-2 * (np.abs(dr) + np.abs(dl)) + 1e-6 * s[1]).all()
            qs = np.exp(lq[j] + np.array([-h, 0.0, h]))
            v, s, _ = og.xfxq2(np.full(3, g.x_knots[i] * 1.21), qs)
            dl, dr = (v[1] - v[0]) / h, (v[2] - v[1]) / h
            assert (np.abs(dr - dl) < 1e-2 * (np.abs(dr) + np.abs(dl)) + 1e-6 * s[1]).all()


# ---------------------------------------------------------------------------
# extrapolation identities
# ---------------------------------------------------------------------------

def test_extrapolation_is_continuous_at_the_grid_edges(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    x0, q2min, q2max = g.x_knots[0], g.q2_knots[0], g.q2_knots[-1]
    qs = np.exp(rng(18).uniform(np.log(q2min), np.log(q2max), 8))
    xs = np.exp(rng(19).uniform(np.log(x0), 0.0, 8))
    d = 1e-9
    for xa, xb, qa, qb in [
        (np.full(8, x0 * (1 - d)), np.full(8, x0), qs, qs),
        (xs, xs, np.full(8, q2min * (1 - d)), np.full(8, q2min)),
        (xs, xs, np.full(8, q2max * (1 + d)), np.full(8, q2max)),
        (np.full(8, x0 * (1 - d)), np.full(8, x0), np.full(8, q2min * (1 - d)), np.full(8, q2min)),
        (np.full(8, x0 * (1 - d)), np.full(8, x0), np.full(8, q2max * (1 + d)), np.full(8, q2max)),
    ]:
        va, s, _ = og.xfxq2(xa, qa)
        vb, _, _ = og.xfxq2(xb, qb)
        assert (np.abs(va - vb) < 1e-6 * s).all()


def test_low_x_reproduces_power_laws(oracle_mod, synth):
    x = synth.geom_knots(1e-5, 1.0, 12)
    subs = [synth.geom_knots(2.0, 1e4, 9)]
    A, a = np.array([0.5, 2.0]), np.array([-0.25, 0.4])

    def fn(xk, q2):
        return A * xk[None, :, None] ** a * (3.0 + 0.2 * np.log(q2))[:, None, None]

    og = oracle_mod.OracleGrid(mk(synth, x, subs, fn, 2))
    xs = np.array([1e-6, 3e-8, 1e-10, 5e-6])
    qs = np.array([2.0, 17.0, 333.0, 1e4])
    v, _, _ = og.xfxq2(xs, qs)
    want = A * xs[:, None] ** a * (3.0 + 0.2 * np.log(qs))[:, None]
    assert np.allclose(v, want, rtol=1e-12, atol=0)


def test_high_q2_reproduces_power_laws(oracle_mod, synth):
    x = synth.geom_knots(1e-5, 1.0, 7)
    subs = [synth.geom_knots(2.0, 50.0, 4), synth.geom_knots(50.0, 1e4, 6)]
    k = np.array([0.3, -0.2])

    def fn(xk, q2):
        return (2.0 + 0.1 * np.log(xk))[None, :, None] ** 2 * 0 + (2.0 - 0.1 * np.log(xk))[None, :, None] \
            * q2[:, None, None] ** k

    og = oracle_mod.OracleGrid(mk(synth, x, subs, fn, 2))
    xs = np.array([1e-5, 0.3, 0.9])
    qs = np.array([2e4, 1e6, 1e9])
    v, _, _ = og.xfxq2(xs, qs)
    want = (2.0 - 0.1 * np.log(xs))[:, None] * qs[:, None] ** k
    assert np.allclose(v, want, rtol=1e-12, atol=0)


def test_negative_values_continue_linearly(oracle_mod, synth):
    x = synth.geom_knots(1e-4, 1.0, 6)
    subs = [synth.geom_knots(2.0, 1e3, 5)]
    og = oracle_mod.OracleGrid(mk(synth, x, subs, lambda xk, q2: -np.ones((5, 6, 1))
                                  - 0.3 * np.log(xk)[None, :, None] ** 2 * np.ones((5, 1, 1)), 1))
    q = np.full(3, 20.0)
    lxs = np.log(1e-4) - np.array([1.0, 2.0, 3.0])
    v, _, _ = og.xfxq2(np.exp(lxs), q)
    # collinear in ln x
    assert abs((v[2, 0] - v[1, 0]) - (v[1, 0] - v[0, 0])) < 1e-12 * np.abs(v).max()
    # high Q^2 with negative values: linear in ln Q^2
    lqs = np.log(1e3) + np.array([1.0, 2.0, 3.0])
    v, _, _ = og.xfxq2(np.full(3, 0.01), np.exp(lqs))
    assert abs((v[2, 0] - v[1, 0]) - (v[1, 0] - v[0, 0])) < 1e-12 * np.abs(v).max()
    # low Q^2 with negative values: gamma = 1, so xf = f0 Q^2 / Q2min
    f0, _, _ = og.xfxq2(np.full(3, 0.01), np.full(3, 2.0))
    qs = np.array([1.5, 0.2, 1e-3])
    v, _, _ = og.xfxq2(np.full(3, 0.01), qs)
    assert np.allclose(v[:, 0], f0[:, 0] * qs / 2.0, rtol=1e-14, atol=0)


def test_low_q2_continuation_slope_and_limit(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    q2min = g.q2_knots[0]
    xs = np.array([1e-6, 1e-3, 0.1, 0.5])
    f0, _, _ = og.xfxq2(xs, np.full(4, q2min))
    f1, _, _ = og.xfxq2(xs, np.full(4, 1.01 * q2min))
    pos = (f0 > 0) & (f1 > 0)
    gam = np.where(pos, np.log(np.where(pos, f1 / f0, 1.0)) / math.log(1.01), 1.0)
    h = 1e-6
    vlo, _, _ = og.xfxq2(xs, np.full(4, q2min * math.exp(-h)))
    slope = (np.log(np.abs(f0)) - np.log(np.abs(vlo))) / h
    assert np.allclose(slope, gam, rtol=1e-4, atol=1e-4)
    vz, _, _ = og.xfxq2(xs, np.full(4, q2min * 1e-12))
    assert (np.abs(vz) <= 1e-10 * np.abs(f0)).all()


# ---------------------------------------------------------------------------
# alpha_s
# ---------------------------------------------------------------------------

def test_alphas_nodes_constant_ends_and_linear_exactness(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    v, _ = og.alphas(g.as_q2)
    assert np.array_equal(v, g.as_vals)
    v, _ = og.alphas([1e-6, g.as_q2[0] * 0.999, g.as_q2[-1] * 1.001, 1e30])
    assert np.array_equal(v, [g.as_vals[0]] * 2 + [g.as_vals[-1]] * 2)
    # nodes linear in ln Q^2 (with a threshold jump) are reproduced exactly
    q = np.array([1.0, 2.0, 5.0, 5.0, 9.0, 40.0, 100.0])
    av = np.where(np.arange(7) < 3, 0.3 - 0.01 * np.log(q), 0.25 - 0.02 * np.log(q))
    og2 = oracle_mod.OracleGrid(x_knots=[1e-3, 1.0], nq=[2], q2_knots=[1.0, 100.0],
                                values=np.ones((2, 2, 1)), as_q2=q, as_vals=av)
    qs = np.exp(rng(20).uniform(0.0, np.log(100.0), 200))
    v, _ = og2.alphas(qs)
    want = np.where(qs < 5.0, 0.3 - 0.01 * np.log(qs), 0.25 - 0.02 * np.log(qs))
    assert np.allclose(v, want, rtol=1e-13, atol=0)
    v, _ = og2.alphas([5.0])
    assert v[0] == av[3]  # the repeated node belongs to the upper subgrid


def test_alphas_tangent_conditions(oracle_mod):
    r = rng(21)
    q = np.array([1.0, 2.0, 3.5, 7.0, 7.0, 12.0, 30.0, 31.0, 90.0])
    av = r.uniform(0.1, 0.3, 9)
    og = oracle_mod.OracleGrid(x_knots=[1e-3, 1.0], nq=[2], q2_knots=[1.0, 90.0],
                               values=np.ones((2, 2, 1)), as_q2=q, as_vals=av)
    lq = np.log(q)
    for a0, a1 in [(0, 3), (4, 8)]:
        sl = _expected_slopes(lq[a0:a1 + 1], av[a0:a1 + 1])
        for j in range(a1 - a0):
            d = lq[a0 + j + 1] - lq[a0 + j]
            ts = np.linspace(0, 1, 9)
            qs = np.exp(lq[a0 + j] + ts * d)
            qs[0] = q[a0 + j]
            qs[-1] = np.nextafter(q[a0 + j + 1], 0) if a0 + j + 1 == 3 else q[a0 + j + 1]
            v, _ = og.alphas(qs)
            p = _fit_cubic(ts, v)
            assert abs(p.deriv()(0) - d * sl[j]) < 1e-7
            assert abs(p.deriv()(1) - d * sl[j + 1]) < 1e-7


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

def test_knot_gradient_partition_of_unity_and_linearity(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    xs, qs = synth.ingrid_samples(g, 40, 22)
    v, _, _ = og.xfxq2(xs, qs)
    for p in range(40):
        f = p % g.nflav
        cot = np.zeros((1, g.nflav))
        cot[0, f] = 1.0
        G = og.knot_grad(xs[p:p + 1], qs[p:p + 1], cot)
        assert abs(G.sum() - 1.0) < 1e-12  # constants are reproduced
        assert abs((G * g.values).sum() - v[p, f]) < 1e-12 * np.abs(G * g.values).sum()
        assert np.count_nonzero(G) <= 16


def test_knot_gradient_outside_grid_matches_finite_differences(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    pts = [(3e-10, 50.0), (0.01, 3e10), (0.2, 0.5), (2e-10, 2e10), (5e-10, 0.3)]
    for (x, q2) in pts:
        for f in (0, 6, 12):
            cot = np.zeros((1, g.nflav))
            cot[0, f] = 1.0
            G = og.knot_grad([x], [q2], cot)
            nz = np.argwhere(G != 0)
            assert len(nz) > 0
            for (row, ix, col) in nz[:: max(1, len(nz) // 6)]:
                h = 1e-7 * abs(g.values[row, ix, col])  # small against the value: no branch flip
                vals = g.values.copy()
                vals[row, ix, col] += h
                vp = oracle_mod.OracleGrid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots,
                                           values=vals).xfxq2([x], [q2], cols=[f])[0][0, 0]
                vals[row, ix, col] -= 2 * h
                vm = oracle_mod.OracleGrid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots,
                                           values=vals).xfxq2([x], [q2], cols=[f])[0][0, 0]
                fd = (vp - vm) / (2 * h)
                assert abs(fd - G[row, ix, col]) <= 1e-6 * max(1.0, abs(fd)), (x, q2, f, row, ix)


def test_x_and_q2_derivatives_match_finite_differences(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    xs, qs = synth.queries_full(300, 23)
    v, s, _ = og.xfxq2(xs, qs)
    for wrt, arr in (("x", xs), ("q2", qs)):
        d = og.dxfxq2(xs, qs, wrt)
        h = 1e-6 * arr
        a_p, a_m = arr + h, arr - h
        args_p = (a_p, qs) if wrt == "x" else (xs, a_p)
        args_m = (a_m, qs) if wrt == "x" else (xs, a_m)
        vp, _, _ = og.xfxq2(*args_p)
        vm, _, _ = og.xfxq2(*args_m)
        fd = (vp - vm) / (2 * h)[:, None]
        # skip points whose stencil crosses a knot, an edge or a threshold within h
        knots = g.x_knots if wrt == "x" else np.concatenate([g.q2_knots, [g.q2_knots[0] * 1.01]])
        near = np.min(np.abs(np.log(arr)[:, None] - np.log(knots)[None, :]), axis=1) < 2e-6
        ok = np.isfinite(fd) & ~near[:, None] & np.isfinite(d)
        err = np.abs(fd - d) / (np.abs(d) + s / arr[:, None])
        assert ok.mean() > 0.95
        assert (err[ok] < 1e-5).all(), wrt


def test_relative_precision_next_to_a_vanishing_knot(oracle_mod, synth):
    """R-ends: within rounding distance of a knot where xf vanishes (x -> 1,
    xf ~ (1 - x)^b) the value keeps its relative precision: it matches the
    exact-rational evaluation relative to |xf| itself, not only to the data
    mass."""
    x = synth.geom_knots(1e-3, 1.0, 6)
    subs = [synth.geom_knots(2.0, 100.0, 5)]
    g = mk(synth, x, subs, lambda xk, q2: ((1.0 - xk) ** 3)[None, :, None] * (1.0 + 0.1 * np.log(q2))[:, None, None], 1)
    og = oracle_mod.OracleGrid(g)
    xs = np.array([np.nextafter(1.0, 0), 1.0 - 1e-12, 1.0 - 1e-9, np.nextafter(x[2], 0)])
    qs = np.array([7.0, 13.0, np.nextafter(100.0, 0), 3.0])
    v, _, _ = og.xfxq2(xs, qs)
    for p in range(len(xs)):
        want = float(_frac_eval(g, xs[p], qs[p], 0))
        assert want != 0.0
        assert abs(v[p, 0] - want) <= 1e-12 * abs(want), (p, v[p, 0], want)
