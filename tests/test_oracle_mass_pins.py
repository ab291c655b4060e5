"""Pins for the oracle's data mass s, the scale of every parity bound
(|gpu - oracle| <= rtol * max(|oracle|, s)).

s is first-order propagation of the data's absolute size through the same
expression that gives the value: a datum contributes |f|, a + b and a - b
give s_a + s_b, a b gives |b| s_a + |a| s_b, a / b gives (s_a + |a/b| s_b)/|b|,
ln a gives s_a / |a| and e^a gives e^a s_a.  For an in-grid point that is
sum_ab P_ab |f_ab|, with P_ab the sum over the expression's paths from knot
(a, b) of the magnitudes of their coefficients; so P_ab >= |d xf / d f_ab|.

Each test checks s against a value derived by hand from the method's
definition (PDFFlow Sec. 2.2: cubic Hermite segments with finite-difference
tangents; the continuation rules of the EXTRAPOLATE box of Fig. 1; Sec. 2.3
for alpha_s), not against the oracle's own arithmetic:

* a grid of constant value C: the secant slopes vanish, the Hermite weights
  of the two knot values sum to one, and the tangent terms carry the mass
  2|C|/d of each secant, so with h10 = t(1-t)^2, -h11 = t^2(1-t),
      s = |C| R_x(t) R_q(u),  R(t) = 1 + a0 t(1-t)^2 + a1 t^2(1-t),
  a0 = 1 + d_i/d_(i-1) at an interior left knot (2 at the first knot of the
  x grid or of a Q subgrid), a1 likewise on the right;
* the log-linear pair rule v = g0 (g1/g0)^p from values at knots (s = |g|
  there) has s = |v| (1 + 2|p|); the linear branch |g0| + |p| (|g0| + |g1|);
* the low-Q^2 rule on a grid constant in Q^2 (gamma = 0, v = f0 rho^(1-rho))
  has s = |v| (1 + rho |ln rho| (1 + R_q(u1)) / ln 1.01), u1 the position of
  1.01 Q2min in the first Q cell;
* bounds on any grid: sum_ab |W_ab f_ab| <= s (W from the forward-mode knot
  derivative), and min |f| s_1 <= s <= max |f| s_1 over the knots read,
  s_1 the constant-grid value for C = 1.

A mutation that scales s, drops a tangent term or takes the wrong neighbour
spacing fails one of them.
"""
import math

import numpy as np

from conftest import rng


def _grid(synth, xk, subs, fn, nflav=1):
    return synth.make_grid(xk, subs, list(range(nflav)), values_fn=fn)


def _rand_knots(r, lo, hi, n):
    inner = np.sort(r.uniform(math.log(lo), math.log(hi), n - 2))
    k = np.exp(np.concatenate([[math.log(lo)], inner, [math.log(hi)]]))
    k[0], k[-1] = lo, hi
    return k


def _factor(l, i, t, first, last):
    """R(t) for cell i of knots l[first..last] (ln values); first/last bound the
    stencil (the x grid, or one Q subgrid)."""
    d = l[i + 1] - l[i]
    a0 = 2.0 if i == first else 1.0 + d / (l[i] - l[i - 1])
    a1 = 2.0 if i + 1 == last else 1.0 + d / (l[i + 2] - l[i + 1])
    tm = 1.0 - t
    return 1.0 + a0 * t * tm * tm + a1 * t * t * tm


def _cell(knots, v):
    """Cell index i with knots[i] <= v < knots[i+1] (last cell closed)."""
    i = int(np.searchsorted(knots, v, side="right")) - 1
    return min(max(i, 0), len(knots) - 2)


def _constant_mass(g, x, q2):
    """|C| = 1 mass of the in-grid point (x, q2), from the definition."""
    lx = np.log(g.x_knots)
    i = _cell(g.x_knots, x)
    t = (math.log(x) - lx[i]) / (lx[i + 1] - lx[i])
    rx = _factor(lx, i, t, 0, g.nx - 1)
    starts = np.concatenate([[0], np.cumsum(g.nq)[:-1]])
    s = int(np.searchsorted(g.q2_knots[starts], q2, side="right")) - 1  # the upper subgrid on a threshold
    j0, j1 = int(starts[s]), int(starts[s] + g.nq[s] - 1)
    lq = np.log(g.q2_knots)
    j = j0 + _cell(g.q2_knots[j0:j1 + 1], q2)
    u = (math.log(q2) - lq[j]) / (lq[j + 1] - lq[j])
    return rx * _factor(lq, j, u, j0, j1)


def _inside_points(r, g, n):
    lx = r.uniform(math.log(g.x_knots[0]), math.log(g.x_knots[-1]), n)
    lq = r.uniform(math.log(g.q2_knots[0]), math.log(g.q2_knots[-1]), n)
    return np.exp(lx), np.exp(lq)


def test_constant_grid_mass_matches_closed_form(oracle_mod, synth):
    r = rng(101)
    for trial in range(4):
        xk = _rand_knots(r, 1e-6, 1.0, 7 + trial)
        b = [2.0, 9.0, 40.0, 3e3]
        subs = [_rand_knots(r, b[0], b[1], 2 + trial), _rand_knots(r, b[1], b[2], 3), _rand_knots(r, b[2], b[3], 6)]
        c = (-1.0) ** trial * r.uniform(0.5, 4.0)
        g = _grid(synth, xk, subs, lambda xx, qq: np.full((qq.shape[0], xx.shape[0], 1), c))
        og = oracle_mod.OracleGrid(g)
        x, q2 = _inside_points(r, g, 400)
        # knots, thresholds and the last knots too
        x = np.concatenate([x, xk, np.full(4, xk[3])])
        q2 = np.concatenate([q2, np.full(len(xk), g.q2_knots[5]), [b[1], b[2], b[3], b[0]]])
        v, s, fl = og.xfxq2(x, q2)
        want = np.array([abs(c) * _constant_mass(g, a, q) for a, q in zip(x, q2)])
        assert not fl.any()
        np.testing.assert_allclose(v[:, 0], c, rtol=1e-14)
        np.testing.assert_allclose(s[:, 0], want, rtol=1e-13)
    # the mass is above |C| strictly inside a cell and equal to it on a knot
    assert (want >= abs(c) * (1 - 1e-15)).all() and want.max() > 1.2 * abs(c)


def test_in_grid_mass_depends_only_on_magnitudes(oracle_mod, synth):
    g = synth.grid_full()
    r = rng(102)
    signs = np.where(r.random(g.values.shape) < 0.5, -1.0, 1.0)
    og = oracle_mod.OracleGrid(g)
    og_abs = oracle_mod.OracleGrid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots, values=np.abs(g.values))
    og_sgn = oracle_mod.OracleGrid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots, values=signs * g.values)
    x, q2 = _inside_points(r, g, 2000)
    _, s, _ = og.xfxq2(x, q2)
    _, s_abs, _ = og_abs.xfxq2(x, q2)
    _, s_sgn, _ = og_sgn.xfxq2(x, q2)
    assert np.array_equal(s, s_abs) and np.array_equal(s, s_sgn)
    # homogeneous of degree one in |f|
    og3 = oracle_mod.OracleGrid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots, values=-3.0 * g.values)
    _, s3, _ = og3.xfxq2(x, q2)
    np.testing.assert_allclose(s3, 3.0 * s, rtol=1e-15)


def test_mass_bounds_on_a_general_grid(oracle_mod, synth):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    r = rng(103)
    x, q2 = _inside_points(r, g, 60)
    v, s, _ = og.xfxq2(x, q2)
    for p in range(len(x)):
        s1 = _constant_mass(g, x[p], q2[p])
        for f in (0, 6, 12):
            cot = np.zeros((1, g.nflav))
            cot[0, f] = 1.0
            W = og.knot_grad(x[p:p + 1], q2[p:p + 1], cot)[:, :, f]  # d xf_f / d f_ab
            lower = float(np.abs(W * g.values[:, :, f]).sum())
            knots = og.knots_read(x[p], q2[p], f)
            mags = np.array([abs(g.values[a, b, f]) for a, b in knots])
            assert 8 <= len(knots) <= 16  # 4 x 4, fewer rows or columns at edges
            assert lower <= s[p, f] * (1 + 1e-13)
            assert abs(v[p, f]) <= s[p, f] * (1 + 1e-15)
            assert mags.min() * s1 * (1 - 1e-13) <= s[p, f] <= mags.max() * s1 * (1 + 1e-13)


def _power_law(xk, q2k, A=2.0, a=-0.3, c=0.4):
    """A x^a (Q^2)^c: positive everywhere."""
    return A * xk[None, :, None] ** a * q2k[:, None, None] ** c


def test_pair_rule_mass_at_knot_sites(oracle_mod, synth):
    r = rng(104)
    xk = _rand_knots(r, 1e-5, 1.0, 9)
    subs = [_rand_knots(r, 2.0, 30.0, 5), _rand_knots(r, 30.0, 1e4, 6)]
    g = _grid(synth, xk, subs, lambda xx, qq: _power_law(xx, qq))
    og = oracle_mod.OracleGrid(g)
    lx, lq = np.log(xk), np.log(g.q2_knots)
    n = g.nrows - 1
    # low x at every Q knot
    x = np.exp(r.uniform(math.log(1e-12), math.log(xk[0]) - 1e-3, 30))
    for q in g.q2_knots:
        v, s, _ = og.xfxq2(x, np.full(x.shape, q))
        p = (np.log(x) - lx[0]) / (lx[1] - lx[0])
        np.testing.assert_allclose(s[:, 0], np.abs(v[:, 0]) * (1 + 2 * np.abs(p)), rtol=1e-13)
    # high Q^2 at every x knot
    q2 = np.exp(r.uniform(lq[-1] + 1e-3, lq[-1] + 8.0, 30))
    pq = (np.log(q2) - lq[n]) / (lq[n - 1] - lq[n])
    for xv in xk:
        v, s, _ = og.xfxq2(np.full(q2.shape, xv), q2)
        np.testing.assert_allclose(s[:, 0], np.abs(v[:, 0]) * (1 + 2 * np.abs(pq)), rtol=1e-13)
    # the corner: the Q rule at both x sites, then the x rule
    v, s, _ = og.xfxq2(x, q2)
    px = (np.log(x) - lx[0]) / (lx[1] - lx[0])
    np.testing.assert_allclose(s[:, 0], np.abs(v[:, 0]) * (1 + 2 * np.abs(px)) * (1 + 2 * np.abs(pq)), rtol=1e-13)


def test_linear_branch_mass(oracle_mod, synth):
    xk = synth.geom_knots(1e-4, 1.0, 8)
    subs = [synth.geom_knots(2.0, 1e3, 6)]

    def fn(xx, qq):  # negative at the lowest x knot, positive at the next
        v = np.ones((qq.shape[0], xx.shape[0], 1))
        v[:, 0, 0] = -0.5 - 0.1 * np.log(qq)
        v[:, 1:, 0] = 1.5 + 0.2 * np.log(qq)[:, None]
        return v

    g = _grid(synth, xk, subs, fn)
    og = oracle_mod.OracleGrid(g)
    x = np.geomspace(1e-9, 0.9e-4, 20)
    for j, q in enumerate(g.q2_knots):
        v, s, _ = og.xfxq2(x, np.full(x.shape, q))
        g0, g1 = g.values[j, 0, 0], g.values[j, 1, 0]
        p = (np.log(x) - math.log(xk[0])) / (math.log(xk[1]) - math.log(xk[0]))
        np.testing.assert_allclose(v[:, 0], g0 + (g1 - g0) * p, rtol=1e-13)
        np.testing.assert_allclose(s[:, 0], abs(g0) + np.abs(p) * (abs(g0) + abs(g1)), rtol=1e-13)


def test_low_q2_rule_mass(oracle_mod, synth):
    r = rng(105)
    xk = _rand_knots(r, 1e-5, 1.0, 8)
    qk = _rand_knots(r, 2.0, 500.0, 6)
    g = _grid(synth, xk, [qk], lambda xx, qq: np.broadcast_to(1.0 + xx[None, :, None] ** -0.2,
                                                              (qq.shape[0], xx.shape[0], 1)).copy())
    og = oracle_mod.OracleGrid(g)
    lq = np.log(qk)
    u1 = math.log(1.01) / (lq[1] - lq[0])
    rq = _factor(lq, 0, u1, 0, len(qk) - 1)
    rho = np.exp(r.uniform(math.log(1e-6), -1e-3, 40))
    for xv in xk:
        v, s, fl = og.xfxq2(np.full(rho.shape, xv), rho * qk[0])
        f0 = 1.0 + xv**-0.2
        np.testing.assert_allclose(v[:, 0], f0 * rho ** (1.0 - rho), rtol=1e-12)
        want = np.abs(v[:, 0]) * (1 + rho * np.abs(np.log(rho)) * (1 + rq) / math.log(1.01))
        np.testing.assert_allclose(s[:, 0], want, rtol=1e-12)


def test_mass_at_least_value_everywhere(oracle_mod, synth):
    """s >= |v| on the benchmark's own query law and the special points."""
    import parity

    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    x, q2 = synth.queries_full(20_000, 3)
    xs, qs = parity.special_points(g)
    v, s, _ = og.xfxq2(np.concatenate([x, xs]), np.concatenate([q2, qs]))
    ok = ~np.isnan(v)
    assert (np.abs(v[ok]) <= s[ok] * (1 + 1e-15)).all()
    # on the query law the mass is a modest multiple of |v| away from zero crossings
    ratio = s[: len(x)] / np.maximum(np.abs(v[: len(x)]), 1e-300)
    assert np.median(ratio) < 2.5


def test_alphas_mass_constant_nodes(oracle_mod, synth):
    r = rng(106)
    q = _rand_knots(r, 2.0, 1e4, 9)
    q = np.concatenate([q[:4], q[3:]])  # a repeated node splits two alpha_s subgrids
    c = 0.2
    og = oracle_mod.OracleGrid(x_knots=[1e-3, 1.0], nq=[2], q2_knots=[2.0, 1e4], values=np.ones((2, 2, 1)),
                               as_q2=q, as_vals=np.full(q.shape, c))
    l = np.log(q)
    pts = np.exp(r.uniform(l[0], l[-1], 300))
    v, s = og.alphas(pts)
    for k, p in enumerate(pts):
        sub = (0, 3) if p < q[4] else (4, len(q) - 1)
        j = sub[0] + _cell(q[sub[0]:sub[1] + 1], p)
        u = (math.log(p) - l[j]) / (l[j + 1] - l[j])
        assert abs(s[k] - c * _factor(l, j, u, sub[0], sub[1])) <= 1e-13 * c
    np.testing.assert_allclose(v, c, rtol=1e-14)
