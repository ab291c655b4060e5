"""GPU adjoint (vector-Jacobian product of xfxq2_all_flavours) against the
oracle's forward-mode gradients and against central finite differences, and
the torch.autograd.Function built on it.  Workload: points of the
three-subgrid query law with standard-normal cotangents (the adjoint config);
the paper has no counterpart."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def full(synth, oracle_mod):
    g = synth.grid_full()
    return g, P.pdf_load_grid(g), oracle_mod.OracleGrid(g)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_vjp(G, x, q2, cot, with_values=True):
    xd, qd, cd = dev(x), dev(q2), dev(cot)
    gx, gq = torch.empty_like(xd), torch.empty_like(qd)
    gv = torch.zeros((G.nrows, G.nx, G.nflav), dtype=torch.float64, device="cuda") if with_values else None
    P.xfxq2_all_flavours_vjp(G, xd, qd, cd, gx, gq, gv)
    torch.cuda.synchronize()
    return gx.cpu().numpy(), gq.cpu().numpy(), (gv.cpu().numpy() if with_values else None)


def min_log_spacing(k):
    d = np.diff(np.log(k))
    return d[d > 0].min()


def test_gradients_match_oracle(full, synth):
    g, G, og = full
    x, q2, cot = synth.adjoint_inputs(4000, g.nflav, 5, 6)
    gx, gq, gv = run_vjp(G, x, q2, cot)
    dx = og.dxfxq2(x, q2, "x")
    dq = og.dxfxq2(x, q2, "q2")
    v, s, fl = og.xfxq2(x, q2)
    ok = ~fl.any(axis=1)
    want_x = (cot * dx).sum(axis=1)
    want_q = (cot * dq).sum(axis=1)
    # scale: the terms of the sum, plus the data-mass scale of a derivative
    # in ln x (ln Q^2), s / (coordinate * smallest knot spacing)
    sx = np.abs(cot * dx).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (x * min_log_spacing(g.x_knots))
    sq = np.abs(cot * dq).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (q2 * min_log_spacing(g.q2_knots))
    ex = np.abs(gx - want_x) / sx
    eq = np.abs(gq - want_q) / sq
    assert ex[ok].max() < 1e-10, ex[ok].max()
    assert eq[ok].max() < 1e-10, eq[ok].max()
    go, gabs = og.knot_grad(x[ok], q2[ok], cot[ok], with_abs=True)
    gv_ok = run_vjp(G, x[ok], q2[ok], cot[ok])[2]
    err = np.abs(gv_ok - go)
    # where no evaluation touches a knot (gabs = 0) the GPU must add exactly nothing
    assert (err <= 1e-10 * gabs + 1e-300).all(), (err / np.maximum(gabs, 1e-300)).max()


def test_gradients_match_central_differences(full, synth):
    g, G, og = full
    x, q2, cot = synth.adjoint_inputs(3000, g.nflav, 15, 16)
    gx, gq, _ = run_vjp(G, x, q2, cot, with_values=False)
    h = 1e-6
    f = lambda a, b: P.xfxq2_all_flavours(G, dev(a), dev(b)).cpu().numpy()  # noqa: E731
    fdx = ((f(x * (1 + h), q2) - f(x * (1 - h), q2)) * cot).sum(axis=1) / (2 * h * x)
    fdq = ((f(x, q2 * (1 + h)) - f(x, q2 * (1 - h))) * cot).sum(axis=1) / (2 * h * q2)
    # skip points whose difference stencil straddles a knot, an edge, a threshold
    # or the 1.01 Q2min site (the interpolant is C1 inside a subgrid only)
    kx = np.log(g.x_knots)
    kq = np.log(np.concatenate([g.q2_knots, [1.01 * g.q2_knots[0]]]))
    far_x = np.min(np.abs(np.log(x)[:, None] - kx[None, :]), axis=1) > 3 * h
    far_q = np.min(np.abs(np.log(q2)[:, None] - kq[None, :]), axis=1) > 3 * h
    v, s, _ = og.xfxq2(x, q2)
    scale_x = np.abs(gx) + (np.abs(cot) * s).sum(axis=1) / x * 1e-3
    scale_q = np.abs(gq) + (np.abs(cot) * s).sum(axis=1) / q2 * 1e-3
    ok = far_x & far_q
    assert ok.mean() > 0.9
    assert (np.abs(fdx - gx)[ok] / scale_x[ok]).max() < 1e-4
    assert (np.abs(fdq - gq)[ok] / scale_q[ok]).max() < 1e-4


def test_invalid_points_give_nan_and_no_knot_gradient(full):
    g, G, og = full
    x = np.array([0.0, 0.5, -1.0, 0.3])
    q2 = np.array([10.0, -1.0, 10.0, 10.0])
    cot = np.ones((4, g.nflav))
    gx, gq, gv = run_vjp(G, x, q2, cot)
    assert np.isnan(gx[:3]).all() and np.isnan(gq[:3]).all()
    assert np.isfinite(gx[3]) and np.isfinite(gq[3])
    _, _, gv1 = run_vjp(G, x[3:], q2[3:], cot[3:])
    assert np.allclose(gv, gv1, rtol=1e-14, atol=0)


def test_autograd_function_and_value_restaging(full, synth):
    g, G, og = full
    x, q2 = synth.ingrid_samples(g, 2000, 17)
    cot = np.random.default_rng(18).standard_normal((2000, g.nflav))
    vals = torch.from_numpy(g.values).cuda().requires_grad_(True)
    xd = dev(x).requires_grad_(True)
    qd = dev(q2).requires_grad_(True)
    out = P.xfxq2_all_flavours_diff(G, xd, qd, vals)
    (out * dev(cot)).sum().backward()
    go = og.knot_grad(x, q2, cot)
    assert np.allclose(vals.grad.cpu().numpy(), go, rtol=1e-10, atol=1e-12 * np.abs(go).max())
    want_x = (cot * og.dxfxq2(x, q2, "x")).sum(axis=1)
    assert np.allclose(xd.grad.cpu().numpy(), want_x, rtol=1e-9, atol=1e-12 * np.abs(want_x).max())
    # staging new values reproduces a freshly loaded grid bit for bit
    new = g.values * 1.5 + 0.25
    P.pdf_grid_set_values(G, torch.from_numpy(new).cuda())
    fresh = P.pdf_load_grid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots, pids=g.pids, values=new,
                            as_q2=g.as_q2, as_vals=g.as_vals)
    a = P.xfxq2_all_flavours(G, dev(x), dev(q2)).cpu().numpy()
    b = P.xfxq2_all_flavours(fresh, dev(x), dev(q2)).cpu().numpy()
    assert np.array_equal(a, b)
    P.pdf_grid_set_values(G, torch.from_numpy(g.values).cuda())  # restore for other tests


def test_full_size_batch_in_the_benchmark_configuration(full, synth):
    """The benchmark's adjoint step (1e6 points, its seeds, one launch of the
    sorted path): continuation warps are of one kind and in-grid warps hold
    runs of one cell.  Per-point gradients are functions of the point alone,
    so a sample of them must match, bit for bit, the same points run as a
    smaller sorted batch (other neighbours, other runs), and the oracle on a
    subsample; the knot gradient must equal the sum of four quarter batches
    up to the rounding of the run contractions and the order of the FP64
    additions."""
    g, G, og = full
    n = 1_000_000
    x, q2, cot = synth.adjoint_inputs(n, g.nflav, 5, 6)
    gx, gq, gv = run_vjp(G, x, q2, cot)
    rng = np.random.default_rng(77)
    sub = np.sort(rng.choice(n, 20_000, replace=False))
    sx, sq, _ = run_vjp(G, x[sub], q2[sub], cot[sub])
    assert np.array_equal(gx[sub], sx, equal_nan=True) and np.array_equal(gq[sub], sq, equal_nan=True)
    few = sub[:1500]
    dx = og.dxfxq2(x[few], q2[few], "x")
    dq = og.dxfxq2(x[few], q2[few], "q2")
    v, s, fl = og.xfxq2(x[few], q2[few])
    ok = ~fl.any(axis=1)
    c = cot[few]
    sxs = np.abs(c * dx).sum(axis=1) + (np.abs(c) * s).sum(axis=1) / (x[few] * min_log_spacing(g.x_knots))
    sqs = np.abs(c * dq).sum(axis=1) + (np.abs(c) * s).sum(axis=1) / (q2[few] * min_log_spacing(g.q2_knots))
    assert (np.abs(gx[few] - (c * dx).sum(axis=1)) / sxs)[ok].max() < 1e-10
    assert (np.abs(gq[few] - (c * dq).sum(axis=1)) / sqs)[ok].max() < 1e-10
    parts = sum(run_vjp(G, x[k::4], q2[k::4], cot[k::4])[2] for k in range(4))
    scale = np.abs(gv).max(axis=(0, 1))  # per flavour
    assert (np.abs(gv - parts) / scale).max() < 1e-11


def test_sorted_batch_matches_oracle_and_small_batches(full, synth):
    """Batches of 2048 points or more are sorted by cell, and the knot-value
    terms of each warp's run of same-cell points are contracted in
    float-float before one atomic per knot and flavour; smaller batches
    scatter point by point.  Both are checked against the oracle's knot
    gradient, on a batch that also holds points on knots, on the last x knot,
    on the top and boundary Q^2 knots, in runs of one cell longer than a
    warp, and invalid and continuation points."""
    g, G, og = full
    n = 24000
    x, q2, cot = synth.adjoint_inputs(n, g.nflav, 25, 26)
    rng = np.random.default_rng(27)
    k = 0
    for xi in (g.x_knots[0], g.x_knots[57], g.x_knots[-2], g.x_knots[-1]):
        for qj in (g.q2_knots[0], g.q2_knots[11], g.q2_knots[12], g.q2_knots[30], g.q2_knots[-1]):
            x[k], q2[k] = xi, qj
            k += 1
    # 100 points in one cell: runs cross tile boundaries
    c0, c1 = np.log(g.x_knots[100]), np.log(g.x_knots[101])
    d0, d1 = np.log(g.q2_knots[20]), np.log(g.q2_knots[21])
    x[k:k + 100] = np.exp(rng.uniform(c0, c1, 100))
    q2[k:k + 100] = np.exp(rng.uniform(d0, d1, 100))
    k += 100
    x[k:k + 3], q2[k:k + 3] = [0.0, 0.5, 2.0], [10.0, -1.0, 10.0]  # invalid
    perm = rng.permutation(n)
    x, q2, cot = x[perm], q2[perm], cot[perm]
    gx, gq, gv = run_vjp(G, x, q2, cot)  # sorted
    parts = [run_vjp(G, x[a:a + 1500], q2[a:a + 1500], cot[a:a + 1500]) for a in range(0, n, 1500)]
    cx = np.concatenate([p[0] for p in parts])
    cq = np.concatenate([p[1] for p in parts])
    cv = sum(p[2] for p in parts)
    valid = np.isfinite(cx)
    assert (~valid).sum() == 3
    assert np.array_equal(np.isfinite(gx), valid) and np.array_equal(np.isfinite(gq), valid)
    # per point: the oracle's forward-mode gradients, for the sorted batch,
    # the small batches and the sorted batch without the knot gradient
    gx2, gq2, _ = run_vjp(G, x, q2, cot, with_values=False)
    assert np.array_equal(np.isfinite(gx2), valid)
    xv, qv, cv_ = x[valid], q2[valid], cot[valid]
    dx, dq = og.dxfxq2(xv, qv, "x"), og.dxfxq2(xv, qv, "q2")
    _, s, _ = og.xfxq2(xv, qv)
    sx = np.abs(cv_ * dx).sum(axis=1) + (np.abs(cv_) * s).sum(axis=1) / (xv * min_log_spacing(g.x_knots))
    sq = np.abs(cv_ * dq).sum(axis=1) + (np.abs(cv_) * s).sum(axis=1) / (qv * min_log_spacing(g.q2_knots))
    # (at x = 1 every value is 0, so there sq = 0 and the error must vanish)
    for ax, aq in ((gx, gq), (cx, cq), (gx2, gq2)):
        assert (np.abs(ax[valid] - (cv_ * dx).sum(axis=1)) <= 1e-10 * sx + 1e-280).all()
        assert (np.abs(aq[valid] - (cv_ * dq).sum(axis=1)) <= 1e-10 * sq + 1e-280).all()
        assert (np.abs(ax[valid] - gx[valid]) <= 1e-13 * sx + 1e-280).all()
        assert (np.abs(aq[valid] - gq[valid]) <= 1e-13 * sq + 1e-280).all()
    go, gabs = og.knot_grad(x[valid], q2[valid], cot[valid], with_abs=True)
    for got in (gv, cv):
        err = np.abs(got - go)
        assert (err <= 1e-10 * gabs + 1e-300).all(), (err / np.maximum(gabs, 1e-300)).max()
    assert (np.abs(gv - cv) <= 1e-12 * gabs + 1e-300).all()


@pytest.mark.parametrize("cls", ["lowx", "highq", "lowq", "lowx_highq", "lowx_lowq"])
def test_sorted_continuation_warps_sum_their_knot_terms(full, synth, cls):
    """Continuation points are sorted by kind; those that take both rules
    (all on the same few knots) by side too, and a warp of 32 of them that
    share their sites sums each knot term over the warp before one atomic.
    Batches of one class against the oracle's knot gradient and against
    small (unsorted) batches."""
    g, G, og = full
    n = 6000
    x, q2 = synth.queries_class(g, cls, n, 41)
    cot = np.random.default_rng(42).standard_normal((n, g.nflav))
    gx, gq, gv = run_vjp(G, x, q2, cot)  # sorted
    parts = [run_vjp(G, x[a:a + 1500], q2[a:a + 1500], cot[a:a + 1500]) for a in range(0, n, 1500)]
    cx = np.concatenate([p[0] for p in parts])
    cq = np.concatenate([p[1] for p in parts])
    cv = sum(p[2] for p in parts)
    assert np.isfinite(gx).all() and np.isfinite(gq).all()
    go, gabs = og.knot_grad(x, q2, cot, with_abs=True)
    assert np.abs(gabs).max() > 0
    for got in (gv, cv):
        err = np.abs(got - go)
        assert (err <= 1e-10 * gabs + 1e-300).all(), (err / np.maximum(gabs, 1e-300)).max()
    assert (np.abs(gv - cv) <= 1e-12 * gabs + 1e-300).all()
    # the per-point gradients: the oracle's, and the same whatever order the
    # points run in (scales as in the tests above)
    dx, dq = og.dxfxq2(x, q2, "x"), og.dxfxq2(x, q2, "q2")
    _, s, _ = og.xfxq2(x, q2)
    sx = np.abs(cot * dx).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (x * min_log_spacing(g.x_knots))
    sq = np.abs(cot * dq).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (q2 * min_log_spacing(g.q2_knots))
    for ax, aq in ((gx, gq), (cx, cq)):
        assert (np.abs(ax - (cot * dx).sum(axis=1)) <= 1e-10 * sx).all()
        assert (np.abs(aq - (cot * dq).sum(axis=1)) <= 1e-10 * sq).all()
    assert (np.abs(gx - cx) <= 1e-13 * sx).all()
    assert (np.abs(gq - cq) <= 1e-13 * sq).all()


def test_sorted_batch_keeps_each_knots_precision(full, synth):
    """Float-float run sums are used only for weights and cotangents of
    moderate size; a point with a weight or cotangent far from 1 (here whole
    flavours scaled by 1e-30 and 1e30, and points within 1e-12 of a knot,
    whose far weights are ~1e-24) scatters in FP64, so every knot's gradient
    keeps its precision relative to its own terms."""
    g, G, og = full
    n = 20000
    x, q2, cot = synth.adjoint_inputs(n, g.nflav, 35, 36)
    cot[:, 0] *= 1e-30
    cot[:, 1] *= 1e30
    rng = np.random.default_rng(37)
    near = rng.choice(n, 64, replace=False)
    ks = rng.integers(1, len(g.x_knots) - 2, 64)
    x[near] = g.x_knots[ks] * (1 + 1e-12 * rng.uniform(0.5, 2.0, 64))
    q2[near] = np.exp(rng.uniform(np.log(g.q2_knots[0]), np.log(g.q2_knots[-1]), 64))
    gx, gq, gv = run_vjp(G, x, q2, cot)
    valid = np.isfinite(gx)
    go, gabs = og.knot_grad(x[valid], q2[valid], cot[valid], with_abs=True)
    err = np.abs(gv - go)
    assert (err <= 1e-10 * gabs + 1e-300).all(), (err / np.maximum(gabs, 1e-300)).max()
    assert np.abs(gv[..., 0]).max() < 1e-20 < np.abs(gv[..., 1]).max() * 1e-40


def test_large_batch_on_a_grid_the_sort_does_not_take(synth, oracle_mod):
    """More than 16 flavours: the contraction's lane layout does not fit, so
    even a large batch runs the unsorted kernel (its per-warp queues fill);
    its gradients against the oracle."""
    full = synth.grid_full()
    pids = list(full.pids) + [22, 23, 24, 25, 26]
    params = synth.flavour_params(len(pids), 41)
    qb = [q * q for q in (synth.Q_RANGE[0], *synth.Q_THRESHOLDS, synth.Q_RANGE[1])]
    subs = [synth.geom_knots(qb[s], qb[s + 1], synth.SUBGRID_KNOTS[s]) for s in range(3)]
    g = synth.make_grid(full.x_knots, subs, pids, params=params)
    assert g.nflav == 18
    G = P.pdf_load_grid(g)
    og = oracle_mod.OracleGrid(g)
    n = 8000
    x, q2, cot = synth.adjoint_inputs(n, g.nflav, 45, 46)
    gx, gq, gv = run_vjp(G, x, q2, cot)
    dx, dq = og.dxfxq2(x, q2, "x"), og.dxfxq2(x, q2, "q2")
    _, s, _ = og.xfxq2(x, q2)
    sx = np.abs(cot * dx).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (x * min_log_spacing(g.x_knots))
    sq = np.abs(cot * dq).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (q2 * min_log_spacing(g.q2_knots))
    assert (np.abs(gx - (cot * dx).sum(axis=1)) <= 1e-10 * sx + 1e-280).all()
    assert (np.abs(gq - (cot * dq).sum(axis=1)) <= 1e-10 * sq + 1e-280).all()
    go, gabs = og.knot_grad(x, q2, cot, with_abs=True)
    assert (np.abs(gv - go) <= 1e-10 * gabs + 1e-300).all()
    G.free()


def test_no_scratch_runs_the_unsorted_kernel(full, synth):
    """With the scratch bound at 0 a batch above the sort threshold takes the
    unsorted kernel (no scratch); its gradients against the oracle and
    against the sorted path's."""
    g, G, og = full
    n = 6000
    x, q2, cot = synth.adjoint_inputs(n, g.nflav, 55, 56)
    sx_, sq_, sv_ = run_vjp(G, x, q2, cot)  # sorted
    before = P.scratch_limit()
    try:
        P.set_scratch_limit(0)
        gx, gq, gv = run_vjp(G, x, q2, cot)
    finally:
        P.set_scratch_limit(before)
    dx, dq = og.dxfxq2(x, q2, "x"), og.dxfxq2(x, q2, "q2")
    _, s, _ = og.xfxq2(x, q2)
    sx = np.abs(cot * dx).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (x * min_log_spacing(g.x_knots))
    sq = np.abs(cot * dq).sum(axis=1) + (np.abs(cot) * s).sum(axis=1) / (q2 * min_log_spacing(g.q2_knots))
    assert (np.abs(gx - (cot * dx).sum(axis=1)) <= 1e-10 * sx + 1e-280).all()
    assert (np.abs(gq - (cot * dq).sum(axis=1)) <= 1e-10 * sq + 1e-280).all()
    go, gabs = og.knot_grad(x, q2, cot, with_abs=True)
    assert (np.abs(gv - go) <= 1e-10 * gabs + 1e-300).all()
    assert (np.abs(gv - sv_) <= 1e-12 * gabs + 1e-300).all()
    assert (np.abs(gx - sx_) <= 1e-13 * sx + 1e-280).all()


def test_sorted_batch_without_private_copies(full, synth):
    """A scratch bound that leaves room for the sort (~8 B per point) but not
    for two copies of the knot gradient keeps the sorted kernel and sends
    the continuation points' knot terms to grad_values directly: the same
    gradients as with the copies, and the oracle's."""
    g, G, og = full
    n = 6000
    x, q2 = synth.queries_class(g, "lowx", n, 61)
    cot = np.random.default_rng(62).standard_normal((n, g.nflav))
    _, _, with_copies = run_vjp(G, x, q2, cot)
    copy_bytes = 8 * G.nrows * G.nx * G.nflav
    before = P.scratch_limit()
    try:
        P.set_scratch_limit(copy_bytes)  # the sort's ~0.1 MB fits, two copies do not
        gx, gq, gv = run_vjp(G, x, q2, cot)
    finally:
        P.set_scratch_limit(before)
    go, gabs = og.knot_grad(x, q2, cot, with_abs=True)
    for got in (gv, with_copies):
        assert (np.abs(got - go) <= 1e-10 * gabs + 1e-300).all()
    assert (np.abs(gv - with_copies) <= 1e-12 * gabs + 1e-300).all()
    assert np.isfinite(gx).all() and np.isfinite(gq).all()
