"""The surrogate with the residual target: the network corrects a base B_f
(bilinear in the scaled coordinates on a uniform 257 x 257 table of the FP64
interpolator), xf_f = B_f + 2^-10 E_f(x) y_f, so that BF16's ~1% error acts
on a term ~1e-3 of xf.  GPU inference and loss against the numpy oracle of the
same network, base and envelope; training, the error map at the 1e-3
threshold, evaluation with fallback against the interpolator; and what the
trained network gains (or loses) against the interpolator alone at that
accuracy.  No counterpart in the paper (growth axis: a learned replacement of
the Sec. 2.2 interpolation where it is accurate enough)."""
import math

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
def setup(synth, oracle_mod):
    from oracle import mlp
    from paper_2009_06635_gb300.surrogate import Surrogate

    g = synth.grid_full()
    G = P.pdf_load_grid(g)
    og = oracle_mod.OracleGrid(g)
    params, freq = synth.surrogate_init(g.nflav, 9)
    scale = 1e-5 * np.abs(g.values).reshape(-1, g.nflav).max(axis=0)
    bounds = (math.log(g.x_knots[0]), math.log(g.x_knots[-1]), math.log(g.q2_knots[0]), math.log(g.q2_knots[-1]))
    env_table = mlp.envelope_table(g.x_knots, g.values, bounds)
    X, Q = mlp.base_nodes(bounds)
    X[0, :], X[-1, :], Q[:, 0], Q[:, -1] = g.x_knots[0], g.x_knots[-1], g.q2_knots[0], g.q2_knots[-1]
    nodes, _, _ = og.xfxq2(X.ravel(), Q.ravel())
    base_table = mlp.base_table(nodes)
    return g, G, Surrogate, params, freq, scale, bounds, env_table, base_table, og


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_base_table_is_the_interpolator_at_its_nodes(setup):
    """On a node the base is the interpolator's value there (rounded to
    float); between nodes its error is the bilinear one, ~1e-3 of the
    envelope."""
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, env_table, base_table, og = setup
    i = np.array([0, 17, 128, 255, 256])
    X, Q = mlp.base_nodes(bounds)
    xs, qs = X[i, i[::-1]], Q[i, i[::-1]]
    xs[0], qs[-1] = g.x_knots[0], g.q2_knots[0]
    b = mlp.base(base_table, xs, qs, bounds)
    v, _, _ = og.xfxq2(xs, qs)
    assert np.all(np.abs(b - v) <= 2.0**-23 * np.abs(v) + 1e-300)
    x, q2 = P.synthetic.ingrid_samples(g, 20_000, 33)
    r = (og.xfxq2(x, q2)[0] - mlp.base(base_table, x, q2, bounds)) / (mlp.RES_EPS * mlp.envelope(env_table, x, bounds))
    print("residual target, quantiles 50/99/100 of |r|:", np.quantile(np.abs(r), [0.5, 0.99, 1.0]))
    assert np.quantile(np.abs(r), 0.5) < 2.0


def test_loss_and_inference_match_oracle(setup, synth):
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, env_table, base_table, og = setup
    s = Surrogate(G, params, freq, max_batch=1024, target="residual")
    x, q2 = synth.ingrid_samples(g, 1000, 34)
    xf, _, _ = og.xfxq2(x, q2)
    env = mlp.envelope(env_table, x, bounds)
    bv = mlp.base(base_table, x, q2, bounds)
    loss, grad = s.loss_grad(dev(x), dev(q2), dev(xf))
    oloss, _ = mlp.loss_grad(params.astype(np.float64), x, q2, xf, scale, freq.astype(np.float64), bounds, g.nflav,
                             bf=True, env=env, base_vals=bv)
    assert abs(loss - oloss) <= 1e-3 * oloss, (loss, oloss)
    from surrogate_bounds import check_inference, check_training_pass

    f64 = freq.astype(np.float64)
    worst = check_training_pass(s, params, x, q2, xf, scale, f64, bounds, g.nflav, grad, "residual", env_table,
                                base_table)
    print("training pass (residual), largest ratio per stage:", {k: round(v, 3) for k, v in worst.items()})
    x, q2 = synth.ingrid_samples(g, 4001, 35)
    out = s.eval(dev(x), dev(q2)).cpu().numpy()
    worst = check_inference(out, params, x, q2, scale, f64, bounds, g.nflav, "residual", env_table, base_table)
    print(f"inference (residual): worst element at {worst:.3f} of its bound")


def gpu_tiles(x, q2, bounds):
    """Error-map tile (tq, tx) of each point from FP32 coordinates computed as
    the GPU does, and whether the point is clear of tile edges (so that an ulp
    of difference in ln cannot move it to the neighbouring tile)."""
    f = np.float32
    lo0, lo1 = f(bounds[0]), f(bounds[2])
    i0, i1 = f(1.0 / (bounds[1] - bounds[0])), f(1.0 / (bounds[3] - bounds[2]))
    z0 = f(2) * (np.log(x.astype(f)) - lo0) * i0 - f(1)
    z1 = f(2) * (np.log(q2.astype(f)) - lo1) * i1 - f(1)
    u0, u1 = (z0.astype(np.float64) + 1) * 32, (z1.astype(np.float64) + 1) * 32
    clear = (np.abs(u0 - np.round(u0)) > 1e-3) & (np.abs(u1 - np.round(u1)) > 1e-3)
    return np.clip(u1.astype(int), 0, 63), np.clip(u0.astype(int), 0, 63), clear


def test_training_reaches_the_threshold_and_serves_points(setup, synth):
    """Trained on interpolator samples, the network passes the 1e-3 error
    threshold on part of the (z0, z1) square and the base alone on another
    part; evaluation with fallback serves each tile the way its map state
    says (network, base alone, or the interpolator), each served point within
    the threshold (checked on fresh points, with the map's tile resolution as
    margin), and base-alone tiles give exactly the base."""
    g, G, Surrogate, params, freq, scale, bounds, env_table, base_table, og = setup
    s = Surrogate(G, params, freq, max_batch=8192, target="residual")
    x, q2 = synth.ingrid_samples(g, 2_000_000, 7)
    xd, qd = dev(x), dev(q2)
    xf0, _, _ = og.xfxq2(x[:1024], q2[:1024])
    l0, _ = s.loss_grad(xd[:1024], qd[:1024], dev(xf0))
    final = s.train(G, xd, qd, batch=8192, steps=3000, lr=2e-3, lr_min=1e-5, warmup=200)
    assert final < 0.5 * l0, (l0, final)
    xv, qv = synth.ingrid_samples(g, 1_000_000, 23)
    stats = s.build_error_map(G, dev(xv), dev(qv), threshold=1e-3)
    print("residual target: error map", stats, "loss", l0, "->", final)
    assert stats["tiles_accepted"] == stats["tiles_network"] + stats["tiles_base_only"]
    assert stats["tiles_network"] > 0 and stats["tiles_accepted"] > 0.25 * 64 * 64, stats
    m = s.tile_map()
    assert int((m != 0).sum()) == stats["tiles_accepted"]
    xt, qt = synth.ingrid_samples(g, 400_000, 24)
    out, nfb = s.eval_fallback(G, dev(xt), dev(qt))
    out = out.cpu().numpy()
    ref = P.xfxq2_all_flavours(G, dev(xt), dev(qt)).cpu().numpy()
    served = ~np.all(out == ref, axis=1)
    assert served.sum() == len(xt) - nfb > 0
    tq, tx, clear = gpu_tiles(xt, qt, bounds)
    state = m[tq, tx]
    assert np.array_equal(served[clear], state[clear] != 0)
    # base-alone tiles: exactly the base (a network of zeros adds nothing to it)
    s0 = Surrogate(G, np.zeros_like(params), freq, max_batch=8192, target="residual")
    b = s0.eval(dev(xt), dev(qt)).cpu().numpy().astype(np.float64)
    k = clear & (state == 2)
    assert np.array_equal(out[k], b[k])
    k = clear & (state == 1)
    assert k.sum() > 0 and not np.array_equal(out[k], b[k])
    err = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), scale), axis=1)
    print(f"served {served.mean():.3f} of the points ({(state[clear] == 1).mean():.3f} by the network, "
          f"{(state[clear] == 2).mean():.3f} by the base alone); worst error on them {err[served].max():.2e}")
    assert err[served].max() < 3e-3, err[served].max()
    assert np.quantile(err[served], 0.999) < 1e-3


def test_gain_over_the_interpolator_at_the_threshold(setup, synth):
    """What the trained network gains over the method without it, at the 1e-3
    threshold: the served fraction and evaluation-with-fallback throughput
    against the FP64 interpolator alone on the same 4e6 in-grid points (both
    FP64 out).  The numbers are reported; on GB300 the interpolator is the
    faster of the two (a stated loss), and the surrogate's value lies in the
    accuracy it reaches at all, not in speed."""
    g, G, Surrogate, params, freq, scale, bounds, env_table, base_table, og = setup
    s = Surrogate(G, params, freq, max_batch=8192, target="residual")
    x, q2 = synth.ingrid_samples(g, 2_000_000, 7)
    s.train(G, dev(x), dev(q2), batch=8192, steps=3000, lr=2e-3, lr_min=1e-5, warmup=200)
    xv, qv = synth.ingrid_samples(g, 1_000_000, 23)
    s.build_error_map(G, dev(xv), dev(qv), threshold=1e-3)
    n = 4_000_000
    xt, qt = synth.ingrid_samples(g, n, 8)
    xd, qd = dev(xt), dev(qt)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = torch.empty((n, g.nflav), dtype=torch.float64, device="cuda")
    t_int = timed(lambda: P.xfxq2_all_flavours(G, xd, qd, out=out))
    _, nfb = s.eval_fallback(G, xd, qd)
    t_sur = timed(lambda: s.eval_fallback(G, xd, qd, out=out))
    served = 1.0 - nfb / n
    # the base alone (a network of zeros): what the network adds to it
    s0 = Surrogate(G, np.zeros_like(params), freq, max_batch=8192, target="residual")
    s0.build_error_map(G, dev(xv), dev(qv), threshold=1e-3)
    _, nfb0 = s0.eval_fallback(G, xd, qd)
    served0 = 1.0 - nfb0 / n
    print(f"residual surrogate with fallback: {t_sur:.3f} ms, interpolator alone {t_int:.3f} ms "
          f"(gain {t_int / t_sur:.2f}x); served at 1e-3: {served:.3f} of {n} in-grid points with the network "
          f"and its base, {served0:.3f} with the base alone")
    # each tile takes the better of network and base, so the trained network
    # serves at least what the base alone does (the same validation points)
    assert served >= served0 and served > 0.25 and t_sur > 0 and t_int > 0
