"""The surrogate with the envelope target (xf_f = E_f(x) y_f): GPU loss,
gradient and fused inference against the numpy oracle of the same network
and envelope, and training with the error map and fallback.  No counterpart
in the paper (growth axis: a learned replacement of the Sec. 2.2
interpolation where it is accurate enough)."""
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
    params, freq = synth.surrogate_init(g.nflav, 9)
    scale = 1e-5 * np.abs(g.values).reshape(-1, g.nflav).max(axis=0)
    bounds = (math.log(g.x_knots[0]), math.log(g.x_knots[-1]), math.log(g.q2_knots[0]), math.log(g.q2_knots[-1]))
    table = mlp.envelope_table(g.x_knots, g.values, bounds)
    return g, G, Surrogate, params, freq, scale, bounds, table, oracle_mod.OracleGrid(g)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_loss_gradient_and_inference_match_oracle(setup, synth):
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, table, og = setup
    s = Surrogate(G, params, freq, max_batch=1024, target="envelope")
    x, q2 = synth.ingrid_samples(g, 1000, 31)
    xf, _, _ = og.xfxq2(x, q2)
    env = mlp.envelope(table, x, bounds)
    loss, grad = s.loss_grad(dev(x), dev(q2), dev(xf))
    oloss, ograd = mlp.loss_grad(params.astype(np.float64), x, q2, xf, scale, freq.astype(np.float64), bounds,
                                 g.nflav, bf=True, env=env)
    assert abs(loss - oloss) <= 1e-3 * oloss, (loss, oloss)
    from surrogate_bounds import check_inference, check_training_pass

    f64 = freq.astype(np.float64)
    worst = check_training_pass(s, params, x, q2, xf, scale, f64, bounds, g.nflav, grad, "envelope", table)
    print("training pass (envelope), largest ratio per stage:", {k: round(v, 3) for k, v in worst.items()})
    x, q2 = synth.ingrid_samples(g, 4001, 32)
    out = s.eval(dev(x), dev(q2)).cpu().numpy()
    worst = check_inference(out, params, x, q2, scale, f64, bounds, g.nflav, "envelope", table)
    print(f"inference (envelope): worst element at {worst:.3f} of its bound")


def test_training_error_map_and_fallback(setup, synth):
    g, G, Surrogate, params, freq, scale, bounds, table, og = setup
    s = Surrogate(G, params, freq, max_batch=8192, target="envelope")
    x, q2 = synth.ingrid_samples(g, 400_000, 7)
    xd, qd = dev(x), dev(q2)
    xf0, _, _ = og.xfxq2(x[:1024], q2[:1024])
    l0, _ = s.loss_grad(xd[:1024], qd[:1024], dev(xf0))
    final = s.train(G, xd, qd, batch=4096, steps=600, lr=2e-3, warmup=50)
    assert final < 0.2 * l0, (l0, final)
    xv, qv = synth.ingrid_samples(g, 200_000, 23)
    stats = s.build_error_map(G, dev(xv), dev(qv), threshold=1e-2)
    print("error map", stats, "loss", l0, "->", final)
    assert stats["tiles_sampled"] == 64 * 64
    xt, qt = synth.queries_full(100_000, 24)
    out, nfb = s.eval_fallback(G, dev(xt), dev(qt))
    out = out.cpu().numpy()
    ref = P.xfxq2_all_flavours(G, dev(xt), dev(qt)).cpu().numpy()
    same = np.all((out == ref) | (np.isnan(out) & np.isnan(ref)), axis=1)
    assert same.sum() >= nfb
    err = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), scale), axis=1)
    err = np.where(np.isnan(ref).any(axis=1), 0.0, err)
    assert err.max() < 5e-2, err.max()
