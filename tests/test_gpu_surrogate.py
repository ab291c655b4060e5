"""GPU surrogate (BF16 tensor-core MLP) against the numpy oracle of the same
network, plus training, the error map and evaluation with fallback to the
interpolator.  The paper has no counterpart (growth axis: a learned
replacement of the Sec. 2.2 interpolation where it is accurate enough)."""
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
    from paper_2009_06635_gb300.surrogate import Surrogate

    g = synth.grid_full()
    G = P.pdf_load_grid(g)
    params, freq = synth.surrogate_init(g.nflav, 9)
    scale = 1e-5 * np.abs(g.values).reshape(-1, g.nflav).max(axis=0)
    bounds = (math.log(g.x_knots[0]), math.log(g.x_knots[-1]), math.log(g.q2_knots[0]), math.log(g.q2_knots[-1]))
    return g, G, Surrogate, params, freq, scale, bounds, oracle_mod.OracleGrid(g)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_loss_and_gradient_match_oracle(setup, synth):
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, og = setup
    s = Surrogate(G, params, freq, max_batch=1024)
    x, q2 = synth.ingrid_samples(g, 1000, 21)
    xf, _, _ = og.xfxq2(x, q2)  # targets from the oracle interpolator
    loss, grad = s.loss_grad(dev(x), dev(q2), dev(xf))
    oloss, ograd = mlp.loss_grad(params.astype(np.float64), x, q2, xf, scale, freq.astype(np.float64), bounds,
                                 g.nflav, bf=True)
    assert abs(loss - oloss) <= 1e-3 * oloss, (loss, oloss)
    # every element of every stage, the gradient included, within the bound
    # its own arithmetic gives, on the GPU's inputs of that stage
    from surrogate_bounds import check_training_pass

    worst = check_training_pass(s, params, x, q2, xf, scale, freq.astype(np.float64), bounds, g.nflav, grad)
    print("training pass, largest ratio to the bound per stage:", {k: round(v, 3) for k, v in worst.items()})


def test_fused_inference_matches_oracle(setup, synth):
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, og = setup
    s = Surrogate(G, params, freq, max_batch=1024)
    x, q2 = synth.ingrid_samples(g, 4001, 22)
    out = s.eval(dev(x), dev(q2)).cpu().numpy().astype(np.float64)
    from surrogate_bounds import check_inference

    worst = check_inference(out, params, x, q2, scale, freq.astype(np.float64), bounds, g.nflav)
    print(f"inference: worst element at {worst:.3f} of its bound")


@pytest.mark.parametrize("target", ["asinh", "envelope"])
def test_fused_inference_with_biases_matches_oracle(setup, synth, target):
    """Every layer with its own random bias per output row (the initial
    network has zero biases): the fused kernel's bias path and row mapping
    against the oracle."""
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, og = setup
    p = params.astype(np.float64).copy()
    rng = np.random.default_rng(41)
    k = 0
    for (o, i) in [(128, 32), (128, 128), (128, 128), (128, 128), (g.nflav, 128)]:
        k += o * i
        p[k:k + o] = rng.uniform(-1.0, 1.0, o)
        k += o
    assert k == p.size
    p32 = p.astype(np.float32)
    s = Surrogate(G, p32, freq, max_batch=1024, target=target)
    x, q2 = synth.ingrid_samples(g, 4001, 23)
    out = s.eval(dev(x), dev(q2)).cpu().numpy().astype(np.float64)
    from surrogate_bounds import check_inference

    table = mlp.envelope_table(g.x_knots, g.values, bounds) if target == "envelope" else None
    worst = check_inference(out, p32, x, q2, scale, freq.astype(np.float64), bounds, g.nflav, target, table)
    print(f"inference with biases ({target}): worst element at {worst:.3f} of its bound")


def test_training_error_map_and_fallback(setup, synth):
    g, G, Surrogate, params, freq, scale, bounds, og = setup
    s = Surrogate(G, params, freq, max_batch=8192)
    x, q2 = synth.ingrid_samples(g, 400_000, 7)
    xd, qd = dev(x), dev(q2)
    xf0, _, _ = og.xfxq2(x[:1024], q2[:1024])
    l0, _ = s.loss_grad(xd[:1024], qd[:1024], dev(xf0))
    final = s.train(G, xd, qd, batch=4096, steps=600, lr=2e-3, warmup=50)
    assert final < 0.2 * l0, (l0, final)
    xv, qv = synth.ingrid_samples(g, 200_000, 23)
    stats = s.build_error_map(G, dev(xv), dev(qv), threshold=1e-3)
    print("error map", stats, "loss", l0, "->", final)
    assert stats["tiles_sampled"] == 64 * 64
    # evaluation with fallback: the interpolator's exact output on fallback points,
    # within the threshold on accepted tiles (checked on fresh points, with margin)
    xt, qt = synth.queries_full(100_000, 24)
    out, nfb = s.eval_fallback(G, dev(xt), dev(qt))
    out = out.cpu().numpy()
    ref = P.xfxq2_all_flavours(G, dev(xt), dev(qt)).cpu().numpy()
    same = np.all((out == ref) | (np.isnan(out) & np.isnan(ref)), axis=1)
    assert same.sum() >= nfb
    err = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), scale), axis=1)
    err = np.where(np.isnan(ref).any(axis=1), 0.0, err)
    assert err.max() < 5e-3, err.max()
    print(f"fallback {nfb} of {len(xt)} points; network served {len(xt) - nfb}")


def test_fused_inference_ragged_sizes_and_unaligned_output(setup, synth):
    """Each output row is a function of its own point alone (per-row dot
    products in a fixed order), so any prefix run on its own -- fewer points
    than a tile, exactly one, ragged tails, more tiles than the grid has
    groups -- must reproduce the full run bit for bit, and so must a run
    whose output starts 4 bytes past a 16-byte boundary (the scalar store
    path of the staged output)."""
    g, G, Surrogate, params, freq, scale, bounds, og = setup
    p = params.astype(np.float64).copy()
    p[128 * 32:128 * 32 + 128] = np.random.default_rng(5).uniform(-0.5, 0.5, 128)  # b1
    s = Surrogate(G, p.astype(np.float32), freq, max_batch=1024)
    x, q2 = synth.ingrid_samples(g, 80_001, 24)
    xd, qd = dev(x), dev(q2)
    full = s.eval(xd, qd).cpu().numpy()
    for n in (1, 31, 127, 128, 129, 255, 257, 1000, 40_000):
        part = s.eval(xd[:n], qd[:n]).cpu().numpy()
        assert np.array_equal(part, full[:n]), n
    n = 1001
    buf = torch.empty(n * g.nflav + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(n, g.nflav)  # 4 bytes past the allocation's alignment
    assert out.data_ptr() % 16 == 4
    s.eval(xd[:n], qd[:n], out=out)
    assert np.array_equal(out.cpu().numpy(), full[:n])


def test_full_size_inference_sampled(setup, synth):
    """The benchmark's inference size and law (1e8 in-grid points, seed 8):
    sampled rows bit for bit against the same points run alone, and against
    the oracle network on a smaller sample."""
    from oracle import mlp

    g, G, Surrogate, params, freq, scale, bounds, og = setup
    p = params.astype(np.float64).copy()
    p[128 * 32:128 * 32 + 128] = np.random.default_rng(6).uniform(-0.5, 0.5, 128)  # b1
    p32 = p.astype(np.float32)
    s = Surrogate(G, p32, freq, max_batch=1024)
    n = 100_000_000
    x, q2 = synth.ingrid_samples(g, n, 8)
    xd, qd = dev(x), dev(q2)
    out = s.eval(xd, qd)
    idx = np.sort(np.random.default_rng(10).choice(n, 20_000, replace=False))
    ti = torch.from_numpy(idx).cuda()
    got = out[ti].cpu().numpy()
    del out
    alone = s.eval(xd[ti], qd[ti]).cpu().numpy()
    assert np.array_equal(got, alone)
    k = idx[:2000]
    from surrogate_bounds import check_inference

    check_inference(got[:2000], p32, x[k], q2[k], scale, freq.astype(np.float64), bounds, g.nflav)


def test_fallback_calls_on_two_streams_from_two_threads(setup, synth):
    """Fallback calls share the surrogate's gather/scatter buffers, and each
    call's gather, interpolation and scatter still run after it returns: a
    call on another stream must wait for them.  Two threads, each with its own
    non-blocking stream and a batch that falls back nearly everywhere (an
    untrained network), must each get what the same call gives alone."""
    import threading

    g, G, Surrogate, params, freq, scale, bounds, og = setup
    s = Surrogate(G, params, freq, max_batch=1024)
    xv, qv = synth.ingrid_samples(g, 50_000, 25)
    s.build_error_map(G, dev(xv), dev(qv), threshold=1e-3)
    batches = [tuple(map(dev, synth.queries_full(n, 70 + k))) for k, n in enumerate((600_001, 400_003))]
    alone = []
    for xd, qd in batches:
        out, nfb = s.eval_fallback(G, xd, qd)
        torch.cuda.synchronize()
        assert nfb > 0.9 * xd.shape[0]
        alone.append(out.cpu())
    res = [[None] * 4 for _ in batches]

    def run(k):
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        xd, qd = batches[k]
        with torch.cuda.stream(st):
            for r in range(4):
                res[k][r], _ = s.eval_fallback(G, xd, qd)
        st.synchronize()

    th = [threading.Thread(target=run, args=(k,)) for k in range(len(batches))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for k in range(len(batches)):
        for r in range(4):
            assert torch.equal(res[k][r].cpu(), alone[k]), (k, r)


def test_grid_with_other_flavours_is_refused(setup, synth):
    """The error map, training and the fallback write [n][nflav] rows of the
    surrogate's width: a grid with another flavour count is an argument
    error, not an out-of-bounds write."""
    g, G, Surrogate, params, freq, scale, bounds, og = setup
    g11 = synth.grid_single_subgrid()
    assert g11.nflav != g.nflav
    G11 = P.pdf_load_grid(g11)
    s = Surrogate(G, params, freq, max_batch=1024)
    x, q2 = synth.ingrid_samples(g, 256, 23)
    xd, qd = dev(x), dev(q2)
    with pytest.raises(P.PdfError, match="flavours differ"):
        s.build_error_map(G11, xd, qd)
    with pytest.raises(P.PdfError, match="flavours differ"):
        s.train(G11, xd, qd, batch=64, steps=1)
    s.build_error_map(G, xd, qd)
    with pytest.raises(P.PdfError, match="flavours differ"):
        s.eval_fallback(G11, xd, qd)
    out, _ = s.eval_fallback(G, xd, qd)  # the matching grid still works
    assert torch.isfinite(out).all()
    s.free()
    G11.free()
