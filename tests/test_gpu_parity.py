"""GPU parity: the CUDA path (called through the C ABI) against the CPU oracle
on the same seeded inputs.  PDFFlow Sec. 2.2 (x f), Sec. 2.3 (alpha_s),
Fig. 1 (continuation), Sec. 4.1 (the PDF load of a Monte Carlo event)."""
import numpy as np
import pytest
import torch

from parity import RTOL_FP32, RTOL_FP64, assert_parity, scaled_err, special_points

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


@pytest.fixture(scope="module")
def single(synth, oracle_mod):
    g = synth.grid_single_subgrid()
    return g, P.pdf_load_grid(g), oracle_mod.OracleGrid(g)


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ---------------------------------------------------------------------------
# FP64, all flavours
# ---------------------------------------------------------------------------

def test_single_subgrid_workload_fp64(single, synth):
    g, G, og = single
    x, q2 = synth.queries_single_subgrid(10_000, 2)
    out = host(P.xfxq2_all_flavours(G, dev(x), dev(q2)))
    v, s, fl = og.xfxq2(x, q2)
    worst, nflag = assert_parity(out, v, s, fl, RTOL_FP64, "single-subgrid fp64")
    assert nflag == 0
    print(f"single-subgrid fp64 worst scaled err {worst:.2e}")


@pytest.mark.parametrize("n", [1, 31, 33, 50_001])
def test_three_subgrid_queries_fp64_ragged(full, synth, n):
    g, G, og = full
    x, q2 = synth.queries_full(n, 3)
    out = host(P.xfxq2_all_flavours(G, dev(x), dev(q2)))
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out, v, s, fl, RTOL_FP64, f"three-subgrid fp64 n={n}")


def test_special_points_fp64(full):
    g, G, og = full
    x, q2 = special_points(g)
    G.reset_invalid_count()
    out = host(P.xfxq2_all_flavours(G, dev(x), dev(q2)))
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out, v, s, fl, RTOL_FP64, "special points fp64")
    assert G.invalid_count() == int(np.isnan(v[:, 0]).sum()) == 9


def test_knots_reproduced_fp64(full):
    g, G, og = full
    X, Q = np.meshgrid(g.x_knots, g.q2_knots)
    out = host(P.xfxq2_all_flavours(G, dev(X.ravel()), dev(Q.ravel())))
    want = g.values.reshape(-1, g.nflav)
    # every knot, the last x knot and the top Q knot included, sits at t = u = 0
    # of its (possibly degenerate) cell: the stored value comes back exactly
    assert np.array_equal(out, want)


def test_single_pid_matches_all_flavour_columns(full, synth):
    g, G, og = full
    x, q2 = synth.queries_full(20_000, 31)
    v, s, fl = og.xfxq2(x, q2)
    xd, qd = dev(x), dev(q2)
    allf = host(P.xfxq2_all_flavours(G, xd, qd))
    for col, pid in enumerate(g.pids):
        one = host(P.xfxq2(G, pid, xd, qd))
        assert np.array_equal(one, allf[:, col], equal_nan=True)
        assert_parity(one, v[:, col], s[:, col], fl[:, col], RTOL_FP64, f"pid {pid}")
    gl = host(P.xfxq2(G, 0, xd, qd))  # pid 0 is the gluon
    assert np.array_equal(gl, allf[:, g.pids.index(21)], equal_nan=True)
    with pytest.raises(P.PdfError):
        P.xfxq2(G, 7, xd, qd)


def test_alphas_fp64(full, single, synth):
    for g, G, og in (full, single):
        q = np.exp(np.random.default_rng(5).uniform(np.log(g.as_q2[0] * 1e-3), np.log(g.as_q2[-1] * 1e3), 20_000))
        q = np.concatenate([q, g.as_q2, [0.0, -1.0, np.nan, np.inf]])
        out = host(P.alphas_q2(G, dev(q)))
        v, s = og.alphas(q)
        assert_parity(out, v, s, np.zeros(v.shape, bool), RTOL_FP64, "alphas fp64")
        assert np.array_equal(out[20_000:20_000 + len(g.as_q2)], g.as_vals)


def test_mc_event_fp64(full, synth):
    g, G, og = full
    x1, x2, s2 = synth.events_mc(20_003, 4)
    out = host(P.pdf_mc_event(G, dev(x1), dev(x2), s2))
    q2 = x1 * x2 * s2
    nf = g.nflav
    for side, xs in ((0, x1), (1, x2)):
        v, s, fl = og.xfxq2(xs, q2)
        assert_parity(out[:, side * nf:(side + 1) * nf], v, s, fl, RTOL_FP64, f"mc side {side}")
    a, sa = og.alphas(q2)
    assert_parity(out[:, 2 * nf], a, sa, np.zeros(a.shape, bool), RTOL_FP64, "mc alphas")
    assert ((q2 < g.q2_knots[0])).mean() > 0.1  # the batch exercises the low-Q^2 continuation


def test_empty_batch_and_host_path(full, synth):
    g, G, og = full
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert P.xfxq2_all_flavours(G, e, e).shape == (0, g.nflav)
    assert P.alphas_q2(G, e).shape == (0,)
    x, q2 = synth.queries_full(2_500_017, 3)
    dout = host(P.xfxq2_all_flavours(G, dev(x), dev(q2)))
    hout, hal = P.xfxq2_all_flavours_host(G, torch.from_numpy(x).pin_memory(), torch.from_numpy(q2).pin_memory(),
                                          with_alphas=True)
    assert np.array_equal(hout.numpy(), dout, equal_nan=True)
    assert np.array_equal(hal.numpy(), host(P.alphas_q2(G, dev(q2))), equal_nan=True)
    hout2 = P.xfxq2_all_flavours_host(G, x[:1000], q2[:1000])  # pageable memory
    assert np.array_equal(hout2.numpy(), dout[:1000], equal_nan=True)


def test_grid_without_alphas(synth):
    g = synth.grid_single_subgrid()
    G = P.pdf_load_grid(x_knots=g.x_knots, nq=g.nq, q2_knots=g.q2_knots, pids=g.pids, values=g.values)
    q = dev(np.array([10.0]))
    with pytest.raises(P.PdfError, match="NO_ALPHAS"):
        P.alphas_q2(G, q)


# ---------------------------------------------------------------------------
# FP32 paths
# ---------------------------------------------------------------------------

def _fp32_errors(out, v, s, fl, nf):
    ok = ~np.isnan(v) & ~fl
    err = np.where(ok, scaled_err(out, v, s), 0.0)
    rel = np.where(ok & (np.abs(v) > 0), np.abs(out - v) / (np.abs(v) + 1e-16), 0.0)
    return err.max(axis=0), rel


def test_fp32_all_flavours(full, synth):
    g, G, og = full
    x, q2 = synth.queries_full(100_000, 3)
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    out = host(P.xfxq2_all_flavours(G, dev(x32, torch.float32), dev(q32, torch.float32))).astype(np.float64)
    v, s, fl = og.xfxq2(x32.astype(np.float64), q32.astype(np.float64))
    per_flav, _ = _fp32_errors(out, v, s, fl, g.nflav)
    print("fp32 worst scaled error per flavour:", " ".join(f"{e:.2e}" for e in per_flav))
    assert (per_flav <= RTOL_FP32).all(), per_flav
    assert np.array_equal(np.isnan(out), np.isnan(v))


def test_fp32_special_points_and_single_pid(full):
    g, G, og = full
    x, q2 = special_points(g)
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    xd, qd = dev(x32, torch.float32), dev(q32, torch.float32)
    out = host(P.xfxq2_all_flavours(G, xd, qd)).astype(np.float64)
    v, s, fl = og.xfxq2(x32.astype(np.float64), q32.astype(np.float64))
    assert_parity(out, v, s, fl, RTOL_FP32, "special points fp32")
    one = host(P.xfxq2(G, 21, xd, qd))
    assert np.array_equal(one, out[:, g.pids.index(21)].astype(np.float32), equal_nan=True)


def test_fp32_alphas_and_mc(full, synth):
    g, G, og = full
    q = np.exp(np.random.default_rng(6).uniform(np.log(0.1), np.log(1e11), 20_000)).astype(np.float32)
    out = host(P.alphas_q2(G, dev(q, torch.float32))).astype(np.float64)
    v, s = og.alphas(q.astype(np.float64))
    assert (scaled_err(out, v, s) <= 1e-6).all()
    x1, x2, s2 = synth.events_mc(10_000, 4)
    a1, a2 = x1.astype(np.float32), x2.astype(np.float32)
    s32 = np.float32(s2)
    out = host(P.pdf_mc_event(G, dev(a1, torch.float32), dev(a2, torch.float32), float(s32))).astype(np.float64)
    q2 = (a1 * a2 * s32).astype(np.float64)  # the kernel's float product
    nf = g.nflav
    for side, xs in ((0, a1), (1, a2)):
        v, s, fl = og.xfxq2(xs.astype(np.float64), q2)
        assert_parity(out[:, side * nf:(side + 1) * nf], v, s, fl, RTOL_FP32, f"mc fp32 side {side}")


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------

def test_full_size_three_subgrid_batch_sampled(full, synth):
    g, G, og = full
    n = 10_000_000
    x, q2 = synth.queries_full(n, 3)
    G.reset_invalid_count()
    out = P.xfxq2_all_flavours(G, dev(x), dev(q2))
    torch.cuda.synchronize()
    assert G.invalid_count() == 0
    assert not torch.isnan(out).any().item()
    idx = np.random.default_rng(7).choice(n, 100_000, replace=False)
    idx = np.concatenate([idx, [0, n - 1]])
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    v, s, fl = og.xfxq2(x[idx], q2[idx])
    assert_parity(got, v, s, fl, RTOL_FP64, "full-size fp64 sample")
    a = P.alphas_q2(G, dev(q2))
    av, asv = og.alphas(q2[idx])
    assert_parity(a[torch.from_numpy(idx).cuda()].cpu().numpy(), av, asv, np.zeros(av.shape, bool),
                  RTOL_FP64, "full-size alphas sample")


def test_full_size_mc_chunk_sampled(full, synth):
    g, G, og = full
    n = 1_000_000
    x1, x2, s2 = synth.events_mc(n, 4)
    out = P.pdf_mc_event(G, dev(x1), dev(x2), s2)
    torch.cuda.synchronize()
    idx = np.random.default_rng(8).choice(n, 20_000, replace=False)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    q2 = x1[idx] * x2[idx] * s2
    nf = g.nflav
    for side, xs in ((0, x1[idx]), (1, x2[idx])):
        v, s, fl = og.xfxq2(xs, q2)
        assert_parity(got[:, side * nf:(side + 1) * nf], v, s, fl, RTOL_FP64, f"mc chunk side {side}")


def test_host_path_and_mc_from_concurrent_threads(full, synth):
    """Host-buffer calls (and Monte Carlo integrations) on one grid from
    several host threads share the grid's staging buffers; the grid
    serialises them, so every thread gets the result of a call made alone."""
    import threading

    g, G, og = full
    xs = [synth.queries_full(1_500_001, 60 + k) for k in range(4)]
    alone = [P.xfxq2_all_flavours_host(G, torch.from_numpy(x).pin_memory(), torch.from_numpy(q).pin_memory()).numpy()
             for x, q in xs]
    mc_alone = P.pdf_mc_integrate(G, 13000.0, 1e-6, 100.0, 4, 2_000_000)
    res, mc = [None] * 4, [None] * 2
    def host_call(k):
        x, q = xs[k]
        res[k] = P.xfxq2_all_flavours_host(G, torch.from_numpy(x).pin_memory(), torch.from_numpy(q).pin_memory())
    def mc_call(k):
        torch.cuda.set_device(0)
        mc[k] = P.pdf_mc_integrate(G, 13000.0, 1e-6, 100.0, 4, 2_000_000)
    threads = [threading.Thread(target=host_call, args=(k,)) for k in range(4)]
    threads += [threading.Thread(target=mc_call, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for k in range(4):
        assert np.array_equal(res[k].numpy(), alone[k], equal_nan=True), k
    want = (mc_alone.sum_w, mc_alone.sum_w2, mc_alone.sum_abs)  # fixed-order device sums
    for k in range(2):
        assert (mc[k].sum_w, mc[k].sum_w2, mc[k].sum_abs) == want, k


def test_full_size_fp32_batch_sampled(full, synth):
    """The FP32 step of the benchmark (the 1e7-point batch rounded to float,
    all flavours + alpha_s in one launch), sampled against the oracle at the
    float inputs."""
    g, G, og = full
    n = 10_000_000
    x, q2 = synth.queries_full(n, 3)
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    out, a = P.xfxq2_all_flavours_alphas(G, torch.from_numpy(x32).cuda(), torch.from_numpy(q32).cuda())
    torch.cuda.synchronize()
    idx = np.concatenate([np.random.default_rng(9).choice(n, 100_000, replace=False), [0, n - 1]])
    ti = torch.from_numpy(idx).cuda()
    xs, qs = x32[idx].astype(np.float64), q32[idx].astype(np.float64)
    v, s, fl = og.xfxq2(xs, qs)
    assert_parity(out[ti].cpu().numpy().astype(np.float64), v, s, fl, RTOL_FP32, "full-size fp32 sample")
    av, asv = og.alphas(qs)
    assert_parity(a[ti].cpu().numpy().astype(np.float64), av, asv, np.zeros(av.shape, bool), RTOL_FP32,
                  "full-size fp32 alphas sample")
