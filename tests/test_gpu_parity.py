"""GPU parity: the CUDA path (called through the C ABI) against the CPU oracle
on the same seeded inputs.  PDFFlow Sec. 2.2 (x f), Sec. 2.3 (alpha_s),
Fig. 1 (continuation), Sec. 4.1 (the PDF load of a Monte Carlo event)."""
import numpy as np
import pytest
import torch

from parity import (FP32_ALPHAS, RTOL_FP64, U32, assert_fp32, assert_parity, eq1_report, scaled_err,
                    special_points)

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


def test_alphas_q_squares_q(full, single):
    """alphas_Q (Fig. 1): the kernel squares Q; the result is alphas_q2 at
    Q * Q bit for bit, in FP64 and FP32, and Q <= 0 is invalid."""
    for g, G, og in (full, single):
        qn = np.sqrt(g.as_q2)
        q = np.exp(np.random.default_rng(15).uniform(np.log(qn[0] * 1e-2), np.log(qn[-1] * 1e2), 20_000))
        q = np.concatenate([q, qn, [0.0, -2.0, np.nan, np.inf, 1e200]])
        G.reset_invalid_count()
        out = host(P.alphas_q(G, dev(q)))
        assert G.invalid_count() == 5
        assert np.isnan(out[-5:]).all() and not np.isnan(out[:-5]).any()
        want = host(P.alphas_q2(G, dev(q[:-5] * q[:-5])))
        assert np.array_equal(out[:-5], want)
        v, s = og.alphas(q[:-5] * q[:-5])
        assert_parity(out[:-5], v, s, np.zeros(v.shape, bool), RTOL_FP64, "alphas_q fp64")
        q32 = q[:-5].astype(np.float32)
        out32 = host(P.alphas_q(G, dev(q32, torch.float32)))
        assert np.array_equal(out32, host(P.alphas_q2(G, dev(q32 * q32, torch.float32))))


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

def test_fp32_all_flavours(full, synth):
    g, G, og = full
    x, q2 = synth.queries_full(100_000, 3)
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    out = host(P.xfxq2_all_flavours(G, dev(x32, torch.float32), dev(q32, torch.float32))).astype(np.float64)
    xs, qs = x32.astype(np.float64), q32.astype(np.float64)
    v, s, fl = og.xfxq2(xs, qs)
    per_flav, per_class = assert_fp32(g, xs, qs, out, v, s, fl, "fp32 all flavours")
    print("fp32 worst scaled error per flavour:", " ".join(f"{e:.2e}" for e in per_flav))
    print("fp32 worst scaled error per class (units of 2^-24):", per_class)
    assert np.array_equal(np.isnan(out), np.isnan(v))


def test_fp32_special_points_and_single_pid(full):
    g, G, og = full
    x, q2 = special_points(g)
    x32, q32 = x.astype(np.float32), q2.astype(np.float32)
    xd, qd = dev(x32, torch.float32), dev(q32, torch.float32)
    out = host(P.xfxq2_all_flavours(G, xd, qd)).astype(np.float64)
    xs, qs = x32.astype(np.float64), q32.astype(np.float64)
    v, s, fl = og.xfxq2(xs, qs)
    _, per_class = assert_fp32(g, xs, qs, out, v, s, fl, "special points fp32")
    print("fp32 special points, worst scaled error per class (units of 2^-24):", per_class)
    one = host(P.xfxq2(G, 21, xd, qd))
    assert np.array_equal(one, out[:, g.pids.index(21)].astype(np.float32), equal_nan=True)


def test_fp32_alphas_and_mc(full, synth):
    g, G, og = full
    q = np.exp(np.random.default_rng(6).uniform(np.log(0.1), np.log(1e11), 20_000)).astype(np.float32)
    out = host(P.alphas_q2(G, dev(q, torch.float32))).astype(np.float64)
    v, s = og.alphas(q.astype(np.float64))
    assert (scaled_err(out, v, s) <= FP32_ALPHAS * U32).all(), scaled_err(out, v, s).max() / U32
    x1, x2, s2 = synth.events_mc(10_000, 4)
    a1, a2 = x1.astype(np.float32), x2.astype(np.float32)
    s32 = np.float32(s2)
    out = host(P.pdf_mc_event(G, dev(a1, torch.float32), dev(a2, torch.float32), float(s32))).astype(np.float64)
    q2 = (a1 * a2 * s32).astype(np.float64)  # the kernel's float product
    nf = g.nflav
    for side, xs in ((0, a1), (1, a2)):
        v, s, fl = og.xfxq2(xs.astype(np.float64), q2)
        assert_fp32(g, xs.astype(np.float64), q2, out[:, side * nf:(side + 1) * nf], v, s, fl, f"mc fp32 side {side}")


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
    worst, _ = assert_parity(got, v, s, fl, RTOL_FP64, "full-size fp64 sample")
    rep = eq1_report(got, v, s, fl)
    print(f"full-size fp64 sample: worst scaled error {worst:.2e}; eq. (1) max {rep['eq1_max']:.2e} "
          f"over {rep['outputs'] - rep['near_zero_excluded']} outputs ({rep['near_zero_excluded']} at zero "
          f"crossings left out); per flavour", " ".join(f"{e:.1e}" for e in rep["eq1_max_per_column"]))
    # away from zero crossings eq. (1) is the scaled error times S/|xf| <= 1e3
    assert rep["eq1_max"] <= RTOL_FP64 * 1e3
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
    per_flav, per_class = assert_fp32(g, xs, qs, out[ti].cpu().numpy().astype(np.float64), v, s, fl,
                                      "full-size fp32 sample")
    print("full-size fp32, worst scaled error per flavour:", " ".join(f"{e:.2e}" for e in per_flav))
    print("full-size fp32, worst scaled error per class (units of 2^-24):", per_class)
    av, asv = og.alphas(qs)
    assert_parity(a[ti].cpu().numpy().astype(np.float64), av, asv, np.zeros(av.shape, bool), FP32_ALPHAS * U32,
                  "full-size fp32 alphas sample")
