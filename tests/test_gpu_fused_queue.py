"""FP64 evaluation as organised for GB300: the fused all-flavour + alpha_s
pass, and the per-warp continuation queue (points needing a continuation
rule are set aside and evaluated 32 at a time), against the oracle and
against the unfused calls.  PDFFlow Sec. 2.1-2.3 and Fig. 1."""
import numpy as np
import pytest
import torch

from parity import RTOL_FP64, assert_parity, special_points

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
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def interleaved(g, n, seed):
    """Every point's class drawn at random: in the grid, x < x0, Q^2 above,
    Q^2 below, and the two corners, so that tiles mix all of them."""
    r = np.random.default_rng(seed)
    x0, xl, q0, q1 = g.x_knots[0], g.x_knots[-1], g.q2_knots[0], g.q2_knots[-1]

    def lu(a, b):
        return np.exp(r.uniform(np.log(a), np.log(b), n))

    kind = r.integers(0, 6, n)
    xin, xlo = lu(x0, xl), lu(1e-10, x0)
    qin, qhi, qlo = lu(q0, q1), lu(q1, 1e3 * q1), lu(1e-3 * q0, q0)
    x = np.where((kind == 1) | (kind == 4) | (kind == 5), xlo, xin)
    q2 = np.choose(kind, [qin, qin, qhi, qlo, qhi, qlo])
    return x, q2


def test_fused_alphas_bitwise_and_parity(full, synth):
    g, G, og = full
    x, q2 = synth.queries_full(50_017, 21)
    sx, sq = special_points(g)
    x, q2 = np.concatenate([x, sx]), np.concatenate([q2, sq])
    xd, qd = dev(x), dev(q2)
    out, al = P.xfxq2_all_flavours_alphas(G, xd, qd)
    out, al = host(out), host(al)
    assert np.array_equal(out, host(P.xfxq2_all_flavours(G, xd, qd)), equal_nan=True)
    assert np.array_equal(al, host(P.alphas_q2(G, qd)), equal_nan=True)
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out, v, s, fl, RTOL_FP64, "fused xf")
    a, sa = og.alphas(q2)
    assert_parity(al, a, sa, np.zeros(a.shape, bool), RTOL_FP64, "fused alphas")


def test_fused_alphas_fp32_bitwise(full, synth):
    g, G, og = full
    x, q2 = synth.queries_full(30_011, 25)
    sx, sq = special_points(g)
    x = np.concatenate([x, sx]).astype(np.float32)
    q2 = np.concatenate([q2, sq]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q2).cuda()
    out, al = P.xfxq2_all_flavours_alphas(G, xd, qd)
    assert out.dtype == torch.float32 and al.dtype == torch.float32
    assert np.array_equal(host(out), host(P.xfxq2_all_flavours(G, xd, qd)), equal_nan=True)
    assert np.array_equal(host(al), host(P.alphas_q2(G, qd)), equal_nan=True)


@pytest.mark.parametrize("n", [1, 31, 33, 1000, 65_537])
def test_queue_heavy_batches(full, n):
    g, G, og = full
    x, q2 = interleaved(g, n, 40 + n)
    xd, qd = dev(x), dev(q2)
    out = host(P.xfxq2_all_flavours(G, xd, qd))
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out, v, s, fl, RTOL_FP64, f"interleaved n={n}")
    # one column through the same queue: identical bits
    col = 3
    one = host(P.xfxq2(G, g.pids[col], xd, qd))
    assert np.array_equal(one, out[:, col], equal_nan=True)


def test_all_points_continued(full):
    g, G, og = full
    n = 100_003
    r = np.random.default_rng(44)
    x = np.exp(r.uniform(np.log(1e-10), np.log(g.x_knots[0]), n))
    q2 = np.exp(r.uniform(np.log(g.q2_knots[0]), np.log(g.q2_knots[-1]), n))
    out = host(P.xfxq2_all_flavours(G, dev(x), dev(q2)))
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out, v, s, fl, RTOL_FP64, "all low-x")
    # and the Monte Carlo layout, where both sides and alpha_s share a row
    x1 = np.exp(r.uniform(np.log(1e-10), 0.0, 20_001))
    x2 = np.exp(r.uniform(np.log(1e-10), 0.0, 20_001))
    s2 = 13000.0**2  # Q^2 from 1.7e-12 to 1.7e8: low-Q^2, low-x and corner continuations
    mc = host(P.pdf_mc_event(G, dev(x1), dev(x2), s2))
    qq = x1 * x2 * s2
    nf = g.nflav
    for side, xs in ((0, x1), (1, x2)):
        v, s, fl = og.xfxq2(xs, qq)
        assert_parity(mc[:, side * nf:(side + 1) * nf], v, s, fl, RTOL_FP64, f"mc side {side}")
    a, sa = og.alphas(qq)
    assert_parity(mc[:, 2 * nf], a, sa, np.zeros(a.shape, bool), RTOL_FP64, "mc alphas")


def test_two_launches_match_one_launch_bit_for_bit(full, synth):
    """Batches of 65536 points or more run as two launches (in-grid and
    invalid points; then the points that need a rule, in class-pure tiles);
    smaller ones as one.  Every point is computed by the same arithmetic from
    its own coordinates, so a large batch must equal its pieces run alone:
    flavours, alpha_s, the invalid count, and the Monte Carlo layout."""
    g, G, og = full
    n = 300_007
    x, q2 = interleaved(g, n, 77)
    sx, sq = special_points(g)
    at = np.random.default_rng(78).choice(n, len(sx), replace=False)
    x[at], q2[at] = sx, sq
    xd, qd = dev(x), dev(q2)
    G.reset_invalid_count()
    out, al = P.xfxq2_all_flavours_alphas(G, xd, qd)
    torch.cuda.synchronize()
    ninv = G.invalid_count()
    G.reset_invalid_count()
    parts = [P.xfxq2_all_flavours_alphas(G, xd[a:a + 40_000], qd[a:a + 40_000]) for a in range(0, n, 40_000)]
    torch.cuda.synchronize()
    assert G.invalid_count() == ninv > 0
    assert np.array_equal(host(out), np.concatenate([host(p[0]) for p in parts]), equal_nan=True)
    assert np.array_equal(host(al), np.concatenate([host(p[1]) for p in parts]), equal_nan=True)
    r = np.random.default_rng(79)
    x1 = np.exp(r.uniform(np.log(1e-10), 0.0, 150_001))
    x2 = np.exp(r.uniform(np.log(1e-10), 0.0, 150_001))
    s2 = 13000.0**2
    mc = host(P.pdf_mc_event(G, dev(x1), dev(x2), s2))
    mcp = np.concatenate([host(P.pdf_mc_event(G, dev(x1[a:a + 30_000]), dev(x2[a:a + 30_000]), s2))
                          for a in range(0, len(x1), 30_000)])
    assert np.array_equal(mc, mcp, equal_nan=True)
