"""Grids at the sizes the C ABI allows and the degenerate cases the method
has, against the oracle on the same points: the largest knot counts (2048 x
knots, 1024 Q rows in four subgrids), the most flavours (64), the smallest
grid (2 x 2 knots: bilinear), and a two-knot subgrid between wider ones
(linear in ln Q^2 there).  PDFFlow Sec. 2.2 (subgrids, edges, thresholds)."""
import numpy as np
import pytest
import torch

from parity import RTOL_FP64, assert_fp32, assert_parity, special_points

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def queries(g, n, seed):
    r = np.random.default_rng(seed)
    lx = r.uniform(np.log(g.x_knots[0]) - 2.0, 0.0, n)
    lq = r.uniform(np.log(g.q2_knots[0]) - 2.0, np.log(g.q2_knots[-1]) + 2.0, n)
    return np.exp(lx), np.exp(lq)


def check(synth, oracle_mod, g, n=20_000, seed=1, fp32=True):
    G = P.pdf_load_grid(g)
    og = oracle_mod.OracleGrid(g)
    x, q2 = queries(g, n, seed)
    sx, sq = special_points(g)
    x, q2 = np.concatenate([x, sx]), np.concatenate([q2, sq])
    out, al = P.xfxq2_all_flavours_alphas(G, dev(x), dev(q2))
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out.cpu().numpy(), v, s, fl, RTOL_FP64, "fp64")
    a, sa = og.alphas(q2)
    assert_parity(al.cpu().numpy(), a, sa, np.zeros(a.shape, bool), RTOL_FP64, "alphas")
    if fp32:
        x32, q32 = x.astype(np.float32), q2.astype(np.float32)
        o32 = P.xfxq2_all_flavours(G, dev(x32, torch.float32), dev(q32, torch.float32)).cpu().numpy()
        xs, qs = x32.astype(np.float64), q32.astype(np.float64)
        v32, s32, fl32 = og.xfxq2(xs, qs)
        assert_fp32(g, xs, qs, o32, v32, s32, fl32, "fp32")
    return G


def test_largest_knot_counts(synth, oracle_mod):
    xk = np.geomspace(1e-9, 1.0, 2048)
    bounds = np.geomspace(1.0, 1e10, 5)
    subs = [np.geomspace(bounds[k], bounds[k + 1], 256) for k in range(4)]  # 1024 rows
    pids = list(range(-7, 0)) + [21] + list(range(1, 9))  # 16 flavours
    g = synth.make_grid(xk, subs, pids, params=synth.flavour_params(len(pids), 31))
    assert len(g.q2_knots) == 1024
    check(synth, oracle_mod, g, n=20_000, seed=2)


def test_largest_knot_counts_in_two_launches(synth, oracle_mod):
    """The same grid (2048 x knots, 1024 Q rows and alpha_s nodes: the most
    shared memory the staged knot and position tables take) with a batch
    above the two-launch threshold (near and far launches)."""
    xk = np.geomspace(1e-9, 1.0, 2048)
    bounds = np.geomspace(1.0, 1e10, 5)
    subs = [np.geomspace(bounds[k], bounds[k + 1], 256) for k in range(4)]
    pids = list(range(-7, 0)) + [21] + list(range(1, 9))
    g = synth.make_grid(xk, subs, pids, params=synth.flavour_params(len(pids), 31))
    assert len(g.as_q2) == 1024
    check(synth, oracle_mod, g, n=70_000, seed=3, fp32=False)


def test_most_flavours(synth, oracle_mod):
    xk = np.geomspace(1e-7, 1.0, 40)
    subs = [np.geomspace(2.0, 20.0, 8), np.geomspace(20.0, 1e6, 12)]
    pids = list(range(1, 65))
    g = synth.make_grid(xk, subs, pids, params=synth.flavour_params(64, 32))
    G = check(synth, oracle_mod, g, n=5_000, seed=3)
    # one column alone equals its all-flavour column
    x, q2 = queries(g, 3000, 4)
    allf = P.xfxq2_all_flavours(G, dev(x), dev(q2)).cpu().numpy()
    assert np.array_equal(P.xfxq2(G, 64, dev(x), dev(q2)).cpu().numpy(), allf[:, 63], equal_nan=True)


def test_smallest_grid_and_a_two_knot_subgrid(synth, oracle_mod):
    pids = [-1, 21, 1]
    g = synth.make_grid([1e-4, 1.0], [[2.0, 50.0]], pids, params=synth.flavour_params(3, 33))
    check(synth, oracle_mod, g, n=5_000, seed=5)
    g = synth.make_grid(np.geomspace(1e-5, 1.0, 30), [np.geomspace(2.0, 4.0, 6), [4.0, 9.0],
                                                      np.geomspace(9.0, 1e5, 10)], pids,
                        params=synth.flavour_params(3, 34))
    check(synth, oracle_mod, g, n=5_000, seed=6)


def test_a_cell_wider_than_2_to_the_100_takes_the_fp64_positions(synth, oracle_mod):
    """In-grid positions are taken in float-float from the knots' binary
    exponents and significands, which needs the exponent difference across a
    cell exact in floats; a grid with a cell spanning 2^100 or more (here Q^2
    from 10 to 1e33) takes the FP64 logarithm for them instead, and must give
    the same parity."""
    pids = [-1, 21, 1]
    g = synth.make_grid(np.geomspace(1e-5, 1.0, 20), [[1.0, 10.0, 1e33]], pids, params=synth.flavour_params(3, 35))
    check(synth, oracle_mod, g, n=5_000, seed=7)
