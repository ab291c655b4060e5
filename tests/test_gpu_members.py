"""Member sets (PDFFlow Sec. 4.3, multi-member evaluation): every member of a
set sharing the knots, evaluated in one launch, against the oracle member by
member."""
import numpy as np
import pytest
import torch

from parity import RTOL_FP64, assert_parity

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_members_match_oracle_member_by_member(synth, oracle_mod):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    g0, vals = synth.grid_members(5)
    G = P.pdf_load_grid(g0, member_values=vals)
    assert G.nmem == 5
    x, q2 = synth.queries_full(20_001, 33)
    xf, qf = synth.fit_points()
    x, q2 = np.concatenate([x, xf]), np.concatenate([q2, qf])
    out = P.xfxq2_all_members(G, dev(x), dev(q2)).cpu().numpy()
    for m in range(5):
        og = oracle_mod.OracleGrid(x_knots=g0.x_knots, nq=g0.nq, q2_knots=g0.q2_knots, values=vals[m])
        v, s, fl = og.xfxq2(x, q2)
        assert_parity(out[m], v, s, fl, RTOL_FP64, f"member {m}")
    # the single-member calls evaluate member 0, bit for bit
    one = P.xfxq2_all_flavours(G, dev(x), dev(q2)).cpu().numpy()
    assert np.array_equal(one, out[0], equal_nan=True)


def test_one_member_set_takes_the_points_kernel(synth, oracle_mod):
    """A set of one member evaluated as a member set gives the bits of the
    all-flavour call on the same grid (it runs the points kernel), and the
    oracle's values."""
    torch.cuda.set_device(0)
    g0, vals = synth.grid_members(1)
    G = P.pdf_load_grid(g0, member_values=vals)
    assert G.nmem == 1
    x, q2 = synth.queries_full(30_011, 34)
    out = P.xfxq2_all_members(G, dev(x), dev(q2)).cpu().numpy()
    assert out.shape == (1, len(x), g0.nflav)
    one = P.xfxq2_all_flavours(G, dev(x), dev(q2)).cpu().numpy()
    assert np.array_equal(one, out[0], equal_nan=True)
    og = oracle_mod.OracleGrid(x_knots=g0.x_knots, nq=g0.nq, q2_knots=g0.q2_knots, values=vals[0])
    v, s, fl = og.xfxq2(x, q2)
    assert_parity(out[0], v, s, fl, RTOL_FP64, "one member")
