"""Sets loaded from LHAPDF6 text files (pdf_load_lhapdf) evaluate exactly as
the same values loaded from memory (pdf_load_grid), for one member and for a
member set.  PDFFlow Sec. 2.2, Sec. 4.3."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_single_member_matches_the_in_memory_load(tmp_path, synth):
    g = synth.grid_full()
    synth.write_lhapdf(g, tmp_path / "SYN")
    G = P.pdf_load_lhapdf(tmp_path / "SYN")
    q = np.sqrt(g.q2_knots)
    aq = np.sqrt(g.as_q2)
    ref = P.pdf_load_grid(x_knots=g.x_knots, nq=g.nq, q2_knots=q * q, pids=g.pids, values=g.values,
                          as_q2=aq * aq, as_vals=g.as_vals)
    x, q2 = synth.queries_full(50_000, 51)
    a, al = P.xfxq2_all_flavours_alphas(G, dev(x), dev(q2))
    b, bl = P.xfxq2_all_flavours_alphas(ref, dev(x), dev(q2))
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy(), equal_nan=True)
    assert np.array_equal(al.cpu().numpy(), bl.cpu().numpy(), equal_nan=True)
    assert G.pids == list(g.pids) and G.nx == len(g.x_knots)


def test_member_set_matches_the_in_memory_load(tmp_path, synth):
    g0, vals = synth.grid_members(4)
    synth.write_lhapdf(g0, tmp_path / "MEM", member_values=vals)
    G = P.pdf_load_lhapdf(tmp_path / "MEM", member=1, nmem=3)
    q = np.sqrt(g0.q2_knots)
    ref = P.pdf_load_grid(x_knots=g0.x_knots, nq=g0.nq, q2_knots=q * q, pids=g0.pids, values=vals[1],
                          member_values=vals[1:4])
    x, q2 = synth.fit_points()
    a = P.xfxq2_all_members(G, dev(x), dev(q2)).cpu().numpy()
    b = P.xfxq2_all_members(ref, dev(x), dev(q2)).cpu().numpy()
    assert a.shape == (3, len(x), g0.nflav)
    assert np.array_equal(a, b, equal_nan=True)
    with pytest.raises(P.PdfError):
        P.pdf_load_lhapdf(tmp_path / "MEM", member=2, nmem=3)  # member 4 does not exist
