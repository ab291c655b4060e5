"""The native LHAPDF6 (lhagrid1) reader on the host: synthetic sets written in
the text format read back exactly, and malformed files are refused with a
message naming the problem.  PDFFlow Sec. 2.2 (LHAPDF files read directly)
and Sec. 2.3 (alpha_s nodes from the metadata).  The device-side load is
checked in tests/test_gpu_lhapdf.py."""
import numpy as np
import pytest

P = pytest.importorskip("paper_2009_06635_gb300")


def expected(g):
    """What the reader must return for grid g: Q^2 knots as sqrt(Q^2)^2."""
    q = np.sqrt(np.asarray(g.q2_knots))
    aq = np.sqrt(np.asarray(g.as_q2))
    return q * q, aq * aq


@pytest.mark.parametrize("which", ["single", "full"])
def test_round_trip_is_exact(tmp_path, synth, which):
    g = synth.grid_single_subgrid() if which == "single" else synth.grid_full()
    paths = synth.write_lhapdf(g, tmp_path / f"SYN_{which}")
    info = tmp_path / f"SYN_{which}" / f"SYN_{which}.info"
    r = P.read_lhapdf(info, paths[0])
    q2, aq2 = expected(g)
    assert np.array_equal(r["x_knots"], g.x_knots)
    assert r["nq"] == list(g.nq)
    assert np.array_equal(r["q2_knots"], q2)
    assert r["pids"] == list(g.pids)
    assert np.array_equal(r["values"], g.values)
    assert np.array_equal(r["as_q2"], aq2) and np.array_equal(r["as_vals"], g.as_vals)


def test_members_and_short_precision(tmp_path, synth):
    g0, vals = synth.grid_members(3)
    paths = synth.write_lhapdf(g0, tmp_path / "MEM", member_values=vals, digits=9)
    assert len(paths) == 3
    info = tmp_path / "MEM" / "MEM.info"
    for m in range(3):
        r = P.read_lhapdf(info, paths[m])
        # 9 significant digits, as many published sets carry
        assert np.allclose(r["values"], vals[m], rtol=1e-8, atol=0)


def write(path, text):
    path.write_text(text)
    return path


def test_malformed_files_are_refused(tmp_path, synth):
    g = synth.grid_single_subgrid()
    paths = synth.write_lhapdf(g, tmp_path / "OK")
    info = tmp_path / "OK" / "OK.info"
    good = open(paths[0]).read()
    lines = good.splitlines()
    cases = {
        "no separator": "PdfType: central\nFormat: lhagrid1\n",
        "short value line": "\n".join(lines[:10] + [" ".join(lines[10].split()[:-1])] + lines[11:]) + "\n",
        "bad number": "\n".join(lines[:6] + ["1.0 abc 2.0"] + lines[7:]) + "\n",
        "unclosed block": "\n".join(lines[:-1]) + "\n",
        "non-integer pid": "\n".join(lines[:5] + [lines[5].replace("21", "21.5")] + lines[6:]) + "\n",
        "pid out of int range": "\n".join(lines[:5] + [lines[5].replace("21", "1e300")] + lines[6:]) + "\n",
    }
    for what, text in cases.items():
        bad = write(tmp_path / "bad.dat", text)
        with pytest.raises(P.PdfError):
            P.read_lhapdf(info, bad)
    # metadata that contradicts the data, or an alpha_s list cut short
    txt = info.read_text()
    bad_info = write(tmp_path / "bad.info", txt.replace("Flavors: [-5", "Flavors: [-6"))
    with pytest.raises(P.PdfError, match="Flavors"):
        P.read_lhapdf(bad_info, paths[0])
    cut = txt.split("AlphaS_Vals: [")[0] + "AlphaS_Vals: [0.1, 0.2]\n"
    with pytest.raises(P.PdfError, match="AlphaS"):
        P.read_lhapdf(write(tmp_path / "cut.info", cut), paths[0])
    with pytest.raises(P.PdfError, match="cannot read"):
        P.read_lhapdf(tmp_path / "missing.info", paths[0])
    # a set without alpha_s metadata reads, with no nodes
    noas = "\n".join(l for l in txt.splitlines() if not l.startswith(("AlphaS", "  "))) + "\n"
    r = P.read_lhapdf(write(tmp_path / "noas.info", noas), paths[0])
    assert len(r["as_q2"]) == 0


def test_comments_and_subgrids_with_other_x_knots(tmp_path, synth):
    g = synth.grid_full()
    paths = synth.write_lhapdf(g, tmp_path / "FULL")
    info = tmp_path / "FULL" / "FULL.info"
    txt = info.read_text().replace("Flavors:", "# a comment line\nFlavors:") + "Extra: [1, 2]  # ignored\n"
    r = P.read_lhapdf(write(tmp_path / "c.info", txt), paths[0])
    assert r["pids"] == list(g.pids)
    # change the x knots of the second subgrid block: refused
    lines = open(paths[0]).read().splitlines()
    seps = [i for i, l in enumerate(lines) if l.strip() == "---"]
    k = seps[1] + 1  # first line of the second block
    xs = lines[k].split()
    xs[3] = repr(float(xs[3]) * 1.0001)
    lines[k] = " ".join(xs)
    with pytest.raises(P.PdfError, match="different x knots"):
        P.read_lhapdf(info, write(tmp_path / "x.dat", "\n".join(lines) + "\n"))


def test_member_range_is_checked_before_any_file_or_device_work(tmp_path):
    """Member files carry four-digit numbers: a range leaving 0..9999 (or one
    whose end overflows an int) is refused with PDF_ERR_ARG before the set
    directory is even opened."""
    import ctypes
    from paper_2009_06635_gb300 import _native
    lib = _native.load()
    h = ctypes.c_void_p(None)
    for first, nmem in ((9999, 2), (-1, 1), (0, 0), (5, 2**31 - 1), (2**31 - 1, 1)):
        rc = lib.pdf_load_lhapdf(str(tmp_path / "NOSET").encode(), first, nmem, ctypes.byref(h))
        assert rc == -6, (first, nmem, rc)
        assert "outside 0..9999" in _native.last_error()
        assert h.value is None
