"""hm_save / hm_load: the built matrix written to a file and read back.

Host part (no GPU): an uncompressed matrix of every format survives the round
trip -- the same cluster and block trees (hm_structure), the same sizes
(hm_info), and saving the loaded matrix gives the same bytes again; damaged
files (truncated, wrong magic, trailing bytes, an index out of range) are
refused with HM_ERR_IO.  GPU part: a compressed matrix is loaded, compressed
again with its saved settings, and gives the saved matrix's product bit for bit.
"""
import os

import numpy as np
import pytest

import synth

N = 600


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


def _same_structure(hm, a, b):
    sa, sb = hm.hm_structure(a.h), hm.hm_structure(b.h)
    for k in range(len(sa)):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k]))
    ia, ib = a.info(), b.info()
    for k in ("n", "format", "nclusters", "nleaves", "nblocks", "nlowrank", "ndense", "depth", "max_rank"):
        assert ia[k] == ib[k], k


@pytest.mark.parametrize("fmt", ["h", "uh", "h2", "uh_sep"])
def test_round_trip_host(hm, tmp_path, fmt):
    M = hm.HMatrix(synth.sphere_points(N), "laplace", 32, 2.0, fmt, 1e-6)
    p1, p2 = str(tmp_path / "a.hm"), str(tmp_path / "b.hm")
    try:
        M.save(p1)
        L = hm.HMatrix.load(p1)
        try:
            _same_structure(hm, M, L)
            L.save(p2)
            assert open(p1, "rb").read() == open(p2, "rb").read()
        finally:
            L.close()
    finally:
        M.close()


def test_damaged_files_refused(hm, tmp_path):
    M = hm.HMatrix(synth.cube_points(N), "matern", 32, 2.0, "h", 1e-4)
    p = str(tmp_path / "m.hm")
    try:
        M.save(p)
    finally:
        M.close()
    good = open(p, "rb").read()
    cases = {"trunc": good[: len(good) // 2], "magic": b"XMAT" + good[4:], "tail": good + b"\0" * 8,
             "empty": b"", "version": good[:4] + b"\x63" + good[5:]}
    for name, data in cases.items():
        q = str(tmp_path / f"{name}.hm")
        open(q, "wb").write(data)
        with pytest.raises(hm.HMError, match="I/O"):
            hm.hm_load(q)
    with pytest.raises(hm.HMError, match="I/O"):
        hm.hm_load(str(tmp_path / "does-not-exist.hm"))
    with pytest.raises(hm.HMError, match="I/O"):
        hm.HMatrix(synth.cube_points(64), "matern", 32, 2.0, "h", 1e-4).save(str(tmp_path / "no" / "dir.hm"))


def test_block_index_out_of_range_refused(hm, tmp_path):
    """A block whose row cluster index is past the tree: refused, not packed."""
    M = hm.HMatrix(synth.sphere_points(256), "laplace", 32, 2.0, "h", 1e-6)
    p = str(tmp_path / "m.hm")
    try:
        M.save(p)
        nc = M.info()["nclusters"]
        nb = M.info()["nblocks"]
    finally:
        M.close()
    data = bytearray(open(p, "rb").read())
    # the blocks array is (row int32, col int32, adm bool) x nb, 12 bytes each with
    # padding, preceded by its uint64 count: find it by the count and the size
    rec = 12
    pat = int(nb).to_bytes(8, "little")
    at = [i for i in range(len(data) - 8) if data[i:i + 8] == pat]
    hit = False
    for i in at:
        first = int.from_bytes(data[i + 8:i + 12], "little")
        if 0 <= first < nc and i + 8 + rec * nb <= len(data):
            bad = bytearray(data)
            bad[i + 8:i + 12] = (nc + 5).to_bytes(4, "little")
            q = str(tmp_path / "bad.hm")
            open(q, "wb").write(bytes(bad))
            try:
                h = hm.hm_load(q)
            except hm.HMError as e:
                assert "I/O" in str(e)
                hit = True
                break
            hm.hm_free(h)
    assert hit


@pytest.mark.gpu
@pytest.mark.parametrize("fmt,codec,eps", [("h", "aflp", 1e-6), ("h2", "fpx", 1e-8), ("uh", "aflp", 1e-4)])
def test_loaded_product_bitwise(hm, tmp_path, fmt, codec, eps):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    n = 2048
    M = hm.HMatrix(synth.sphere_points(n), "laplace", 32, 2.0, fmt, eps)
    p = str(tmp_path / "c.hm")
    x = torch.from_numpy(synth.rhs(n)[:, 0].copy()).cuda()
    try:
        M.compress(eps, codec, True)
        M.save(p)
        y0 = torch.zeros(n, dtype=torch.float64, device="cuda")
        M.matvec(1.0, x, 0.0, y0)
        torch.cuda.synchronize()
    finally:
        M.close()
    L = hm.HMatrix.load(p)
    try:
        assert L.info()["codec"] == hm.CODECS[codec] and L.info()["eps"] == eps
        y1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        L.matvec(1.0, x, 0.0, y1)
        torch.cuda.synchronize()
        assert L.sync_status() == 0
        assert np.array_equal(y0.cpu().numpy().view(np.uint64), y1.cpu().numpy().view(np.uint64))
    finally:
        L.close()
    os.remove(p)
