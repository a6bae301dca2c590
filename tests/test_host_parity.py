"""Host-side parity of libhm with the oracle (no GPU needed).

* Cluster tree and block tree: integer / index work, bit-exact.
* Codec encoders: the packed bytes of hm_codec_encode equal the oracle's codes
  bit for bit (AFLP, FPX, raw) on seeded inputs with zeros, signs, ties and
  wide dynamic ranges.
"""
import numpy as np
import pytest

import synth
from oracle import codec as ocd
from oracle import trees


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    return _hm


def _oracle_structure(pts, leaf, eta):
    ct = trees.build_cluster_tree(pts, leaf)
    bl = trees.build_block_tree(ct, eta)
    cl = np.array([[c.start, c.end, c.level, c.parent] for c in ct.clusters])
    b = np.array([[x.row, x.col, int(x.adm)] for x in bl])
    return ct.perm, cl, b


@pytest.mark.parametrize("case", ["sphere2048", "sphere5000", "cube3000", "dupes", "lattice"])
def test_trees_bit_exact(hm, case):
    if case == "sphere2048":
        pts, leaf, kern = synth.sphere_points(2048), 32, "laplace"
    elif case == "sphere5000":
        pts, leaf, kern = synth.sphere_points(5000), 64, "laplace"
    elif case == "cube3000":
        pts, leaf, kern = synth.cube_points(3000), 64, "matern"
    elif case == "lattice":                 # 9 x 9 x 9 grid: points lie on the bisection midpoints
        g = np.arange(9, dtype=np.float64) / 8.0
        pts = np.ascontiguousarray(np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3))
        leaf, kern = 8, "matern"
    else:                                   # repeated points force the degenerate split
        base = synth.cube_points(50)
        pts, leaf, kern = np.ascontiguousarray(np.repeat(base, 7, axis=0)), 4, "matern"
    h = hm.hm_build(pts, kern, leaf, 2.0, "h", 1e-4)
    try:
        perm, cl, bl, rk = hm.hm_structure(h)
    finally:
        hm.hm_free(h)
    operm, ocl, obl = _oracle_structure(pts, leaf, 2.0)
    assert np.array_equal(perm, operm)
    assert np.array_equal(cl, ocl)
    assert np.array_equal(bl, obl)
    assert np.all((rk >= 0) == (bl[:, 2] == 1))


@pytest.mark.parametrize("adm", ["hodlr", "blr"])
def test_trees_bit_exact_other_admissibility(hm, adm):
    pts = synth.sphere_points(2048)
    h = hm.hm_build(pts, "laplace", 32, 2.0, "h", 1e-4, adm=adm)
    try:
        perm, cl, bl, rk = hm.hm_structure(h)
    finally:
        hm.hm_free(h)
    ct = trees.build_cluster_tree(pts, 32)
    ob = trees.build_block_tree(ct, 2.0, adm)
    assert np.array_equal(bl, np.array([[x.row, x.col, int(x.adm)] for x in ob]))
    assert np.all((rk >= 0) == (bl[:, 2] == 1))


def _cases():
    out = []
    for seed in range(6):
        for dr in (1.0, 3.0, 1e2, 1e5, 1e12):
            out.append(synth.codec_values(257, dr, zero_frac=0.05, seed=100 + seed + int(np.log10(dr + 1))))
    out.append(np.zeros(17))
    out.append(np.array([-0.0, 0.0, 1.0, -1.0]))
    out.append(np.array([1.0, 16.0 - 2.0 ** -20]))
    out.append(np.array([1.0, 3e40, -2.0]))                 # forces FPX e11 promotion
    out.append(np.array([1e-300, 1e-200, 5e-324, -7.0]))    # AFLP s overflows: raw FP64
    out.append(np.array([1.0, -np.finfo(np.float64).max]))   # AFLP s / FPX e11 round to 2^1024
    return out


@pytest.mark.parametrize("codec", ["aflp", "fpx", "none"])
def test_codec_encode_bit_exact(hm, codec):
    keys = [1, 5, 8, 9, 14, 20, 23, 24, 27, 33, 40, 47, 52] if codec != "none" else [52]
    for v in _cases():
        for key in keys:
            packed, hdr = hm.hm_codec_encode(v, codec, key)
            c = ocd.compress(v, codec, key)
            B = c["B"]
            assert hdr["B"] == B
            codes = np.zeros(v.size, dtype=np.uint64)
            for b in range(B):
                codes |= packed[b::B].astype(np.uint64) << np.uint64(8 * b)
            assert np.array_equal(codes, c["codes"].astype(np.uint64)), (codec, key, v[:4])
            if codec == "aflp":
                if c["raw"]:
                    assert hdr["fmt"] == 3
                else:
                    assert (hdr["fmt"], hdr["e"], hdr["m"]) == (2, c["e"], c["mp"])
                    assert hdr["vmin"] == c["vmin"]
            elif codec == "fpx":
                assert hdr["fmt"] == (0 if c["e"] == 8 else 1) and hdr["m"] == c["m"]
