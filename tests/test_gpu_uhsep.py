"""UH with separate row and column coupling matrices (HM_FMT_UH_SEP, the variant
discussed after Alg. 5) on the GPU against the oracle's form of the same
variant: product and adjoint within 4 eps for AFLP and FPX, several
right-hand sides through the multi-RHS panels, and equality (to rounding) with
the single-coupling UH product of the same bases."""
import numpy as np
import pytest

import synth
from oracle import hmatrix, matvec, nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N = 2048
EPS = 1e-6


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


@pytest.fixture(scope="module")
def oracle():
    h = hmatrix.build_h(synth.sphere_points(N), "laplace", 32, 2.0, EPS)
    return nested.build_uniform_sep(h)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cols(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda().t().contiguous().t()


@pytest.mark.parametrize("codec", ["aflp", "fpx"])
def test_uhsep_product_and_adjoint(hm, oracle, codec):
    pts = synth.sphere_points(N)
    x = synth.rhs(N, 1, seed=91)[:, 0]
    y0 = synth.rhs(N, 1, seed=92)[:, 0]
    ref = matvec.uhsep_mvm(oracle, 0.5, x, -1.0, y0)
    refa = matvec.uhsep_mvm(oracle, 0.5, x, -1.0, y0, adjoint=True)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "uh_sep", EPS)
    try:
        M.compress(EPS, codec)
        xd = torch.from_numpy(x.copy()).cuda()
        outs = []
        for _ in range(2):
            yd = torch.from_numpy(y0.copy()).cuda()
            M.matvec(0.5, xd, -1.0, yd)
            outs.append(yd.cpu().numpy())
        ya = torch.from_numpy(y0.copy()).cuda()
        M.matvec(0.5, xd, -1.0, ya, adjoint=True)
        assert M.sync_status() == 0
        assert rel(outs[0], ref) <= 4 * EPS
        assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
        assert rel(ya.cpu().numpy(), refa) <= 4 * EPS
    finally:
        M.close()


def test_uhsep_multi_rhs_and_single_coupling(hm, oracle):
    pts = synth.sphere_points(N)
    r = 19
    x = synth.rhs(N, r, seed=93)
    ref = matvec.uhsep_mvm(oracle, 1.0, x, 0.0)
    outs = {}
    for fmt in ("uh_sep", "uh"):
        M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, EPS)
        try:
            M.compress(EPS, "none")   # uncompressed factors: the two forms agree to rounding
            yd = cols(np.zeros_like(x))
            M.matvec(1.0, cols(x), 0.0, yd)
            outs[fmt] = yd.cpu().numpy()
            assert M.sync_status() == 0
        finally:
            M.close()
    for k in range(r):
        assert rel(outs["uh_sep"][:, k], ref[:, k]) <= 4 * EPS, k
    assert rel(outs["uh_sep"], outs["uh"]) <= 1e-11
