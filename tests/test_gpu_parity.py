"""GPU parity of libhm against the CPU oracle (through the C ABI).

* K0 decode: bit-exact with the oracle's decoder for every codec and width.
* Products: y := alpha*M*x + beta*y for H, UH, H^2 at N = 2048 (several
  tiles, ragged leaves) within 4*eps relative of the oracle's uncompressed
  FP64 product -- the stated accuracy of the compressed product -- and, at the benchmark's full
  size (N = 131072), on sampled rows of the exact dense product.
* Determinism (no atomics), host path, beta = 0, multi-RHS, error word.
"""
import json

import numpy as np
import pytest

import synth
from oracle import codec as ocd
from oracle import hmatrix, kernels, matvec, nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ K0 decode
@pytest.mark.parametrize("codec", ["aflp", "fpx", "none"])
def test_decode_bit_exact(hm, codec):
    keys = [1, 6, 9, 14, 20, 23, 27, 33, 44, 52] if codec != "none" else [52]
    for seed in range(4):
        for dr in (1.0, 1e2, 1e6, 1e15):
            v = synth.codec_values(3001, dr, zero_frac=0.03, seed=500 + seed)
            for key in keys:
                packed, hdr = hm.hm_codec_encode(v, codec, key)
                d_in = torch.from_numpy(packed).cuda()
                d_out = torch.empty(v.size, dtype=torch.float64, device="cuda")
                hm.hm_codec_decode(d_in.data_ptr(), v.size, hdr, d_out.data_ptr())
                torch.cuda.synchronize()
                got = d_out.cpu().numpy()
                want = ocd.decompress(ocd.compress(v, codec, key))
                assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (codec, key, dr)


# ------------------------------------------------------------------ products at N = 2048
N = 2048


@pytest.fixture(scope="module")
def problem():
    pts = synth.sphere_points(N)
    x = synth.rhs(N, 3)
    y0 = synth.rhs(N, 3, seed=77)
    return pts, x, y0


_oracle_cache = {}


def oracle_ref(pts, fmt, eps, x, alpha, y0, beta):
    key = (fmt, eps)
    if key not in _oracle_cache:
        h = hmatrix.build_h(pts, "laplace", 32, 2.0, eps)
        m = h if fmt == "h" else (nested.build_uniform(h) if fmt == "uh" else nested.build_h2(h))
        _oracle_cache[key] = m
    m = _oracle_cache[key]
    f = {"h": matvec.h_mvm, "uh": matvec.uh_mvm, "h2": matvec.h2_mvm}[fmt]
    return f(m, alpha, x, beta, y0)


def run_gpu(hm, pts, fmt, eps, codec, x, alpha, y0, beta, valr=True):
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, codec, valr)
        xd = torch.from_numpy(np.asfortranarray(x)).cuda()
        yd = torch.from_numpy(np.asfortranarray(y0)).cuda()
        xd = xd.t().contiguous().t() if xd.dim() == 2 else xd
        yd = yd.t().contiguous().t() if yd.dim() == 2 else yd
        M.matvec(alpha, xd, beta, yd)
        torch.cuda.synchronize()
        assert M.sync_status() == 0
        return yd.cpu().numpy(), M.info()
    finally:
        M.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("codec", ["none", "aflp", "fpx"])
def test_h_matvec_within_4eps(hm, problem, eps, codec):
    pts, x, y0 = problem
    ref = oracle_ref(pts, "h", eps, x[:, 0], 1.0, y0[:, 0], 1.0)
    got, info = run_gpu(hm, pts, "h", eps, codec, x[:, 0], 1.0, y0[:, 0], 1.0)
    assert rel(got, ref) <= 4 * eps
    if codec != "none":
        assert info["bytes_values"] < info["bytes_fp64"] / 2


@pytest.mark.parametrize("fmt", ["uh", "h2"])
@pytest.mark.parametrize("eps,codec", [(1e-6, "aflp"), (1e-6, "fpx"), (1e-6, "none"), (1e-8, "aflp"),
                                       (1e-4, "fpx")])
def test_uh_h2_matvec_within_4eps(hm, problem, fmt, eps, codec):
    pts, x, y0 = problem
    ref = oracle_ref(pts, fmt, eps, x[:, 0], 1.0, y0[:, 0], 1.0)
    got, _ = run_gpu(hm, pts, fmt, eps, codec, x[:, 0], 1.0, y0[:, 0], 1.0)
    assert rel(got, ref) <= 4 * eps


def test_alpha_beta_multi_rhs(hm, problem):
    pts, x, y0 = problem
    eps = 1e-6
    ref = oracle_ref(pts, "h", eps, x, 0.7, y0, -0.3)
    got, _ = run_gpu(hm, pts, "h", eps, "aflp", x, 0.7, y0, -0.3)
    for r in range(3):
        assert rel(got[:, r], ref[:, r]) <= 4 * eps


def test_beta_zero_ignores_y(hm, problem):
    pts, x, _ = problem
    eps = 1e-6
    y0 = np.full(N, np.nan)
    ref = oracle_ref(pts, "h", eps, x[:, 0], 1.0, np.zeros(N), 0.0)
    got, _ = run_gpu(hm, pts, "h", eps, "fpx", x[:, 0], 1.0, y0, 0.0)
    assert np.all(np.isfinite(got))
    assert rel(got, ref) <= 4 * eps


def test_compressed_matches_oracle_compressed_product(hm, problem):
    """Same eps and codec on both sides: the two compressed products agree to ~eps."""
    from oracle import compress
    pts, x, y0 = problem
    eps = 1e-6
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, eps)
    ref = matvec.h_mvm(compress.compress_h(h, "aflp"), 1.0, x[:, 0], 1.0, y0[:, 0])
    got, _ = run_gpu(hm, pts, "h", eps, "aflp", x[:, 0], 1.0, y0[:, 0], 1.0)
    assert rel(got, ref) <= 4 * eps


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
def test_deterministic_and_host_path(hm, problem, fmt):
    pts, x, y0 = problem
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, 1e-6)
    try:
        M.compress(1e-6, "aflp")
        xd = torch.from_numpy(x[:, 0].copy()).cuda()
        outs = []
        for _ in range(20):
            yd = torch.from_numpy(y0[:, 0].copy()).cuda()
            M.matvec(1.0, xd, 1.0, yd)
            outs.append(yd.cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))
        yh = np.asfortranarray(y0[:, 0].copy())
        M.matvec_host(1.0, np.asfortranarray(x[:, 0]), 1.0, yh)
        assert np.array_equal(yh.view(np.uint64), outs[0].view(np.uint64))
        assert M.sync_status() == 0
    finally:
        M.close()


@pytest.mark.parametrize("fmt", ["h", "h2"])
def test_graph_replay_bitwise(hm, problem, fmt):
    """CUDA-graph replay equals direct launches bit for bit; new arguments re-capture."""
    pts, x, y0 = problem
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, 1e-6)
    try:
        M.compress(1e-6, "aflp")
        xd = torch.from_numpy(x[:, 0].copy()).cuda()
        ya = torch.from_numpy(y0[:, 0].copy()).cuda()
        M.matvec(0.5, xd, 1.0, ya)
        M.graph(True)
        for alpha in (0.5, 0.5, 2.0):
            yb = torch.from_numpy(y0[:, 0].copy()).cuda()
            M.matvec(alpha, xd, 1.0, yb)
            yb = yb.cpu().numpy()
            if alpha == 0.5:
                assert np.array_equal(yb.view(np.uint64), ya.cpu().numpy().view(np.uint64))
        ref = oracle_ref(pts, fmt, 1e-6, x[:, 0], 2.0, y0[:, 0], 1.0)
        assert rel(yb, ref) <= 4e-6
    finally:
        M.close()


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
def test_launch_shapes_and_autotune(hm, problem, fmt):
    """Every launch shape (warps x stages per warp, with its own split of the
    work into warp ranges) gives a product within 4 eps of the oracle and is
    bitwise reproducible; the autotuner keeps one of them per launch."""
    pts, x, y0 = problem
    eps = 1e-6
    ref = oracle_ref(pts, fmt, eps, x[:, 0], 1.0, y0[:, 0], 1.0)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp")
        xd = torch.from_numpy(x[:, 0].copy()).cuda()
        for shape in range(hm.NSHAPES):
            M.set_launch_shapes(shape)
            outs = []
            for _ in range(3):
                yd = torch.from_numpy(y0[:, 0].copy()).cuda()
                M.matvec(1.0, xd, 1.0, yd)
                outs.append(yd.cpu().numpy())
            assert rel(outs[0], ref) <= 4 * eps
            for o in outs[1:]:
                assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))
        M.autotune(2)
        shapes = M.launch_shapes()
        assert len(shapes) == M.info()["nlaunches"]
        assert all(s in (-1, 0, 1, 2) for s in shapes) and any(s >= 0 for s in shapes)
        yd = torch.from_numpy(y0[:, 0].copy()).cuda()
        M.matvec(1.0, xd, 1.0, yd)
        assert rel(yd.cpu().numpy(), ref) <= 4 * eps
        assert M.sync_status() == 0
    finally:
        M.close()


def test_tuning_record_cache(hm, problem, tmp_path):
    """The autotuner's choices (launch shapes, launch mode, multi-RHS engine) round
    trip through a tuning record: a cache file written by one matrix is applied to
    an identical one without timing, a record of another launch program or with a
    value out of range is refused and leaves the settings as they were."""
    pts, x, y0 = problem
    eps = 1e-6
    ref = oracle_ref(pts, "h", eps, x[:, 0], 1.0, y0[:, 0], 1.0)
    cache = tmp_path / "tuning.json"
    A = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    B = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    U = hm.HMatrix(pts, "laplace", 32, 2.0, "uh", eps)
    try:
        for M in (A, B, U):
            M.compress(eps, "aflp")
        A.autotune(2, cache=str(cache))
        rec = A.tuning()
        nl = A.info()["nlaunches"]
        assert len(rec) == 7 + nl and rec[4] == nl
        assert all(rec[5 + i] == s for i, s in enumerate(A.launch_shapes()) if s >= 0)
        assert rec[5 + nl] == A.persistent_mode() and rec[6 + nl] == A.multi_rhs_engine()
        assert len(json.loads(cache.read_text())) == 1
        # B differs from A's record before, and takes it from the cache without timing
        B.set_launch_shapes((rec[5] + 1) % hm.NSHAPES)
        B.autotune(2, cache=str(cache))
        assert B.tuning() == rec
        assert len(json.loads(cache.read_text())) == 1
        xd = torch.from_numpy(x[:, 0].copy()).cuda()
        yd = torch.from_numpy(y0[:, 0].copy()).cuda()
        B.matvec(1.0, xd, 1.0, yd)
        assert rel(yd.cpu().numpy(), ref) <= 4 * eps
        # another launch program (UH) refuses A's record; bad values are refused
        before = U.tuning()
        assert not U.set_tuning(rec)
        bad = list(rec)
        bad[5] = 7
        assert not B.set_tuning(bad) and not B.set_tuning(rec[:-1]) and not B.set_tuning(bad[:4])
        bad = list(rec)
        bad[6 + nl] = 2
        assert not B.set_tuning(bad)
        assert U.tuning() == before and B.tuning() == rec
        # a second program adds its own record to the same file
        U.autotune(2, cache=str(cache))
        assert len(json.loads(cache.read_text())) == 2
        assert B.sync_status() == 0 and U.sync_status() == 0
    finally:
        for M in (A, B, U):
            M.close()


@pytest.mark.parametrize("fmt", ["h", "uh", "h2", "uh_sep"])
@pytest.mark.parametrize("eps", [1e-6, 1e-8])
def test_persistent_launch_equals_per_launch(hm, problem, fmt, eps):
    """The persistent forms -- runs of row-chunk launches as one dataflow launch
    (mode 1), and the whole product, forward, coupling and backward passes
    included, as ONE cooperative launch with grid barriers between its phases
    (mode 2) -- give the per-launch result bit for bit (same warp ranges of
    shape 0, same order of every sum), within 4 eps of the oracle, also
    replayed from a CUDA graph."""
    pts, x, y0 = problem
    ref = oracle_ref(pts, "uh" if fmt == "uh_sep" else fmt, eps, x[:, 0], 0.75, y0[:, 0], -0.5)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp")
        M.set_launch_shapes(0)
        xd = torch.from_numpy(x[:, 0].copy()).cuda()
        outs = []
        for persistent, graph in ((0, False), (1, False), (1, True), (1, True), (2, False), (2, True), (2, True),
                                  (0, False)):
            M.persistent(persistent)
            M.graph(graph)
            yd = torch.from_numpy(y0[:, 0].copy()).cuda()
            M.matvec(0.75, xd, -0.5, yd)
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
        assert M.sync_status() == 0
        assert rel(outs[0], ref) <= 4 * eps
        for o in outs[1:]:
            assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))
    finally:
        M.close()


def test_matern_cube(hm):
    pts = synth.cube_points(3000)
    x = synth.rhs(3000)[:, 0]
    eps = 1e-6
    h = hmatrix.build_h(pts, "matern", 64, 2.0, eps)
    ref = matvec.h_mvm(h, 1.0, x)
    M = hm.HMatrix(pts, "matern", 64, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp")
        xd = torch.from_numpy(x.copy()).cuda()
        yd = torch.zeros(3000, dtype=torch.float64, device="cuda")
        M.matvec(1.0, xd, 0.0, yd)
        assert rel(yd.cpu().numpy(), ref) <= 4 * eps
    finally:
        M.close()


# ------------------------------------------------------------------ full size, sampled rows
@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
def test_full_size_sampled_rows(hm, fmt):
    """N = 131072 sphere, eps = 1e-6, AFLP: 256 sampled rows against the exact dense rows.

    Each sampled output is the plain definition sum_j a_ij x_j (oracle kernels),
    computed row by row.  The H approximation differs from the exact matrix by
    about eps relative (per block), so the bound is 4 eps on the sampled rows.
    """
    n, eps = 131072, 1e-6
    pts = synth.sphere_points(n)
    x = synth.rhs(n)[:, 0]
    M = hm.HMatrix(pts, "laplace", 64, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp")
        xd = torch.from_numpy(x.copy()).cuda()
        yd = torch.zeros(n, dtype=torch.float64, device="cuda")
        M.matvec(1.0, xd, 0.0, yd)
        y = yd.cpu().numpy()
        assert M.sync_status() == 0
    finally:
        M.close()
    rows = np.random.default_rng(5).choice(n, 256, replace=False)
    param = kernels.default_param("laplace", n)
    ye = np.array([kernels.entries("laplace", pts, np.array([i]), np.arange(n), param)[0] @ x for i in rows])
    assert rel(y[rows], ye) <= 4 * eps
