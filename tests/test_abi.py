"""The C-ABI library builds, loads and exports every entry point include/hm.h declares.

No GPU work is done here (CPU-only checks).
"""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_03456_gb300 import build, hm
    build.build()
    return hm.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    from paper_2405_03456_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(hm_[a-z_0-9]+)", out))
    decl = declared_symbols()
    assert len(decl) >= 11
    assert set(decl) <= exported, set(decl) - exported
    for name in decl:
        assert hasattr(lib, name)


def test_binding_covers_header():
    from paper_2405_03456_gb300 import hm
    assert sorted(hm.DECLARED) == declared_symbols()


def test_status_strings(lib):
    for code, text in [(0, b"ok"), (1, b"invalid argument"), (8, b"data outside the decodable range")]:
        assert lib.hm_status_str(code) == text


def test_argument_errors_without_gpu(lib):
    from paper_2405_03456_gb300 import hm
    pts = np.zeros((4, 3))
    with pytest.raises(hm.HMError):
        hm.hm_build(pts, leaf_size=0)
    with pytest.raises(hm.HMError):
        hm.hm_build(pts, eps_build=2.0)
    bad = pts.copy()
    bad[0, 0] = np.nan
    with pytest.raises(hm.HMError):
        hm.hm_build(bad)
    assert lib.hm_matvec(None, 1.0, None, 1, 0.0, None, 1, 1, None) == 1
    assert lib.hm_free(None) == 0


def test_newer_entry_points_check_arguments_and_order(lib):
    """Adjoint, persistent launches and the admissibility / format enums reject bad
    input before any device work."""
    import ctypes as C

    from paper_2405_03456_gb300 import hm
    pts = np.random.default_rng(3).uniform(-1, 1, (64, 3))
    for bad in ({"adm": 3}, {"fmt": 4}):
        p = hm.hm_build_params(0, 0.0, 16, 2.0, bad.get("fmt", 0), 1e-6, 1, bad.get("adm", 0))
        h = C.c_void_p()
        assert lib.hm_build(C.byref(p), pts.ctypes.data, 64, C.byref(h)) == 1
    assert lib.hm_matvec_adjoint(None, 1.0, None, 1, 0.0, None, 1, 1, None) == 1
    assert lib.hm_persistent(None, 1) == 1
    h = hm.hm_build(pts, leaf_size=16, nthreads=1)
    try:
        buf = np.zeros(64)
        # built but not compressed: call order violated, nothing reaches the device
        assert lib.hm_matvec_adjoint(h, 1.0, buf.ctypes.data, 64, 0.0, buf.ctypes.data, 64, 1, None) == 4
        assert lib.hm_matvec_adjoint(h, 1.0, buf.ctypes.data, 64, 0.0, buf.ctypes.data, 64, 65, None) == 1
        assert lib.hm_persistent(h, 0) == 0 and lib.hm_persistent(h, 1) == 0 and lib.hm_persistent(h, 2) == 0
        assert lib.hm_persistent(h, 3) == 1 and lib.hm_persistent(h, -1) == 1
        eng = C.c_int32(-1)
        assert lib.hm_multi_rhs_engine(h, C.byref(eng)) == 0 and eng.value == 1
        assert lib.hm_set_multi_rhs_engine(h, 0) == 0 and lib.hm_multi_rhs_engine(h, C.byref(eng)) == 0
        assert eng.value == 0
        assert lib.hm_set_multi_rhs_engine(h, 2) == 1 and lib.hm_set_multi_rhs_engine(h, -1) == 1
        assert lib.hm_set_multi_rhs_engine(None, 0) == 1 and lib.hm_multi_rhs_engine(h, None) == 1
        rec = (C.c_int32 * 16)()
        n = C.c_int32(-1)
        # tuning records: argument errors first, then call order (not compressed)
        assert lib.hm_tuning(None, rec, 16, C.byref(n)) == 1 and lib.hm_tuning(h, None, 4, C.byref(n)) == 1
        assert lib.hm_tuning(h, rec, -1, C.byref(n)) == 1 and lib.hm_tuning(h, rec, 16, None) == 1
        assert lib.hm_tuning(h, rec, 16, C.byref(n)) == 4
        assert lib.hm_set_tuning(h, rec, 6) == 1 and lib.hm_set_tuning(h, None, 16) == 1
        assert lib.hm_set_tuning(None, rec, 16) == 1 and lib.hm_set_tuning(h, rec, 16) == 4
    finally:
        assert lib.hm_free(h) == 0
