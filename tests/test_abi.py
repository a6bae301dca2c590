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
