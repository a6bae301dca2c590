"""Host check of the H-LU triangular-solve program, without a GPU.

``tests/lu_check.cpp`` (linked against the library's host objects) factors the
Matern covariance matrix with the library's own host elimination, packs both
factors, checks every packed column and index against the payload and the
vectors, and replays the solve's work list in list order in FP64 -- requiring
every dependency to be met when its item starts, which is the condition under
which the GPU's persistent launch (warps taking items in list order, each
waiting only for earlier items) cannot stall.  The replayed solution must be
within eps of a dense LU solve with partial pivoting of the exact matrix, and
its residual within eps / 100 relative to ||A|| ||x||.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from paper_2405_03456_gb300 import build as hbuild

HOST = ["trees.cpp", "linalg.cpp", "build.cpp", "codec.cpp", "program.cpp", "lu_factor.cpp"]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    hbuild.build()
    tmp = tmp_path_factory.mktemp("lu_check")
    exe = str(tmp / "lu_check")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lu_check.cpp")
    inc = os.path.join(hbuild.HERE, "..", "include")
    objs = [os.path.join(hbuild.OUT, f + ".o") for f in HOST]
    subprocess.run(["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-I", hbuild.CSRC, "-I", inc,
                    src] + objs + ["-o", exe], check=True)
    n = 1000
    path = tmp / "cube.bin"
    path.write_bytes(np.ascontiguousarray(synth.cube_points(n)).tobytes() +
                     np.ascontiguousarray(synth.rhs(n)[:, 0]).tobytes())
    return exe, str(path), n


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("codec", [0, 1, 2])
def test_lu_program_replay(checker, eps, codec):
    exe, path, n = checker
    r = subprocess.run([exe, path, str(n), "1", repr(eps), str(codec), "32"], stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    vals = dict(line.split()[:2] for line in r.stdout.splitlines() if line.split()[0] in ("diff", "residual"))
    assert float(vals["diff"]) <= eps, vals
    assert float(vals["residual"]) <= eps / 100, vals
