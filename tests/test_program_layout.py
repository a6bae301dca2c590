"""Host check of the launch program, for every launch shape, without a GPU.

``tests/program_check.cpp`` is linked against the library's host objects.  It
builds a matrix, packs it and builds its launch program, and checks the program
in two ways.  First, every copy descriptor and every vector index the kernels
would touch is checked against the buffers the library allocates.  Second, the
launches are replayed in FP64, and the replay must give the same y on a second
pass.  The replayed product is compared with the FP64 product of the matrix as
the host stores it in its format (H blocks, or bases and couplings):

* uncompressed: equal up to FP64 rounding (1e-13), which pins the program's
  indices, scales and emit modes for every format;
* compressed: within eps, the codecs' rounding only (measured at most 0.18 eps
  over formats, codecs and eps 1e-4..1e-8).

The program of the transposed matrix, which the adjoint product runs, is
checked the same way.  Its replay is compared with M^T x, computed from the
original matrix's blocks.

The runs of row-chunk launches that the library fuses into one persistent
launch (the H2 sweeps, the two coupling stages of separate couplings) are also
replayed as dataflow.  Warps step in random order with 1 to 1000 warps, and each
piece waits for the chunk versions of its dependencies.  No order may stall with
work left, which would be a hang, and none may change y by a bit, which would be
a race.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from paper_2405_03456_gb300 import build as hbuild

HOST = ["trees.cpp", "linalg.cpp", "build.cpp", "codec.cpp", "program.cpp"]
FORMATS = {"h": 0, "uh": 1, "h2": 2, "uh_sep": 3}
CODECS = {"none": 0, "aflp": 1, "fpx": 2}
ADMS = {"std": 0, "hodlr": 1, "blr": 2}

# (points, n, format, eps, codec, leaf, nsm, adm)
CASES = [("sphere", 3000, f, 1e-6, c, 32, 152, "std") for f in FORMATS for c in CODECS] + [
    ("sphere", 2048, "h", 1e-8, "aflp", 32, 152, "std"),        # float-float tier
    ("sphere", 2048, "h2", 1e-8, "fpx", 32, 152, "std"),
    ("sphere", 3000, "uh_sep", 1e-8, "aflp", 64, 152, "std"),
    ("sphere", 3000, "h", 1e-6, "aflp", 32, 7, "std"),          # few SMs: long ranges, shared chunks
    ("sphere", 3000, "h2", 1e-6, "aflp", 32, 3, "std"),
    ("sphere", 3000, "h", 1e-6, "aflp", 32, 152, "hodlr"),
    ("sphere", 3000, "uh", 1e-6, "fpx", 32, 152, "blr"),
    ("cube", 3000, "h2", 1e-4, "aflp", 32, 152, "std"),         # Matern
    ("cube", 2048, "h", 1e-8, "fpx", 32, 152, "blr"),
]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    hbuild.build()
    tmp = tmp_path_factory.mktemp("program_check")
    exe = str(tmp / "program_check")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "program_check.cpp")
    inc = os.path.join(hbuild.HERE, "..", "include")
    objs = [os.path.join(hbuild.OUT, f + ".o") for f in HOST]
    subprocess.run(["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-I", hbuild.CSRC, "-I", inc,
                    src] + objs + ["-o", exe], check=True)
    return exe, tmp


def _run(checker, pts_kind, n, fmt, eps, codec, leaf, nsm, adm, adjoint=False):
    exe, tmp = checker
    path = tmp / f"{pts_kind}{n}.bin"
    if not path.exists():
        pts = synth.sphere_points(n) if pts_kind == "sphere" else synth.cube_points(n)
        x = synth.rhs(n)[:, 0]
        path.write_bytes(np.ascontiguousarray(pts).tobytes() + np.ascontiguousarray(x).tobytes())
    kernel = 0 if pts_kind == "sphere" else 1
    return subprocess.run([exe, str(path), str(n), str(FORMATS[fmt]), repr(eps), str(CODECS[codec]), str(leaf),
                           str(nsm), str(ADMS[adm]), str(kernel), str(int(adjoint))],
                          stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_program_layout_and_replay(checker, case):
    pts_kind, n, fmt, eps, codec, leaf, nsm, adm = case
    r = _run(checker, *case)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    errs = [float(line.split()[-1]) for line in r.stdout.splitlines() if line.startswith("shape")]
    assert len(errs) == 4                                  # three warp shapes and the multi-RHS shape
    bound = 1e-13 if codec == "none" else eps
    assert max(errs) <= bound, (errs, bound)
    runs = [int(line.split()[-1]) for line in r.stdout.splitlines() if line.startswith("persistent runs")]
    assert len(runs) == 1
    if fmt in ("h2", "uh_sep"):
        assert runs[0] >= 1                                # the dataflow replay ran


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("codec", ["none", "fpx"])
def test_adjoint_program(checker, fmt, codec):
    # the adjoint product runs the program of the transposed matrix: its replay
    # must give M^T x computed from the original matrix's blocks
    eps = 1e-6
    r = _run(checker, "sphere", 3000, fmt, eps, codec, 32, 152, "std", adjoint=True)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    errs = [float(line.split()[-1]) for line in r.stdout.splitlines() if line.startswith("shape")]
    assert len(errs) == 4 and max(errs) <= (1e-13 if codec == "none" else eps), errs


@pytest.mark.parametrize("fmt,adm,codec", [("h", "hodlr", "aflp"), ("uh", "blr", "aflp"), ("h2", "blr", "none")])
def test_adjoint_program_other_admissibility(checker, fmt, adm, codec):
    eps = 1e-6
    r = _run(checker, "sphere", 3000, fmt, eps, codec, 32, 152, adm, adjoint=True)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    errs = [float(line.split()[-1]) for line in r.stdout.splitlines() if line.startswith("shape")]
    assert len(errs) == 4 and max(errs) <= (1e-13 if codec == "none" else eps), errs


HEADLINE = [(131072, f, eps, c, adj) for (f, eps, c, adj) in [
    ("h", 1e-6, "aflp", False), ("uh", 1e-6, "aflp", False), ("h2", 1e-6, "aflp", False),
    ("uh_sep", 1e-6, "aflp", False), ("h", 1e-8, "aflp", False), ("h", 1e-4, "fpx", False),
    ("h", 1e-6, "none", False), ("h", 1e-6, "aflp", True)]]


@pytest.mark.skipif(os.environ.get("HM_CHECK_FULL") != "1", reason="full-size check: set HM_CHECK_FULL=1 "
                    "(about 2 minutes and 6 GB of host memory per case)")
@pytest.mark.parametrize("case", HEADLINE, ids=lambda c: "-".join(map(str, c)))
def test_program_layout_headline_size(checker, case):
    # the sphere workload the benchmark times: N = 131072, leaf 64
    n, fmt, eps, codec, adjoint = case
    r = _run(checker, "sphere", n, fmt, eps, codec, 64, 152, "std", adjoint=adjoint)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    errs = [float(line.split()[-1]) for line in r.stdout.splitlines() if line.startswith("shape")]
    assert len(errs) == 4 and max(errs) <= (1e-13 if codec == "none" else eps), errs


def test_persistent_dependency_analysis_on_hand_built_programs(checker):
    # seq_dependencies on small programs: which chunk a multiplier run reads, the
    # versions it waits for, and the cases that must keep the launches separate
    exe, tmp = checker
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seqdeps_check.cpp")
    inc = os.path.join(hbuild.HERE, "..", "include")
    objs = [os.path.join(hbuild.OUT, f + ".o") for f in HOST]
    sd = str(tmp / "seqdeps_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fopenmp", "-I", hbuild.CSRC, "-I", inc, src] + objs + ["-o", sd],
                   check=True)
    r = subprocess.run([sd], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_h2_hodlr_basis_rank_above_the_kernel_limit(checker):
    # HODLR's top-level blocks need H2 bases of rank > 128: the program is not
    # built (hm_compress reports HM_ERR_CAPACITY)
    r = _run(checker, "sphere", 3000, "h2", 1e-6, "aflp", 32, 152, "hodlr")
    assert r.returncode == 1 and "build_program failed" in r.stdout


@pytest.mark.parametrize("fmt", list(FORMATS))
def test_fanout_folded_into_segment_sums(checker, fmt):
    # the fan-out right after the segment sums (H: the multipliers of the W factors)
    # is folded into them; a fan-out of row-chunk outputs (UH / H^2 backward) stays.
    # The replay above checks the values; here the launch list.
    r = _run(checker, "sphere", 3000, fmt, 1e-6, "aflp", 32, 152, "std")
    assert r.returncode == 0 and r.stdout.rstrip().endswith("ok"), r.stdout[-2000:]
    kinds = [line.split()[2] for line in r.stdout.splitlines() if line.startswith("launch ")]
    assert kinds[:2] == ["gather", "cdot"]
    for i, k in enumerate(kinds):
        if k == "fanout":
            assert kinds[i - 1] == "rgemv"
    if fmt == "h":
        assert kinds == ["gather", "cdot", "gsum", "rgemv"]
    else:
        assert "fanout" in kinds
