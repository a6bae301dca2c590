"""Compile libhm (host C++ + sm_103a CUDA) in-tree into ``_build/libhm.so``.

Translation units compile in parallel; the CUDA file is compiled for sm_103a
only.  Host code is built with -ffp-contract=off: the tree construction and the
codec encoders must round every operation as written (their results are
compared bit for bit with the oracle's).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhm.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = shutil.which("nvcc") or os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CPP = ["trees.cpp", "linalg.cpp", "build.cpp", "codec.cpp", "program.cpp", "matrix.cpp", "persist.cpp", "lu_factor.cpp", "hlu.cpp"]
CU = ["kernels.cu", "mrhs.cu", "mrhs_tc.cu", "noalloc.cu", "hlu.cu"]
HDRS = ["hm_internal.h", "dev_types.h", "program.h", "decode.cuh"]


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    inc = ["-I" + os.path.join(CUDA, "include"), "-I" + CSRC]
    hdrs = [os.path.join(CSRC, h) for h in HDRS] + [os.path.join(HERE, "..", "include", "hm.h")]
    jobs = []
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        cmd = ["g++", "-std=c++17", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-Wall",
               "-Wno-unused-function"] + inc + ["-c", src, "-o", obj]
        jobs.append((obj, [src] + hdrs, cmd))
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        cmd = [NVCC, "-std=c++17", "-O3", "-lineinfo"] + ARCH + ["-Xcompiler", "-fPIC"] + inc + \
              ["-c", src, "-o", obj]
        jobs.append((obj, [src] + hdrs, cmd))
    todo = [j for j in jobs if force or _stale(j[0], j[1])]
    with cf.ThreadPoolExecutor(max_workers=len(todo) or 1) as ex:
        for out in ex.map(lambda j: _run(j[2]), todo):
            if verbose and out:
                print(out)
    objs = [j[0] for j in jobs]
    if force or todo or not os.path.exists(LIB):
        cmd = [NVCC, "-shared"] + ARCH + ["-o", LIB + ".tmp"] + objs + \
              ["-Xcompiler", "-fopenmp", "-lgomp", "-lpthread"]
        _run(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
