"""Thin ctypes binding of libhm (include/hm.h): argument marshalling only.

Every entry point keeps the C name.  Device buffers are plain pointers (for
example ``torch.Tensor.data_ptr()`` of CUDA tensors) and streams are raw
``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).  The
library must be built (``paper_2405_03456_gb300.build.build()``); loading fails
loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HM_FMT_H, HM_FMT_UH, HM_FMT_H2, HM_FMT_UH_SEP = 0, 1, 2, 3
HM_CODEC_NONE, HM_CODEC_AFLP, HM_CODEC_FPX = 0, 1, 2
HM_KERNEL_LAPLACE, HM_KERNEL_MATERN15, HM_KERNEL_LAPLACE_W = 0, 1, 2
FORMATS = {"h": HM_FMT_H, "uh": HM_FMT_UH, "h2": HM_FMT_H2, "uh_sep": HM_FMT_UH_SEP}
CODECS = {"none": HM_CODEC_NONE, "aflp": HM_CODEC_AFLP, "fpx": HM_CODEC_FPX}
KERNELS = {"laplace": HM_KERNEL_LAPLACE, "matern": HM_KERNEL_MATERN15, "laplace_w": HM_KERNEL_LAPLACE_W}

DECLARED = ["hm_build", "hm_compress", "hm_matvec", "hm_matvec_host", "hm_free", "hm_info",
            "hm_status_str", "hm_sync_status", "hm_structure", "hm_codec_encode", "hm_codec_decode",
            "hm_profile", "hm_profile_read", "hm_alg_bytes", "hm_matvec_host_noalloc", "hm_graph",
            "hm_autotune", "hm_launch_shapes", "hm_set_launch_shapes", "hm_persistent", "hm_matvec_adjoint",
            "hm_decompress_debug", "hm_save", "hm_load", "hm_lu_build", "hm_lu_compress", "hm_lu_solve",
            "hm_lu_sync_status", "hm_lu_info", "hm_lu_free", "hm_persistent_mode", "hm_set_multi_rhs_engine",
            "hm_multi_rhs_engine", "hm_tuning", "hm_set_tuning"]
NSHAPES = 3
HM_NOALLOC_MAX_ENTRIES = 1 << 20
KERNEL_KINDS = ["gather", "cdot", "gsum", "rgemv", "fanout"]


class hm_build_params(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("kparam", C.c_double), ("leaf_size", C.c_int32),
                ("eta", C.c_double), ("format", C.c_int32), ("eps_build", C.c_double),
                ("nthreads", C.c_int32), ("adm", C.c_int32)]


class hm_info_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("format", C.c_int32), ("codec", C.c_int32), ("valr", C.c_int32),
                ("eps", C.c_double), ("nclusters", C.c_int64), ("nleaves", C.c_int64),
                ("nblocks", C.c_int64), ("nlowrank", C.c_int64), ("ndense", C.c_int64),
                ("depth", C.c_int32), ("max_rank", C.c_int32), ("bytes_fp64", C.c_int64),
                ("bytes_payload", C.c_int64), ("bytes_values", C.c_int64), ("bytes_meta", C.c_int64),
                ("bytes_workspace", C.c_int64), ("bytes_lowrank_fp64", C.c_int64),
                ("bytes_dense_fp64", C.c_int64), ("nlaunches", C.c_int64), ("tier", C.c_int32),
                ("nunits", C.c_int64), ("bytes_inline_meta", C.c_int64), ("bytes_alg", C.c_int64),
                ("bytes_by_width", C.c_int64 * 8)]


class hm_codec_header(C.Structure):
    _fields_ = [("B", C.c_int32), ("fmt", C.c_int32), ("e", C.c_int32), ("m", C.c_int32),
                ("vmin", C.c_double)]


class hm_kernel_stat(C.Structure):
    _fields_ = [("ms", C.c_double), ("launches", C.c_int64), ("bytes", C.c_int64)]


class HMError(RuntimeError):
    pass


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> C.CDLL:
    """Load libhm; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise HMError(f"libhm is not built ({p}); run paper_2405_03456_gb300.build.build()")
    L = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "hm_build": ([C.POINTER(hm_build_params), vp, i64, C.POINTER(vp)], i32),
        "hm_compress": ([vp, dbl, i32, i32], i32),
        "hm_matvec": ([vp, dbl, vp, i64, dbl, vp, i64, i64, vp], i32),
        "hm_matvec_host": ([vp, dbl, vp, dbl, vp, i64, vp], i32),
        "hm_free": ([vp], i32),
        "hm_info": ([vp, C.POINTER(hm_info_t)], i32),
        "hm_status_str": ([i32], C.c_char_p),
        "hm_sync_status": ([vp, vp], i32),
        "hm_structure": ([vp, vp, vp, vp, vp], i32),
        "hm_codec_encode": ([vp, i64, i32, i32, vp, i64, C.POINTER(hm_codec_header)], i32),
        "hm_codec_decode": ([vp, i64, C.POINTER(hm_codec_header), vp, vp], i32),
        "hm_profile": ([vp, i32], i32),
        "hm_persistent": ([vp, i32], i32),
        "hm_matvec_adjoint": ([vp, dbl, vp, i64, dbl, vp, i64, i64, vp], i32),
        "hm_profile_read": ([vp, C.POINTER(hm_kernel_stat), i32], i32),
        "hm_alg_bytes": ([vp, C.POINTER(i64)], i32),
        "hm_matvec_host_noalloc": ([vp, dbl, vp, dbl, vp, i64, vp], i32),
        "hm_graph": ([vp, i32], i32),
        "hm_autotune": ([vp, i32, vp], i32),
        "hm_launch_shapes": ([vp, vp, i32, C.POINTER(i32)], i32),
        "hm_set_launch_shapes": ([vp, i32], i32),
        "hm_persistent_mode": ([vp, C.POINTER(i32)], i32),
        "hm_set_multi_rhs_engine": ([vp, i32], i32),
        "hm_tuning": ([vp, vp, i32, C.POINTER(i32)], i32),
        "hm_set_tuning": ([vp, vp, i32], i32),
        "hm_multi_rhs_engine": ([vp, C.POINTER(i32)], i32),
        "hm_decompress_debug": ([vp, i32, i64, i64, i64, vp, vp, vp, vp, C.POINTER(i64), vp], i32),
        "hm_save": ([vp, C.c_char_p], i32),
        "hm_lu_build": ([C.POINTER(hm_build_params), vp, i64, C.POINTER(vp)], i32),
        "hm_lu_compress": ([vp, dbl, i32, i32], i32),
        "hm_lu_solve": ([vp, vp, i64, vp, i64, i64, vp], i32),
        "hm_lu_sync_status": ([vp, vp], i32),
        "hm_lu_info": ([vp, vp, i32], i32),
        "hm_lu_free": ([vp], i32),
        "hm_load": ([C.c_char_p, C.POINTER(vp)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def check(status: int, what: str = "") -> None:
    if status != 0:
        msg = load().hm_status_str(status).decode()
        raise HMError(f"{what}: {msg} ({status})")


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- C entry points
ADMS = {"std": 0, "hodlr": 1, "blr": 2}


def hm_build(pts: np.ndarray, kernel: str = "laplace", leaf_size: int = 64, eta: float = 2.0,
             fmt: str = "h", eps_build: float = 1e-6, kparam: float = 0.0, nthreads: int = 0,
             adm: str = "std") -> int:
    p = hm_build_params(KERNELS[kernel], kparam, leaf_size, eta, FORMATS[fmt], eps_build, nthreads, ADMS[adm])
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    h = C.c_void_p()
    check(load().hm_build(C.byref(p), _ptr(pts), pts.shape[0], C.byref(h)), "hm_build")
    return h.value


def hm_compress(h: int, eps: float, codec: str = "aflp", valr: bool = True) -> None:
    check(load().hm_compress(h, eps, CODECS[codec], 1 if valr else 0), "hm_compress")


def hm_matvec(h: int, alpha: float, x_ptr: int, ldx: int, beta: float, y_ptr: int, ldy: int,
              nrhs: int = 1, stream: int = 0) -> None:
    check(load().hm_matvec(h, alpha, x_ptr, ldx, beta, y_ptr, ldy, nrhs, stream), "hm_matvec")


def hm_matvec_adjoint(h: int, alpha: float, x_ptr: int, ldx: int, beta: float, y_ptr: int, ldy: int,
                      nrhs: int = 1, stream: int = 0) -> None:
    check(load().hm_matvec_adjoint(h, alpha, x_ptr, ldx, beta, y_ptr, ldy, nrhs, stream), "hm_matvec_adjoint")


def hm_matvec_host(h: int, alpha: float, x: np.ndarray, beta: float, y: np.ndarray, stream: int = 0) -> None:
    """x, y: host FP64 arrays of shape (n,) or (n, nrhs), Fortran order (y updated in place)."""
    assert x.dtype == np.float64 and y.dtype == np.float64 and x.flags.f_contiguous and y.flags.f_contiguous
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    check(load().hm_matvec_host(h, alpha, _ptr(x), beta, _ptr(y), nrhs, stream), "hm_matvec_host")


def hm_matvec_host_noalloc(h: int, alpha: float, x: np.ndarray, beta: float, y: np.ndarray,
                           stream: int = 0) -> None:
    """As hm_matvec_host, staged through libhm's fixed device array (no allocation)."""
    assert x.dtype == np.float64 and y.dtype == np.float64 and x.flags.f_contiguous and y.flags.f_contiguous
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    check(load().hm_matvec_host_noalloc(h, alpha, _ptr(x), beta, _ptr(y), nrhs, stream),
          "hm_matvec_host_noalloc")


def hm_free(h: int) -> None:
    check(load().hm_free(h), "hm_free")


def hm_info(h: int) -> dict:
    o = hm_info_t()
    check(load().hm_info(h, C.byref(o)), "hm_info")
    out = {f: getattr(o, f) for f, _ in hm_info_t._fields_}
    out["bytes_by_width"] = list(o.bytes_by_width)
    return out


def hm_sync_status(h: int, stream: int = 0) -> int:
    return load().hm_sync_status(h, stream)


def hm_structure(h: int):
    info = hm_info(h)
    n, nc, nb = info["n"], info["nclusters"], info["nblocks"]
    perm = np.empty(n, dtype=np.int64)
    cl = np.empty((nc, 4), dtype=np.int64)
    bl = np.empty((nb, 3), dtype=np.int64)
    rk = np.empty(nb, dtype=np.int32)
    check(load().hm_structure(h, _ptr(perm), _ptr(cl), _ptr(bl), _ptr(rk)), "hm_structure")
    return perm, cl, bl, rk


def hm_codec_encode(v: np.ndarray, codec: str, key: int):
    """Host encode; returns (packed uint8 array, header dict)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(max(8 * v.size, 8), dtype=np.uint8)
    hdr = hm_codec_header()
    check(load().hm_codec_encode(_ptr(v), v.size, CODECS[codec], key, _ptr(out), out.size, C.byref(hdr)),
          "hm_codec_encode")
    h = {"B": hdr.B, "fmt": hdr.fmt, "e": hdr.e, "m": hdr.m, "vmin": hdr.vmin}
    return out[: v.size * hdr.B].copy(), h


def hm_codec_decode(packed_ptr: int, n: int, hdr: dict, out_ptr: int, stream: int = 0) -> None:
    """Device decode (kernel K0) of n packed values into FP64 device memory."""
    h = hm_codec_header(hdr["B"], hdr["fmt"], hdr["e"], hdr["m"], hdr["vmin"])
    check(load().hm_codec_decode(packed_ptr, n, C.byref(h), out_ptr, stream), "hm_codec_decode")


def hm_graph(h: int, enable: bool) -> None:
    check(load().hm_graph(h, 1 if enable else 0), "hm_graph")


def hm_persistent(h: int, mode: int) -> None:
    check(load().hm_persistent(h, int(mode)), "hm_persistent")


def hm_autotune(h: int, reps: int = 5, stream: int = 0) -> None:
    check(load().hm_autotune(h, reps, stream), "hm_autotune")


def hm_launch_shapes(h: int) -> list:
    cnt = C.c_int32()
    check(load().hm_launch_shapes(h, None, 0, C.byref(cnt)), "hm_launch_shapes")
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    check(load().hm_launch_shapes(h, _ptr(out), cnt.value, C.byref(cnt)), "hm_launch_shapes")
    return [int(v) for v in out[: cnt.value]]


def hm_set_launch_shapes(h: int, shape: int) -> None:
    check(load().hm_set_launch_shapes(h, shape), "hm_set_launch_shapes")


def hm_profile(h: int, enable: bool) -> None:
    check(load().hm_profile(h, 1 if enable else 0), "hm_profile")


def hm_profile_read(h: int) -> dict:
    nk = len(KERNEL_KINDS)
    arr = (hm_kernel_stat * nk)()
    check(load().hm_profile_read(h, arr, nk), "hm_profile_read")
    return {KERNEL_KINDS[i]: {"ms": arr[i].ms, "launches": arr[i].launches, "bytes": arr[i].bytes}
            for i in range(nk)}


def hm_alg_bytes(h: int) -> int:
    b = C.c_int64()
    check(load().hm_alg_bytes(h, C.byref(b)), "hm_alg_bytes")
    return b.value


def hm_decompress_debug(h: int, tier: int, u0: int = 0, u1: int = 1 << 62, stream: int = 0) -> dict:
    """Decode units [u0, u1) of the resident payload with the product kernels'
    decoders of `tier` (0 FP32, 1 float-float): per value its code, format word,
    and the GPU's head and tail (numpy arrays, payload order)."""
    L = load()
    n = C.c_int64()
    check(L.hm_decompress_debug(h, tier, u0, u1, 0, None, None, None, None, C.byref(n), stream),
          "hm_decompress_debug")
    cnt = n.value
    head = np.zeros(max(cnt, 1), dtype=np.float32)
    tail = np.zeros(max(cnt, 1), dtype=np.float32)
    code = np.zeros(max(cnt, 1), dtype=np.uint64)
    fmt = np.zeros(max(cnt, 1), dtype=np.uint16)
    check(L.hm_decompress_debug(h, tier, u0, u1, cnt, _ptr(head), _ptr(tail), _ptr(code), _ptr(fmt), C.byref(n),
                                stream), "hm_decompress_debug")
    return {"head": head[:cnt], "tail": tail[:cnt], "code": code[:cnt], "fmt": fmt[:cnt]}


def hm_save(h: int, path: str) -> None:
    check(load().hm_save(h, os.fsencode(path)), "hm_save")


def hm_load(path: str) -> int:
    h = C.c_void_p()
    check(load().hm_load(os.fsencode(path), C.byref(h)), "hm_load")
    return h.value


class HLU:
    """Owns one hm_lu handle: H-LU factors of a kernel matrix and their triangular solves."""

    INFO = ["n", "bytes_payload", "bytes_values", "bytes_fp64", "items", "leaves", "lowrank_blocks"]

    def __init__(self, pts, kernel="matern", leaf_size=32, eta=2.0, eps_build=1e-6, kparam=0.0, nthreads=0,
                 adm="std"):
        p = hm_build_params(KERNELS[kernel], kparam, leaf_size, eta, 0, eps_build, nthreads, ADMS[adm])
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        h = C.c_void_p()
        check(load().hm_lu_build(C.byref(p), _ptr(pts), pts.shape[0], C.byref(h)), "hm_lu_build")
        self.h = h.value
        self.n = pts.shape[0]

    def compress(self, eps, codec="aflp", valr=True):
        check(load().hm_lu_compress(self.h, eps, CODECS[codec], 1 if valr else 0), "hm_lu_compress")
        return self

    def solve(self, b, x, stream=None):
        """x := U^-1 L^-1 b for CUDA FP64 tensors of shape (n,) or (n, r), column-major."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        ldb = b.shape[0] if nrhs == 1 else b.stride(1)
        ldx = x.shape[0] if nrhs == 1 else x.stride(1)
        check(load().hm_lu_solve(self.h, b.data_ptr(), ldb, x.data_ptr(), ldx, nrhs, stream), "hm_lu_solve")
        return x

    def sync_status(self, stream=0):
        return load().hm_lu_sync_status(self.h, stream)

    def info(self):
        out = np.zeros(7, dtype=np.int64)
        check(load().hm_lu_info(self.h, _ptr(out), 7), "hm_lu_info")
        return dict(zip(self.INFO, out.tolist()))

    def close(self):
        if self.h:
            load().hm_lu_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience object
class HMatrix:
    """Owns one hm_matrix handle; products take CUDA tensors (torch) or host arrays."""

    def __init__(self, pts, kernel="laplace", leaf_size=64, eta=2.0, fmt="h", eps_build=1e-6,
                 kparam=0.0, nthreads=0, adm="std"):
        self.h = hm_build(pts, kernel, leaf_size, eta, fmt, eps_build, kparam, nthreads, adm)
        self.n = pts.shape[0]

    @classmethod
    def load(cls, path):
        """A matrix written by save() (compressed again on the current device if it was)."""
        self = cls.__new__(cls)
        self.h = hm_load(path)
        self.n = hm_info(self.h)["n"]
        return self

    def save(self, path):
        hm_save(self.h, path)

    def compress(self, eps, codec="aflp", valr=True):
        hm_compress(self.h, eps, codec, valr)
        return self

    def matvec(self, alpha, x, beta, y, stream=None, adjoint=False):
        """y := alpha*M*x + beta*y (adjoint: alpha*M^H*x + beta*y) for CUDA FP64
        tensors x, y of shape (n,) or (n, r) column-major."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        # a single column's leading dimension is n (the stride of a size-1 dimension is arbitrary)
        ldx = x.shape[0] if nrhs == 1 else x.stride(1)
        ldy = y.shape[0] if nrhs == 1 else y.stride(1)
        assert x.dtype == torch.float64 and y.dtype == torch.float64 and x.is_cuda and y.is_cuda
        assert x.dim() == 1 or x.stride(0) == 1
        assert y.dim() == 1 or y.stride(0) == 1
        f = hm_matvec_adjoint if adjoint else hm_matvec
        f(self.h, alpha, x.data_ptr(), ldx, beta, y.data_ptr(), ldy, nrhs, stream)
        return y

    def matvec_host(self, alpha, x, beta, y, stream=0):
        hm_matvec_host(self.h, alpha, x, beta, y, stream)
        return y

    def info(self):
        return hm_info(self.h)

    def alg_bytes(self):
        return hm_alg_bytes(self.h)

    def graph(self, enable=True):
        hm_graph(self.h, enable)
        return self

    def persistent_mode(self):
        m = C.c_int32()
        check(load().hm_persistent_mode(self.h, C.byref(m)), "hm_persistent_mode")
        return m.value

    def multi_rhs_engine(self, engine=None):
        """Set (0: tensor cores, 1: FP32 pipes) and/or return the multi-RHS row-chunk engine."""
        if engine is not None:
            check(load().hm_set_multi_rhs_engine(self.h, int(engine)), "hm_set_multi_rhs_engine")
        m = C.c_int32()
        check(load().hm_multi_rhs_engine(self.h, C.byref(m)), "hm_multi_rhs_engine")
        return m.value

    def persistent(self, enable=True):
        """0 / False: one launch per step; 1 / True: runs of row-chunk steps fused
        (the default); 2: the whole product as one persistent launch."""
        hm_persistent(self.h, int(enable))
        return self

    def autotune(self, reps=5, stream=0, cache=None):
        """Time the launch shapes, launch modes and multi-RHS engines and keep the
        fastest.  cache: a JSON file of tuning records (one per device and launch
        program); a record found there is applied instead of timing, a new one is
        added to it."""
        if cache is None:
            hm_autotune(self.h, reps, stream)
            return self
        import json
        import os
        try:
            with open(cache) as f:
                recs = json.load(f)
        except (OSError, ValueError):
            recs = {}
        rec = self.tuning()
        key = f"{rec[2] & 0xffffffff:08x}{rec[3] & 0xffffffff:08x}"
        if key in recs and self.set_tuning(recs[key]):
            return self
        hm_autotune(self.h, reps, stream)
        recs[key] = self.tuning()
        tmp = f"{cache}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(recs, f)
        os.replace(tmp, cache)
        return self

    def tuning(self):
        """The current tuning record (list of int)."""
        n = C.c_int32()
        check(load().hm_tuning(self.h, None, 0, C.byref(n)), "hm_tuning")
        buf = (C.c_int32 * n.value)()
        check(load().hm_tuning(self.h, buf, n.value, C.byref(n)), "hm_tuning")
        return list(buf)

    def set_tuning(self, rec):
        """Apply a tuning record; False if it belongs to another device or program."""
        buf = (C.c_int32 * len(rec))(*rec)
        return load().hm_set_tuning(self.h, buf, len(rec)) == 0

    def launch_shapes(self):
        return hm_launch_shapes(self.h)

    def set_launch_shapes(self, shape):
        hm_set_launch_shapes(self.h, shape)
        return self

    def profile(self, enable=True):
        hm_profile(self.h, enable)

    def profile_read(self):
        return hm_profile_read(self.h)

    def structure(self):
        return hm_structure(self.h)

    def sync_status(self, stream=0):
        return hm_sync_status(self.h, stream)

    def close(self):
        if self.h:
            hm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
