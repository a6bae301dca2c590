#!/usr/bin/env python
"""Benchmark: compressed H-matrix-vector product on one GB300 (libhm).

Workload: Laplace single-layer point kernel on N = 131072 jittered Fibonacci
points of the unit sphere, binary geometric bisection (leaf 64), standard
admissibility eta = 2, H format built at eps; one FP64 right-hand side
x ~ U(-1, 1).  For eps in {1e-4, 1e-6, 1e-8} the matrix is packed with AFLP
(VALR), FPX (VALR) and uncompressed FP64, and each variant is timed; the
headline is AFLP at eps = 1e-6.

A step is one product y := M x + y (gather / decode / low-rank forward /
row-chunk accumulation / scatter: every kernel of the path), timed with CUDA
events on the launching stream.  The packed matrix (> 0.5 GB) is larger than
the 129 MB L2, so no flush is needed between steps.  ``value`` is the
method's algorithmic bytes per product (packed codes and their inline metadata,
24 N for x and y, 16 per coefficient of the coefficient vectors) divided by
the median step time, summed over ranks; the layout's intermediate traffic is
reported beside it, not counted in it.

``--impl reference`` times the CPU oracle (Alg. 1 with Alg. 8 decompression)
on all host cores (one process per core) over a bounded random block sample of
the same workload; ``cpu_baseline`` in the GPU line is the same measurement.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed H-matvec GB/s and matvecs/s vs uncompressed FP64 GPU at eps; p50/p99"
N_DEFAULT = 131072
EPS_LIST = (1e-4, 1e-6, 1e-8)
HEADLINE = (1e-6, "aflp")


def workload_name(n):
    return f"laplace-sphere N={n} leaf=64 eta=2 H-format, AFLP/FPX VALR vs FP64, 1 FP64 RHS"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed loops run."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _cpu_worker(p, nw, budget_bytes, passes, warmup, barrier, q, n=N_DEFAULT, kind="laplace"):
    """One oracle process (one BLAS thread): builds its share of the block
    sample, then times Alg. 1 + Alg. 8 passes over it in step with the others."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    try:
        import synth
        from oracle import baseline
        h, ch, nblocks = baseline.sample_h(n, HEADLINE[0], HEADLINE[1], budget_bytes, part=(p, nw), kind=kind)
        ab = baseline.alg_bytes(ch)
        xp = synth.rhs(n)[:, 0][ch.h.ct.perm]
        import numpy as np
        yp = np.zeros(n)
        for _ in range(warmup):
            baseline.run_pass(ch, xp, yp)
        ts = []
        for _ in range(passes):
            barrier.wait(timeout=900)
            t0 = time.perf_counter()
            baseline.run_pass(ch, xp, yp)
            ts.append(time.perf_counter() - t0)
        q.put((p, ab, len(h.blocks), nblocks, ts, None))
    except Exception as e:  # noqa: BLE001
        try:
            barrier.abort()
        except Exception:  # noqa: BLE001
            pass
        q.put((p, 0, 0, 0, [], repr(e)[:300]))


def cpu_baseline_parallel(budget_mb_per_worker: float, passes: int, warmup: int, workers: int = 0,
                          timeout: float = 1200.0, n: int = N_DEFAULT, kind: str = "laplace") -> dict:
    """The oracle as it stands on all host cores: nw spawned processes (one per
    core), each timing Alg. 1 + Alg. 8 over a disjoint share of one random
    block sample of the headline workload; a pass is timed from a common
    barrier to the slowest process's end.  value = the sample's algorithmic
    bytes / the median pass time."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    nw = workers or nproc
    ctx = mp.get_context("spawn")   # fresh interpreters: no CUDA state is inherited
    barrier = ctx.Barrier(nw)
    q = ctx.Queue()
    budget = budget_mb_per_worker * 1e6 * nw
    procs = [ctx.Process(target=_cpu_worker, args=(p, nw, budget, passes, warmup, barrier, q, n, kind), daemon=True)
             for p in range(nw)]
    t0 = time.perf_counter()
    for pr in procs:
        pr.start()
    res = []
    try:
        for _ in range(nw):
            res.append(q.get(timeout=timeout))
    finally:
        for pr in procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()
    errs = [r[5] for r in res if r[5]]
    if errs:
        raise RuntimeError("oracle worker failed: " + errs[0])
    ab = sum(r[1] for r in res)
    nb = sum(r[2] for r in res)
    per_pass = [max(r[4][k] for r in res) for k in range(passes)]
    med = statistics.median(per_pass)
    return {"value": ab / med / 1e9, "unit": "GB/s", "cores": nw, "nproc": nproc, "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": (f"{nb} of {res[0][3]} leaf blocks (<= 2^20 entries, random, seed 3) of the N={n} "
                       f"{'sphere Laplace' if kind == 'laplace' else 'cube Matern'} H-matrix at eps=1e-6, AFLP "
                       f"VALR, split over {nw} processes (one per core, one "
                       f"BLAS thread each); Alg. 1 + Alg. 8 decode in FP64, {passes} passes from a common "
                       f"barrier, {ab / 1e6:.2f} MB algorithmic per pass"),
            "pass_s_median": med, "wall_s": round(time.perf_counter() - t0, 1), "alg_bytes": ab}


# ------------------------------------------------------------------ GPU arm
def time_variant(torch, M, x, y, steps, warmup, stream, world=1, adjoint=False):
    for _ in range(warmup):
        M.matvec(1.0, x, 1.0, y, stream=stream.cuda_stream, adjoint=adjoint)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        for a, b in ev:
            a.record(stream)
            M.matvec(1.0, x, 1.0, y, stream=stream.cuda_stream, adjoint=adjoint)
            b.record(stream)
        end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    per = sorted(a.elapsed_time(b) for a, b in ev)
    total = start.elapsed_time(end)
    return per, total


def time_multi_rhs(torch, M, n, r_list, steps, warmup, stream, seed=5):
    """Products Y := M X of r right-hand sides (panels of 32, on the multi-RHS
    engine the autotuner chose): median ms and right-hand sides per second for each r."""
    import numpy as np
    import synth
    out = {}
    for r in r_list:
        X = torch.from_numpy(np.asfortranarray(synth.rhs(n, r, seed=seed + r))).cuda().t().contiguous().t()
        Y = torch.zeros_like(X)
        for _ in range(warmup):
            M.matvec(1.0, X, 0.0, Y, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for a, b in ev:
                a.record(stream)
                M.matvec(1.0, X, 0.0, Y, stream=stream.cuda_stream)
                b.record(stream)
        torch.cuda.synchronize()
        per = sorted(a.elapsed_time(b) for a, b in ev)
        med = statistics.median(per)
        out[str(r)] = {"ms_p50": round(med, 4), "ms_p99": round(pct(per, 0.99), 4),
                       "rhs_per_s": round(r / (med * 1e-3), 1)}
        del X, Y
    return out


def profiled_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` from the committed ncu record, if that
    record was taken on this workload with the current kernel sources."""
    import hashlib
    try:
        rec = dict(ln.split(" ", 1) for ln in open(os.path.join(ROOT, "profiles", "k_rstream_traffic.txt")).read()
                   .strip().splitlines())
        src = b"".join(open(os.path.join(ROOT, "paper_2405_03456_gb300", "csrc", f), "rb").read()
                       for f in ("kernels.cu", "decode.cuh", "dev_types.h"))
    except OSError:
        return None
    if rec.get("kernel") != kernel or f"N={n} " not in rec.get("workload", ""):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("sources_sha256_prefix"):
        return None
    return int(rec["bytes_per_launch"])


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's step time (every rank takes part; replicas only: the
    ranks run independent copies of the workload and exchange nothing else)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(alg_bytes: int, ms: float, world: int) -> float:
    """Algorithmic bytes all ranks moved per step over the slowest rank's time."""
    return alg_bytes / (ms * 1e-3) / 1e9 * world


def pct(v, q):
    i = min(len(v) - 1, max(0, int(round(q * (len(v) - 1)))))
    return v[i]


def serving_draw(nmin: int, nmax: int, count: int = 8, seed: int = 5, budget_gb: float = 120.0):
    """Seeded draw of the resident matrices of the serving workload: kernel
    alternating Laplace sphere / Matern cube, N log-uniform in [nmin, nmax]
    (rounded to 1024), eps uniform in {1e-4, 1e-6, 1e-8}."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(2.0 ** rng.uniform(np.log2(nmin), np.log2(nmax)) / 1024.0)) * 1024
        eps = float(rng.choice([1e-4, 1e-6, 1e-8]))
        out.append(("laplace" if i % 2 == 0 else "matern", max(n, 1024), eps))
    return out


def serving_leg(torch, hm, nmin, nmax, reqs_per_point):
    """Continuous batching of a seeded Poisson stream of 1..32-RHS requests on 8
    resident compressed H-matrices (hm_matvec panels on 4 slot streams, admitted
    by an HBM budget): closed-loop capacity, then offered loads of 25..120 % of it;
    throughput and p50/p99 latency per load."""
    import numpy as np
    import synth
    from paper_2405_03456_gb300.serving import GpuExecutor, Request, Scheduler
    draw = serving_draw(nmin, nmax)
    ex = GpuExecutor(nslots=4, max_rhs=64)
    sch_budget = int(120e9)
    Ms, mats, X = {}, {}, {}
    t0 = time.perf_counter()
    resident = 0
    for mid, (kern, n, eps) in enumerate(draw):
        pts = synth.sphere_points(n) if kern == "laplace" else synth.cube_points(n)
        M = hm.HMatrix(pts, kern, 64, 2.0, "h", eps).compress(eps, "aflp", True)
        M.graph(False)
        info = M.info()
        Ms[mid] = M
        mats[mid] = {"kernel": kern, "n": n, "eps": eps, "payload_mb": round(info["bytes_payload"] / 1e6, 1)}
        resident += info["bytes_payload"] + info["bytes_meta"] + info["bytes_workspace"]
        ex.add(mid, M)
        X[mid] = np.asfortranarray(np.random.default_rng(100 + mid).uniform(-1.0, 1.0, (n, 32)))
    build_s = time.perf_counter() - t0

    def stream_of(rate, count, seed):
        rng = np.random.default_rng(seed)
        t, out = 0.0, []
        for k in range(count):
            t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
            mid = int(rng.integers(len(draw)))
            r = int(rng.integers(1, 33))
            out.append(Request(k, mid, X[mid][:, :r], t))
        return out

    def run(rate, seed):
        sch = Scheduler(ex, budget_bytes=sch_budget, nslots=4, max_batch_rhs=64)
        for mid, M in Ms.items():
            info = M.info()
            sch.add_matrix(mid, mats[mid]["n"], info["bytes_payload"] + info["bytes_meta"] + info["bytes_workspace"])
        sch.run(stream_of(rate, reqs_per_point, seed))
        st = sch.stats()
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}

    run(0.0, 1)                                    # warm-up (graphs off: first launches, staging)
    cap = run(0.0, 2)                              # closed loop: every request at t = 0
    sat = cap["requests_per_s"]
    points = []
    for frac in (0.25, 0.5, 0.75, 0.9, 1.0, 1.2):
        st = run(frac * sat, 10 + int(frac * 100))
        st["offered_requests_per_s"] = round(frac * sat, 1)
        points.append(st)
    for M in Ms.values():
        M.close()
    return {"workload": (f"8 resident H-matrices (Laplace sphere / Matern cube alternating, N log-uniform in "
                         f"[{nmin}, {nmax}], eps in {{1e-4, 1e-6, 1e-8}}, AFLP VALR, seed 5), Poisson "
                         f"requests of U{{1..32}} FP64 right-hand sides, host buffers (copies included), "
                         f"4 slot streams, batches of <= 64 RHS, HBM budget 120 GB"),
            "matrices": mats, "resident_gb": round(resident / 1e9, 2), "build_s": round(build_s, 1),
            "requests_per_point": reqs_per_point, "closed_loop": cap, "by_load": points}


def gpu_arm(args, rank, world):
    import numpy as np
    import torch
    import synth
    from paper_2405_03456_gb300 import build as libbuild
    from paper_2405_03456_gb300 import hm

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    libbuild.build()
    hm.load()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    n = args.n
    pts = synth.sphere_points(n)
    xh = synth.rhs(n)[:, 0].copy()
    stream = torch.cuda.Stream()
    x = torch.from_numpy(xh).cuda()
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    results = {}
    clocks = ClockSampler(torch.cuda.current_device())
    headline = None
    eps_list = [float(e) for e in args.eps.split(",")]
    codecs = args.codecs.split(",")
    clocks_started = False
    for eps in eps_list:
        M = hm.HMatrix(pts, "laplace", 64, 2.0, "h", eps)
        for codec in codecs:
            M.compress(eps, codec, True)
            if not args.no_tune:
                M.autotune(5, stream.cuda_stream)
            if args.mr_engine != "auto":    # the multi-RHS engine, fixed instead of autotuned
                M.multi_rhs_engine({"tcgen05": 0, "fp32": 1}[args.mr_engine])
            M.graph(not args.no_graph)
            info = M.info()
            ab = info["bytes_alg"]          # the method's bytes (codes, their metadata, vectors)
            lb = M.alg_bytes()              # what the launches move, intermediates included
            if not clocks_started:
                clocks.start()
                clocks_started = True
            per, total = time_variant(torch, M, x, y, args.steps, args.warmup, stream, world)
            med = statistics.median(per)
            r = {"ms_p50": med, "ms_p99": pct(per, 0.99), "ms_mean": total / args.steps,
                 "gbs": ab / (med * 1e-3) / 1e9, "matvecs_per_s": 1e3 / med, "alg_bytes": ab, "layout_bytes": lb,
                 "payload_bytes": info["bytes_payload"], "value_bytes": info["bytes_values"],
                 "fp64_bytes": info["bytes_fp64"], "tier": info["tier"], "launches": info["nlaunches"],
                 "shapes": [s for s in M.launch_shapes() if s >= 0]}
            results[(eps, codec)] = r
            if (eps, codec) == HEADLINE:
                headline = dict(r)
                # roofline: per-kernel CUDA events on the launching stream
                M.profile(True)
                for _ in range(min(args.steps, 200)):
                    M.matvec(1.0, x, 1.0, y, stream=stream.cuda_stream)
                prof = M.profile_read()
                if not args.no_multi_rhs:   # precision / multi-RHS form on the same matrix
                    M.profile(False)
                    headline["by_nrhs"] = time_multi_rhs(torch, M, n, (1, 8, 32, 64), max(5, min(50, args.steps // 10)),
                                                         3, stream)
                    headline["multi_rhs_engine"] = ("tensor cores (tcgen05)", "FP32 pipes")[M.multi_rhs_engine()]
                    M.profile(True)
                M.profile(False)
                headline["kernels"] = prof
                # e2e: host buffers, copies inside the timed region
                xp = torch.from_numpy(xh.copy()).pin_memory().numpy()
                yp = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
                for _ in range(3):
                    M.matvec_host(1.0, xp, 1.0, yp, stream=stream.cuda_stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                esteps = max(1, min(args.steps, 500))
                e0.record(stream)
                for _ in range(esteps):
                    M.matvec_host(1.0, xp, 1.0, yp, stream=stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ems = e0.elapsed_time(e1) / esteps
                headline["e2e"] = {"value": ab / (ems * 1e-3) / 1e9 * world, "unit": "GB/s",
                                   "ms_per_step": ems, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n}
                # adjoint product y := M^H x + y on the same matrix (transposed matrix built on first use)
                aper, _ = time_variant(torch, M, x, y, max(20, min(args.steps, 200)), 3, stream, world, adjoint=True)
                amed = statistics.median(aper)
                headline["adjoint"] = {"ms_p50": round(amed, 4), "ms_p99": round(pct(aper, 0.99), 4),
                                       "gbs": round(ab / (amed * 1e-3) / 1e9, 1),
                                       "note": "M^H x on the same compressed matrix (transpose built on first use, "
                                               "launch shape 0); GB/s counts the forward product's algorithmic bytes"}
        M.close()
    # uniform-H and H^2 formats of the same problem (one persistent graph-captured product each)
    fmt_results = {}
    for fmt in [f for f in args.formats.split(",") if f]:
        eps = HEADLINE[0]
        M = hm.HMatrix(pts, "laplace", 64, 2.0, fmt, eps)
        for codec in ("none", "aflp"):
            M.compress(eps, codec, True)
            if not args.no_tune:
                M.autotune(5, stream.cuda_stream)
            M.graph(not args.no_graph)
            info = M.info()
            ab = info["bytes_alg"]
            per, total = time_variant(torch, M, x, y, args.steps, args.warmup, stream, world)
            med = statistics.median(per)
            mode = M.persistent_mode()
            fmt_results[(fmt, codec)] = {"ms_p50": med, "ms_p99": pct(per, 0.99), "gbs": ab / (med * 1e-3) / 1e9,
                                         "payload_bytes": info["bytes_payload"], "value_bytes": info["bytes_values"],
                                         "fp64_bytes": info["bytes_fp64"], "launches": info["nlaunches"],
                                         "persistent_mode": mode}
            if codec != "none":   # the whole product as ONE persistent launch (forward, coupling, backward)
                M.persistent(2)
                per2, _ = time_variant(torch, M, x, y, max(20, min(args.steps, 200)), 3, stream, world)
                fmt_results[(fmt, codec)]["one_launch_ms_p50"] = statistics.median(per2)
                M.persistent(mode)
        M.close()
    matern = None
    if args.matern:   # Matern nu = 1.5 covariance on the unit cube: multi-RHS products
        import numpy as np
        nm = args.matern
        t0 = time.perf_counter()
        M = hm.HMatrix(synth.cube_points(nm), "matern", 64, 2.0, "h", 1e-6, 0.1)
        M.compress(1e-6, "aflp", True)
        build_s = time.perf_counter() - t0
        if not args.no_tune:
            M.autotune(3, stream.cuda_stream)
        M.graph(not args.no_graph)
        info = M.info()
        xm = torch.from_numpy(synth.rhs(nm)[:, 0].copy()).cuda()
        ym = torch.zeros_like(xm)
        reps = max(5, min(50, args.steps))
        per, _ = time_variant(torch, M, xm, ym, reps, 3, stream, world)
        ab = info["bytes_alg"]
        single = {"ms_p50": round(statistics.median(per), 4), "gbs": round(ab / (statistics.median(per) * 1e-3) / 1e9, 1),
                  "hbm_frac": round(ab / (statistics.median(per) * 1e-3) / 1e9 / hbm_peak, 3)}
        matern = {"workload": f"matern-1.5 l=0.1 N={nm} uniform unit cube, leaf=64 eta=2 H eps=1e-6 AFLP VALR",
                  "payload_mb": round(info["bytes_payload"] / 1e6, 1), "fp64_mb": round(info["bytes_fp64"] / 1e6, 1),
                  "build_s": round(build_s, 1), "single_rhs": single,
                  "by_nrhs": time_multi_rhs(torch, M, nm, (1, 8, 32, 64), max(3, min(20, args.steps // 20)), 2,
                                            stream),
                  "multi_rhs_engine": ("tensor cores (tcgen05)", "FP32 pipes")[M.multi_rhs_engine()]}
        M.compress(1e-6, "none", True)   # the uncompressed FP64 product of the same matrix
        if not args.no_tune:
            M.autotune(3, stream.cuda_stream)
        per, _ = time_variant(torch, M, xm, ym, reps, 3, stream, world)
        matern["fp64_ms_p50"] = round(statistics.median(per), 4)
        if not args.no_cpu:   # the oracle on the host cores, a block sample of the same matrix
            try:
                cb = cpu_baseline_parallel(args.cpu_budget_mb, args.cpu_passes, 1, n=nm, kind="matern")
                matern["cpu_baseline"] = {k: (round(v, 5) if isinstance(v, float) else v) for k, v in cb.items()}
            except Exception as e:  # noqa: BLE001
                matern["cpu_baseline"] = {"value": None, "sample": f"failed: {e}"[:300]}
        matern["speedup_vs_fp64"] = round(statistics.median(per) / single["ms_p50"], 3)
        M.close()
    adm_legs = None
    if args.adm_legs:   # HODLR / BLR block trees of the sphere problem: huge top-level blocks vs a flat tiling
        adm_legs = {}
        na = args.adm_legs
        pa = synth.sphere_points(na)
        xa = torch.from_numpy(synth.rhs(na)[:, 0].copy()).cuda()
        ya = torch.zeros_like(xa)
        for adm in ("hodlr", "blr"):
            t0 = time.perf_counter()
            M = hm.HMatrix(pa, "laplace", 64, 2.0, "h", 1e-6, adm=adm)
            M.compress(1e-6, "aflp", True)
            build_s = time.perf_counter() - t0
            if not args.no_tune:
                M.autotune(3, stream.cuda_stream)
            M.graph(not args.no_graph)
            info = M.info()
            ab = info["bytes_alg"]
            per, _ = time_variant(torch, M, xa, ya, max(20, min(args.steps, 200)), 3, stream, world)
            med = statistics.median(per)
            adm_legs[adm] = {"ms_p50": round(med, 4), "gbs": round(ab / (med * 1e-3) / 1e9, 1),
                             "hbm_frac": round(ab / (med * 1e-3) / 1e9 / hbm_peak, 3),
                             "payload_mb": round(info["bytes_payload"] / 1e6, 1), "max_rank": info["max_rank"],
                             "nblocks": info["nblocks"], "build_s": round(build_s, 1)}
            M.close()
        adm_legs["workload"] = f"laplace sphere N={na}, leaf 64, H eps=1e-6 AFLP VALR; HODLR and BLR block trees"
    serving = None
    if args.serving != "none":
        lo, hi = (16384, 1048576) if args.serving == "full" else (16384, 131072)
        serving = serving_leg(torch, hm, lo, hi, args.serving_requests)
    clk = clocks.stop()

    # ------------------------------------------------------------ multi-rank reduction
    med = max_over_ranks(headline["ms_p50"], world)
    if rank != 0:
        return None
    ab = headline["alg_bytes"]
    value = whole_job_gbs(ab, med, world)
    prof = headline["kernels"]
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dk = prof[dom]
    per_launch_bytes = dk["bytes"] / max(dk["launches"], 1)
    per_launch_ms = dk["ms"] / max(dk["launches"], 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    tot_ms = sum(p["ms"] for p in prof.values())
    by_eps = {}
    for (eps, codec), r in results.items():
        base = results.get((eps, "none"))
        # the uncompressed FP64 product at the HBM roof: its bytes at the measured peak
        roof_ms = base["alg_bytes"] / (hbm_peak * 1e9) * 1e3 if base else None
        by_eps.setdefault(f"{eps:g}", {})[codec] = {
            "gbs": round(r["gbs"], 1), "matvecs_per_s": round(r["matvecs_per_s"], 1),
            "ms_p50": round(r["ms_p50"], 4), "ms_p99": round(r["ms_p99"], 4),
            "alg_mb": round(r["alg_bytes"] / 1e6, 1),
            "intermediate_mb": round((r["layout_bytes"] - r["alg_bytes"]) / 1e6, 1),
            "payload_mb": round(r["payload_bytes"] / 1e6, 1), "fp64_mb": round(r["fp64_bytes"] / 1e6, 1),
            "compression_ratio": round(r["fp64_bytes"] / max(r["value_bytes"], 1), 3),
            "speedup_vs_fp64": round(base["ms_p50"] / r["ms_p50"], 3) if base else None,
            "speedup_vs_fp64_at_roof": round(roof_ms / r["ms_p50"], 3) if base else None,
            "hbm_frac": round(r["gbs"] / hbm_peak, 3), "tier": "ff" if r["tier"] else "f32",
            "launch_shapes": r["shapes"]}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(med, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/ff decode of AFLP codes, f64 y",
        "data": "synthetic (seeded jittered Fibonacci sphere, x ~ U(-1,1))",
        "config": config_of(n, world),
        "matvecs_per_s": round(1e3 / med * world, 1), "ms_p50": round(med, 5),
        "ms_p99": round(headline["ms_p99"], 5),
        "hbm_frac": round(value / world / hbm_peak, 4),
        "bytes": {"alg_per_step": ab, "intermediate_per_step": headline["layout_bytes"] - ab,
                  "payload": headline["payload_bytes"], "codes": headline["value_bytes"],
                  "definition": "value = alg_per_step / median step time: packed codes + their inline metadata "
                                "(unit headers, per-column decode parameters and scales) + 24 N (x read, y read "
                                "and written) + 16 per coefficient (t_b written once and read once); "
                                "intermediate_per_step = the layout's extra traffic (copy descriptors, per-piece "
                                "input segments and multiplier runs, segment partials, fan-out slots), counted in "
                                "the per-kernel figures only"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak,
                     "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": profiled_traffic(dom, n),
                     "alg_bytes_per_launch": int(per_launch_bytes),
                     "peak_source": peak_src + " (MEASURED_PEAKS hbm_gbs copy bandwidth)",
                     "share": round(dk["ms"] / tot_ms, 3) if tot_ms else None,
                     "kernels": {k: {"ms_per_launch": round(v["ms"] / max(v["launches"], 1), 5),
                                     "launches": v["launches"],
                                     "gbs": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                                 for k, v in prof.items()}},
        "e2e": headline["e2e"],
        "adjoint": headline.get("adjoint"),
        "gpu_launches": int(headline["launches"] * args.steps),
        "clocks": clk,
        "by_eps": by_eps,
        "by_nrhs": {"workload": "the headline matrix, Y := M X with r right-hand sides (panels of 32 on the "
                               "multi-RHS engine the autotuner chose: FP32 pipes, or tcgen05 tensor cores with exact "
                               "BF16 limbs; per-piece FP32 sums, float-float across pieces; r < 9 as single products)",
                    "engine": headline.get("multi_rhs_engine"),
                    **headline.get("by_nrhs", {})},
        "by_format": {f"{f}-{c}": {"gbs": round(r["gbs"], 1), "ms_p50": round(r["ms_p50"], 4),
                                   "ms_p99": round(r["ms_p99"], 4), "payload_mb": round(r["payload_bytes"] / 1e6, 1),
                                   "compression_ratio": round(r["fp64_bytes"] / max(r["value_bytes"], 1), 3),
                                   "hbm_frac": round(r["gbs"] / hbm_peak, 3), "launches": r["launches"],
                                   "persistent_mode": r["persistent_mode"],
                                   "one_launch_ms_p50": (round(r["one_launch_ms_p50"], 4)
                                                         if "one_launch_ms_p50" in r else None),
                                   "speedup_vs_fp64": round(fmt_results[(f, "none")]["ms_p50"] / r["ms_p50"], 3)}
                      for (f, c), r in fmt_results.items()},
    }
    if matern is not None:
        line["matern_multi_rhs"] = matern
    if serving is not None:
        line["serving"] = serving
    if adm_legs is not None:
        line["hodlr_blr"] = adm_legs
    if not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline_parallel(args.cpu_budget_mb, args.cpu_passes, 1)
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {e}"[:300]}
    return line


# ------------------------------------------------------------------ reference arm
def config_of(n, world):
    """The workload's config (both arms report the same one)."""
    return {"workload": workload_name(n), "n": n, "eps": HEADLINE[0], "codec": "aflp-valr", "format": "H",
            "nrhs": 1, "parallelism": "replicas" if world > 1 else "single-gpu",
            "l2": "inputs larger than L2 (packed matrix ~0.96 GB vs 129 MB L2), no flush"}


def reference_arm(args, rank, world):
    """The oracle (the paper's Alg. 1 with Alg. 8 decode, FP64) on all host
    cores; each step is one pass over a bounded block sample of the workload."""
    if rank != 0:
        return None
    # size the per-step sample so that the whole run stays within a few minutes
    budget_mb = max(0.5, min(8.0, 200.0 / max(args.steps + args.warmup, 1)))
    cb = cpu_baseline_parallel(budget_mb, args.steps, args.warmup)
    value = cb["value"]
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(cb["pass_s_median"] * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded jittered Fibonacci sphere, x ~ U(-1,1))", "config": config_of(N_DEFAULT, world),
            "cpu_baseline": {"value": round(value, 5), "unit": "GB/s", "cores": cb["cores"], "nproc": cb["nproc"],
                             "cpu_model": cb["cpu_model"], "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": round(value, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": cb["wall_s"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--eps", default=",".join(f"{e:g}" for e in EPS_LIST))
    ap.add_argument("--codecs", default="none,aflp,fpx")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--formats", default="uh,uh_sep,h2")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuning)")
    ap.add_argument("--no-multi-rhs", action="store_true", help="skip the multi-RHS timings")
    ap.add_argument("--mr-engine", default="auto", choices=["auto", "tcgen05", "fp32"],
                    help="multi-RHS engine of the headline matrices (auto: the autotuner's choice)")
    ap.add_argument("--adm-legs", type=int, default=0,
                    help="also time HODLR and BLR H-matrices of the sphere problem at this N (opt-in)")
    ap.add_argument("--serving", default="small", choices=["none", "small", "full"],
                    help="serving leg: small = N in [16384, 131072] (default), full = [16384, 1048576] (slow to "
                         "build), none")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--matern", type=int, default=524288,
                    help="Matern cube leg (single and multi-RHS products) with this many points; 0 skips it "
                         "(the host build takes minutes)")
    ap.add_argument("--cpu-budget-mb", type=float, default=8.0, help="oracle sample per host core (MB of FP64)")
    ap.add_argument("--cpu-passes", type=int, default=10)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        line = reference_arm(args, rank, world)
        print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
        dist.barrier()
    line = gpu_arm(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
