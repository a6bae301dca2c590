"""Request serving: continuous batching of matvec requests on resident matrices.

Several compressed H-matrices stay resident in HBM.  Requests (matrix id, a
host block of 1..32 right-hand sides, arrival time) are admitted while the
memory they need fits the budget; each matrix has a FIFO queue.  Whenever a
stream slot is free and a matrix has no product in flight, the queued
requests of that matrix (up to 64 right-hand sides) are packed into one
multi-RHS product y := M X on that slot's stream: upload of X, hm_matvec,
download of Y.  Requests that arrive while others run wait only for their
matrix and a slot, so products of different matrices overlap on the device
and later arrivals join the next launch ("continuous batching").  Products of
one matrix never overlap, because they share its device workspace.  A request
may ask for the adjoint product y := M^H X instead (hm_matvec_adjoint); a launch
packs consecutive requests of one direction only, so the FIFO order of every
matrix is kept.

The scheduler is host logic with a pluggable executor: ``GpuExecutor`` runs
the products through libhm on CUDA streams; tests drive the same scheduler
with a deterministic fake executor on the CPU.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

MAX_BATCH_RHS = 64


@dataclass
class Request:
    rid: int
    mid: int                      # matrix id
    x: np.ndarray                 # (n, r) FP64 host, Fortran order
    arrival: float                # seconds from the start of the run
    admitted: float = -1.0
    done: float = -1.0
    y: np.ndarray | None = None
    adjoint: bool = False         # y := M^H x instead of M x

    @property
    def r(self) -> int:
        return 1 if self.x.ndim == 1 else self.x.shape[1]


@dataclass
class Launch:
    mid: int
    slot: int
    reqs: list
    handle: object = None


@dataclass
class MatrixSlot:
    mid: int
    n: int
    resident_bytes: int
    queue: list = field(default_factory=list)
    busy: bool = False
    adjoint: bool = False         # serves M^H x requests (its transposed copy is resident too)


class Scheduler:
    """Admission by memory budget, per-matrix FIFO queues, continuous batching."""

    def __init__(self, executor, budget_bytes: int, nslots: int = 4, max_batch_rhs: int = MAX_BATCH_RHS):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.nslots = nslots
        self.max_rhs = max_batch_rhs
        self.mats: dict[int, MatrixSlot] = {}
        self.used = 0                 # resident matrices + staging
        self.queued_bytes = 0         # host-side request data waiting for a launch
        self.free_slots = list(range(nslots))
        self.inflight: list[Launch] = []
        self.backlog: list[Request] = []
        self.finished: list[Request] = []
        self.launches = 0
        self.rhs_launched = 0

    # -------------------------------------------------------------- matrices
    def add_matrix(self, mid: int, n: int, resident_bytes: int, adjoint: bool = False) -> None:
        """Register a resident matrix; refuses it if the budget would be exceeded.
        adjoint: the matrix also serves M^H x requests, which run on its transposed
        copy (the same codes rearranged), counted as a second resident_bytes."""
        need = resident_bytes * (2 if adjoint else 1) + self.ex.staging_bytes(n, self.max_rhs)
        if self.used + need > self.budget:
            raise MemoryError(f"matrix {mid}: {need} bytes exceed the remaining budget "
                              f"{self.budget - self.used}")
        self.used += need
        self.mats[mid] = MatrixSlot(mid, n, resident_bytes, adjoint=adjoint)

    # -------------------------------------------------------------- requests
    def _req_bytes(self, req: Request) -> int:
        return 16 * self.mats[req.mid].n * req.r

    def submit(self, req: Request, now: float) -> None:
        """Admit a request if its data fits next to what is queued, else keep it in the backlog."""
        if req.r < 1 or req.r > self.max_rhs or req.mid not in self.mats:
            raise ValueError(f"request {req.rid}: bad matrix or RHS count")
        if req.adjoint and not self.mats[req.mid].adjoint:
            raise ValueError(f"request {req.rid}: matrix {req.mid} was registered without adjoint support")
        if self.backlog or self.used + self.queued_bytes + self._req_bytes(req) > self.budget:
            self.backlog.append(req)
            return
        self._admit(req, now)

    def _admit(self, req: Request, now: float) -> None:
        req.admitted = now
        self.queued_bytes += self._req_bytes(req)
        self.mats[req.mid].queue.append(req)

    def _drain_backlog(self, now: float) -> None:
        while self.backlog and self.used + self.queued_bytes + self._req_bytes(self.backlog[0]) <= self.budget:
            self._admit(self.backlog.pop(0), now)

    # -------------------------------------------------------------- launches
    def _start(self, now: float) -> None:
        while self.free_slots:
            ready = [m for m in self.mats.values() if m.queue and not m.busy]
            if not ready:
                return
            m = min(ready, key=lambda m: m.queue[0].arrival)       # oldest waiting request first
            adj = m.queue[0].adjoint                                 # one direction per launch
            batch, r = [], 0
            while m.queue and m.queue[0].adjoint == adj and r + m.queue[0].r <= self.max_rhs:
                req = m.queue.pop(0)
                batch.append(req)
                r += req.r
            slot = self.free_slots.pop(0)
            m.busy = True
            L = Launch(m.mid, slot, batch)
            L.handle = self.ex.launch(m.mid, slot, [q.x for q in batch], adjoint=adj)
            self.inflight.append(L)
            self.launches += 1
            self.rhs_launched += r

    def _poll(self, now_fn) -> int:
        done = 0
        for L in list(self.inflight):
            ys = self.ex.poll(L.handle)
            if ys is None:
                continue
            t = now_fn()
            for req, yv in zip(L.reqs, ys):
                req.y = yv
                req.done = t
                self.queued_bytes -= self._req_bytes(req)
                self.finished.append(req)
            self.mats[L.mid].busy = False
            self.free_slots.append(L.slot)
            self.inflight.remove(L)
            done += 1
        return done

    def run(self, requests: list, clock=None, idle_sleep: float = 0.0) -> list:
        """Serve requests (sorted by arrival) against `clock()` seconds; returns them when done."""
        clock = clock or _WallClock()
        pending = sorted(requests, key=lambda q: q.arrival)
        i = 0
        while i < len(pending) or self.inflight or self.backlog or any(m.queue for m in self.mats.values()):
            now = clock()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i], now)
                i += 1
            self._drain_backlog(now)
            self._start(now)
            progressed = self._poll(clock)
            if not progressed and idle_sleep:
                time.sleep(idle_sleep)
            if hasattr(clock, "advance") and not progressed:
                nxt = pending[i].arrival if i < len(pending) else None
                clock.advance(self.ex, nxt)
        return self.finished

    # -------------------------------------------------------------- metrics
    def stats(self) -> dict:
        lat = np.array([q.done - q.arrival for q in self.finished])
        t0 = min(q.arrival for q in self.finished)
        t1 = max(q.done for q in self.finished)
        rhs = sum(q.r for q in self.finished)
        return {"requests": len(self.finished), "rhs": rhs, "launches": self.launches,
                "mean_batch_rhs": self.rhs_launched / max(self.launches, 1),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3), "seconds": t1 - t0,
                "requests_per_s": len(self.finished) / max(t1 - t0, 1e-12),
                "rhs_per_s": rhs / max(t1 - t0, 1e-12)}


class _WallClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def __call__(self) -> float:
        return time.perf_counter() - self.t0


def poisson_requests(mats: dict, rate: float, count: int, seed: int, rhs_max: int = 32,
                     adjoint_frac: float = 0.0) -> list:
    """Seeded Poisson arrivals (rate per second), matrix uniform, RHS count U{1..rhs_max}, x ~ U(-1,1);
    a fraction adjoint_frac of the requests asks for M^H x (drawn only when adjoint_frac > 0)."""
    rng = np.random.default_rng(seed)
    mids = sorted(mats)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        mid = mids[int(rng.integers(len(mids)))]
        r = int(rng.integers(1, rhs_max + 1))
        x = np.asfortranarray(rng.uniform(-1.0, 1.0, (mats[mid], r)))
        adj = bool(rng.random() < adjoint_frac) if adjoint_frac > 0 else False
        out.append(Request(k, mid, x, t, adjoint=adj))
    return out


# ---------------------------------------------------------------------- GPU executor
class GpuExecutor:
    """Runs packed products through libhm: one CUDA stream per slot, pinned staging per matrix."""

    def __init__(self, nslots: int, max_rhs: int = MAX_BATCH_RHS):
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(nslots)]
        self.max_rhs = max_rhs
        self.mats = {}

    @staticmethod
    def staging_bytes(n: int, max_rhs: int) -> int:
        return 2 * 8 * n * max_rhs          # device X and Y blocks

    def add(self, mid: int, M, prepare_adjoint: bool = False) -> None:
        """Register M; prepare_adjoint builds its transposed matrix now (one adjoint
        product of zeros), so that no adjoint request waits for it."""
        torch = self.torch
        n = M.n
        if prepare_adjoint:
            z = torch.zeros(n, dtype=torch.float64, device="cuda")
            M.matvec(1.0, z, 0.0, torch.zeros_like(z), adjoint=True)
            torch.cuda.synchronize()
        self.mats[mid] = {
            "M": M, "n": n,
            "dx": torch.empty((self.max_rhs, n), dtype=torch.float64, device="cuda"),
            "dy": torch.empty((self.max_rhs, n), dtype=torch.float64, device="cuda"),
            "hx": torch.empty((self.max_rhs, n), dtype=torch.float64).pin_memory(),
            "hy": torch.empty((self.max_rhs, n), dtype=torch.float64).pin_memory(),
        }

    def launch(self, mid: int, slot: int, xs: list, adjoint: bool = False):
        from . import hm
        torch = self.torch
        e = self.mats[mid]
        st = self.streams[slot]
        n = e["n"]
        cols = [x.reshape(n, -1) for x in xs]
        r = sum(c.shape[1] for c in cols)
        hx = e["hx"].numpy()
        k = 0
        for c in cols:                      # row j of hx = right-hand side j (column-major X)
            hx[k:k + c.shape[1]] = c.T
            k += c.shape[1]
        with torch.cuda.stream(st):
            e["dx"][:r].copy_(e["hx"][:r], non_blocking=True)
            f = hm.hm_matvec_adjoint if adjoint else hm.hm_matvec
            f(e["M"].h, 1.0, e["dx"].data_ptr(), n, 0.0, e["dy"].data_ptr(), n, r, st.cuda_stream)
            e["hy"][:r].copy_(e["dy"][:r], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, mid, [c.shape[1] for c in cols])

    def poll(self, handle):
        ev, mid, widths = handle
        if not ev.query():
            return None
        hy = self.mats[mid]["hy"].numpy()
        out, k = [], 0
        for w in widths:
            out.append(np.asfortranarray(hy[k:k + w].T.copy()))
            k += w
        return out
