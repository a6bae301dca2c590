"""Serving scheduler (continuous batching, admission by memory budget).

Host logic on the CPU with a deterministic fake executor and clock; the GPU
test at the end serves real compressed matrices and checks that every result
is the same alone and in the mix.
"""
import numpy as np
import pytest

import synth
from paper_2405_03456_gb300.serving import MAX_BATCH_RHS, Request, Scheduler, poisson_requests


class FakeExecutor:
    """y = A_mid @ x on the CPU; a product of r RHS takes a + b*r seconds of fake time."""

    def __init__(self, mats, a=1e-3, b=1e-4):
        self.A = {mid: np.random.default_rng(mid).standard_normal((n, n)) for mid, n in mats.items()}
        self.a, self.b = a, b
        self.now = 0.0
        self.log = []            # (mid, start, end, r)

    @staticmethod
    def staging_bytes(n, max_rhs):
        return 2 * 8 * n * max_rhs

    def launch(self, mid, slot, xs, adjoint=False):
        r = sum(x.reshape(x.shape[0], -1).shape[1] for x in xs)
        end = self.now + self.a + self.b * r
        self.log.append((mid, self.now, end, r))
        return (end, mid, xs, adjoint)

    def poll(self, h):
        end, mid, xs, adjoint = h
        if self.now < end:
            return None
        a = self.A[mid].T if adjoint else self.A[mid]
        return [a @ x for x in xs]

    def next_finish(self):
        return min((e for (_, _, e, _) in self.log if e > self.now), default=None)


class FakeClock:
    def __init__(self, ex):
        self.ex = ex

    def __call__(self):
        return self.ex.now

    def advance(self, ex, next_arrival):
        cand = [t for t in (ex.next_finish(), next_arrival) if t is not None]
        if cand:
            ex.now = max(ex.now, min(cand))


def make(mats, budget=10**12, nslots=2, adjoint=False):
    ex = FakeExecutor(mats)
    sch = Scheduler(ex, budget, nslots=nslots)
    for mid, n in mats.items():
        sch.add_matrix(mid, n, resident_bytes=1000, adjoint=adjoint)
    return ex, sch


def test_results_and_continuous_batching():
    mats = {0: 40, 1: 30, 2: 50}
    ex, sch = make(mats)
    reqs = poisson_requests(mats, rate=5000.0, count=200, seed=4)
    done = sch.run(reqs, clock=FakeClock(ex))
    assert len(done) == 200
    for q in done:
        assert np.allclose(q.y, ex.A[q.mid] @ q.x, rtol=1e-12, atol=1e-12)
        assert q.done >= q.arrival
    st = sch.stats()
    assert st["mean_batch_rhs"] > 20          # later arrivals joined the next launch
    assert all(r <= MAX_BATCH_RHS for (_, _, _, r) in ex.log)
    # one matrix never has two products in flight; different matrices do overlap
    overlap_diff = False
    for i, (m1, s1, e1, _) in enumerate(ex.log):
        for (m2, s2, e2, _) in ex.log[i + 1:]:
            if s2 < e1 and s1 < e2:
                assert m1 != m2
                overlap_diff = True
    assert overlap_diff


def test_budget_admission_and_backlog():
    mats = {0: 64}
    ex = FakeExecutor(mats)
    need = 1000 + FakeExecutor.staging_bytes(64, MAX_BATCH_RHS)
    with pytest.raises(MemoryError):
        Scheduler(ex, need - 1).add_matrix(0, 64, 1000)
    # room for the matrix plus 40 queued RHS of data: the rest waits in the backlog
    sch = Scheduler(ex, need + 16 * 64 * 40, nslots=1)
    sch.add_matrix(0, 64, 1000)
    reqs = [Request(k, 0, np.asfortranarray(np.ones((64, 16)) * k), 0.0) for k in range(6)]
    done = sch.run(reqs, clock=FakeClock(ex))
    assert [q.rid for q in sorted(done, key=lambda q: q.done)] == list(range(6))
    assert max(r for (_, _, _, r) in ex.log) <= 32      # at most 2 requests (40 RHS of room) admitted at once
    for q in done:
        assert np.allclose(q.y, ex.A[0] @ q.x)


def test_adjoint_requests_one_direction_per_launch():
    """Mixed M x and M^H x requests: every result is its own direction's product,
    a launch never mixes directions, and each matrix serves its requests in
    arrival order."""
    mats = {0: 24, 1: 36}
    ex, sch = make(mats, adjoint=True)
    reqs = poisson_requests(mats, rate=5000.0, count=150, seed=6, adjoint_frac=0.4)
    assert 20 < sum(q.adjoint for q in reqs) < 130
    launched = []
    orig = ex.launch

    def spy(mid, slot, xs, adjoint=False):
        launched.append((mid, adjoint, [id(x) for x in xs]))
        return orig(mid, slot, xs, adjoint=adjoint)

    ex.launch = spy
    done = sch.run(reqs, clock=FakeClock(ex))
    assert len(done) == 150
    by_x = {id(q.x): q for q in reqs}
    for mid, adjoint, xs in launched:
        assert all(by_x[x].adjoint == adjoint and by_x[x].mid == mid for x in xs)
    for q in done:
        a = ex.A[q.mid].T if q.adjoint else ex.A[q.mid]
        assert np.allclose(q.y, a @ q.x, rtol=1e-12, atol=1e-12)
    for mid in mats:
        order = [by_x[x].rid for (m, _, xs) in launched if m == mid for x in xs]
        assert order == sorted(order)


def test_rejects_bad_requests():
    ex, sch = make({0: 8})
    with pytest.raises(ValueError):
        sch.submit(Request(0, 5, np.zeros((8, 1)), 0.0), 0.0)
    with pytest.raises(ValueError):
        sch.submit(Request(1, 0, np.zeros((8, MAX_BATCH_RHS + 1)), 0.0), 0.0)
    with pytest.raises(ValueError):                          # registered without adjoint support
        sch.submit(Request(2, 0, np.zeros((8, 1)), 0.0, adjoint=True), 0.0)


def test_adjoint_support_counts_the_transposed_copy():
    ex = FakeExecutor({0: 8, 1: 8})
    stage = ex.staging_bytes(8, MAX_BATCH_RHS)
    sch = Scheduler(ex, budget_bytes=3000 + 2 * stage, nslots=2)
    sch.add_matrix(0, 8, resident_bytes=1000, adjoint=True)     # 2000 + staging
    assert sch.used == 2000 + stage
    with pytest.raises(MemoryError):
        sch.add_matrix(1, 8, resident_bytes=1000, adjoint=True)
    sch.add_matrix(1, 8, resident_bytes=1000)                    # fits without its transpose
    assert sch.used == 3000 + 2 * stage


def test_stats_by_hand():
    # one matrix, one slot; products take 1 ms + 0.1 ms per RHS of fake time
    ex = FakeExecutor({0: 8})
    sch = Scheduler(ex, budget_bytes=10**9, nslots=1)
    sch.add_matrix(0, 8, 1000)
    x = lambda r: np.asfortranarray(np.ones((8, r)))
    ex.now = 0.5                                      # the stream starts at 0.5 s
    reqs = [Request(0, 0, x(2), 0.5), Request(1, 0, x(3), 0.5), Request(2, 0, x(1), 0.51)]
    sch.run(reqs, clock=FakeClock(ex))
    # requests 0 and 1 share one launch ending 1.5 ms later; request 2 runs alone, 0.51 s .. 0.5111 s
    st = sch.stats()
    assert (st["requests"], st["rhs"], st["launches"]) == (3, 6, 2)
    assert st["mean_batch_rhs"] == 3.0
    assert st["p50_ms"] == pytest.approx(1.5) and st["max_ms"] == pytest.approx(1.5)
    assert st["p99_ms"] == pytest.approx(1.5)
    assert st["seconds"] == pytest.approx(0.0111)
    assert st["requests_per_s"] == pytest.approx(3 / 0.0111) and st["rhs_per_s"] == pytest.approx(6 / 0.0111)


def test_oldest_waiting_request_goes_first():
    # the slot is busy with matrix 2; meanwhile matrix 1 gets a request before matrix 0
    ex = FakeExecutor({0: 8, 1: 8, 2: 8})
    sch = Scheduler(ex, budget_bytes=10**9, nslots=1)
    for mid in (0, 1, 2):
        sch.add_matrix(mid, 8, 1000)
    x = np.asfortranarray(np.ones((8, 1)))
    sch.run([Request(0, 2, x, 0.0), Request(1, 1, x, 1e-4), Request(2, 0, x, 2e-4)], clock=FakeClock(ex))
    assert [mid for (mid, _, _, _) in ex.log] == [2, 1, 0]


def test_batch_fills_exactly_max_rhs():
    ex = FakeExecutor({0: 8})
    sch = Scheduler(ex, budget_bytes=10**9, nslots=1)
    sch.add_matrix(0, 8, 1000)
    x = lambda r: np.asfortranarray(np.ones((8, r)))
    reqs = [Request(0, 0, x(1), 0.0), Request(1, 0, x(MAX_BATCH_RHS - 8), 1e-4), Request(2, 0, x(8), 1e-4),
            Request(3, 0, x(1), 1e-4)]
    sch.run(reqs, clock=FakeClock(ex))
    assert [r for (_, _, _, r) in ex.log] == [1, MAX_BATCH_RHS, 1]


def test_admission_at_the_exact_budget():
    ex = FakeExecutor({0: 8})
    need = 1000 + FakeExecutor.staging_bytes(8, MAX_BATCH_RHS)
    sch = Scheduler(ex, need + 16 * 8 * MAX_BATCH_RHS, nslots=1)
    sch.add_matrix(0, 8, 1000)
    sch.submit(Request(0, 0, np.zeros((8, MAX_BATCH_RHS)), 0.0), 0.0)   # the largest request, exactly fitting
    assert not sch.backlog and sch.queued_bytes == 16 * 8 * MAX_BATCH_RHS
    sch.submit(Request(1, 0, np.zeros((8, 1)), 0.0), 0.0)                # one more RHS does not fit
    assert [q.rid for q in sch.backlog] == [1]
    # two requests that each fill the budget: the second leaves the backlog once the first is done
    sch = Scheduler(ex, need + 16 * 8 * MAX_BATCH_RHS, nslots=1)
    sch.add_matrix(0, 8, 1000)
    x = np.asfortranarray(np.ones((8, MAX_BATCH_RHS)))
    done = sch.run([Request(0, 0, x, 0.0), Request(1, 0, x, 0.0)], clock=FakeClock(ex))
    assert [q.rid for q in done] == [0, 1]


def test_poisson_request_ranges():
    reqs = poisson_requests({0: 8, 1: 8}, rate=1000.0, count=2000, seed=3, rhs_max=4, adjoint_frac=0.5)
    rs = sorted({q.r for q in reqs})
    assert rs == [1, 2, 3, 4]
    assert sorted({q.mid for q in reqs}) == [0, 1]
    arr = np.array([q.arrival for q in reqs])
    assert np.all(np.diff(arr) > 0) and 1.5 < arr[-1] < 2.5          # 2000 arrivals at 1000 per second
    assert 800 < sum(q.adjoint for q in reqs) < 1200
    assert not any(q.adjoint for q in poisson_requests({0: 8}, 1000.0, 200, seed=3))
    assert all(q.adjoint for q in poisson_requests({0: 8}, 1000.0, 200, seed=3, adjoint_frac=1.0))


@pytest.mark.gpu
def test_gpu_serving_alone_equals_mix():
    """Four resident matrices of every format (H, UH, H^2, UH with separate
    couplings; AFLP and FPX; eps 1e-4 .. 1e-8), a Poisson stream with 30 %
    adjoint requests: products of different matrices -- the UH / H^2 / UH_SEP
    ones as persistent cooperative launches -- run concurrently on three slot
    streams.  Every result must lie within 4 eps of the same request computed
    alone (one product of just its columns, on the default stream) and within
    4 eps of the CPU oracle's product of the uncompressed matrix."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from oracle import hmatrix, matvec, nested
    from paper_2405_03456_gb300 import build, hm
    from paper_2405_03456_gb300.serving import GpuExecutor
    build.build()
    specs = {0: ("laplace", 2048, 1e-6, "h", "aflp"), 1: ("matern", 3000, 1e-4, "uh", "fpx"),
             2: ("laplace", 4096, 1e-8, "h2", "aflp"), 3: ("laplace", 2048, 1e-6, "uh_sep", "fpx")}
    ex = GpuExecutor(nslots=3)
    sch = Scheduler(ex, budget_bytes=8 << 30, nslots=3)
    Ms, oracles = {}, {}
    for mid, (kern, n, eps, fmt, codec) in specs.items():
        pts = synth.sphere_points(n) if kern == "laplace" else synth.cube_points(n)
        M = hm.HMatrix(pts, kern, 64, 2.0, fmt, eps).compress(eps, codec)
        Ms[mid] = M
        info = M.info()
        sch.add_matrix(mid, n, info["bytes_payload"] + info["bytes_meta"] + info["bytes_workspace"], adjoint=True)
        ex.add(mid, M, prepare_adjoint=True)
        h = hmatrix.build_h(pts, kern, 64, 2.0, eps)
        if fmt == "h":
            oracles[mid] = (h, matvec.h_mvm, matvec.h_mvm_adjoint)
        elif fmt == "h2":
            oracles[mid] = (nested.build_h2(h), matvec.h2_mvm, matvec.h2_mvm_adjoint)
        else:   # separate couplings: the same product as single couplings (uncompressed, to 1e-13)
            oracles[mid] = (nested.build_uniform(h), matvec.uh_mvm, matvec.uh_mvm_adjoint)
    reqs = poisson_requests({m: s[1] for m, s in specs.items()}, rate=20000.0, count=80, seed=8, adjoint_frac=0.3)
    done = sch.run(reqs)
    assert len(done) == 80
    st = sch.stats()
    assert st["mean_batch_rhs"] > 1 and any(q.adjoint for q in done) and not all(q.adjoint for q in done)
    for q in done:
        eps = specs[q.mid][2]
        n = specs[q.mid][1]
        xd = torch.from_numpy(np.asfortranarray(q.x.reshape(n, -1))).cuda().t().contiguous().t()
        yd = torch.zeros_like(xd)
        Ms[q.mid].matvec(1.0, xd, 0.0, yd, adjoint=q.adjoint)
        torch.cuda.synchronize()
        alone = yd.cpu().numpy().reshape(q.y.shape)
        m, f, fa = oracles[q.mid]
        ref = (fa if q.adjoint else f)(m, 1.0, q.x, 0.0)
        assert np.linalg.norm(q.y - alone) <= 4 * eps * np.linalg.norm(alone), (q.mid, q.adjoint)
        assert np.linalg.norm(q.y - ref) <= 4 * eps * np.linalg.norm(ref), (q.mid, q.adjoint)
    for M in Ms.values():
        assert M.sync_status() == 0
        M.close()
