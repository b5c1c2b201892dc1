"""Host logic of the request loop (admission by HBM budget, arrival order,
completion handling, statistics) with a fake device backend; no GPU."""
import numpy as np
import pytest

from paper_2001_06113_gb300.serve import Backend, Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3          # every clock read advances 1 ms
        return self.t


class FakeBackend(Backend):
    """A solve takes `nsteps` polls after it starts; workspace = points * 10 bytes."""

    def __init__(self):
        self.log = []
        self.live = 0
        self.max_live_bytes = 0

    def prepare(self, req):
        return {"req": req, "left": None, "bytes": req.points * 10}

    def workspace_bytes(self, h):
        return h["bytes"]

    def start(self, h):
        h["left"] = h["req"].nsteps
        self.live += h["bytes"]
        self.max_live_bytes = max(self.max_live_bytes, self.live)
        self.log.append(("start", h["req"].rid))

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def finish(self, h):
        self.live -= h["bytes"]
        self.log.append(("finish", h["req"].rid))
        return np.full(3, h["req"].rid, dtype=np.complex128)

    def release(self, h):
        if h["left"] is not None:
            self.live -= h["bytes"]


class Inst:
    def __init__(self, shape, nsteps):
        self.shape = shape
        self.nsteps = nsteps


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(n):
        t += rng.exponential(0.005)
        out.append(Request(i, t, Inst((int(rng.choice([64, 256, 1024])),), int(rng.integers(2, 20)))))
    return out


def test_admission_respects_budget_and_order():
    reqs = _requests(60)
    be = FakeBackend()
    budget = 1024 * 10 * 3                      # at most three of the largest at once
    srv = Server(be, budget, max_active=8, clock=FakeClock(), idle_sleep=0)
    st = srv.run(reqs)
    assert be.max_live_bytes <= budget and srv.peak_bytes <= budget
    assert srv.peak_active <= 8
    starts = [rid for kind, rid in be.log if kind == "start"]
    assert starts == sorted(starts)             # admitted in arrival order
    for r in reqs:
        assert r.admitted >= r.arrival and r.finished > r.admitted
        assert r.result[0] == r.rid
    assert st["requests"] == 60 and st["p99_s"] >= st["p50_s"] > 0
    assert st["point_steps"] == sum(r.points * r.nsteps for r in reqs)


def test_requests_overlap_when_memory_allows():
    reqs = [Request(i, 0.0, Inst((64,), 50)) for i in range(10)]
    be = FakeBackend()
    srv = Server(be, 10 ** 9, max_active=16, clock=FakeClock(), idle_sleep=0)
    srv.run(reqs)
    assert srv.peak_active == 10                # all in flight together
    kinds = [k for k, _ in be.log]
    assert kinds[:10] == ["start"] * 10


def test_oversize_request_rejected():
    be = FakeBackend()
    srv = Server(be, 100, clock=FakeClock(), idle_sleep=0)
    with pytest.raises(ValueError):
        srv.run([Request(0, 0.0, Inst((64,), 3))])


class FailingBackend(FakeBackend):
    """Start fails for some requests (as a device allocation failure would);
    the result of others is not finite."""

    def __init__(self, fail_start=(), fail_finish=()):
        super().__init__()
        self.fail_start, self.fail_finish = set(fail_start), set(fail_finish)
        self.released = []

    def start(self, h):
        if h["req"].rid in self.fail_start:
            raise MemoryError("no device memory for the workspace")
        super().start(h)

    def finish(self, h):
        if h["req"].rid in self.fail_finish:
            self.live -= h["bytes"]
            raise FloatingPointError("non-finite values in the mode state")
        return super().finish(h)

    def release(self, h):
        self.released.append(h["req"].rid)
        super().release(h)


def test_failures_stay_with_their_request():
    reqs = _requests(30, seed=1)
    be = FailingBackend(fail_start={3, 7}, fail_finish={11})
    srv = Server(be, 1024 * 10 * 4, max_active=8, clock=FakeClock(), idle_sleep=0)
    st = srv.run(reqs)
    assert st["failed"] == 3 and st["completed"] == 27 and st["cancelled"] == 0
    assert reqs[3].error.startswith("start") and reqs[11].error.startswith("finish")
    assert 3 in be.released and 7 in be.released
    assert all(r.result is not None for r in reqs if r.error is None)
    assert be.live == 0                               # every workspace given back


def test_cancellation_waiting_and_active():
    reqs = [Request(i, 0.0, Inst((1024,), 40)) for i in range(4)]
    reqs[0].cancel_after = 0.005                      # active: runs out, result dropped
    reqs[3].cancel_after = 0.0                        # still waiting (budget): never starts
    be = FakeBackend()
    srv = Server(be, 1024 * 10 * 2, max_active=8, clock=FakeClock(), idle_sleep=0)
    st = srv.run(reqs)
    assert st["cancelled"] == 2 and st["completed"] == 2
    assert reqs[0].result is None and reqs[0].admitted is not None
    assert reqs[3].admitted is None
    assert ("start", 3) not in be.log and be.live == 0


def test_trace_routes_free_space_by_precision():
    """requests_from_trace: periodic classes in mixed precision; free space in
    FP64 on the eps = 1e-10 contour or with FP32 transforms on the contour for
    eps = 1e-4 with FP32 sums (smaller H, same nu = 8 n)."""
    pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import math
    import synth
    from paper_2001_06113_gb300.serve import requests_from_trace
    trace = synth.serve_requests(seed=3, rate=80.0, duration=0.2, T_range=(0.01, 0.02), sizes_1d=(1024,),
                                 sizes_2d=(128,), sizes_free=(64,))
    f64 = requests_from_trace(trace)
    f32 = requests_from_trace(trace, free_precision="mixed")
    assert any(r.bc == "free" for r in f64)
    for a, b in zip(f64, f32):
        assert a.bc == b.bc
        if a.bc != "free":
            assert a.precision == b.precision == "mixed"
            continue
        assert (a.precision, b.precision) == ("fp64", "mixed")
        assert a.free["nu"] == b.free["nu"] == [8 * n for n in a.inst.shape]
        # same ||V|| and phi_max, machine epsilon 2^-52 at 1e-10 against 2^-23 at 1e-4
        d = a.inst.dim
        lhs = a.free["H"] * 2 * d                        # = log(eps / ((1 + |V|) eps_m)) / (1 + phimax)
        rhs = b.free["H"] * 2 * d
        ratio = (lhs - rhs) / (math.log(1e-10 / 1e-4) + 29 * math.log(2.0))
        assert 0.0 < ratio <= 1.0 + 1e-12                 # = 1 / (1 + phimax)
