"""Host logic of the served request stream (no GPU): admission order, slot
and HBM-budget limits, rejection of requests that can never fit, overlap of
the rod and shell iterations, and per-request results that do not depend on
what else is resident."""
import dataclasses
import threading
import time

import numpy as np

from paper_2510_10256_gb300.serve import Request, Server, StepResult, poisson_requests


@dataclasses.dataclass
class FakeScene:
    kind: str
    n: int
    meta: dict = dataclasses.field(default_factory=dict)
    p: np.ndarray = dataclasses.field(default_factory=lambda: np.ones((3, 4)))


class FakeEngine:
    """Footprint n bytes; a step sleeps a little and returns values that
    depend only on the request and the step (as the real pass must)."""

    def __init__(self, budget, step_s=0.002):
        self.budget = budget
        self.step_s = step_s
        self.live = {}
        self.created = []
        self.max_live_bytes = 0
        self.max_live = 0
        self.concurrent = 0
        self.max_concurrent = 0
        self.lock = threading.Lock()

    def footprint(self, req):
        return req.scene.n

    def create(self, req):
        with self.lock:
            h = {"req": req, "step": 0}
            self.live[id(h)] = req.scene.n
            self.created.append(req.rid)
            self.max_live_bytes = max(self.max_live_bytes, sum(self.live.values()))
            self.max_live = max(self.max_live, len(self.live))
            assert sum(self.live.values()) <= self.budget
        return h

    def run_step(self, kind, handles):
        with self.lock:
            self.concurrent += 1
            self.max_concurrent = max(self.max_concurrent, self.concurrent)
        time.sleep(self.step_s)
        out = []
        for h in handles:
            assert h["req"].kind == kind
            out.append(StepResult(energy=float(h["req"].rid), alpha=1.0 / (1 + h["step"])))
            h["step"] += 1
        with self.lock:
            self.concurrent -= 1
        return out, 10 * len(handles)

    def release(self, h):
        with self.lock:
            del self.live[id(h)]


def _reqs(n, rate=2000.0, steps=3, seed=3):
    pool = [FakeScene("rod", 100), FakeScene("rod", 300), FakeScene("shell", 200), FakeScene("shell", 500)]
    return poisson_requests(pool, n, rate, steps, seed)


def test_every_request_completes_within_limits():
    reqs = _reqs(40)
    eng = FakeEngine(budget=1200)
    rep = Server(eng, hbm_budget=1200, max_slots=5, keep_results=True).run(reqs)
    assert rep["steps"] == 40 * 3 and rep["requests"] == 40 and not rep["rejected"]
    assert eng.max_live <= 5 and eng.max_live_bytes <= 1200
    assert rep["max_resident"] <= 5
    assert rep["peak_reserved_bytes"] <= 1200
    assert not eng.live  # everything released
    # FIFO admission: scenes are created in arrival order
    order = [r.rid for r in sorted(reqs, key=lambda r: (r.arrival, r.rid))]
    assert eng.created == order
    # results depend only on the request and the step
    for r in reqs:
        res = rep["results"][r.rid]
        assert [x.alpha for x in res] == [1.0, 0.5, 1.0 / 3]
        assert all(x.energy == float(r.rid) for x in res)
    assert rep["pairs"] == 10 * rep["steps"]
    lat = rep["step_latency_ms"]
    assert lat["p50"] is not None and lat["p99"] >= lat["p50"] > 0


def test_batching_and_overlap():
    reqs = _reqs(30, rate=5000.0, steps=4)
    eng = FakeEngine(budget=10_000, step_s=0.004)
    rep = Server(eng, hbm_budget=10_000, max_slots=16).run(reqs)
    # several requests share an iteration, and rods and shells run at once
    assert rep["iterations"] < rep["steps"]
    assert rep["max_resident"] > 2
    assert eng.max_concurrent == 2


def test_oversized_request_is_rejected_not_stalled():
    pool = [FakeScene("rod", 100), FakeScene("shell", 5000)]
    reqs = [Request(0, 0.0, pool[0], 2), Request(1, 0.0, pool[1], 2), Request(2, 0.001, pool[0], 2)]
    eng = FakeEngine(budget=1000)
    rep = Server(eng, hbm_budget=1000, max_slots=4).run(reqs)
    assert rep["rejected"] == [1]
    assert rep["steps"] == 4


def test_budget_blocks_admission_until_memory_frees():
    pool = [FakeScene("shell", 600)]
    reqs = [Request(i, 0.0, pool[0], 2) for i in range(4)]
    eng = FakeEngine(budget=1000)
    rep = Server(eng, hbm_budget=1000, max_slots=4).run(reqs)
    assert eng.max_live == 1 and rep["steps"] == 8


def test_poisson_stream_is_seeded():
    pool = [FakeScene("rod", 10), FakeScene("shell", 20)]
    a = poisson_requests(pool, 200, 200.0, 10, 5)
    b = poisson_requests(pool, 200, 200.0, 10, 5)
    assert [(r.arrival, r.scene.kind, r.seed) for r in a] == [(r.arrival, r.scene.kind, r.seed) for r in b]
    gaps = np.diff([r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 200.0) < 0.3 / 200.0
    kinds = [r.kind for r in a]
    assert 60 < kinds.count("rod") < 140


def test_plain_form_runs_fifo_one_request_at_a_time():
    """run_plain, the comparison arm of the served stream: the same trace in
    arrival order, one request and one single-scene step at a time."""
    from paper_2510_10256_gb300.serve import run_plain
    reqs = _reqs(12, rate=4000.0, steps=3)
    eng = FakeEngine(budget=10_000, step_s=0.001)
    rep = run_plain(eng, reqs)
    assert rep["steps"] == 12 * 3 and rep["iterations"] == rep["steps"]
    assert eng.max_live == 1 and eng.max_concurrent == 1 and not eng.live
    assert eng.created == [r.rid for r in sorted(reqs, key=lambda r: (r.arrival, r.rid))]
    assert rep["pairs"] == 10 * rep["steps"]
    lat = rep["step_latency_ms"]
    assert lat["p99"] >= lat["p50"] > 0
    # the served form batches the same trace into fewer iterations
    served = Server(FakeEngine(budget=10_000, step_s=0.001), hbm_budget=10_000, max_slots=16).run(reqs)
    assert served["steps"] == rep["steps"] and served["iterations"] < rep["iterations"]


def test_budget_is_charged_from_the_memory_really_held():
    """An engine that reports the device memory its resident requests really
    hold (live_bytes) is charged that, not the smaller footprint estimate:
    here every scene holds five times its estimate, so while the first
    request is resident (1000 of an 1100 budget) nothing else is admitted,
    which the estimates alone (200 each) would allow."""
    pool = [FakeScene("shell", 200)]
    # the first request is resident (3 steps of 20 ms) when the others arrive
    reqs = [Request(i, 0.0 if i == 0 else 0.02, pool[0], 3) for i in range(4)]

    class Heavy(FakeEngine):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            self.events = []

        def create(self, req):
            h = super().create(req)
            with self.lock:
                self.events.append(("create", req.rid))
            return h

        def release(self, h):
            with self.lock:
                self.events.append(("release", h["req"].rid))
            super().release(h)

        def live_bytes(self):
            with self.lock:
                return 5 * sum(self.live.values())

    eng = Heavy(budget=10_000, step_s=0.02)
    rep = Server(eng, hbm_budget=1100, max_slots=4).run(reqs)
    assert rep["steps"] == 12
    assert eng.events[:2] == [("create", 0), ("release", 0)], eng.events
    assert rep["peak_live_bytes"] >= 1000
    # without the report the estimates alone let the others in beside the first
    eng2 = Heavy(budget=10_000, step_s=0.02)
    eng2.live_bytes = None
    Server(eng2, hbm_budget=1100, max_slots=4).run(reqs)
    assert eng2.events[1][0] == "create", eng2.events
