"""Scheduling logic of the continuous-batching service, on a fake engine and clock (CPU)."""
import pytest

from paper_1002_3028_gb300 import inputs as I
from paper_1002_3028_gb300.serve import Engine, serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeEngine(Engine):
    """Steps cost 1 us per thousand active nodes; a retired copy takes 0.5 ms."""

    def __init__(self, clock):
        self.clock = clock
        self.active = {}
        self.steps_done = {}
        self.used = 0
        self.max_used = 0
        self.admit_order = []
        self.log = []

    def bytes_needed(self, req):
        return req.workload.nodes * 100

    def admit(self, req):
        self.active[req.rid] = req
        self.steps_done[req.rid] = 0
        self.used += self.bytes_needed(req)
        self.max_used = max(self.max_used, self.used)
        self.admit_order.append(req.rid)
        self.log.append(("admit", req.rid, self.clock()))
        return req.rid

    def step(self, n):
        for rid in self.active:
            self.steps_done[rid] += n
        self.clock.t += n * 1e-6 * sum(r.workload.nodes for r in self.active.values()) / 1000.0

    def retire(self, rid):
        req = self.active.pop(rid)
        self.log.append(("retire", rid, self.clock()))
        return [rid, self.clock() + 5e-4, req]

    def done(self, token):
        if self.clock() >= token[1]:
            if token[2] is not None:
                self.used -= self.bytes_needed(token[2])
                token[2] = None
            return True
        return False


def small_stream(n=60, rate=400.0, seed=3):
    reqs = I.request_stream(count=n, rate_per_s=rate, seed=seed, min_steps=50, max_steps=400)
    return reqs


def test_every_request_gets_its_steps_and_memory_stays_in_budget():
    clock = FakeClock()
    eng = FakeEngine(clock)
    reqs = small_stream()
    budget = 4 * max(eng.bytes_needed(r) for r in reqs)
    stats = serve(reqs, eng, budget, chunk=64, clock=clock, sleep=clock.sleep)
    assert len(stats.results) == len(reqs)
    for r in reqs:
        assert eng.steps_done[r.rid] == r.workload.steps
    assert eng.max_used <= budget
    assert eng.used == 0
    # first in, first out
    assert eng.admit_order == sorted(eng.admit_order, key=lambda rid: reqs[rid].arrival_s)
    for res in stats.results:
        assert res.finished_s >= res.admitted_s >= res.arrival_s
    assert stats.lups == sum(r.workload.nodes * r.workload.steps for r in reqs)


def test_requests_join_while_others_run():
    clock = FakeClock()
    eng = FakeEngine(clock)
    reqs = small_stream(n=30, rate=2000.0)
    stats = serve(reqs, eng, 1e18, chunk=32, clock=clock, sleep=clock.sleep)
    # some request was admitted while an earlier one was still running
    spans = {r.rid: (r.admitted_s, r.finished_s) for r in stats.results}
    overlap = any(spans[a][0] < spans[b][0] < spans[a][1] for a in spans for b in spans if a != b)
    assert overlap
    assert stats.percentile(99) >= stats.percentile(50) > 0


def test_budget_limits_concurrency():
    clock = FakeClock()
    eng = FakeEngine(clock)
    reqs = small_stream(n=20, rate=1e6)  # all arrive at once
    one = max(eng.bytes_needed(r) for r in reqs)
    stats = serve(reqs, eng, one, chunk=64, clock=clock, sleep=clock.sleep)
    # a request waits until the memory of earlier ones has come back; all complete
    assert eng.max_used <= one
    assert len(stats.results) == len(reqs) and eng.used == 0


def test_oversize_request_is_refused():
    clock = FakeClock()
    eng = FakeEngine(clock)
    reqs = small_stream(n=3)
    with pytest.raises(ValueError):
        serve(reqs, eng, 1.0, clock=clock, sleep=clock.sleep)


class QueueingFakeEngine(FakeEngine):
    """Steps are only enqueued; the device catches up when the host waits on a fence."""

    def __init__(self, clock):
        super().__init__(clock)
        self.enqueued = 0
        self.completed = 0
        self.max_in_flight = 0

    def step(self, n):
        for rid in self.active:
            self.steps_done[rid] += n
        self.enqueued += 1
        self.max_in_flight = max(self.max_in_flight, self.enqueued - self.completed)

    def fence(self):
        return self.enqueued

    def wait(self, fence):
        if fence > self.completed:
            self.clock.t += (fence - self.completed) * 1e-4
            self.completed = fence


@pytest.mark.parametrize("ahead", [1, 2, 4])
def test_host_runs_a_bounded_number_of_chunks_ahead(ahead):
    clock = FakeClock()
    eng = QueueingFakeEngine(clock)
    reqs = small_stream(n=40, rate=2000.0)
    stats = serve(reqs, eng, 1e18, chunk=16, clock=clock, sleep=clock.sleep, ahead=ahead)
    assert len(stats.results) == len(reqs)
    for r in reqs:
        assert eng.steps_done[r.rid] == r.workload.steps
    # after each chunk the host waits until at most `ahead` chunks are queued
    assert eng.max_in_flight == ahead + 1
    assert eng.enqueued - eng.completed <= ahead
