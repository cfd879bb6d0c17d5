"""Scheduling logic of the continuous-batching server, on the CPU.

A fake backend stands in for the GPU: a batch of requests takes a fixed
time per request after launch on a simulated clock, and its exact memory is
a given number of bytes per request.  The tests check that every request
completes once, that the memory admitted never exceeds the cap, that the
batch-size and in-flight limits hold, and that requests arriving while
batches run join later batches.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1804_01698_gb300.serve import Request, Server, Stats, Completion, serve_one_by_one, upper_bound_bytes


class SimClock:
    """Simulated time: every read advances it by `tick` seconds."""

    def __init__(self, tick=1e-4):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t


class FakeOperand:
    def __init__(self, nrows, nnz):
        self.nrows, self.nnz = nrows, nnz


class FakeBackend:
    vsize = 8

    def __init__(self, clock, per_request_s=2e-3, bytes_per_request=1000):
        self.clock = clock
        self.per_request_s = per_request_s
        self.bytes_per_request = bytes_per_request
        self.live = 0          # bytes of launched, unreleased batches
        self.max_live = 0
        self.max_running = 0
        self.running = set()
        self.batch_sizes = []
        self.next_id = 0

    def prepare(self, reqs):
        h = {"id": self.next_id, "reqs": list(reqs), "end": None}
        self.next_id += 1
        self.batch_sizes.append(len(reqs))
        return h

    def bytes(self, h):
        return self.bytes_per_request * len(h["reqs"])

    def launch(self, h):
        h["end"] = self.clock.t + self.per_request_s * len(h["reqs"])
        self.live += self.bytes(h)
        self.max_live = max(self.max_live, self.live)
        self.running.add(h["id"])
        self.max_running = max(self.max_running, len(self.running))

    def done(self, h):
        return self.clock.t >= h["end"]

    def wait(self, h):
        self.clock.t = max(self.clock.t, h["end"])

    def results(self, h):
        return [("C", r.rid) for r in h["reqs"]]

    def release(self, h):
        if h["end"] is not None:             # launched
            self.live -= self.bytes(h)
        self.running.discard(h["id"])


def make_requests(n, rate, seed=0, flop=10):
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n)) if rate else np.zeros(n)
    return [Request(i, FakeOperand(4, 4), FakeOperand(4, 4), float(arrivals[i]), flop) for i in range(n)]


def test_every_request_completes_once_with_its_result():
    clock = SimClock()
    be = FakeBackend(clock)
    reqs = make_requests(200, rate=2000.0, seed=1)
    st = Server(be, mem_cap=1 << 30, max_batch=16).run(reqs, keep_results=True, clock=clock)
    assert sorted(c.rid for c in st.completions) == list(range(200))
    for c in st.completions:
        assert c.result == ("C", c.rid)
        assert c.done >= c.start >= c.arrival - 1e-12
    assert be.live == 0


def test_arrivals_during_running_batches_join_later_batches():
    clock = SimClock()
    be = FakeBackend(clock, per_request_s=1e-3)
    reqs = make_requests(300, rate=5000.0, seed=2)
    st = Server(be, mem_cap=1 << 30, max_batch=64).run(reqs, clock=clock)
    assert st.batches == len(be.batch_sizes)
    assert 1 < st.batches < 300, "requests were neither batched nor spread over several batches"
    assert max(be.batch_sizes) > 1
    assert sum(be.batch_sizes) == 300


def test_batch_size_and_inflight_limits_hold():
    clock = SimClock()
    be = FakeBackend(clock)
    reqs = make_requests(500, rate=0, seed=3)     # all arrive at once
    st = Server(be, mem_cap=1 << 40, max_batch=7, max_inflight=2).run(reqs, clock=clock)
    assert max(be.batch_sizes) <= 7
    assert be.max_running <= 2
    assert len(st.completions) == 500


def test_admitted_memory_never_exceeds_the_cap():
    clock = SimClock()
    be = FakeBackend(clock, bytes_per_request=1000)
    reqs = make_requests(400, rate=0, seed=4, flop=1)
    cap = 5500           # at most five requests' exact memory at once
    st = Server(be, mem_cap=cap, max_batch=64, max_inflight=8).run(reqs, clock=clock)
    assert be.max_live <= cap
    assert be.live == 0
    assert len(st.completions) == 400
    assert max(be.batch_sizes) > 5          # the first batch was too large and given back


def test_upper_bound_splits_batches_before_the_symbolic_pass():
    clock = SimClock()
    be = FakeBackend(clock, bytes_per_request=1)
    reqs = make_requests(40, rate=0, seed=5, flop=1000)
    ub = upper_bound_bytes(reqs[0], be.vsize)
    cap = 4 * ub
    Server(be, mem_cap=cap, max_batch=64).run(reqs, clock=clock)
    assert max(be.batch_sizes) == 4


def test_a_request_larger_than_the_cap_still_runs_alone():
    clock = SimClock()
    be = FakeBackend(clock, bytes_per_request=10_000)
    reqs = make_requests(3, rate=0, seed=6)
    st = Server(be, mem_cap=100, max_batch=64).run(reqs, clock=clock)
    assert be.batch_sizes == [1, 1, 1]
    assert be.max_running == 1
    assert len(st.completions) == 3


def test_one_by_one_baseline_runs_each_request_alone():
    clock = SimClock()
    be = FakeBackend(clock)
    reqs = make_requests(50, rate=1000.0, seed=7)
    st = serve_one_by_one(be, reqs, keep_results=True, clock=clock)
    assert be.batch_sizes == [1] * 50
    assert [c.rid for c in st.completions] == list(range(50))
    assert st.batches == 50


def test_batching_beats_one_by_one_under_load_on_a_fixed_cost_backend():
    """With a per-launch cost, a saturated server that batches finishes
    sooner than one launch per request."""

    class LaunchCost(FakeBackend):
        def launch(self, h):
            super().launch(h)
            h["end"] += 5e-3

    reqs = make_requests(100, rate=0, seed=8)
    c1 = SimClock()
    batched = Server(LaunchCost(c1), mem_cap=1 << 30, max_batch=32).run(reqs, clock=c1)
    c2 = SimClock()
    alone = serve_one_by_one(LaunchCost(c2), reqs, clock=c2)
    assert batched.wall < alone.wall
    assert batched.percentile(99) < alone.percentile(99)


@pytest.mark.parametrize("n", [1, 2, 10, 101])
def test_percentiles_are_nearest_rank_of_the_latencies(n):
    rng = np.random.default_rng(n)
    lat = rng.exponential(1.0, size=n)
    st = Stats(completions=[Completion(i, 0.0, 0.0, float(lat[i]), 0) for i in range(n)], wall=1.0)
    s = np.sort(lat)
    for q in (0, 50, 99, 100):
        assert st.percentile(q) == s[int(round(q / 100 * (n - 1)))]
    assert st.summary()["requests"] == n
    assert Stats().percentile(50) != Stats().percentile(50)    # NaN when empty
