"""The bench's serving harness (open-loop Poisson load into msir_server) on
the CPU: a fake one-slot FIFO server and a fake clock that advances only
when the harness sleeps."""

import numpy as np
import pytest

import bench
from synth import poisson_arrivals, serving_pool


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeServer:
    """One request at a time, first come first served; a request of size n
    takes service * n seconds once it starts."""

    def __init__(self, clock, service=1e-4):
        self.clock, self.service = clock, service
        self.free_at = 0.0
        self.done_at, self.submitted_at = {}, {}
        self.next = 1

    def submit(self, A, b, spec):
        tk = self.next
        self.next += 1
        now = self.clock()
        start = max(now, self.free_at)
        self.free_at = start + self.service * A.shape[0]
        self.done_at[tk], self.submitted_at[tk] = self.free_at, now
        return tk

    def poll(self, tk, n):
        if self.clock() >= self.done_at[tk]:
            lat = (self.done_at[tk] - self.submitted_at[tk]) * 1e3
            return 2, np.zeros(n), {"cged": True, "call_status": 0}, lat
        return 1, None, None, None


def _systems(sizes):
    return [(np.zeros((n, n)), np.zeros(n), "fp16,fp32,fp64") for n in sizes]


def test_poisson_arrivals_rate_and_order():
    times, picks = poisson_arrivals(200.0, 50.0, 512, seed=0)
    assert all(0 < a < b < 50.0 for a, b in zip(times, times[1:]))
    assert abs(len(times) / 50.0 - 200.0) < 4 * np.sqrt(200.0 / 50.0) * 2  # within a few sigma
    assert min(picks) >= 0 and max(picks) < 512
    assert (times, picks) == poisson_arrivals(200.0, 50.0, 512, seed=0)


def test_serving_pool_ranges():
    pool = serving_pool(300, seed=0)
    ns = [p[0] for p in pool]
    ks = [p[1] for p in pool]
    assert 256 <= min(ns) and max(ns) <= 8192
    assert 1e2 <= min(ks) and max(ks) <= 1e10
    assert {p[2] for p in pool} == {"fp16,fp32,fp64", "bf16,fp32,fp64", "fp32,fp64,dd"}
    assert len({p[3] for p in pool}) == 300


def test_underloaded_server_finishes_everything_with_service_latency():
    clk = FakeClock()
    srv = FakeServer(clk, service=1e-4)
    systems = _systems([10, 20])
    times = [0.1 * (i + 1) for i in range(20)]       # one arrival every 0.1 s
    picks = [i % 2 for i in range(20)]
    recs = bench.run_serving(srv, systems, times, picks, duration_s=3.0, byte_cap=10 ** 12,
                             clock=clk, sleep=clk.sleep)
    assert len(recs) == 20 and all(r["status"] == "done" for r in recs)
    for r in recs:  # a request waits for nothing: latency = its own service time
        assert r["latency_ms"] == pytest.approx(1e-4 * r["n"] * 1e3, rel=1e-9)
    summ = bench.serving_summary(recs, warmup_s=1.0, duration_s=3.0)
    assert summ["arrivals"] == 11 and summ["unfinished"] == 0 and summ["rejected"] == 0
    assert summ["solves_per_s"] == pytest.approx(11 / 2.0)
    assert summ["all_converged"]


def test_overloaded_server_queues_and_the_byte_cap_rejects():
    clk = FakeClock()
    srv = FakeServer(clk, service=0.01)             # a size-100 request takes 1 s
    systems = _systems([100])
    times = [0.01 * (i + 1) for i in range(300)]    # 100 arrivals per second
    picks = [0] * 300
    cap = 5 * bench.request_bytes(100)              # at most 5 outstanding
    recs = bench.run_serving(srv, systems, times, picks, duration_s=3.0, byte_cap=cap,
                             clock=clk, sleep=clk.sleep)
    accepted = [r for r in recs if r["status"] != "rejected"]
    assert len(recs) == 300 - sum(t >= 3.0 for t in times)
    assert sum(r["status"] == "rejected" for r in recs) > 0
    # at no arrival were more than 5 requests outstanding
    events = sorted([(r["t"], 1) for r in accepted] + [(r["t_done"], -1) for r in accepted if r["t_done"]])
    level = 0
    for _, d in events:
        level += d
        assert level <= 5
    done = [r for r in recs if r["status"] == "done"]
    assert 1 <= len(done) <= 3  # one slot, 1 s each, 3 s of run
    summ = bench.serving_summary(recs, warmup_s=0.0, duration_s=3.0)
    assert summ["unfinished"] == len(accepted) - len(done)
    assert summ["latency_ms"]["samples"] == len(done)


def test_server_back_pressure_counts_as_rejected():
    """A submission the server refuses with MSIR_ERR_BUSY (its bound on held
    host copies or on queued work) or MSIR_ERR_NOMEM (no host memory for the
    copy) is a rejected arrival, not an error of the harness; any other error
    propagates."""
    import bench

    class Refusing:
        def __init__(self, codes):
            self.calls = 0
            self.codes = list(codes)

        def submit(self, A, b, spec):
            self.calls += 1
            err = RuntimeError("server_submit: refused")
            err.code = self.codes.pop(0)
            raise err

        def poll(self, t, n):
            raise AssertionError("nothing was queued")

    A = np.eye(4)
    srv = Refusing([-7, -2])
    clock = iter([0.0, 0.0, 0.5, 0.6, 1.5, 2.5, 3.0]).__next__
    recs = bench.run_serving(srv, [(A, np.ones(4), "fp16,fp32,fp64")], [0.1, 0.4], [0, 0], 1.0, None,
                             clock=clock, sleep=lambda s: None)
    assert srv.calls == 2 and [r["status"] for r in recs] == ["rejected", "rejected"]
    srv = Refusing([-1])
    clock = iter([0.0, 0.0, 0.5, 0.6, 1.5, 2.5, 3.0]).__next__
    with pytest.raises(RuntimeError):
        bench.run_serving(srv, [(A, np.ones(4), "fp16,fp32,fp64")], [0.1], [0], 1.0, None,
                          clock=clock, sleep=lambda s: None)
