"""Continuous-batching policy of the server, on the CPU with a simulated executor and clock."""
import numpy as np

from paper_2512_08887_gb300.serve import Request, Scheduler, poisson_requests, run_loop


class FakeClock:
    """Each reading advances simulated time by `dt` seconds."""

    def __init__(self, dt=2e-6):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class SimExecutor:
    """Batches finish `cost(batch)` simulated seconds after submission; checks the invariants."""

    def __init__(self, clock, slots, per_request_s, units):
        self.clock, self.free, self.per, self.units = clock, slots, per_request_s, units
        self.inflight, self.max_inflight = [], 0

    def can_submit(self):
        return self.free > 0

    def submit(self, batch, now):
        active = {r.array for _, b in self.inflight for r in b}
        assert not active & {r.array for r in batch}, "an array is in two in-flight batches"
        self.free -= 1
        self.inflight.append((self.clock.t + 1e-5 + self.per * len(batch), batch))
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def poll(self):
        done = [b for t, b in self.inflight if t <= self.clock.t]
        self.inflight = [(t, b) for t, b in self.inflight if t > self.clock.t]
        self.free += len(done)
        return done


def _setup(rate, count=400, arrays=6, budget=10**9, max_per_array=4, slots=3):
    reqs = poisson_requests(rate, count, [[None]] * arrays, seed=3)
    req_bytes = [1 << (20 + a) for a in range(arrays)]
    sched = Scheduler(req_bytes, budget, max_per_array)
    clock = FakeClock()
    ex = SimExecutor(clock, slots, 5e-5, [100 * (a + 1) for a in range(arrays)])
    return reqs, sched, ex, clock


def test_every_request_completes_and_latency_is_positive():
    reqs, sched, ex, clock = _setup(rate=2e4)
    stats = run_loop(reqs, sched, ex, clock=clock)
    assert stats["requests"] == len(reqs)
    assert all(r.t_done >= r.t_arrival for r in reqs)
    assert all(r.t_admit >= r.t_arrival for r in reqs)
    assert sched.mem_used == 0 and not sched.busy and not sched.pending


def test_bursts_are_batched_and_overlap_on_streams():
    reqs, sched, ex, clock = _setup(rate=1e6)       # everything arrives almost at once
    stats = run_loop(reqs, sched, ex, clock=clock)
    assert stats["mean_batch"] > 3
    assert ex.max_inflight > 1


def test_memory_budget_is_never_exceeded():
    budget = 40 << 20
    reqs, sched, ex, clock = _setup(rate=1e6, budget=budget)
    run_loop(reqs, sched, ex, clock=clock)
    assert 0 < sched.peak_mem <= budget


def test_per_array_order_is_arrival_order_and_capacity_is_respected():
    reqs, sched, ex, clock = _setup(rate=5e5, max_per_array=2)
    run_loop(reqs, sched, ex, clock=clock)
    for a in range(6):
        mine = [r for r in reqs if r.array == a]
        assert [r.batch_id for r in mine] == sorted(r.batch_id for r in mine)
    counts = {}
    for r in reqs:
        counts[(r.batch_id, r.array)] = counts.get((r.batch_id, r.array), 0) + 1
    assert max(counts.values()) <= 2


def test_large_request_is_not_starved_by_small_ones():
    # Array 1 needs 3/4 of the budget: it must get in before later small requests pile up.
    sched = Scheduler([1, 75], 100, max_per_array=64)
    big = Request(0, 1, None, 0.0)
    sched.arrive(Request(9, 0, None, 0.0))
    sched.busy.add(0)                                   # array 0 in flight
    sched.mem_used = 30
    sched.arrive(big)
    for k in range(10):
        sched.arrive(Request(10 + k, 0, None, 0.0))
    assert sched.form_batch(0.0) == []                  # big does not fit yet; nothing jumps it
    sched.busy.clear()
    sched.mem_used = 0
    b = sched.form_batch(0.0)
    assert big in b


def test_poisson_arrivals_have_the_requested_rate():
    reqs = poisson_requests(1e3, 5000, [[None]] * 4, seed=1)
    t = np.array([r.t_arrival for r in reqs])
    assert abs(len(t) / t[-1] / 1e3 - 1) < 0.05


class FailingExecutor(SimExecutor):
    """A SimExecutor whose k-th submission raises (a host-side injected failure: the library or a
    malformed request refusing the batch) before anything runs."""

    def __init__(self, *a, fail_on=(3,), **kw):
        super().__init__(*a, **kw)
        self.calls, self.fail_on = 0, set(fail_on)

    def submit(self, batch, now):
        self.calls += 1
        if self.calls in self.fail_on:
            raise RuntimeError("injected: fbst_batch_enqueue failed")
        super().submit(batch, now)


def test_failed_batches_are_reported_and_the_rest_is_served():
    reqs = poisson_requests(5e4, 300, [[None]] * 5, seed=8)
    sched = Scheduler([1 << 20] * 5, 1 << 30, max_per_array=4)
    clock = FakeClock()
    ex = FailingExecutor(clock, 3, 5e-5, [100] * 5, fail_on=(2, 5, 9))
    stats = run_loop(reqs, sched, ex, clock=clock)
    failed = [r for r in reqs if r.error is not None]
    assert failed and all("injected" in r.error for r in failed)
    assert stats["failed"] == len(failed) and stats["requests"] == len(reqs)
    # Every other request was served after the failures, and the bookkeeping is clean.
    assert all(r.t_done is not None and r.t_done >= r.t_admit for r in reqs if r.error is None)
    assert max(r.batch_id for r in failed) < max(r.batch_id for r in reqs if r.error is None)
    assert sched.mem_used == 0 and not sched.busy and not sched.pending
    assert stats["beam_samples_per_s"] > 0


def test_batch_bytes_stay_within_one_stream_arena():
    reqs = poisson_requests(1e6, 200, [[None]] * 6, seed=4)
    req_bytes = [1 << (20 + a % 3) for a in range(6)]
    cap = 5 << 20
    sched = Scheduler(req_bytes, 1 << 30, max_per_array=8, max_batch_bytes=cap)
    clock = FakeClock()
    run_loop(reqs, sched, SimExecutor(clock, 3, 5e-5, [100] * 6), clock=clock)
    per_batch = {}
    for r in reqs:
        per_batch[r.batch_id] = per_batch.get(r.batch_id, 0) + req_bytes[r.array]
    assert max(per_batch.values()) <= cap and len(per_batch) > 1
