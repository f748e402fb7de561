"""Host logic of the continuous-batching server, with a CPU stand-in engine:
admission by memory and resident limits, FIFO order, per-request step
counts, cohort halving, error propagation, time limits and the report."""
import threading
import time

import numpy as np
import pytest

from paper_2504_12908_b300.serving import Cohort, Engine, Request, Server, poisson_arrivals


class FakeCohort(Cohort):
    def __init__(self, eng, reqs):
        self.eng, self.reqs = eng, reqs
        self.steps = np.zeros(len(reqs), int)
        with eng.lock:
            eng.used += eng.cohort_bytes([r.scene for r in reqs])
            eng.resident += len(reqs)
            eng.peak_used = max(eng.peak_used, eng.used)
            eng.peak_resident = max(eng.peak_resident, eng.resident)
            eng.opened.append([r.rid for r in reqs])
        if eng.fail_rid is not None and any(r.rid == eng.fail_rid for r in reqs):
            raise RuntimeError("cohort failed to open")

    def step(self, env_ids, k):
        time.sleep(self.eng.step_s)
        for i in env_ids:
            assert self.steps[i] == k          # every env steps 0, 1, 2, ... in order
            self.steps[i] += 1
        return np.zeros(len(env_ids), np.int32)

    def final_state(self, i):
        r = self.reqs[i]
        return np.full((2, 3), float(r.rid)), np.full((1, 12), float(self.steps[i]))

    def close(self):
        with self.eng.lock:
            self.eng.used -= self.eng.cohort_bytes([r.scene for r in self.reqs])
            self.eng.resident -= len(self.reqs)


class FakeEngine(Engine):
    """scene = its workspace bytes (an int); free memory = capacity - used."""

    def __init__(self, capacity, step_s=0.001, fail_rid=None):
        self.capacity, self.step_s, self.fail_rid = capacity, step_s, fail_rid
        self.used = 0
        self.resident = 0
        self.peak_used = 0
        self.peak_resident = 0
        self.opened = []
        self.lock = threading.Lock()

    def cohort_bytes(self, scenes):
        return int(sum(scenes)) + 1000          # a fixed per-context overhead

    def free_bytes(self):
        with self.lock:
            return self.capacity - self.used

    def open(self, requests):
        return FakeCohort(self, requests)


def _reqs(n, size=10_000, steps=5, rate=None, seed=0):
    arr = poisson_arrivals(n, rate, seed) if rate else np.zeros(n)
    return [Request(rid=i, scene=size, delta=lambda k: np.zeros((1, 3)), n_steps=steps, arrival=float(arr[i]))
            for i in range(n)]


def test_every_request_completes_with_its_own_step_count():
    reqs = _reqs(30)
    for i, r in enumerate(reqs):
        r.n_steps = 1 + i % 7
    eng = FakeEngine(capacity=10**9)
    rep = Server(eng, max_cohort=8, max_cohorts=3, mem_reserve=0).run(reqs, realtime=False)
    assert rep.completed == rep.admitted == 30 and rep.backlog == 0
    assert rep.env_steps == sum(r.n_steps for r in reqs)
    for r in reqs:
        res = rep.results[r.rid]
        assert res.status == 0 and res.steps == r.n_steps
        assert res.final_y[0, 0] == r.n_steps             # stepped exactly n_steps times
        assert np.all(res.final_x == r.rid)
    assert eng.used == 0 and eng.resident == 0            # every cohort closed


def test_resident_and_cohort_limits_hold():
    eng = FakeEngine(capacity=10**9, step_s=0.002)
    rep = Server(eng, max_resident=10, max_cohort=4, max_cohorts=8, mem_reserve=0).run(_reqs(40), realtime=False)
    assert rep.completed == 40
    assert eng.peak_resident <= 10 and rep.max_resident <= 10
    assert max(len(c) for c in eng.opened) <= 4


def test_memory_limit_holds_and_oversized_cohorts_are_halved():
    # room for 3 requests (3 x 10 000 + 1000) beside a 20 000-byte reserve
    eng = FakeEngine(capacity=51_000 + 20_000)
    rep = Server(eng, max_cohort=16, max_cohorts=4, mem_reserve=20_000).run(_reqs(12), realtime=False)
    assert rep.completed == 12
    assert eng.peak_used <= 51_000
    assert max(len(c) for c in eng.opened) <= 4                # 16 -> 8 -> 4 -> 2 ... halving


def test_admission_is_fifo_in_arrival_order():
    reqs = _reqs(25, rate=2000.0, seed=3)
    eng = FakeEngine(capacity=10**9)
    Server(eng, max_cohort=5, max_cohorts=2, mem_reserve=0).run(reqs)
    order = [rid for c in eng.opened for rid in c]
    arrival = {r.rid: r.arrival for r in reqs}
    assert order == sorted(order, key=lambda rid: (arrival[rid], rid))
    assert sorted(order) == list(range(25))


def test_a_request_that_never_fits_stays_in_the_backlog_until_the_time_limit():
    eng = FakeEngine(capacity=5_000)                          # one request needs 11 000
    rep = Server(eng, max_cohort=4, mem_reserve=0).run(_reqs(3), time_limit=0.05, realtime=False)
    assert rep.admitted == 0 and rep.backlog == 3 and rep.env_steps == 0


def test_errors_in_a_cohort_surface_from_run():
    eng = FakeEngine(capacity=10**9, fail_rid=7)
    with pytest.raises(RuntimeError, match="cohort failed"):
        Server(eng, max_cohort=4, max_cohorts=2, mem_reserve=0).run(_reqs(12), realtime=False)


def test_report_latency_percentiles_are_env_weighted():
    srv = Server(FakeEngine(capacity=10**9))
    srv._step_samples = [(1.0, 1), (10.0, 99)]               # 99 of 100 env-steps took 10 ms
    rep = srv._report(1.0, 0, 0, 0, 0)
    assert rep.step_ms_p50 == 10.0 and rep.step_ms_p99 == 10.0
    assert rep.env_steps == 100 and rep.env_steps_per_s == 100.0


def test_poisson_arrivals_have_the_requested_rate():
    a = poisson_arrivals(20000, 2000.0, 4000)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 20000 - 1 / 2000.0) < 0.02 / 2000.0 * 5
