"""Host logic of the continuous-batching server, with a CPU stand-in engine:
per-slot admission (a finished request's slot takes the next waiting
request of its size class at once), one pool per size class, resident and
memory limits, FIFO order within a class, per-request step counts, error
propagation, time limits and the report."""
import threading
import time

import numpy as np
import pytest

from paper_2504_12908_b300.serving import Engine, Pool, Request, Server, poisson_arrivals


class FakePool(Pool):
    def __init__(self, eng, scene, n_slots, max_steps):
        self.eng, self.n_slots = eng, n_slots
        self.key = eng.class_key(scene)
        self.bytes = eng.pool_bytes(scene, n_slots)
        self.req = [None] * n_slots
        self.k = np.zeros(n_slots, int)
        self.loads = []                                  # (slot, rid) in load order
        with eng.lock:
            eng.used += self.bytes
            eng.peak_used = max(eng.peak_used, eng.used)
            eng.pools.append(self)
        if eng.fail_key is not None and self.key == eng.fail_key:
            raise RuntimeError("pool failed to open")

    def load(self, slot, req):
        assert self.eng.class_key(req.scene) == self.key   # only its own size class
        self.req[slot] = req
        self.k[slot] = 0
        self.loads.append((slot, req.rid))
        with self.eng.lock:
            self.eng.order.append(req.rid)

    def step(self, slots, ks):
        time.sleep(self.eng.step_s)
        with self.eng.lock:
            self.eng.resident_now = sum(r is not None for p in self.eng.pools for r in p.req)
            self.eng.peak_resident = max(self.eng.peak_resident, self.eng.resident_now)
        for s, k in zip(slots, ks):
            assert self.req[s] is not None and self.k[s] == k   # each slot steps its script in order
            self.k[s] += 1
        return np.zeros(len(slots), np.int32)

    def final_state(self, slot):
        r = self.req[slot]
        x, y = np.full((2, 3), float(r.rid)), np.full((1, 12), float(self.k[slot]))
        self.req[slot] = None
        return x, y

    def close(self):
        with self.eng.lock:
            self.eng.used -= self.bytes


class FakeEngine(Engine):
    """scene = (size class, bytes per env); free memory = capacity - used."""

    def __init__(self, capacity, step_s=0.001, fail_key=None):
        self.capacity, self.step_s, self.fail_key = capacity, step_s, fail_key
        self.used = 0
        self.peak_used = 0
        self.peak_resident = 0
        self.resident_now = 0
        self.pools = []
        self.order = []
        self.lock = threading.Lock()

    def class_key(self, scene):
        return scene[0]

    def pool_bytes(self, scene, n_slots):
        return scene[1] * n_slots + 1000          # a fixed per-context overhead

    def free_bytes(self):
        with self.lock:
            return self.capacity - self.used

    def open_pool(self, scene, n_slots, max_steps):
        return FakePool(self, scene, n_slots, max_steps)


def _reqs(n, classes=1, size=10_000, steps=5, rate=None, seed=0):
    arr = poisson_arrivals(n, rate, seed) if rate else np.zeros(n)
    return [Request(rid=i, scene=(i % classes, size), delta=lambda k: np.zeros((1, 3)), n_steps=steps,
                    arrival=float(arr[i])) for i in range(n)]


def test_every_request_completes_with_its_own_step_count():
    reqs = _reqs(30, classes=3)
    for i, r in enumerate(reqs):
        r.n_steps = 1 + i % 7
    eng = FakeEngine(capacity=10**9)
    rep = Server(eng, slots_per_pool=4, mem_reserve=0).run(reqs, realtime=False)
    assert rep.completed == rep.admitted == 30 and rep.backlog == 0
    assert rep.env_steps == sum(r.n_steps for r in reqs)
    assert rep.pools == 3 and rep.slots == 12               # one pool per size class
    for r in reqs:
        res = rep.results[r.rid]
        assert res.status == 0 and res.steps == r.n_steps
        assert res.final_y[0, 0] == r.n_steps               # stepped exactly n_steps times
        assert np.all(res.final_x == r.rid)
    assert eng.used == 0                                    # every pool closed


def test_a_finished_slot_takes_the_next_request_of_its_class():
    # 2 slots, 6 requests of one class with different lengths: a short
    # request's slot is reused while the long one is still running
    reqs = _reqs(6, steps=3)
    reqs[0].n_steps = 20
    eng = FakeEngine(capacity=10**9, step_s=0.002)
    rep = Server(eng, slots_per_pool=2, mem_reserve=0).run(reqs, realtime=False)
    assert rep.completed == 6 and rep.pools == 1 and rep.slots == 2
    assert rep.slot_reuses == 4
    loads = eng.pools[0].loads
    assert [rid for _, rid in loads] == [0, 1, 2, 3, 4, 5]
    # every later request went into slot 1 (slot 0 held the long request)
    assert all(s == 1 for s, rid in loads if rid >= 2)
    # request 0 was still running when the others finished
    assert rep.results[0].finished >= max(rep.results[i].finished for i in range(1, 6))


def test_resident_limit_holds():
    eng = FakeEngine(capacity=10**9, step_s=0.002)
    rep = Server(eng, max_resident=5, slots_per_pool=4, mem_reserve=0).run(_reqs(40, classes=3), realtime=False)
    assert rep.completed == 40
    assert rep.max_resident <= 5 and eng.peak_resident <= 5


def test_memory_limit_sizes_the_pools():
    # room for 4 slots (4 x 10 000 + 1000) beside a 20 000-byte reserve
    eng = FakeEngine(capacity=51_000 + 20_000)
    rep = Server(eng, slots_per_pool=16, mem_reserve=20_000).run(_reqs(12), realtime=False)
    assert rep.completed == 12
    assert eng.peak_used <= 51_000
    assert [p.n_slots for p in eng.pools] == [4]            # 16 -> 8 -> 4 halving


def test_admission_is_fifo_within_a_class():
    reqs = _reqs(25, classes=2, rate=2000.0, seed=3)
    eng = FakeEngine(capacity=10**9)
    Server(eng, slots_per_pool=3, mem_reserve=0).run(reqs)
    arrival = {r.rid: r.arrival for r in reqs}
    for c in (0, 1):
        order = [rid for rid in eng.order if rid % 2 == c]
        assert order == sorted(order, key=lambda rid: (arrival[rid], rid))
    assert sorted(eng.order) == list(range(25))


def test_a_request_that_never_fits_stays_in_the_backlog_until_the_time_limit():
    eng = FakeEngine(capacity=5_000)                          # one slot needs 11 000
    rep = Server(eng, slots_per_pool=4, mem_reserve=0).run(_reqs(3), time_limit=0.05, realtime=False)
    assert rep.admitted == 0 and rep.backlog == 3 and rep.env_steps == 0


def test_errors_in_a_pool_surface_from_run():
    eng = FakeEngine(capacity=10**9, fail_key=1)
    with pytest.raises(RuntimeError, match="pool failed"):
        Server(eng, slots_per_pool=4, mem_reserve=0).run(_reqs(12, classes=2), realtime=False)


def test_report_latency_percentiles_are_env_weighted():
    srv = Server(FakeEngine(capacity=10**9))
    srv._step_samples = [(1.0, 1), (10.0, 99)]               # 99 of 100 env-steps took 10 ms
    rep = srv._report(1.0, 0, 0, [])
    assert rep.step_ms_p50 == 10.0 and rep.step_ms_p99 == 10.0
    assert rep.env_steps == 100 and rep.env_steps_per_s == 100.0


def test_poisson_arrivals_have_the_requested_rate():
    a = poisson_arrivals(20000, 2000.0, 4000)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 20000 - 1 / 2000.0) < 0.02 / 2000.0 * 5


class ChunkPool(FakePool):
    """Advances up to `chunk` steps per call (slot i at most remaining[i]),
    as the GPU pools' rollouts do."""

    def advance(self, slots, ks, remaining, chunk):
        taken = np.zeros(len(slots), np.int64)
        for j, (s, k, rem) in enumerate(zip(slots, ks, remaining)):
            assert self.req[s] is not None and self.k[s] == k and rem == self.req[s].n_steps - k
            n = min(chunk, rem)
            self.k[s] += n
            taken[j] = n
        time.sleep(self.eng.step_s)
        return np.zeros(len(slots), np.int32), taken


class ChunkEngine(FakeEngine):
    def open_pool(self, scene, n_slots, max_steps):
        return ChunkPool(self, scene, n_slots, max_steps)


def test_chunked_calls_advance_each_slot_to_its_own_last_step():
    reqs = [Request(rid=i, scene=("a", 10), n_steps=n, arrival=0.0) for i, n in enumerate([1, 5, 7, 3, 8, 2])]
    eng = ChunkEngine(capacity=10_000)
    rep = Server(eng, slots_per_pool=3, mem_reserve=0, chunk=4).run(reqs, realtime=False)
    assert rep.completed == len(reqs) and rep.backlog == 0
    assert rep.env_steps == sum(r.n_steps for r in reqs)
    for r in reqs:
        res = rep.results[r.rid]
        assert res.steps == r.n_steps and res.status == 0
        assert float(res.final_y[0, 0]) == r.n_steps        # the pool's own step count
