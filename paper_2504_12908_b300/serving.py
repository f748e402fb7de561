"""Continuous-batching request loop around the batched IPC step.

A request is one environment (a scene of gel + affine bodies, a kinematic
script and a number of steps) that arrives at some time.  The server keeps
resident *pools*: one library context per size class (the topology of a
request: mesh sizes, connectivity, body vertex counts) with a fixed number
of env slots.  Admission is per slot:

* arrived requests wait in a FIFO queue of their size class;
* a pool is opened for a class when requests of that class wait and device
  memory (``ipc_workspace_bytes`` of the pool against the free memory minus
  a reserve) and the pool limit allow; its slot count is the largest that
  fits, up to ``slots_per_pool``;
* the moment a slot's request has run its last step, the next waiting
  request of that class is loaded into the slot (``ipc_reset_env``: the new
  scene's material, rest geometry and bodies replace the old ones in place,
  state back to rest) and steps from the next batched step on;
* every pool is stepped by its own host thread on its own CUDA stream (the
  C-ABI calls release the GIL), so pools of different classes overlap on
  the device; each call advances the pool's occupied slots, every slot at
  its own script step: one batched step, or with ``chunk`` > 1 up to
  ``chunk`` steps as one rollout (``ipc_rollout``: every slot on its own step
  schedule inside one graph, a slot stops at its request's last step), so a
  slot whose step converges fast does not wait for the slowest slot of the
  pool at every step.  A freed slot is refilled between calls.

The engine behind the loop is pluggable (``Engine``): ``GpuEngine`` drives
the library; the tests drive the scheduling logic with a CPU stand-in.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque
from typing import Callable, Deque, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    """One environment to simulate.

    delta(k) -> (n_bodies, 3): translation of each driven body's rest
    placement at step k (the scripted targets; bodies keep A = I).
    Instead of scene and delta a request may carry build() -> (scene, delta),
    called when the request first arrives."""
    rid: int
    scene: object = None
    delta: Optional[Callable[[int], np.ndarray]] = None
    n_steps: int = 1
    arrival: float = 0.0          # seconds after the start of the run
    build: Optional[Callable[[], tuple]] = None
    state: Optional[tuple] = None  # (x, v, y, ydot) to start from; None = the scene's rest state

    def materialize(self) -> "Request":
        if self.scene is None and self.build is not None:
            self.scene, self.delta = self.build()
            self.build = None
        return self


@dataclasses.dataclass
class RequestResult:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int                    # steps taken (n_steps unless the run was cut)
    status: int                   # first non-OK per-env status, else 0
    slot: tuple = ()              # (pool index, slot index) it ran in
    final_x: Optional[np.ndarray] = None   # gel vertex positions after the last step
    final_y: Optional[np.ndarray] = None   # body DoFs after the last step


@dataclasses.dataclass
class ServeReport:
    wall_s: float
    env_steps: int
    env_steps_per_s: float
    step_ms_p50: float            # latency of the batched step calls, weighted by envs
    step_ms_p99: float
    completion_s_p50: Optional[float]
    completion_s_p99: Optional[float]
    queue_s_p50: Optional[float]
    queue_s_p99: Optional[float]
    queue_s_max: Optional[float]
    admitted: int
    completed: int                # ran all their steps with status OK
    arrived: int
    backlog: int                  # arrived, not admitted at the end
    pools: int                    # resident contexts opened (one per size class)
    slots: int                    # env slots over all pools
    slot_reuses: int              # requests loaded into a slot a previous request used
    max_resident: int             # most requests in slots at once
    max_active_pools: int         # pools stepping at the same time (overlap)
    results: Dict[int, RequestResult]

    def summary(self) -> dict:
        d = dataclasses.asdict(self)
        d.pop("results")
        return d


class Pool:
    """Engine-side handle of one resident context with env slots."""

    n_slots: int = 0

    def load(self, slot: int, req: Request) -> None:
        raise NotImplementedError

    def step(self, slots: Sequence[int], ks: Sequence[int]) -> np.ndarray:   # per-slot status
        raise NotImplementedError

    def advance(self, slots: Sequence[int], ks: Sequence[int], remaining: Sequence[int], chunk: int):
        """Up to `chunk` steps of each listed slot (slot i at most
        remaining[i]); returns (per-slot status, per-slot steps taken).
        Default: one batched step."""
        st = np.asarray(self.step(slots, ks))
        return st, np.ones(len(slots), dtype=np.int64)

    def final_state(self, slot: int):
        raise NotImplementedError

    def close(self) -> None:
        raise NotImplementedError


class Engine:
    def class_key(self, scene) -> object:
        raise NotImplementedError

    def pool_bytes(self, scene, n_slots: int) -> int:
        raise NotImplementedError

    def free_bytes(self) -> int:
        raise NotImplementedError

    def open_pool(self, scene, n_slots: int, max_steps: int) -> Pool:
        raise NotImplementedError


def topology_key(scene) -> tuple:
    """Size class of a scene: what ipc_reset_env requires to be equal."""
    tets = np.ascontiguousarray(scene.gel_tets)
    bodies = tuple((b.rest_x.shape[0], b.tris.shape[0], bool(b.driven), hash(np.ascontiguousarray(b.tris).tobytes()))
                   for b in scene.bodies)
    return (scene.gel_x.shape[0], hash(tets.tobytes()), hash(np.asarray(scene.pinned).tobytes()),
            hash(np.asarray(scene.attach).tobytes()), hash(np.asarray(scene.gel_obj).tobytes()),
            None if scene.self_contact is None else tuple(bool(v) for v in scene.self_contact), bodies)


class GpuEngine(Engine):
    """The library on one GPU: one context and one CUDA stream per pool,
    whole steps as CUDA graphs."""

    def __init__(self, params, device: str = "cuda:0", graphs: bool = True):
        import torch

        from . import ipc
        self._torch, self._ipc = torch, ipc
        self.params = params
        self.device = torch.device(device)
        self.graphs = graphs

    def class_key(self, scene):
        return topology_key(scene)

    def pool_bytes(self, scene, n_slots):
        return self._ipc.workspace_bytes([scene] * n_slots, self.params)

    def free_bytes(self) -> int:
        torch = self._torch
        free, _ = torch.cuda.mem_get_info(self.device)
        # memory held by torch's caching allocator but unused is free to us
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return int(free + cached)

    def open_pool(self, scene, n_slots, max_steps):
        return _GpuPool(self, scene, n_slots, max_steps)


class _GpuPool(Pool):
    def __init__(self, eng: GpuEngine, scene, n_slots: int, max_steps: int):
        torch, ipc = eng._torch, eng._ipc
        self.torch, self.ipc = torch, ipc
        self.n_slots = n_slots
        self.stream = torch.cuda.Stream(eng.device)
        self.envs = ipc.Envs([scene] * n_slots, eng.params, device=str(eng.device), stream=self.stream)
        self.graphs = eng.graphs
        if eng.graphs:
            self.envs.set_graph_mode(2)
        mb = max(self.envs.max_bodies, 1)
        # every slot's script, resident on the device: [slot][step][body][12]
        with torch.cuda.stream(self.stream):
            self.dev_tg = torch.zeros((n_slots, max_steps, mb, 12), dtype=torch.float64, device=eng.device)
        self.max_steps = max_steps

    def load(self, slot, req):
        torch = self.torch
        self.envs.reset_env(slot, req.scene)
        if req.state is not None:
            st = self.envs.set_state(slot, *req.state)
            if st != self.ipc.IPC_OK:
                raise self.ipc.IpcError(st, f"request {req.rid}: initial state rejected")
        rest = self.envs.rest_y(slot)
        nb = rest.shape[0]
        tg = np.zeros((self.max_steps,) + tuple(self.dev_tg.shape[2:]))
        for k in range(min(req.n_steps, self.max_steps)):
            t = rest.copy()
            t[:, :3] += np.asarray(req.delta(k), dtype=np.float64).reshape(-1, 3)[:nb]
            tg[k, :nb] = t
        with torch.cuda.stream(self.stream):
            self.dev_tg[slot].copy_(torch.as_tensor(tg), non_blocking=False)

    def _targets(self, slots, ks, n):
        """[n][n_slots][bodies][12]: step ks[i] + j of listed slot i's script
        (clamped to the script's end); other slots get step 0."""
        torch = self.torch
        dev = self.dev_tg.device
        with torch.cuda.stream(self.stream):
            k_all = torch.zeros(self.n_slots, dtype=torch.long, device=dev)
            k_all[torch.as_tensor(list(slots), device=dev)] = torch.as_tensor(list(ks), dtype=torch.long, device=dev)
            kk = (k_all[None, :] + torch.arange(n, device=dev)[:, None]).clamp_(max=self.max_steps - 1)
            return self.dev_tg[torch.arange(self.n_slots, device=dev)[None, :], kk].contiguous()

    def step(self, slots, ks):
        self.envs.set_targets_all_device(self._targets(slots, ks, 1)[0])
        status, _ = self.envs.step(list(slots))
        return status

    def advance(self, slots, ks, remaining, chunk):
        """Up to `chunk` steps per slot as one rollout (every slot on its own
        step schedule inside one graph) when graphs are on; else one step."""
        n = int(min(chunk, max(remaining)))
        if not self.graphs or n <= 1:
            return super().advance(slots, ks, remaining, chunk)
        tab = self._targets(slots, ks, n)
        status, taken, _ = self.envs.rollout(n, tab, env_ids=list(slots), steps_per_env=list(remaining))
        return status, taken

    def final_state(self, slot):
        x, _, y, _ = self.envs.get_state(slot)
        return x, y

    def close(self):
        self.envs.close()
        self.dev_tg = None


class _PoolState:
    def __init__(self, index, key, pool, n_slots):
        self.index, self.key, self.pool = index, key, pool
        self.req: List[Optional[Request]] = [None] * n_slots
        self.k = np.zeros(n_slots, int)
        self.status = np.zeros(n_slots, np.int32)
        self.admitted = np.zeros(n_slots)
        self.used = np.zeros(n_slots, bool)
        self.closed = False


class Server:
    """Per-slot admission and stepping loop (see the module docstring)."""

    def __init__(self, engine: Engine, max_resident: int = 4096, slots_per_pool: int = 256,
                 max_pools: int = 32, mem_reserve: int = 2 << 30, keep_state: bool = True,
                 poll_s: float = 0.002, chunk: int = 1):
        self.engine = engine
        self.chunk = max(1, int(chunk))       # steps per pool call (a rollout when > 1)
        self.max_resident = max_resident
        self.slots_per_pool = slots_per_pool
        self.max_pools = max_pools
        self.mem_reserve = mem_reserve
        self.keep_state = keep_state
        self.poll_s = poll_s
        self._lock = threading.Lock()
        self._stop = threading.Event()          # stop stepping (hard limit)
        self._closed = threading.Event()        # no further admission
        self._queues: Dict[object, Deque[Request]] = {}
        self._resident = 0
        self._peak_resident = 0
        self._active = 0
        self._peak_active = 0
        self._reuses = 0
        self._step_samples: List[tuple] = []      # (ms, envs in the call)
        self._results: Dict[int, RequestResult] = {}
        self._errors: List[BaseException] = []
        self._n_steps: Dict[int, int] = {}

    # ---------------------------------------------------------------- slots
    def _fill(self, ps: _PoolState, t0: float) -> None:
        """Load waiting requests of the pool's class into its free slots."""
        for s in range(len(ps.req)):
            if ps.req[s] is not None or self._closed.is_set():
                continue
            with self._lock:
                q = self._queues.get(ps.key)
                if not q or self._resident >= self.max_resident:
                    return
                r = q.popleft()
                self._resident += 1
                self._peak_resident = max(self._peak_resident, self._resident)
                if ps.used[s]:
                    self._reuses += 1
            ps.pool.load(s, r)
            ps.req[s], ps.k[s], ps.status[s] = r, 0, 0
            ps.admitted[s] = time.perf_counter() - t0
            ps.used[s] = True

    def _finish(self, ps: _PoolState, s: int, now: float) -> None:
        r = ps.req[s]
        x = y = None
        if self.keep_state:
            x, y = ps.pool.final_state(s)
        res = RequestResult(rid=r.rid, arrival=r.arrival, admitted=float(ps.admitted[s]), finished=now,
                            steps=int(ps.k[s]), status=int(ps.status[s]), slot=(ps.index, s),
                            final_x=x, final_y=y)
        with self._lock:
            self._results[r.rid] = res
            self._resident -= 1
        ps.req[s] = None

    def _run_pool(self, ps: _PoolState, t0: float) -> None:
        try:
            while True:
                self._fill(ps, t0)
                occ = [s for s, r in enumerate(ps.req) if r is not None]
                if not occ:
                    with self._lock:
                        empty = not self._queues.get(ps.key)
                    if self._closed.is_set() or self._stop.is_set() or (empty and self._admission_done):
                        return
                    time.sleep(self.poll_s)
                    continue
                if self._stop.is_set():
                    now = time.perf_counter() - t0
                    for s in occ:
                        self._finish(ps, s, now)
                    return
                with self._lock:
                    self._active += 1
                    self._peak_active = max(self._peak_active, self._active)
                ts = time.perf_counter()
                remaining = [int(ps.req[s].n_steps - ps.k[s]) for s in occ]
                st, taken = ps.pool.advance(occ, [int(ps.k[s]) for s in occ], remaining, self.chunk)
                ms = 1e3 * (time.perf_counter() - ts)
                now = time.perf_counter() - t0
                n_env_steps = int(np.sum(taken))
                with self._lock:
                    self._active -= 1
                    # per-step latency of the call: its time over the most steps one slot took
                    self._step_samples.append((ms / max(int(np.max(taken)), 1), n_env_steps))
                for j, s in enumerate(occ):
                    ps.k[s] += int(taken[j])
                    if st[j] != 0:
                        ps.status[s] = st[j]
                    if ps.k[s] >= ps.req[s].n_steps or st[j] != 0:
                        self._finish(ps, s, now)
        except BaseException as exc:  # surfaced by run()
            with self._lock:
                self._errors.append(exc)
        finally:
            ps.pool.close()
            ps.closed = True

    # ---------------------------------------------------------------- main loop
    def _open_pool(self, key, scene, max_steps, n_pools) -> Optional[_PoolState]:
        n = self.slots_per_pool
        free = self.engine.free_bytes() - self.mem_reserve
        while n > 0 and self.engine.pool_bytes(scene, n) > free:
            n //= 2
        if n == 0:
            return None
        return _PoolState(n_pools, key, self.engine.open_pool(scene, n, max_steps), n)

    def run(self, requests: Sequence[Request], time_limit: Optional[float] = None,
            realtime: bool = True, hard_limit: Optional[float] = None) -> ServeReport:
        """Serve `requests` (arrival times relative to the start).  With
        realtime=False every request counts as arrived at t = 0.  With a
        time_limit, admission stops at that time and the run ends when the
        loaded requests finish; with a hard_limit, stepping stops at that
        time too (the requests in slots then count as not completed)."""
        self._stop.clear()
        self._closed.clear()
        self._admission_done = False
        queue = sorted(requests, key=lambda r: (r.arrival if realtime else 0.0, r.rid))
        self._n_steps = {r.rid: r.n_steps for r in queue}
        max_steps = max([r.n_steps for r in queue] + [1])
        t0 = time.perf_counter()
        live: Dict[object, _PoolState] = {}      # open pools by size class
        opened: List[_PoolState] = []
        threads: List[threading.Thread] = []
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            stop_admitting = time_limit is not None and now >= time_limit
            if stop_admitting:
                self._closed.set()
            while not stop_admitting and nxt < len(queue) and (not realtime or queue[nxt].arrival <= now):
                r = queue[nxt].materialize()
                with self._lock:
                    self._queues.setdefault(self.engine.class_key(r.scene), deque()).append(r)
                nxt += 1
            self._admission_done = nxt == len(queue)
            # a pool for every class with waiting requests (memory and the
            # pool limit permitting); closed pools give their memory back
            for key in [k for k, ps in live.items() if ps.closed]:
                del live[key]
            if not stop_admitting:
                with self._lock:
                    want = [(k, q[0].scene) for k, q in self._queues.items() if q and k not in live]
                for key, scene in want:
                    if len(live) >= self.max_pools:
                        break
                    ps = self._open_pool(key, scene, max_steps, len(opened))
                    if ps is None:
                        continue
                    live[key] = ps
                    opened.append(ps)
                    th = threading.Thread(target=self._run_pool, args=(ps, t0), daemon=True)
                    th.start()
                    threads.append(th)
            with self._lock:
                err = list(self._errors)
                waiting = sum(len(q) for q in self._queues.values())
            if err:
                self._stop.set()
                for th in threads:
                    th.join()
                raise err[0]
            alive = any(th.is_alive() for th in threads)
            if not alive and (stop_admitting or (nxt == len(queue) and waiting == 0)):
                break
            if (not alive and not live and nxt == len(queue) and waiting and not opened and time_limit is None
                    and hard_limit is None):
                raise RuntimeError("no pool fits in device memory")
            if hard_limit is not None and now >= hard_limit:
                self._stop.set()
                self._closed.set()
            time.sleep(self.poll_s)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        with self._lock:
            waiting = sum(len(q) for q in self._queues.values())
        arrived = len(queue) if not realtime else nxt
        return self._report(wall, arrived, waiting + (len(queue) - nxt), opened)

    def _report(self, wall, arrived, backlog, pools) -> ServeReport:
        res = self._results
        env_steps = int(sum(n for _, n in self._step_samples))
        if self._step_samples:
            ms = np.array([m for m, _ in self._step_samples])
            w = np.array([n for _, n in self._step_samples], dtype=np.float64)
            order = np.argsort(ms)
            cw = np.cumsum(w[order]) / w.sum()
            p50 = float(ms[order][np.searchsorted(cw, 0.50)])
            p99 = float(ms[order][min(np.searchsorted(cw, 0.99), len(ms) - 1)])
        else:
            p50 = p99 = float("nan")
        comp = np.array([r.finished - r.arrival for r in res.values()])
        queue = np.array([r.admitted - r.arrival for r in res.values()])

        def pct(a, q):
            return float(np.percentile(a, q)) if len(a) else None
        return ServeReport(
            wall_s=wall, env_steps=env_steps, env_steps_per_s=env_steps / wall if wall > 0 else 0.0,
            step_ms_p50=p50, step_ms_p99=p99,
            completion_s_p50=pct(comp, 50), completion_s_p99=pct(comp, 99),
            queue_s_p50=pct(queue, 50), queue_s_p99=pct(queue, 99),
            queue_s_max=float(queue.max()) if len(queue) else None,
            admitted=len(res),
            completed=sum(1 for r in res.values() if r.status == 0 and r.steps == self._n_steps.get(r.rid, r.steps)),
            arrived=arrived, backlog=backlog, pools=len(pools),
            slots=int(sum(len(p.req) for p in pools)), slot_reuses=self._reuses,
            max_resident=self._peak_resident, max_active_pools=self._peak_active, results=dict(res))


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
