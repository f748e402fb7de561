"""Continuous-batching request loop around the batched IPC step.

A request is one environment (a scene of gel + affine bodies, a kinematic
script and a number of steps) that arrives at some time.  The server keeps
every admitted environment resident on the GPU until its last step and
admits waiting requests whenever a cohort slot and device memory are free:

* a cohort is a group of requests admitted together into one library
  context (one `ipc_create_envs`, one workspace, one CUDA stream);
* each cohort is stepped by its own host thread (the C-ABI calls release the
  GIL), so cohorts admitted at different times overlap on the device;
* admission takes the oldest waiting requests, up to the cohort size limit,
  the resident-environment limit and what the free device memory holds
  (`ipc_workspace_bytes` of the candidate cohort against the free memory
  minus a reserve); a cohort that does not fit is halved until it does;
* a finished cohort closes its context and returns its workspace, which
  lets the next requests in.

Every environment of a cohort is stepped by the same `ipc_step` call; an
env whose script ended is left out of the env-id list (`ipc_step` takes a
subset), so requests of different lengths can share a cohort.

The engine behind the loop is pluggable (`Engine`): `GpuEngine` drives the
library; the tests drive the scheduling logic with a CPU stand-in.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    """One environment to simulate.

    delta(k) -> (n_bodies, 3): translation of each driven body's rest
    placement at step k (the scripted targets; bodies keep A = I).
    Instead of scene and delta a request may carry build() -> (scene, delta),
    called when the request is first considered for admission."""
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
    cohorts: int
    max_resident: int
    max_active_cohorts: int       # cohorts stepping at the same time (overlap)
    results: Dict[int, RequestResult]

    def summary(self) -> dict:
        d = dataclasses.asdict(self)
        d.pop("results")
        return d


class Cohort:
    """Engine-side handle of one admitted cohort."""

    def step(self, env_ids: Sequence[int], k: int) -> np.ndarray:   # per-env status
        raise NotImplementedError

    def final_state(self, i: int):
        raise NotImplementedError

    def close(self) -> None:
        raise NotImplementedError


class Engine:
    def cohort_bytes(self, scenes: Sequence) -> int:
        raise NotImplementedError

    def free_bytes(self) -> int:
        raise NotImplementedError

    def open(self, requests: Sequence[Request]) -> Cohort:
        raise NotImplementedError


class GpuEngine(Engine):
    """The library on one GPU: one context and one CUDA stream per cohort."""

    def __init__(self, params, device: str = "cuda:0", graphs: bool = True):
        import torch

        from . import ipc
        self._torch, self._ipc = torch, ipc
        self.params = params
        self.device = torch.device(device)
        self.graphs = graphs

    def cohort_bytes(self, scenes: Sequence) -> int:
        return self._ipc.workspace_bytes(list(scenes), self.params)

    def free_bytes(self) -> int:
        torch = self._torch
        free, _ = torch.cuda.mem_get_info(self.device)
        # memory held by torch's caching allocator but unused is free to us
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return int(free + cached)

    def open(self, requests: Sequence[Request]) -> Cohort:
        return _GpuCohort(self, requests)


class _GpuCohort(Cohort):
    def __init__(self, eng: GpuEngine, requests: Sequence[Request]):
        torch, ipc = eng._torch, eng._ipc
        self.stream = torch.cuda.Stream(eng.device)
        self.envs = ipc.Envs([r.scene for r in requests], eng.params, device=str(eng.device),
                             stream=self.stream)
        if eng.graphs:
            self.envs.set_graph_mode(True)
        for i, r in enumerate(requests):
            if r.state is not None:
                st = self.envs.set_state(i, *r.state)
                if st != ipc.IPC_OK:
                    raise ipc.IpcError(st, f"request {r.rid}: initial state rejected")
        n, mb = len(requests), self.envs.max_bodies
        n_steps = max(r.n_steps for r in requests)
        # the whole script of every env, resident on the device
        tg = np.zeros((n_steps, n, mb, 12))
        for i, r in enumerate(requests):
            rest = self.envs.rest_y(i)
            nb = rest.shape[0]
            for k in range(r.n_steps):
                t = rest.copy()
                dl = np.asarray(r.delta(k), dtype=np.float64).reshape(-1, 3)
                t[:, :3] += dl[:nb]
                tg[k, i, :nb] = t
        with torch.cuda.stream(self.stream):
            self.dev_tg = torch.as_tensor(tg, device=eng.device)

    def step(self, env_ids: Sequence[int], k: int) -> np.ndarray:
        self.envs.set_targets_all_device(self.dev_tg[k])
        status, _ = self.envs.step(list(env_ids))
        return status

    def final_state(self, i: int):
        x, _, y, _ = self.envs.get_state(i)
        return x, y

    def close(self) -> None:
        self.envs.close()
        self.dev_tg = None


class Server:
    """Admission and stepping loop (see the module docstring)."""

    def __init__(self, engine: Engine, max_resident: int = 4096, max_cohort: int = 512,
                 max_cohorts: int = 8, mem_reserve: int = 2 << 30, keep_state: bool = True,
                 poll_s: float = 0.002):
        self.engine = engine
        self.max_resident = max_resident
        self.max_cohort = max_cohort
        self.max_cohorts = max_cohorts
        self.mem_reserve = mem_reserve
        self.keep_state = keep_state
        self.poll_s = poll_s
        self._lock = threading.Lock()
        self._stop = threading.Event()
        self._resident = 0
        self._active = 0
        self._peak_active = 0
        self._step_samples: List[tuple] = []      # (ms, envs in the call)
        self._results: Dict[int, RequestResult] = {}
        self._errors: List[BaseException] = []
        self._n_steps: Dict[int, int] = {}

    # ---------------------------------------------------------------- admission
    def _admit(self, waiting: List[Request]) -> List[Request]:
        """Largest FIFO prefix of `waiting` that fits the limits (may be empty)."""
        with self._lock:
            room = min(self.max_cohort, self.max_resident - self._resident)
            slots = self.max_cohorts - self._active
        if room <= 0 or slots <= 0 or not waiting:
            return []
        n = min(room, len(waiting))
        for r in waiting[:n]:
            r.materialize()
        free = self.engine.free_bytes() - self.mem_reserve
        while n > 0:
            if self.engine.cohort_bytes([r.scene for r in waiting[:n]]) <= free:
                return waiting[:n]
            n //= 2
        return []

    # ---------------------------------------------------------------- stepping
    def _run_cohort(self, reqs: List[Request], t0: float, admitted_at: float):
        try:
            coh = self.engine.open(reqs)
            status = np.zeros(len(reqs), np.int32)
            done_at = [None] * len(reqs)
            taken = np.zeros(len(reqs), int)
            n_max = max(r.n_steps for r in reqs)
            for k in range(n_max):
                ids = [i for i, r in enumerate(reqs) if k < r.n_steps and status[i] == 0]
                if not ids or self._stop.is_set():
                    break
                ts = time.perf_counter()
                st = coh.step(ids, k)
                ms = 1e3 * (time.perf_counter() - ts)
                now = time.perf_counter() - t0
                with self._lock:
                    self._step_samples.append((ms, len(ids)))
                for j, i in enumerate(ids):
                    taken[i] += 1
                    if st[j] != 0:
                        status[i] = st[j]
                    if k == reqs[i].n_steps - 1 or st[j] != 0:
                        done_at[i] = now
            finished = time.perf_counter() - t0
            for i, r in enumerate(reqs):
                x = y = None
                if self.keep_state:
                    x, y = coh.final_state(i)
                res = RequestResult(rid=r.rid, arrival=r.arrival, admitted=admitted_at,
                                    finished=done_at[i] if done_at[i] is not None else finished,
                                    steps=int(taken[i]), status=int(status[i]), final_x=x, final_y=y)
                with self._lock:
                    self._results[r.rid] = res
            coh.close()
        except BaseException as exc:  # surfaced by run()
            with self._lock:
                self._errors.append(exc)
        finally:
            with self._lock:
                self._resident -= len(reqs)
                self._active -= 1

    def run(self, requests: Sequence[Request], time_limit: Optional[float] = None,
            realtime: bool = True, hard_limit: Optional[float] = None) -> ServeReport:
        """Serve `requests` (arrival times relative to the start).  With
        realtime=False every request counts as arrived at t = 0.  With a
        time_limit, admission stops at that time and the run ends when the
        admitted cohorts finish; with a hard_limit, cohorts stop stepping at
        that time too (their requests count as not completed)."""
        self._stop.clear()
        queue = sorted(requests, key=lambda r: (r.arrival if realtime else 0.0, r.rid))
        self._n_steps = {r.rid: r.n_steps for r in queue}
        t0 = time.perf_counter()
        threads: List[threading.Thread] = []
        nxt = 0
        waiting: List[Request] = []
        cohorts = 0
        peak = 0
        while True:
            now = time.perf_counter() - t0
            while nxt < len(queue) and (not realtime or queue[nxt].arrival <= now):
                waiting.append(queue[nxt])
                nxt += 1
            stop_admitting = time_limit is not None and now >= time_limit
            if not stop_admitting:
                batch = self._admit(waiting)
                if batch:
                    waiting = waiting[len(batch):]
                    with self._lock:
                        self._resident += len(batch)
                        self._active += 1
                        peak = max(peak, self._resident)
                        self._peak_active = max(self._peak_active, self._active)
                    cohorts += 1
                    th = threading.Thread(target=self._run_cohort, args=(batch, t0, now), daemon=True)
                    th.start()
                    threads.append(th)
                    continue
            with self._lock:
                active = self._active
                err = list(self._errors)
            if err:
                for th in threads:
                    th.join()
                raise err[0]
            if active == 0 and (stop_admitting or (nxt == len(queue) and not waiting)):
                break
            if hard_limit is not None and now >= hard_limit:
                self._stop.set()
            time.sleep(self.poll_s)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        return self._report(wall, len(queue) if not realtime else nxt, len(waiting) + (len(queue) - nxt),
                            cohorts, peak)

    def _report(self, wall, arrived, backlog, cohorts, peak) -> ServeReport:
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
            arrived=arrived, backlog=backlog, cohorts=cohorts, max_resident=peak,
            max_active_cohorts=self._peak_active, results=dict(res))


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
