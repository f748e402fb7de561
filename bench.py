#!/usr/bin/env python
"""Throughput of the batched ABD-IPC step: env-steps/s.

Workload (the uniform-batch configuration): 256 environments, each a
40x40x6-vertex neo-Hookean gel (20x20x4 mm, 9600 vertices, 38 025 tets,
bottom pinned) pressed by a driven level-2 icosphere (162 vertices, r = 4 mm)
with a seeded press-then-slide script, dt = 1e-3 s, dhat = 1e-4 m, FP64.
One bench step = one ipc_step over all envs (time step k of every env's
script).  The working set (~24 GB) is far larger than L2 (126 MB), so no
explicit flush is needed between steps.

Outputs ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s"
WORKLOAD = "uniform batch: 256 envs x (gel 40x40x6 + ABD icosphere L2, press/slide)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=256)
    ap.add_argument("--precision", type=int, default=1,
                    help="1: time FP64 then mixed (headline); 0: FP64 only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-env", action="store_true", help="skip the per-env FP64 GPU comparison")
    ap.add_argument("--only-mixed", action="store_true",
                    help="time only the mixed path (profiling runs); no FP64 comparison")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "serving", "uneven", "self_contact", "grasp", "single", "broadphase"],
                    help="batch: the uniform 256-env batch (default); serving: the Poisson request stream; "
                         "uneven: 512 config-2 envs of different sizes in one launch; "
                         "self_contact: 1024 two-block pads pressed together (gel self-contact); "
                         "grasp: 1024 two-finger grasps (config 3); single: config 0, one env, FP64")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serving: admission window (s)")
    ap.add_argument("--serve-hard", type=float, default=60.0, help="serving: stop stepping at this time (s)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--req-steps", type=int, default=200, help="serving: steps per request")
    ap.add_argument("--max-resident", type=int, default=4096)
    ap.add_argument("--slots-per-pool", type=int, default=256, help="serving: env slots per size-class pool")
    ap.add_argument("--max-pools", type=int, default=32)
    ap.add_argument("--no-graphs", action="store_true", help="serving: plain launches instead of PCG graphs")
    ap.add_argument("--serve-chunk", type=int, default=8, help="serving: steps per pool call (rollout when > 1)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--pcg-window", type=int, default=None,
                    help="rollout: PCG iterations per loop iteration (even; 0 = whole solves; default: the library's)")
    ap.add_argument("--pcg-fused", type=int, default=None, choices=(0, 1, 2),
                    help="1 / 2: one fused kernel per PCG iteration (update items in ready / env order), "
                         "0: three kernels (default: the library's)")
    ap.add_argument("--pcg-iters-per-launch", type=int, default=None,
                    help="fused PCG kernel: iterations per launch (default: the library's)")
    ap.add_argument("--no-lockstep", action="store_true", help="skip the lock-step timing beside the rollout")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel profiling pass")
    return ap.parse_args()


def max_over_ranks(ms: float, world: int, device) -> float:
    """The timed region of the slowest rank (every rank gets it)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(envs_per_rank: int, steps: int, world: int, ms: float) -> float:
    """env-steps/s of the whole job: every rank advanced its own envs (weak
    scaling over independent envs), divided by the slowest rank's time."""
    return envs_per_rank * steps * world / (ms / 1e3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ workload
def build_workload(n_envs, precision, pcg_window=None, pcg_fused=None, pcg_ipl=None):
    import scenes
    scene, params, deltas = scenes.config1_batch(n_envs)
    params.precision = precision
    if pcg_window is not None:
        params.rollout_pcg_window = pcg_window
    if pcg_fused is not None:
        params.pcg_fused = pcg_fused
    if pcg_ipl is not None:
        params.pcg_iters_per_launch = pcg_ipl
    return scene, params, deltas


def targets_for(envs, deltas, step, com):
    """[n_envs][1][12] rest placement of the icosphere translated by its script."""
    t = np.zeros((len(deltas), 1, 12))
    for e, dl in enumerate(deltas):
        t[e, 0, :3] = com + dl(step)[0]
        t[e, 0, 3:] = np.eye(3).T.ravel()
    return t


# ------------------------------------------------------------------ CPU oracle sample
_ORACLE_CHILD = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
import scenes
from oracle import OracleEnv
from oracle import distance as ods
for k in ("PP", "PE", "PT", "EE", "X"):
    ods._sym(k)          # symbolic set-up outside the timed sample
z = np.load({inp!r})
env_i, step_i = int(z["env"]), int(z["step"])
scene, params, deltas = scenes.config1_batch(env_i + 1)
params.precision = 0
env = OracleEnv(scene, params)
t0 = time.perf_counter()
x, v, y, yd, st = env.step(z["x"], z["v"], z["y"], z["yd"], env.targets_from_delta(deltas[env_i](step_i)))
dt = time.perf_counter() - t0
np.savez({out!r}, x=x, y=y, seconds=dt, status=st.status, newton=st.newton_iters)
"""


def oracle_steps_parallel(states, cores):
    """The FP64 oracle advancing each given env of the workload by one step,
    one env per child process (BLAS/OpenMP pools at one thread), `cores`
    processes at a time.  states: list of (env, step, x, v, y, yd).  Returns
    (wall seconds, per-env result dicts).  Children are fresh interpreters
    (no CUDA context is forked)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    tmp = tempfile.mkdtemp(prefix="oracle_")
    jobs = []
    for i, (e, k, x, v, y, yd) in enumerate(states):
        inp, out = os.path.join(tmp, f"in{i}.npz"), os.path.join(tmp, f"out{i}.npz")
        np.savez(inp, env=e, step=k, x=x, v=v, y=y, yd=yd)
        jobs.append((inp, out))
    t0 = time.perf_counter()
    running, results, queue = [], {}, list(enumerate(jobs))
    while queue or running:
        while queue and len(running) < cores:
            i, (inp, out) = queue.pop(0)
            code = _ORACLE_CHILD.format(root=ROOT, inp=inp, out=out)
            running.append((i, out, subprocess.Popen([sys.executable, "-c", code], env=env,
                                                     stdout=subprocess.DEVNULL, stderr=subprocess.PIPE)))
        time.sleep(0.05)
        still = []
        for i, out, pr in running:
            if pr.poll() is None:
                still.append((i, out, pr))
                continue
            if pr.returncode != 0:
                raise RuntimeError("oracle child failed: " + pr.stderr.read().decode()[-2000:])
            z = np.load(out)
            results[i] = {k: z[k] for k in z.files}
        running = still
    wall = time.perf_counter() - t0
    return wall, [results[i] for i in range(len(jobs))]


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    """The reference arm of this tier: the FP64 oracle on the host cores, on
    a bounded sample of the same workload (each bench step: one step, from
    the rest state, of `cores` envs in parallel processes)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import scenes
    cores = max(1, min(os.cpu_count() or 1, 16))
    scene, params, deltas = scenes.config1_batch(1)
    from oracle import OracleEnv
    x, v, y, yd = OracleEnv(scene, params).rest_state()
    times = []
    for k in range(args.warmup + args.steps):
        states = [((k * cores + j) % args.envs, 0, x, v, y, yd) for j in range(cores)]
        wall, _ = oracle_steps_parallel(states, cores)
        if k >= args.warmup:
            times.append(wall)
    ms = 1e3 * float(np.mean(times))
    value = cores / float(np.mean(times))
    sample = (f"{cores} envs x 1 time step (step 0 of each env's script) per bench step, one env per process on "
              f"{cores} of {os.cpu_count()} host cores ({cpu_model()}), oracle FP64, BLAS threads = 1")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "envs_per_step": cores, "cache": "inputs larger than L2 (per env ~95 MB)"},
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ ours
def kernel_bytes(genv, tot):
    """Algorithmic bytes of every kernel class over a run with the counters
    `tot` (what each class must move at least for the work it did, per the
    units in the design notes: 3x3 blocks and rows per PCG iteration, tets
    and rows per Newton iteration, pairs per evaluation)."""
    sz = genv.system_sizes(0)
    nv, nb, ns = genv.sizes[0]
    rows = nv + 4 * nb
    T = sz["tets"]
    blocks = sz["real_blocks"]
    hs = 4 if getattr(genv.params, "precision", 0) else 8   # Hessian / matrix value bytes
    vb = 12 if hs == 4 else 24                               # a PCG row of z, d or q
    pcg, newt = tot["pcg_iters"], tot["newton_env_iters"]
    n_ls = max(newt - tot["env_steps"], 0)                   # line searches: iterations that did not stop
    ls_evals = tot["ls_trials"] + n_ls                       # trials + the energy at alpha = 0
    # contact vertices, at least: the coated gel surface and the body vertices
    n_cv = ns + sum(len(b.rest_x) for b in genv.scenes[0].bodies)
    out = {
        # matrix values + columns, z and d_{k-1} read, d_k and q written per row
        "pcg_matvec": pcg * (blocks * (9 * hs + 4) + rows * 4 * vb),
        # per active pair and PCG iteration: its packed 78-entry Hessian, the 4 points' z and d_{k-1}
        # rows gathered, 12 FP64 contact entries scattered
        "pair_matvec": tot.get("act_pair_iters", 0) * (78 * hs + 4 * 2 * vb + 12 * 8),
        # p and r read + written (FP64), d_k and q read, the 6-entry inverse block, z written
        # (the fused iteration kernel, pcg_iter, does the work of the three PCG classes)
        "pcg_update": pcg * rows * (4 * 24 + 2 * vb + 6 * hs + vb),
        # indices, positions, Dm^-1, volume read; FP64 gradient and the Hessian written
        "tet_elastic": newt * T * (16 + 96 + 72 + 8 + 96 + 144 * hs),
        # every element block read once, every real block written once
        "assemble": newt * (T * 144 * hs + blocks * (9 * hs + 4)),
        # per static pair: 4 ids, 4 points, weight + mollifier read; packed Hessian (78) and gradient written
        "barrier": tot["pair_evals"] * (16 + 96 + 16 + 78 * hs + 96),
        # per swept pair: 8 points x 3 x 8 B x 2 (x, p)
        "accd": tot["swept_pairs"] * 384,
        # per energy evaluation: per tet ids + positions + Dm^-1 + volume, per row x, p, xt, per swept pair its points
        "ls_energy": ls_evals * (T * (16 + 96 + 72 + 8 + 8) + rows * (72 + 8)) + tot["swept_pairs"] * 200,
        # per Newton iteration: gradient gather (12 per tet corner) + x, xt, qc, g per row
        "gradient": newt * (T * 4 * 24 + rows * 4 * 24),
        # per body and Newton iteration: state, target, 12x12 Hessian and gradient
        "body_abd": newt * nb * (4 * 96 + 144 * 8 + 96),
        # per Newton iteration: each row's diagonal block read and its 6-entry inverse written; each
        # body's 12x12 block read and its inverse written (FP64)
        "precond": newt * (rows * 15 * hs + nb * 2 * 144 * 8),
        # per search: the contact vertices' positions read (x for the static search of a Newton
        # iteration, x and p for the swept search of a line search), each candidate pair written
        # (4 ids, kind, weight, mollifier threshold)
        "broad_phase": (newt + n_ls) * n_cv * 24 + n_ls * n_cv * 24 + (tot["pair_evals"] + tot["swept_pairs"]) * 36,
    }
    # per Newton iteration: g read, r, p, z and d_{-1} written, the 6-entry inverse read
    out["pcg_init"] = newt * rows * (24 + 48 + 2 * vb + 6 * hs)
    # per Newton iteration: p read per row (x and the target on attached rows, left out)
    out["newton_check"] = newt * rows * 24
    # per step: x and v read, the predicted position written
    out["predict"] = tot["env_steps"] * rows * 72
    # per search: each contact vertex's row (gel) or body state and rest point read, its position written
    out["cv_pos"] = (newt + n_ls) * n_cv * 48
    out["pcg_iter"] = out["pcg_matvec"] + out["pair_matvec"] + out["pcg_update"]
    return out


def time_steps(genv, dev_tg, k0, steps, stream):
    """Steps k0 .. k0 + steps - 1 (device-resident targets), CUDA events on
    the context's stream around each step; per-step statuses and counters."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tot = {"pcg_iters": 0, "newton_env_iters": 0, "ls_trials": 0, "newton_max": 0, "max_pairs": 0,
           "al_env_updates": 0, "ccd_limited": 0, "alpha_sum": 0.0, "accd_iters": 0, "accd_iters_max": 0,
           "pair_evals": 0, "swept_pairs": 0, "act_pair_iters": 0, "env_steps": 0, "graph_loop_iters": 0,
           "graph_pcg_launches": 0}
    statuses = []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        genv.set_targets_all_device(dev_tg[k0 + i])
        st, s = genv.step()
        ev[i][1].record(stream)
        statuses.append(st)
        for key in ("pcg_iters", "newton_env_iters", "ls_trials", "al_env_updates", "ccd_limited", "alpha_sum",
                    "accd_iters", "pair_evals", "swept_pairs", "act_pair_iters"):
            tot[key] += s[key]
        tot["newton_max"] = max(tot["newton_max"], s["newton_iters"])
        tot["max_pairs"] = max(tot["max_pairs"], s["max_pairs"])
        tot["accd_iters_max"] = max(tot["accd_iters_max"], s["accd_iters_max"])
        tot["env_steps"] += len(st)
        tot["graph_loop_iters"] += s["loop_iters"]
        tot["graph_pcg_launches"] += s["pcg_launches"]
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev], tot, statuses


def time_rollout(genv, dev_tg, k0, steps, stream):
    """Steps k0 .. k0 + steps - 1 as one rollout (every env on its own
    schedule, device-resident targets), CUDA events on the context's stream
    around it; per-env statuses and the summed counters."""
    import torch
    tab = dev_tg[k0:k0 + steps]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    genv.rollout(steps, tab, wait=False)
    t1.record(stream)
    st, taken, s = genv.rollout_results()
    torch.cuda.synchronize()
    tot = {k: s[k] for k in ("pcg_iters", "newton_env_iters", "ls_trials", "al_env_updates", "ccd_limited",
                             "alpha_sum", "accd_iters", "pair_evals", "swept_pairs", "act_pair_iters")}
    tot.update({"newton_max": s["newton_iters"], "max_pairs": s["max_pairs"], "accd_iters_max": s["accd_iters_max"],
                "env_steps": int(np.sum(taken)), "graph_loop_iters": s["loop_iters"],
                "graph_pcg_launches": s["pcg_launches"]})
    return t0.elapsed_time(t1), tot, st, taken


def snapshot(genv):
    return [genv.get_state(e) for e in range(genv.n_envs)]


def restore(genv, snap):
    for e, st in enumerate(snap):
        r = genv.set_state(e, *st)
        if r != 0:
            raise RuntimeError(f"set_state({e}) -> {r}")


def per_step_error(g64, g32, tg, body_radius, states=None):
    """Spec'd error of the mixed form: one step of both paths from the same
    input state (`states`, else the FP64 path's current state; every env),
    largest vertex difference over all gel vertices and body vertices,
    relative to the gel box diagonal.  Body vertices are bounded through the
    12 DoF: |dp| + R * sum_j |dA_ij| for points within radius R of the
    frame."""
    n = len(g64.sizes)
    for e in range(n):
        st = g64.get_state(e) if states is None else states[e]
        for g in (g64, g32):
            assert g.set_state(e, *st) == 0
    for g in (g64, g32):
        g.set_targets_all_device(tg)
    s64, _ = g64.step()
    s32, _ = g32.step()
    diag = float(np.linalg.norm(np.array([0.02, 0.02, 0.004])))
    errs = np.zeros(n)
    for e in range(n):
        x64, _, y64, _ = g64.get_state(e)
        x32, _, y32, _ = g32.get_state(e)
        errs[e] = state_diff(x64, y64, x32, y32, body_radius) / diag
    return errs, int(np.sum(s64 != 0) + np.sum(s32 != 0))


def error_distribution(errs):
    errs = np.concatenate(errs)
    return {"max": float(errs.max()), "p99": float(np.percentile(errs, 99)), "median": float(np.median(errs)),
            "env_steps_above_1e-4": int(np.sum(errs > 1e-4)), "env_steps": int(errs.size)}


def state_diff(xa, ya, xb, yb, body_radius):
    d = float(np.abs(xa - xb).max())
    dy = np.abs(np.asarray(ya) - np.asarray(yb)).reshape(-1, 4, 3)   # [p, a0, a1, a2] per body
    if dy.size:
        d = max(d, float((dy[:, 0, :] + body_radius * dy[:, 1:, :].sum(axis=1)).max()))
    return d


# DRAM traffic of one mat-vec launch (dram__bytes_read.sum +
# dram__bytes_write.sum under ncu: the first launch of the 24-env case, every
# env in its first PCG iteration, inputs larger than L2) and the
# env-iterations that launch processed; reported, scaled to the average
# launch by env-iterations, only while the kernel's source is the one that
# was measured (hash of its text).
MATVEC_TRAFFIC = {"env_iters": 24, "bytes": 116996352 + 3195136,
                  "source_sha256": "6c0cc14516947417a70839a2ad4f2b3dd6f6613b6cc979217d68974595a0b7c9"}


def _function_text(src: str, signature: str) -> str:
    """The text of the function whose definition starts at `signature` (up
    to its closing brace at column 0)."""
    i = src.index(signature)
    j = src.index("\n}\n", i)
    return src[i:j + 3]


def _kernel_source_hash(parts) -> str:
    """Hash of (file, signature or None for the whole file) source parts."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2504_12908_b300", "csrc")
    h = hashlib.sha256()
    for f, sig in parts:
        src = open(os.path.join(csrc, f)).read()
        h.update((src if sig is None else _function_text(src, sig)).encode())
    return h.hexdigest()


MATVEC_PARTS = [("pcgvec.cuh", None), ("kernels_pcg.cu", "__device__ __forceinline__ void matvec_rows("),
                ("kernels_pcg.cu", "__global__ void __launch_bounds__(128) k_pcg_matvec(")]


def _matvec_source_hash() -> str:
    return _kernel_source_hash(MATVEC_PARTS)


def matvec_traffic_per_launch(env_iters_per_launch):
    if MATVEC_TRAFFIC["bytes"] is None or _matvec_source_hash() != MATVEC_TRAFFIC["source_sha256"]:
        return None
    return MATVEC_TRAFFIC["bytes"] / MATVEC_TRAFFIC["env_iters"] * env_iters_per_launch


# The same for the fused PCG kernel as the bench runs it (k_pcg_multi: 8
# iterations of contact terms, SELL mat-vec and update per launch): DRAM
# bytes of its third launch in the 24-env case (mid-solve, ~180 of its 192
# env-iterations run: counted from its FP64 instructions at 23.25 per row
# and iteration), scaled by env-iterations.
PCG_ITER_TRAFFIC = {"env_iters": 179.73, "bytes": 922980096 + 133039616, "source_sha256": "32b2347407bcfb0359651f38d18ec402c9e53d4005e7196b8e55ac856ae6c319"}
PCG_ITER_PARTS = [("pcgvec.cuh", None), ("fpconv.cuh", None),
                  ("kernels_pcg.cu", "__device__ __forceinline__ void matvec_rows("),
                  ("kernels_pcg.cu", "__device__ __forceinline__ void matvec_pairs("),
                  ("kernels_pcg.cu", "__device__ __forceinline__ void update_rows("),
                  ("kernels_pcg.cu", "k_pcg_multi(Dev d")]


def pcg_iter_traffic_per_launch(env_iters_per_launch):
    if PCG_ITER_TRAFFIC["bytes"] is None or _kernel_source_hash(PCG_ITER_PARTS) != PCG_ITER_TRAFFIC["source_sha256"]:
        return None
    return PCG_ITER_TRAFFIC["bytes"] / PCG_ITER_TRAFFIC["env_iters"] * env_iters_per_launch


# FP64 floating-point operations per unit of work of the FP64-heavy kernel
# classes in the mixed mode (dadd + dmul + 2 dfma thread instructions of one
# launch under ncu, divided by the units that launch processed: the first
# launch of each kernel in a process, every env active).  Reported, as an
# ALU roofline against the measured FP64 FMA rate, only while the kernel
# sources are the ones that were measured (hash of their text).
FP64_FLOPS_PER_UNIT = {
    "tet_elastic": (242.0, "0657c712ffa87872172c39c9433c5f8809afe6af23538ae1311894e1c2e972ad"),
    "body_abd": (4920.0, "176a85a7dc5c0d3c979f3de3ea30e78cb61eee8f864c11b05d2bc3a3ad460833"),
    "pcg_iter": (23.25, "32b2347407bcfb0359651f38d18ec402c9e53d4005e7196b8e55ac856ae6c319"),
}
ALU_UNIT = {"tet_elastic": "tet per Newton iteration", "body_abd": "body per Newton iteration",
            "pcg_iter": "row per PCG iteration"}
ALU_PARTS = {
    "tet_elastic": [("physics.cuh", None), ("common.cuh", None),
                    ("kernels_solver.cu", "__global__ void __launch_bounds__(64) k_tet(")],
    "body_abd": [("physics.cuh", None), ("common.cuh", None),
                 ("kernels_solver.cu", "__global__ void __launch_bounds__(128) k_body(")],
    "pcg_iter": PCG_ITER_PARTS,
}


def alu_rooflines(genv, prof, tot, fp64_tflops):
    """FP64 GFLOP/s of the ALU-bound classes from their flop counts per unit
    and their profiled time, against the measured FP64 FMA rate."""
    if fp64_tflops is None:
        return None
    sz = genv.system_sizes(0)
    nv, nb, _ = genv.sizes[0]
    units = {"tet_elastic": tot["newton_env_iters"] * sz["tets"], "body_abd": tot["newton_env_iters"] * nb,
             "pcg_iter": tot["pcg_iters"] * (nv + 4 * nb)}
    out = {}
    for k, (per, sha) in FP64_FLOPS_PER_UNIT.items():
        if per is None or k not in prof or prof[k][1] <= 0 or sha != _kernel_source_hash(ALU_PARTS[k]):
            continue
        gf = per * units[k] / (prof[k][1] / 1e3) / 1e9
        out[k] = {"bound": "alu", "achieved": round(gf, 1), "peak": round(1e3 * fp64_tflops, 1), "unit": "GFLOP/s (FP64)",
                  "frac": round(gf / (1e3 * fp64_tflops), 4), "flops_per_unit": per, "unit_of_work": ALU_UNIT[k]}
    return out


def roofline_of(genv, prof, tot):
    """Per-class time shares (profile pass) and GB/s of algorithmic bytes;
    the roofline line for the dominant class."""
    kb = kernel_bytes(genv, tot)
    peak, peak_kind = measured_peaks()
    tot_ms = max(sum(v[1] for v in prof.values()), 1e-9)
    kernels = {}
    for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        if n == 0:
            continue
        row = {"launches": n, "ms": round(ms, 3), "share": round(ms / tot_ms, 4)}
        if name in kb and ms > 0:
            row["GB/s"] = round(kb[name] / (ms / 1e3) / 1e9, 1)
            row["frac_of_hbm"] = round(kb[name] / (ms / 1e3) / 1e9 / peak, 4)
        kernels[name] = row
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    rk = dom if dom in kb else "pcg_matvec"
    n, ms = prof[rk]
    achieved = kb[rk] / (ms / 1e3) / 1e9
    traffic = None
    if rk == "pcg_matvec":
        traffic = matvec_traffic_per_launch(tot["pcg_iters"] / max(n, 1))
    elif rk == "pcg_iter":
        traffic = pcg_iter_traffic_per_launch(tot["pcg_iters"] / max(n, 1))
    roof = {"kernel": rk, "dominant_kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
            "bytes_per_launch": kb[rk] / max(n, 1), "env_iters_per_launch": tot["pcg_iters"] / max(n, 1),
            "share_of_step": kernels[rk]["share"]}
    return roof, kernels


def per_env_fp64(scene, params, deltas, snap64, k0, envs, steps, device, graph_mode=0):
    """The plain per-environment FP64 GPU path: each env alone in its own
    context (one env per ipc_step), started from the batch's FP64 state at
    step k0; env-steps/s over the sample (host clock, synchronised)."""
    import torch

    from paper_2504_12908_b300 import ipc
    prm = type(params)(**params.__dict__)
    prm.precision = 0
    n, t = 0, 0.0
    ms = []
    for e in envs:
        g = ipc.Envs([scene], prm, device=device, stream=torch.cuda.Stream() if graph_mode else None)
        if graph_mode:
            g.set_graph_mode(graph_mode)
        com = g.body_com(0, 0)
        assert g.set_state(0, *snap64[e]) == 0
        tg = targets_for(None, [deltas[e]], 0, com)   # shape only
        torch.cuda.synchronize()
        for k in range(k0, k0 + steps):
            tg = targets_for(None, [deltas[e]], k, com)
            g.set_targets_all(tg)
            t0 = time.perf_counter()
            g.step()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            t += dt
            ms.append(1e3 * dt)
            n += 1
        g.close()
    return {"value": n / t, "unit": METRIC, "ms_per_env_step": {"p50": float(np.percentile(ms, 50)),
                                                               "p99": float(np.percentile(ms, 99))},
            "sample": f"{len(envs)} envs x {steps} steps (steps {k0}-{k0 + steps - 1}), each env alone in its own "
                      f"context, FP64, " + ("whole-step graphs" if graph_mode == 2 else "plain launches")}


def run_precision(args, scene, params, deltas, precision, local, world, dev_tg, lockstep=True):
    """One precision mode on the batch: warm-up, autotune, snapshot at the
    first timed step, then the timed regions (no profiling): the K steps as
    one rollout (every env on its own schedule, the headline), and, when
    `lockstep`, as K batched whole-step graphs from the same snapshot (the
    per-step latencies)."""
    import torch

    from paper_2504_12908_b300 import ipc
    prm = type(params)(**params.__dict__)
    prm.precision = precision
    stream = torch.cuda.Stream(device=f"cuda:{local}")
    genv = ipc.Envs([scene] * args.envs, prm, device=f"cuda:{local}", stream=stream)
    genv.set_graph_mode(2)
    for k in range(args.warmup):
        genv.set_targets_all_device(dev_tg[k])
        genv.step()
    tuning = genv.autotune() if not args.no_autotune else None
    genv.rollout(0, dev_tg[args.warmup:args.warmup])   # captures the rollout graph; no step
    snap = snapshot(genv)
    torch.cuda.synchronize()
    lock = None
    if lockstep:
        if world > 1:
            torch.distributed.barrier()
        ms, step_ms, tot, statuses = time_steps(genv, dev_tg, args.warmup, args.steps, stream)
        ms = max_over_ranks(ms, world, f"cuda:{local}")
        lock = {"value": whole_job_rate(args.envs, args.steps, world, ms), "ms_total": ms, "step_ms": step_ms,
                "tot": tot, "n_bad": int(sum(int(np.sum(s_ != 0)) for s_ in statuses))}
        restore(genv, snap)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = genv.launch_count()
    ms, tot, st, taken = time_rollout(genv, dev_tg, args.warmup, args.steps, stream)
    clk = clocks.stop()
    end = snapshot(genv) if precision == 0 else None
    launches = genv.launch_count() - l0
    ms = max_over_ranks(ms, world, f"cuda:{local}")
    n_bad = int(np.sum(st != 0)) + int(np.sum(taken != args.steps))
    return {"genv": genv, "stream": stream, "snap": snap, "value": whole_job_rate(args.envs, args.steps, world, ms),
            "ms_total": ms, "tot": tot, "clocks": clk, "launches": launches, "n_bad": n_bad,
            "tuning": tuning, "lock": lock, "end": end}


def run_ours(args):
    import torch

    from paper_2504_12908_b300.build import build

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build()
    scene, params, deltas = build_workload(args.envs, 0, args.pcg_window, args.pcg_fused, args.pcg_iters_per_launch)
    n_total = args.warmup + args.steps
    dev = f"cuda:{local}"

    # targets of every step (device-resident for the timed region)
    from paper_2504_12908_b300 import ipc
    probe = ipc.Envs([scene], params, device=dev)
    com = probe.body_com(0, 0)
    probe.close()
    dev_tg = torch.as_tensor(np.stack([targets_for(None, deltas, k, com) for k in range(n_total + 1)]),
                             dtype=torch.float64, device=dev)
    precisions = [0] if args.precision == 0 else ([1] if args.only_mixed else [0, 1])
    results = {}
    for prec in precisions:
        # batched FP64 is timed as a rollout only (its lock-step form is the
        # slower of the two)
        results[prec] = run_precision(args, scene, params, deltas, prec, local, world, dev_tg,
                                      lockstep=(prec == precisions[-1] and not args.no_lockstep))
    hp = precisions[-1]
    head = results[hp]
    genv, stream = head["genv"], head["stream"]

    roof = kernels = alu = fma = None
    if not args.no_profile:
        # per-class shares: the same rollout again from the snapshot, with
        # per-kernel CUDA events (the same loop as plain launches driven from the
        # host); not part of the timed region
        restore(genv, head["snap"])
        genv.profile_enable(True)
        genv.profile_reset()
        _, taken_p, s_p = genv.rollout(args.steps, dev_tg[args.warmup:n_total])
        prof = genv.profile()
        genv.profile_enable(False)
        tot_p = {"pcg_iters": s_p["pcg_iters"], "newton_env_iters": s_p["newton_env_iters"],
                 "ls_trials": s_p["ls_trials"], "pair_evals": s_p["pair_evals"], "swept_pairs": s_p["swept_pairs"],
                 "accd_iters": s_p["accd_iters"], "act_pair_iters": s_p["act_pair_iters"],
                 "env_steps": int(np.sum(taken_p))}
        roof, kernels = roofline_of(genv, prof, tot_p)
        try:
            fma = ipc.fma_peaks(dev)
        except Exception:  # noqa: BLE001 - reported as unavailable
            fma = None
        alu = alu_rooflines(genv, prof, tot_p, fma["fp64_tflops"] if fma else None)

    # e2e through the public API on the same steps: every step's targets
    # copied in from pinned host memory, the rollout, and the per-env
    # statuses, step counts and final coated surfaces copied out
    e2e = e2e_lock = None
    if not args.no_e2e:
        restore(genv, head["snap"])
        mb = max(genv.max_bodies, 1)
        host_tg = torch.empty((args.steps, args.envs, mb, 12), dtype=torch.float64, pin_memory=True)
        dev_tab = torch.empty((args.steps, args.envs, mb, 12), dtype=torch.float64, device=dev)
        n_out = sum(s_[2] for s_ in genv.sizes)
        host_out = torch.empty((n_out, 3), dtype=torch.float64, pin_memory=True)
        tg_np, out_np = host_tg.numpy(), host_out.numpy()
        for i in range(args.steps):
            tg_np[i] = targets_for(None, deltas, args.warmup + i, com)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            dev_tab.copy_(host_tg, non_blocking=True)
        genv.rollout(args.steps, dev_tab, wait=False)
        st_e, taken_e, _ = genv.rollout_results()
        genv.read_gel_surface_all(out_np)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": args.envs * args.steps * world / dt, "unit": METRIC,
               "h2d_bytes_per_step": int(tg_np.nbytes // args.steps),
               "d2h_bytes_per_step": int((out_np.nbytes + st_e.nbytes + taken_e.nbytes) // args.steps),
               "steps": f"{args.warmup}-{n_total - 1} (the timed steps, from the same state) as one rollout: "
                        f"every step's targets in from pinned host memory, statuses, step counts and final "
                        f"coated surfaces out; bytes per step = the call's bytes / steps",
               "status_not_ok": int(np.sum(st_e != 0) + np.sum(taken_e != args.steps))}
        # the same through K batched ipc_step calls: targets in and coated
        # surfaces out every step
        restore(genv, head["snap"])
        host_tg1 = torch.empty((args.envs, mb, 12), dtype=torch.float64, pin_memory=True)
        tg1 = host_tg1.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            tg1[:] = targets_for(None, deltas, args.warmup + i, com)
            genv.set_targets_all(tg1)
            genv.step(wait=False)
            genv.read_gel_surface_all(out_np)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_lock = {"value": args.envs * args.steps * world / dt, "unit": METRIC,
                    "h2d_bytes_per_step": int(tg1.nbytes), "d2h_bytes_per_step": int(out_np.nbytes)}

    rel_err = err_dist = plain64 = oracle_cmp = cpu = None
    if 0 in results:
        g64 = results[0]["genv"]
        snap64 = results[0]["snap"]
        if len(precisions) == 2:
            # one step of both paths from the same input states: every env at
            # the first timed step (the FP64 snapshot) and after the timed steps
            e_first, _ = per_step_error(g64, genv, dev_tg[args.warmup], 4e-3, states=snap64)
            for e in range(args.envs):   # the FP64 path's end of the timed region, as it was
                assert g64.set_state(e, *results[0]["end"][e]) == 0
            e_last, _ = per_step_error(g64, genv, dev_tg[n_total], 4e-3)
            err_dist = error_distribution([e_first, e_last])
            rel_err = err_dist["max"]
        # the metric's comparison: the plain per-environment FP64 GPU path
        if rank == 0 and not args.no_per_env:
            plain64 = per_env_fp64(scene, params, deltas, snap64, args.warmup, [0, 1], min(args.steps, 10), dev)
        # the FP64 oracle on the host cores: one step of `cores` envs from the
        # FP64 batch's state at the first timed step; the mixed path's step
        # from the same state is compared with it
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cores = max(1, min(os.cpu_count() or 1, 16))
            picks = list(range(cores))
            states = [(e, args.warmup) + tuple(snap64[e]) for e in picks]
            wall, res = oracle_steps_parallel(states, cores)
            cpu = {"value": cores / wall, "unit": METRIC, "cores": cores, "kind": "oracle",
                   "sample": f"{cores} envs x 1 step (step {args.warmup}, the first timed step, from the FP64 "
                             f"batch's state), one env per process on {cores} of {os.cpu_count()} host cores "
                             f"({cpu_model()}), FP64 oracle, BLAS threads = 1, {wall:.1f} s wall"}
            # the mixed path from the same inputs
            diag = float(np.linalg.norm(np.array([0.02, 0.02, 0.004])))
            for e in picks:
                assert genv.set_state(e, *snap64[e]) == 0
            genv.set_targets_all_device(dev_tg[args.warmup])
            st32, _ = genv.step(picks)
            errs = [state_diff(r["x"], r["y"], genv.get_state(e)[0], genv.get_state(e)[2], 4e-3) / diag
                    for e, r in zip(picks, res)]
            oracle_cmp = {"max": float(np.max(errs)), "median": float(np.median(errs)), "envs": len(picks),
                          "oracle_status_not_ok": int(sum(int(r["status"]) != 0 for r in res)),
                          "mixed_status_not_ok": int(np.sum(st32 != 0)),
                          "def": "one step from the FP64 batch's state at the first timed step: mixed path vs "
                                 "FP64 oracle (same solver parameters), max vertex difference / gel bbox diagonal"}
        g64.close()
    genv.close()

    if rank == 0:
        fp = results.get(0, head)
        lock = head["lock"]
        out = {"metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": head["ms_total"] / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if hp == 0 else "f32+f64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "envs": args.envs * world, "envs_per_gpu": args.envs,
                          "gel_vertices": 9600, "tets": 38025, "timed_steps": f"{args.warmup}-{n_total - 1}",
                          "precision": "fp64" if hp == 0 else
                          "mixed: FP32 element/contact Hessians + mat-vec; FP64 gradient, distances, CCD, energies, PCG residual",
                          "execution": "the timed steps as one rollout (ipc_rollout: one CUDA graph, device-side "
                                       "Newton / PCG / line-search loops, every env on its own step schedule); "
                                       "ms_per_step = rollout time / steps",
                          "cache": "inputs larger than L2 (~24 GB working set per GPU)", "parallelism": f"envs x{world}"},
               "latency_ms": None if lock is None else
                             {"p50": float(np.percentile(lock["step_ms"], 50)),
                              "p99": float(np.percentile(lock["step_ms"], 99)),
                              "def": "per batched step (lock-step ipc_step whole-step graphs, all envs), CUDA events"},
               "lockstep": None if lock is None else
                           {"value": lock["value"], "ms_per_step": lock["ms_total"] / args.steps,
                            "iterations": lock["tot"], "status_not_ok": lock["n_bad"],
                            "execution": "K batched ipc_step calls, whole step as one CUDA graph each"},
               "speedup_vs_lockstep": head["value"] / lock["value"] if lock else None,
               "fp64": None if 0 not in results else
                       {"value": fp["value"], "ms_per_step": fp["ms_total"] / args.steps,
                        "execution": "the same rollout in FP64", "iterations": fp["tot"],
                        "status_not_ok": fp["n_bad"]},
               "speedup_vs_fp64": head["value"] / fp["value"] if (0 in results and hp == 1) else None,
               "per_env_fp64": plain64,
               "speedup_vs_per_env_fp64": head["value"] / plain64["value"] if plain64 else None,
               "rel_err_vs_fp64": rel_err,
               "rel_err_def": "one step of both paths from the same input state, every env at the first timed "
                              "step and after the timed steps, max vertex difference / gel bbox diagonal",
               "rel_err_per_env": err_dist,
               "rel_err_vs_oracle": oracle_cmp,
               "status_not_ok": head["n_bad"],
               "iterations": head["tot"],
               "launch_shapes": head["tuning"],
               "roofline": roof, "kernels": kernels, "alu_rooflines": alu, "fma_peaks_tflops": fma,
               "clocks": head["clocks"], "gpu_launches": int(head["launches"]),
               "e2e": e2e, "e2e_lockstep": e2e_lock, "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args):
    """The serving stream: Poisson arrivals of config-2-style requests,
    loaded into the env slots of resident per-size-class pools as slots free
    up (memory-sized pools, one stream and host thread each), mixed
    precision, whole steps as CUDA graphs.  Compared with the same kind of
    requests stepped one by one in plain FP64 (a bounded sample)."""
    import torch

    import scenes
    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build
    from paper_2504_12908_b300.serving import GpuEngine, Request, Server, poisson_arrivals
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    build()
    n_req = int(args.rate * args.serve_seconds) + 1
    arr = poisson_arrivals(n_req, args.rate, 4000)

    def make(rid):
        def b():
            sc = scenes.config4_request(rid, n_steps=args.req_steps)
            return sc.scene, sc.delta
        return b
    reqs = [Request(rid=i, n_steps=args.req_steps, arrival=float(arr[i]), build=make(i)) for i in range(n_req)]
    prm = scenes.SolverParams()
    prm.precision = 1
    eng = GpuEngine(prm, device=f"cuda:{local}", graphs=not args.no_graphs)
    srv = Server(eng, max_resident=args.max_resident, slots_per_pool=args.slots_per_pool,
                 max_pools=args.max_pools, keep_state=False, chunk=1 if args.no_graphs else args.serve_chunk)
    clocks = ClockSampler(local)
    clocks.start()
    rep = srv.run(reqs, time_limit=args.serve_seconds, hard_limit=args.serve_hard)
    clk = clocks.stop()
    # plain FP64, one request at a time (bounded sample: 3 requests x 10 steps)
    p64 = scenes.SolverParams()
    one_ms = []
    for rid in range(3):
        sc = scenes.config4_request(rid, n_steps=args.req_steps)
        g = ipc.Envs([sc.scene], p64)
        for k in range(10):
            t = g.rest_y(0)
            t[:, :3] += sc.delta(k)[:, :3]
            g.set_targets(0, t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step()
            torch.cuda.synchronize()
            one_ms.append(1e3 * (time.perf_counter() - t0))
        g.close()
    one = 1e3 / float(np.mean(one_ms))
    summ = rep.summary()
    out = {"metric": "env-steps/s (serving stream)", "value": rep.env_steps_per_s, "unit": "env-steps/s",
           "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "serving: Poisson %.0f req/s of config-2-style envs x %d steps, window %.0f s"
                      % (args.rate, args.req_steps, args.serve_seconds),
                      "max_resident": args.max_resident, "slots_per_pool": args.slots_per_pool,
                      "max_pools": args.max_pools, "graphs": not args.no_graphs,
                      "steps_per_call": 1 if args.no_graphs else args.serve_chunk},
           "latency_ms": {"p50": rep.step_ms_p50, "p99": rep.step_ms_p99},
           "serving": {k: v for k, v in summ.items()},
           "fp64_one_by_one": {"value": one, "unit": "env-steps/s", "step_ms_mean": float(np.mean(one_ms)),
                               "sample": "3 requests x 10 steps, each alone in its own context, plain FP64"},
           "speedup_vs_fp64_one_by_one": rep.env_steps_per_s / one if one > 0 else None,
           "clocks": clk}
    print(json.dumps(out), flush=True)


def _mixed_vs_fp64(args, scs):
    """Step one batch of scenarios in mixed precision and in plain FP64 (the
    same scripted targets; K timed steps after W warm-up steps)."""
    import torch

    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build
    import scenes
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    build()
    n = len(scs)
    out = {}
    for prec in (0, 1):
        prm = scenes.SolverParams()
        prm.precision = prec
        g = ipc.Envs([sc.scene for sc in scs], prm, device=f"cuda:{local}", stream=torch.cuda.Stream())
        g.set_graph_mode(2)
        rest = [g.rest_y(e) for e in range(n)]
        mb = g.max_bodies

        def targets(k):
            t = np.zeros((n, mb, 12))
            for e, sc in enumerate(scs):
                r = rest[e].copy()
                r[:, :3] += sc.delta(k)[:, :3]
                t[e, :r.shape[0]] = r
            return t
        tg = [targets(k) for k in range(args.warmup + args.steps)]
        for k in range(args.warmup):
            g.set_targets_all(tg[k])
            g.step()
        if prec == 1 and not args.no_autotune:
            g.autotune()
        dev_tab = torch.as_tensor(np.stack(tg[args.warmup:args.warmup + args.steps]), dtype=torch.float64,
                                  device=f"cuda:{local}")
        g.rollout(0, dev_tab[:0])              # captures the rollout graph; no step
        snap = snapshot(g)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        bad, newton_max, pcg = 0, 0, 0
        ev0.record(g.stream)
        for k in range(args.warmup, args.warmup + args.steps):
            g.set_targets_all(tg[k])
            st, stt = g.step()
            bad += int(np.sum(st != 0))
            newton_max = max(newton_max, stt["newton_iters"])
            pcg += stt["pcg_iters"]
        ev1.record(g.stream)
        torch.cuda.synchronize()
        ms_lock = ev0.elapsed_time(ev1)
        restore(g, snap)
        ms_roll, tot_r, st_r, taken_r = time_rollout(g, dev_tab, 0, args.steps, g.stream)
        out[prec] = {"value": n * args.steps / (ms_roll / 1e3), "ms_per_step": ms_roll / args.steps,
                     "status_not_ok": int(np.sum(st_r != 0) + np.sum(taken_r != args.steps)),
                     "newton_max": tot_r["newton_max"], "pcg_iters": tot_r["pcg_iters"],
                     "execution": "the timed steps as one rollout (every env on its own step schedule)",
                     "lockstep": {"value": n * args.steps / (ms_lock / 1e3), "ms_per_step": ms_lock / args.steps,
                                  "status_not_ok": bad, "newton_max": newton_max, "pcg_iters": pcg,
                                  "execution": "K batched steps, whole step as one CUDA graph each"}}
        g.close()
        torch.cuda.empty_cache()
    return out


def _batch_line(args, out, metric, workload):
    return {"metric": metric, "value": out[1]["value"], "unit": "env-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out[1]["ms_per_step"],
            "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload, "cache": "inputs larger than L2"},
            "fp64": out[0], "mixed": out[1], "speedup_vs_fp64": out[1]["value"] / out[0]["value"]}


def run_grasp(args):
    """Config 3 at size: 1024 two-finger grasps (two 32x32x6 pads on driven
    ABD fingers closing at 10 mm/s on a free level-4 icosphere, r = 10 mm,
    under gravity), mixed precision vs plain FP64, whole-step graphs.  Per
    env the initial gap of config3(env) as a rigid shift of each finger with
    its pad.  Reports env-steps/s of both paths, the mixed-vs-FP64 one-step
    error over all envs, and e2e through host buffers."""
    import torch

    import scenes
    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    build()
    n = args.envs if args.envs != 256 else 1024
    scene, params, shifts, delta = scenes.config3_batch(n)
    pad = np.asarray(scene.gel_obj)
    n_total = args.warmup + args.steps
    out = {}
    keep = {}
    for prec in (0, 1):
        prm = scenes.SolverParams(**params.__dict__)
        prm.precision = prec
        stream = torch.cuda.Stream()
        g = ipc.Envs([scene] * n, prm, device=f"cuda:{local}", stream=stream)
        g.set_graph_mode(2)
        rest_y = g.rest_y(0)
        x0, v0, y0, yd0 = g.get_state(0)
        tg = np.zeros((n_total + 1, n, g.max_bodies, 12))
        for e, (s0, s1) in enumerate(shifts):
            x = x0.copy()
            x[pad == 0, 0] += s0
            x[pad == 1, 0] += s1
            y = y0.copy()
            y[0, 0] += s0
            y[1, 0] += s1
            assert g.set_state(e, x, None, y, None) == 0
            for k in range(n_total + 1):
                t = rest_y.copy()
                t[:, :3] += delta(k)[:, :3]
                t[0, 0] += s0
                t[1, 0] += s1
                tg[k, e] = t
        dev_tg = torch.as_tensor(tg, dtype=torch.float64, device=f"cuda:{local}")
        for k in range(args.warmup):
            g.set_targets_all_device(dev_tg[k])
            g.step()
        if not args.no_autotune:
            g.autotune()
        g.rollout(0, dev_tg[:0])                 # captures the rollout graph; no step
        snap = snapshot(g)
        ms, step_ms, tot, statuses = time_steps(g, dev_tg, args.warmup, args.steps, stream)
        restore(g, snap)
        ms_r, tot_r, st_r, taken_r = time_rollout(g, dev_tg, args.warmup, args.steps, stream)
        out[prec] = {"value": n * args.steps / (ms_r / 1e3), "ms_per_step": ms_r / args.steps,
                     "status_not_ok": int(np.sum(st_r != 0) + np.sum(taken_r != args.steps)),
                     "newton_max": tot_r["newton_max"], "pcg_iters": tot_r["pcg_iters"],
                     "execution": "the timed steps as one rollout (every env on its own step schedule)",
                     "lockstep": {"value": n * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                                  "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                                                 "p99": float(np.percentile(step_ms, 99))},
                                  "status_not_ok": int(sum(int(np.sum(s_ != 0)) for s_ in statuses)),
                                  "newton_max": tot["newton_max"], "pcg_iters": tot["pcg_iters"]}}
        if prec == 0:
            keep["x64"] = [g.get_state(e) for e in range(n)]
            g.close()
            torch.cuda.empty_cache()
        else:
            keep["g"], keep["snap"], keep["dev_tg"], keep["tg"] = g, snap, dev_tg, tg
    g = keep["g"]
    # one step of the mixed path from each FP64 end state vs the FP64 path's
    # next step is not available here (its context is closed): the error is
    # measured against a fresh FP64 context on a sample of envs
    diag = float(np.linalg.norm(np.array([0.04, 0.02, 0.02])))
    sample = list(range(0, n, max(1, n // 16)))
    prm64 = scenes.SolverParams(**params.__dict__)
    g64 = ipc.Envs([scene] * len(sample), prm64, device=f"cuda:{local}")
    errs = []
    for i, e in enumerate(sample):
        assert g64.set_state(i, *keep["x64"][e]) == 0
        assert g.set_state(e, *keep["x64"][e]) == 0
    g64.set_targets_all(keep["tg"][n_total][sample])
    g64.step()
    g.set_targets_all_device(keep["dev_tg"][n_total])
    g.step(sample)
    for i, e in enumerate(sample):
        a, b = g64.get_state(i), g.get_state(e)
        errs.append(state_diff(a[0], a[2], b[0], b[2], 10e-3) / diag)
    g64.close()
    # e2e on the mixed path: the timed steps again from the snapshot, pinned
    # host targets in and coated surfaces out every step
    restore(g, keep["snap"])
    host_tg = torch.empty((n, g.max_bodies, 12), dtype=torch.float64, pin_memory=True)
    host_out = torch.empty((sum(s_[2] for s_ in g.sizes), 3), dtype=torch.float64, pin_memory=True)
    tg_np, out_np = host_tg.numpy(), host_out.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        tg_np[:] = keep["tg"][args.warmup + i]
        g.set_targets_all(tg_np)
        g.step(wait=False)
        g.read_gel_surface_all(out_np)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    g.close()
    line = {"metric": "env-steps/s (two-finger grasp batch)", "value": out[1]["value"], "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out[1]["ms_per_step"],
            "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"two-finger grasp: {n} envs x (2 gel pads 32x32x6 on driven ABD fingers + "
                                   f"free ABD icosphere L4, r = 10 mm)", "timed_steps": f"{args.warmup}-{n_total - 1}",
                       "execution": "the timed steps as one rollout (one CUDA graph, every env on its own step "
                                    "schedule); lock-step whole-step graphs beside it", "cache": "inputs larger than L2"},
            "fp64": out[0], "mixed": out[1], "speedup_vs_fp64": out[1]["value"] / out[0]["value"],
            "rel_err_vs_fp64": {"max": float(np.max(errs)), "median": float(np.median(errs)), "envs": len(sample),
                                "def": "one step from the FP64 end state, mixed vs FP64, max vertex difference / "
                                       "scene bbox diagonal (40 x 20 x 20 mm)"},
            "e2e": {"value": n * args.steps / dt, "unit": METRIC, "h2d_bytes_per_step": int(tg_np.nbytes),
                    "d2h_bytes_per_step": int(out_np.nbytes)}}
    print(json.dumps(line), flush=True)


def run_single(args):
    """Config 0: one env (9x9x3 gel, 8 mm ABD cube driven down at 5 mm/s),
    FP64, 20 steps from rest, plain launches and whole-step graphs."""
    import torch

    import scenes
    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build
    build()
    sc = scenes.config0()
    res = {}
    for mode in (0, 2):
        g = ipc.Envs([sc.scene], sc.params, stream=torch.cuda.Stream())
        g.set_graph_mode(mode)
        rest = g.rest_y(0)
        ms, bad = [], 0
        for k in range(sc.n_steps):
            t = rest.copy()
            t[:, :3] += sc.delta(k)[:, :3]
            g.set_targets(0, t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, _ = g.step()
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            bad += int(st[0] != 0)
        g.close()
        res[mode] = {"value": len(ms) / (sum(ms) / 1e3), "ms_per_step": float(np.mean(ms)),
                     "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
                     "status_not_ok": bad}
    line = {"metric": "env-steps/s (single env)", "value": res[2]["value"], "unit": METRIC, "n_gpus": 1,
            "steps": sc.n_steps, "warmup": 0, "ms_per_step": res[2]["ms_per_step"], "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single env: gel 9x9x3 + 8 mm ABD cube driven down at 5 mm/s, 20 steps from rest",
                       "cache": "working set within L2"},
            "graph_step": res[2], "plain_launches": res[0]}
    print(json.dumps(line), flush=True)


def run_broadphase(args):
    """Candidate-search time against surface size: one gel pad of n x n x 3
    vertices with self-contact on (every pair of its own non-adjacent
    primitives is a candidate query), n = 10, 20, 40, 80, and the level-4
    icosphere of the grasp against a 32 x 32 x 6 pad; static and swept
    searches from a perturbed state, per-call time from CUDA events.  The
    brute-force search this replaces is quadratic in the pad's primitives."""
    import torch

    import scenes
    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build
    build()
    rows = []
    cases = [("pad %dx%dx3, self-contact" % (n, n), scenes.self_contact_pad(n)) for n in (10, 20, 40, 80)]
    cases.append(("pad 32x32x6 + icosphere L4 (r = 10 mm)", scenes.pad_and_sphere(32, 6, 4)))
    for name, sc in cases:
        g = ipc.Envs([sc], scenes.SolverParams())
        n_cv = sc.gel_x.shape[0] + sum(b.rest_x.shape[0] for b in sc.bodies)
        rng = np.random.default_rng(7)
        X = np.concatenate([sc.gel_x] + [b.rest_x for b in sc.bodies])
        X = X + rng.normal(scale=2e-6, size=X.shape)
        Xe = X + rng.normal(scale=1e-5, size=X.shape)
        g.debug_pairs(0, X, Xe)
        g.profile_enable(True)
        g.profile_reset()
        reps = 10
        n_pairs = 0
        for _ in range(reps):
            n_pairs = len(g.debug_pairs(0, X, None))
            g.debug_pairs(0, X, Xe)
        prof = g.profile()
        g.close()
        ms = prof["broad_phase"][1] / (2 * reps)
        rows.append({"case": name, "contact_vertices": int(n_cv), "ms_per_search": round(ms, 4),
                     "static_candidates": int(n_pairs), "us_per_vertex": round(1e3 * ms / n_cv, 4)})
    print(json.dumps({"metric": "broad-phase ms per candidate search", "unit": "ms", "data": "synthetic",
                      "rows": rows}), flush=True)


def run_uneven(args):
    """512 config-2 envs of different sizes stepped together: mixed vs plain
    FP64 on the same batch (press phase steps after the warm-up)."""
    import scenes
    out = _mixed_vs_fp64(args, [scenes.config2(e) for e in range(512)])
    print(json.dumps(_batch_line(args, out, "env-steps/s (uneven batch)",
                                 "uneven batch: 512 config-2 envs (gel {16,24,32,48}^2 x {4,6}, icosphere L1-3)")),
          flush=True)


def run_self_contact(args):
    """Gel self-contact batch: 1024 envs of one pad made of two blocks that a
    driven cube presses together (seeded press depth per env), mixed vs
    plain FP64."""
    import scenes
    scs = [scenes.self_contact_scene(depth=float(np.random.default_rng(6000 + e).uniform(5e-5, 1.5e-4)))
           for e in range(1024)]
    out = _mixed_vs_fp64(args, scs)
    line = _batch_line(args, out, "env-steps/s (self-contact batch)",
                       "self-contact batch: 1024 envs x (two-block pad, 82 gel vertices, 125 tets, "
                       "self-contact on) + driven 3 mm cube")
    line["config"]["cache"] = "working set within L2 (small envs)"
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "self_contact":
        run_self_contact(args)
    elif args.workload == "grasp":
        run_grasp(args)
    elif args.workload == "single":
        run_single(args)
    elif args.workload == "broadphase":
        run_broadphase(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
