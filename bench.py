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
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=256)
    ap.add_argument("--precision", type=int, default=1,
                    help="1: time FP64 then mixed (headline); 0: FP64 only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only-mixed", action="store_true",
                    help="time only the mixed path (profiling runs); no FP64 comparison")
    ap.add_argument("--workload", default="batch", choices=["batch", "serving", "uneven", "self_contact"],
                    help="batch: the uniform 256-env batch (default); serving: the Poisson request stream; "
                         "uneven: 512 config-2 envs of different sizes in one launch; "
                         "self_contact: 1024 two-block pads pressed together (gel self-contact)")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serving: admission window (s)")
    ap.add_argument("--serve-hard", type=float, default=60.0, help="serving: stop stepping at this time (s)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--req-steps", type=int, default=200, help="serving: steps per request")
    ap.add_argument("--max-resident", type=int, default=4096)
    ap.add_argument("--max-cohort", type=int, default=256)
    ap.add_argument("--max-cohorts", type=int, default=8)
    ap.add_argument("--no-graphs", action="store_true", help="serving: plain launches instead of PCG graphs")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
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
def build_workload(n_envs, precision):
    import scenes
    scene, params, deltas = scenes.config1_batch(n_envs)
    params.precision = precision
    return scene, params, deltas


def targets_for(envs, deltas, step, com):
    """[n_envs][1][12] rest placement of the icosphere translated by its script."""
    t = np.zeros((len(deltas), 1, 12))
    for e, dl in enumerate(deltas):
        t[e, 0, :3] = com + dl(step)[0]
        t[e, 0, 3:] = np.eye(3).T.ravel()
    return t


# ------------------------------------------------------------------ CPU oracle sample
_ORACLE_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import scenes
from oracle import OracleEnv
from oracle import distance as ods
for k in ("PP", "PE", "PT", "EE", "X"):
    ods._sym(k)          # symbolic set-up outside the timed sample
scene, params, deltas = scenes.config1_batch({env} + 1)
env = OracleEnv(scene, params)
x, v, y, yd = env.rest_state()
t0 = time.perf_counter()
x, v, y, yd, st = env.step(x, v, y, yd, env.targets_from_delta(deltas[{env}]({step})))
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "status": st.status, "newton": st.newton_iters}}))
"""


def oracle_sample_seconds(env_index=0, step_index=0):
    """Wall time of the FP64 oracle advancing one env of the workload by one
    step, in a child process with every BLAS/OpenMP pool at one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    code = _ORACLE_SAMPLE.format(root=ROOT, env=env_index, step=step_index)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["seconds"], d


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    times = []
    for k in range(args.warmup + args.steps):
        dt, st = oracle_sample_seconds(k % args.envs, 0)
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = 1.0 / float(np.mean(times))
    sample = "1 env x 1 time step (step 0 of env k's script) per bench step, oracle FP64, BLAS threads = 1"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "envs_per_step": 1, "cache": "inputs larger than L2 (per env ~95 MB)"},
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ ours
def kernel_bytes(genv, stats_tot, prof):
    """Algorithmic bytes of the main kernel classes over the timed region
    (what each kernel must move at minimum for the work it did)."""
    sz = genv.system_sizes(0)
    nv, nb, _ = genv.sizes[0]
    rows_real = nv + 4 * nb
    T = sz["tets"]
    hs = 4 if getattr(genv.params, "precision", 0) else 8   # Hessian / matrix value bytes
    out = {}
    # SELL SpMV per env-iteration: 9 values + 4 B column per real block; per
    # row the own direction read, q written (16 B FP32 rows in mixed mode,
    # 24 B FP64 rows otherwise), the FP64 contact part qc read and cleared
    vb = 16 if hs == 4 else 24
    spmv_env_iter = sz["real_blocks"] * (9 * hs + 4) + rows_real * (2 * vb + 48)
    out["sell_spmv"] = stats_tot["pcg_iters"] * spmv_env_iter
    # PCG update: p (FP64) read + written, d and q read, r (FP64) read +
    # written, the 6-entry symmetric P^-1 block, z written
    out["pcg_update"] = stats_tot["pcg_iters"] * rows_real * (48 + 2 * vb + 48 + 6 * hs + vb)
    # PCG direction: z and d read, d written
    out["pcg_dir"] = stats_tot["pcg_iters"] * rows_real * 3 * vb
    # elastic element kernel: 4 indices + 4 positions + Dm^-1 + vol read,
    # 12 FP64 gradient and 144 Hessian values written
    out["tet_elastic"] = stats_tot["newton_env_iters"] * T * (16 + 96 + 72 + 8 + 96 + 144 * hs)
    # assembly: every element block read once, every real block written once
    out["assemble"] = stats_tot["newton_env_iters"] * (T * 144 * hs + sz["real_blocks"] * (9 * hs + 4))
    return out, spmv_env_iter


def time_precision(args, scene, params, deltas, precision, local, world, profile=True):
    """Warm-up + timed region for one precision mode; returns a result dict
    and leaves the Envs open (caller closes)."""
    import torch

    from paper_2504_12908_b300 import ipc
    prm = type(params)(**params.__dict__)
    prm.precision = precision
    genv = ipc.Envs([scene] * args.envs, prm, device=f"cuda:{local}")
    com = genv.body_com(0, 0)
    n_total = args.warmup + args.steps
    dev_tg = torch.as_tensor(np.stack([targets_for(None, deltas, k, com) for k in range(n_total + args.steps)]),
                             dtype=torch.float64, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()

    def one_step(k):
        genv.set_targets_all_device(dev_tg[k])
        return genv.step()

    for k in range(args.warmup):
        one_step(k)
    tuning = genv.autotune() if not args.no_autotune else None
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if profile:
        genv.profile_enable(True)
        genv.profile_reset()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = genv.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tot = {"pcg_iters": 0, "newton_env_iters": 0, "ls_trials": 0, "newton_max": 0, "max_pairs": 0,
           "al_env_updates": 0, "ccd_limited": 0, "alpha_sum": 0.0, "accd_iters": 0, "accd_iters_max": 0}
    statuses = []
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        st, s = one_step(args.warmup + i)
        ev[i][1].record(stream)
        statuses.append(st)
        tot["pcg_iters"] += s["pcg_iters"]
        tot["newton_env_iters"] += s["newton_env_iters"]
        tot["ls_trials"] += s["ls_trials"]
        tot["newton_max"] = max(tot["newton_max"], s["newton_iters"])
        tot["max_pairs"] = max(tot["max_pairs"], s["max_pairs"])
        tot["al_env_updates"] += s["al_env_updates"]
        tot["ccd_limited"] += s["ccd_limited"]
        tot["alpha_sum"] += s["alpha_sum"]
        tot["accd_iters"] += s["accd_iters"]
        tot["accd_iters_max"] = max(tot["accd_iters_max"], s["accd_iters_max"])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = genv.launch_count() - launches0
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), world, f"cuda:{local}")
    prof = genv.profile() if profile else {}
    genv.profile_enable(False)
    step_ms = [a_.elapsed_time(b_) for a_, b_ in ev]
    n_bad = int(sum(int(np.sum(s_ != 0)) for s_ in statuses))
    return {"genv": genv, "value": whole_job_rate(args.envs, args.steps, world, ms_total), "ms_total": ms_total,
            "step_ms": step_ms, "tot": tot, "prof": prof, "clocks": clk, "launches": launches, "n_bad": n_bad,
            "statuses": statuses, "deltas": deltas, "com": com, "n_total": n_total, "dev_tg": dev_tg,
            "tuning": tuning}


def per_step_error(g64, g32, tg, body_radius):
    """Spec'd error of the mixed form: one step of both paths from the same
    input state (the FP64 path's current state, every env), largest vertex
    difference over all gel vertices and body vertices, relative to the
    gel box diagonal.  Body vertices are bounded through the 12 DoF:
    |dp| + R * sum_j |dA_ij| for points within radius R of the frame."""
    n = len(g64.sizes)
    for e in range(n):
        st = g64.get_state(e)
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
        d = float(np.abs(x64 - x32).max())
        dy = np.abs(np.asarray(y64) - np.asarray(y32)).reshape(-1, 4, 3)   # [p, a0, a1, a2] per body
        if dy.size:
            d = max(d, float((dy[:, 0, :] + body_radius * dy[:, 1:, :].sum(axis=1)).max()))
        errs[e] = d / diag
    dist = {"max": float(errs.max()), "p99": float(np.percentile(errs, 99)), "median": float(np.median(errs)),
            "envs_above_1e-4": int(np.sum(errs > 1e-4)), "envs": n}
    return float(errs.max()), dist, int(np.sum(s64 != 0) + np.sum(s32 != 0))


# DRAM traffic of one SpMV launch with every env of the 256-env workload
# active: dram__bytes_read.sum + dram__bytes_write.sum of the first k_spmv
# launch of `bench.py --only-mixed --steps 1 --warmup 1` under ncu.  Reported only while
# the kernel's source is the one that was measured (hash of its text).
# (measured with 4 slots in flight per lane)
SPMV_TRAFFIC = {"envs": 256, "bytes": 1275934208 + 90306816,
                "source_sha256": "830203d985315711f5332876ced428e43c65ae8bc3a3b875c54921744617e589"}


def _spmv_source_hash() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2504_12908_b300", "csrc")
    src = open(os.path.join(csrc, "kernels_solver.cu")).read()
    c = src.index("__global__ void __launch_bounds__(128) k_spmv(Dev d")
    d = src.index("\n}\n", c)
    vec = open(os.path.join(csrc, "pcgvec.cuh")).read()
    return hashlib.sha256((vec + src[c:d]).encode()).hexdigest()


def spmv_traffic_per_launch(stats_tot, launches):
    """Measured DRAM bytes scaled to the average launch of the timed region
    (envs active per launch = env-iterations / launches), or None."""
    if SPMV_TRAFFIC["bytes"] is None or _spmv_source_hash() != SPMV_TRAFFIC["source_sha256"]:
        return None
    active = stats_tot["pcg_iters"] / max(launches, 1)
    return SPMV_TRAFFIC["bytes"] / SPMV_TRAFFIC["envs"] * active


def roofline_of(genv, res):
    kb, _ = kernel_bytes(genv, res["tot"], res["prof"])
    prof = res["prof"]
    peak, peak_kind = measured_peaks()
    tot_ms = max(sum(v[1] for v in prof.values()), 1e-9)
    kernels = {}
    for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        if n == 0:
            continue
        row = {"launches": n, "ms": round(ms, 3), "share": round(ms / tot_ms, 4)}
        if name in kb and ms > 0:
            row["GB/s"] = round(kb[name] / (ms / 1e3) / 1e9, 1)
        kernels[name] = row
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    # the roofline is reported for the dominant kernel with an HBM bound
    hbm = [k for k in kernels if k in kb]
    rk = dom if dom in kb else (hbm[0] if hbm else None)
    roof = {"kernel": rk, "dominant_kernel": dom}
    if rk is not None:
        n, ms = prof[rk]
        achieved = kb[rk] / (ms / 1e3) / 1e9
        tuned_u = (res.get("tuning") or {}).get("spmv_unroll", 4)
        traffic = spmv_traffic_per_launch(res["tot"], n) if (rk == "sell_spmv" and tuned_u == 4) else None
        roof.update({"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                     "bytes_per_launch": kb[rk] / max(n, 1), "share_of_step": kernels[rk]["share"]})
    return roof, kernels


def run_ours(args):
    import torch

    from paper_2504_12908_b300.build import build

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build()
    scene, params, deltas = build_workload(args.envs, 0)

    # plain FP64 path (the comparison), then the mixed-precision path (headline)
    precisions = [0] if args.precision == 0 else ([1] if args.only_mixed else [0, 1])
    results = {}
    surf = {}
    for prec in precisions:
        res = time_precision(args, scene, params, deltas, prec, local, world)
        surf[prec] = res["genv"].read_gel_surface_all()
        results[prec] = res
    head = results[precisions[-1]]
    genv = head["genv"]
    roof, kernels = roofline_of(genv, head)
    rel_err = traj_err = err_dist = None
    if len(precisions) == 2:
        diag = float(np.linalg.norm(np.array([0.02, 0.02, 0.004])))
        # trajectories after warm-up + timed steps (divergence accumulates)
        traj_err = float(np.abs(surf[1] - surf[0]).max() / diag)
        # the per-step error from the same input state, checked after timing
        rel_err, err_dist, n_bad_err = per_step_error(results[0]["genv"], genv, head["dev_tg"][head["n_total"]], 4e-3)
        results[0]["genv"].close()
        torch.cuda.empty_cache()
        # the e2e leg continues from a state the error check has moved on
        head["n_total"] += 1

    # e2e on the headline path: pinned host targets in, coated surfaces out
    e2e = None
    if not args.no_e2e:
        mb = genv.max_bodies
        host_tg = torch.empty((args.envs, mb, 12), dtype=torch.float64, pin_memory=True)
        n_out = sum(s_[2] for s_ in genv.sizes)
        host_out = torch.empty((n_out, 3), dtype=torch.float64, pin_memory=True)
        tg_np, out_np = host_tg.numpy(), host_out.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            k = head["n_total"] + i
            tg_np[:] = targets_for(None, deltas, k, head["com"])
            genv.set_targets_all(tg_np)
            genv.step()
            genv.read_gel_surface_all(out_np)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": args.envs * args.steps * world / dt, "unit": METRIC,
               "h2d_bytes_per_step": int(tg_np.nbytes), "d2h_bytes_per_step": int(out_np.nbytes)}
    genv.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, st = oracle_sample_seconds(0, 0)
        cpu = {"value": 1.0 / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"1 env x 1 step (step 0) of the same workload, FP64 oracle, {dt:.1f} s, BLAS threads = 1"}

    if rank == 0:
        hp = precisions[-1]
        fp = results.get(0, head)
        out = {"metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": head["ms_total"] / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if hp == 0 else "f32+f64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "envs": args.envs * world, "envs_per_gpu": args.envs,
                          "gel_vertices": 9600, "tets": 38025,
                          "precision": "fp64" if hp == 0 else
                          "mixed: FP32 element/contact Hessians + mat-vec; FP64 gradient, distances, CCD, energies, PCG residual",
                          "cache": "inputs larger than L2 (~24 GB working set per GPU)", "parallelism": f"envs x{world}"},
               "latency_ms": {"p50": float(np.percentile(head["step_ms"], 50)),
                              "p99": float(np.percentile(head["step_ms"], 99))},
               "fp64": None if 0 not in results else
                       {"value": fp["value"], "ms_per_step": fp["ms_total"] / args.steps,
                        "latency_ms": {"p50": float(np.percentile(fp["step_ms"], 50)),
                                       "p99": float(np.percentile(fp["step_ms"], 99))},
                        "iterations": fp["tot"], "status_not_ok": fp["n_bad"]},
               "speedup_vs_fp64": head["value"] / fp["value"] if (0 in results and hp == 1) else None,
               "rel_err_vs_fp64": rel_err,
               "rel_err_def": "one step of both paths from the same input state (every env), max vertex "
                              "difference / gel bbox diagonal",
               "rel_err_per_env": err_dist,
               "traj_err_vs_fp64": traj_err,
               "status_not_ok": head["n_bad"],
               "iterations": head["tot"],
               "launch_shapes": head["tuning"],
               "roofline": roof, "kernels": kernels, "clocks": head["clocks"], "gpu_launches": int(head["launches"]),
               "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args):
    """The serving stream: Poisson arrivals of config-2-style requests,
    admitted into cohorts by free device memory, mixed precision, PCG inner
    loop as captured CUDA graphs.  Compared with the same kind of requests
    stepped one by one in plain FP64 (a bounded sample)."""
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
    srv = Server(eng, max_resident=args.max_resident, max_cohort=args.max_cohort,
                 max_cohorts=args.max_cohorts, keep_state=False)
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
                      "max_resident": args.max_resident, "max_cohort": args.max_cohort,
                      "max_cohorts": args.max_cohorts, "graphs": not args.no_graphs},
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
        g = ipc.Envs([sc.scene for sc in scs], prm, device=f"cuda:{local}")
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
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        bad = 0
        ev0.record()
        for k in range(args.warmup, args.warmup + args.steps):
            g.set_targets_all(tg[k])
            st, _ = g.step()
            bad += int(np.sum(st != 0))
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        out[prec] = {"value": n * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps, "status_not_ok": bad}
        g.close()
        torch.cuda.empty_cache()
    return out


def _batch_line(args, out, metric, workload):
    return {"metric": metric, "value": out[1]["value"], "unit": "env-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out[1]["ms_per_step"],
            "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload, "cache": "inputs larger than L2"},
            "fp64": out[0], "mixed": out[1], "speedup_vs_fp64": out[1]["value"] / out[0]["value"]}


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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
