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
WORKLOAD = "uniform batch: 256 envs x (gel 40x40x6 + ABD icosphere L2, press/slide), FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=256)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


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
def oracle_sample_seconds(scene, params, delta, step_index=0):
    """Wall time of the FP64 oracle advancing one env by one step, BLAS at 1 thread."""
    from threadpoolctl import threadpool_limits

    from oracle import OracleEnv
    from oracle import distance as ods
    for k in ("PP", "PE", "PT", "EE", "X"):
        ods._sym(k)   # symbolic set-up outside the timed sample
    with threadpool_limits(1):
        env = OracleEnv(scene, params)
        x, v, y, yd = env.rest_state()
        t0 = time.perf_counter()
        x, v, y, yd, st = env.step(x, v, y, yd, env.targets_from_delta(delta(step_index)))
        dt = time.perf_counter() - t0
    return dt, st


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    scene, params, deltas = build_workload(args.envs, 0)
    times = []
    for k in range(args.warmup + args.steps):
        dt, st = oracle_sample_seconds(scene, params, deltas[k % len(deltas)], 0)
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
    """Algorithmic bytes of the main kernel classes over the timed region."""
    sz = genv.system_sizes(0)
    nv, nb, _ = genv.sizes[0]
    rows_real = nv + 4 * nb
    n_envs = genv.n_envs
    T = sz["tets"]
    out = {}
    # SELL SpMV: 72 B values + 4 B column per real block; per row d, qc read,
    # q, qc written (24 B each)
    spmv_env_iter = sz["real_blocks"] * 76 + rows_real * 96
    out["sell_spmv"] = stats_tot["pcg_iters"] * spmv_env_iter
    # PCG update: reads p, d, r, q, P^-1 (72), writes p, r, z
    out["pcg_update"] = stats_tot["pcg_iters"] * rows_real * (4 * 24 + 72 + 3 * 24)
    out["pcg_dir"] = stats_tot["pcg_iters"] * rows_real * 72
    # elastic element kernel: x of 4 vertices, Dm^-1, vol, indices; writes
    # 12 gradient + 144 Hessian doubles
    out["tet_elastic"] = stats_tot["newton_env_iters"] * T * (16 + 96 + 72 + 8 + 96 + 1152)
    # assembly: reads the 16 element blocks of every tet once, writes every
    # real block once (72 B) and reads its column (4 B)
    out["assemble"] = stats_tot["newton_env_iters"] * (T * 16 * 72 + sz["real_blocks"] * 76)
    return out, spmv_env_iter


def run_ours(args):
    import torch

    from paper_2504_12908_b300 import ipc
    from paper_2504_12908_b300.build import build

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build()
    scene, params, deltas = build_workload(args.envs, args.precision)
    genv = ipc.Envs([scene] * args.envs, params, device=f"cuda:{local}")
    com = genv.body_com(0, 0)
    n_steps_total = args.warmup + args.steps
    dev_tg = torch.as_tensor(np.stack([targets_for(None, deltas, k, com) for k in range(n_steps_total + args.steps)]),
                             dtype=torch.float64, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()

    def one_step(k):
        genv.set_targets_all_device(dev_tg[k])
        return genv.step()

    # warm-up
    for k in range(args.warmup):
        st, _ = one_step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    genv.profile_enable(True)
    genv.profile_reset()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = genv.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tot = {"pcg_iters": 0, "newton_env_iters": 0, "ls_trials": 0, "newton_max": 0, "max_pairs": 0}
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
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = genv.launch_count() - launches0
    ms_total = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([ms_total], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    prof = genv.profile()
    genv.profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ok = all(np.all(s == 0) for s in statuses)
    value = args.envs * args.steps * world / (ms_total / 1e3)

    # roofline of the dominant kernel class
    kb, spmv_env_iter = kernel_bytes(genv, tot, prof)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peak, peak_kind = measured_peaks()
    kernels = {}
    for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        if n == 0:
            continue
        row = {"launches": n, "ms": round(ms, 3), "share": round(ms / max(sum(v[1] for v in prof.values()), 1e-9), 4)}
        if name in kb and ms > 0:
            row["GB/s"] = round(kb[name] / (ms / 1e3) / 1e9, 1)
        kernels[name] = row
    if dom in kb:
        n, ms = prof[dom]
        achieved = kb[dom] / (ms / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind,
                "bytes_per_launch": kb[dom] / max(n, 1)}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}

    # e2e: host targets in pinned memory, one H2D + step + one D2H per step
    e2e = None
    if not args.no_e2e:
        mb = genv.max_bodies
        host_tg = torch.empty((args.envs, mb, 12), dtype=torch.float64, pin_memory=True)
        n_out = sum(s[2] for s in genv.sizes)
        host_out = torch.empty((n_out, 3), dtype=torch.float64, pin_memory=True)
        tg_np, out_np = host_tg.numpy(), host_out.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            k = n_steps_total + i
            tg_np[:] = targets_for(None, deltas, k, com)
            genv.set_targets_all(tg_np)
            genv.step()
            genv.read_gel_surface_all(out_np)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": args.envs * args.steps * world / dt, "unit": METRIC,
               "h2d_bytes_per_step": int(tg_np.nbytes), "d2h_bytes_per_step": int(out_np.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, st = oracle_sample_seconds(scene, params, deltas[0], 0)
        cpu = {"value": 1.0 / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"1 env x 1 step (step 0) of the same workload, FP64 oracle, {dt:.1f} s, BLAS threads = 1"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f32+f64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "envs": args.envs * world, "envs_per_gpu": args.envs,
                          "gel_vertices": 9600, "tets": 38025, "precision": "fp64" if args.precision == 0 else "mixed",
                          "cache": "inputs larger than L2 (~24 GB working set per GPU)", "parallelism": f"envs x{world}"},
               "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
               "all_status_ok": bool(ok),
               "iterations": {"newton_env_iters": tot["newton_env_iters"], "pcg_env_iters": tot["pcg_iters"],
                              "newton_max": tot["newton_max"], "ls_trials": tot["ls_trials"],
                              "max_pairs": tot["max_pairs"]},
               "roofline": roof, "kernels": kernels, "clocks": clk, "gpu_launches": int(launches),
               "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    genv.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
