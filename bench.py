#!/usr/bin/env python
"""Stein ICP registration throughput on GB300.

One step = one full pass of the hot path over one problem: build the voxel
grid of the reference cloud (sicp_set_reference) and run the Stein ICP loop
(sicp_register: minibatch selection, T iterations of transform + grid nearest
neighbour + per-particle gradient + Stein/Adam update, FP64 moments).  The
default workload is the Kinect-scale scene: 50,000-point reference from a
640x480 depth render, 10,000-point source from an offset view, 100 particles,
minibatch 300, 150 iterations, exact grid search.

Metric: particle.point NN+gradient evaluations per second (K*m*T per step,
summed over ranks); SVGD iterations per second are reported beside it.

Under torchrun each rank registers its own problem (a different seed) on its
own GPU: the problems are independent, so there is no data-path collective
(weak scaling); only the timing maximum is reduced across ranks.

`--impl reference` times the FP64 CPU oracle (the method stated plainly in
double precision) on the same workload, on a bounded number of iterations
per step, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kinect", choices=["kinect", "box", "lidar", "batched"])
    ap.add_argument("--profile-stride", type=int, default=5,
                    help="time the gradient and Stein kernels of every s-th iteration with CUDA events")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_problem(workload: str, seed: int):
    from paper_2106_03287_gb300 import synth
    if workload == "batched":
        return synth.make_batched_problems(seed), dict(synth.WORKLOADS["batched"])
    if workload == "kinect":
        d = synth.make_kinect_problem(seed)
    elif workload == "box":
        d = synth.make_box_problem(seed)
    else:
        d = synth.make_lidar_problem(seed)
    return d, dict(synth.WORKLOADS[workload])


def workload_config(workload, d, cfg, nn_mode_name):
    return {"workload": workload, "reference_points": int(d["ref"].shape[0]),
            "source_points": int(d["src"].shape[0]), "particles": int(d["particles"].shape[0]),
            "minibatch": cfg["m"], "iterations": cfg["T"], "adam_lr": cfg["lr"], "nn": nn_mode_name}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def grad_kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_grid.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2106_03287_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_query():
    """DRAM bytes per query of the gradient kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "k_grad_grid_kinect.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("source_hash") != grad_kernel_source_hash():
        return None
    return rec["dram_bytes"] / rec["queries"]


def cpu_baseline(d, cfg, budget_s=15.0):
    """The oracle as it stands, on a bounded number of iterations of the same workload."""
    import oracle as O
    ref, src = d["ref"], d["src"]
    th = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    p = O.Params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0)
    K = th.shape[0]
    t0 = time.perf_counter()
    O.step(ref, src, th, mom, vel, p, 0)
    first = time.perf_counter() - t0
    n = max(1, min(cfg["T"] - 1, int(budget_s / max(first, 1e-6))))
    t0 = time.perf_counter()
    for t in range(1, 1 + n):
        O.step(ref, src, th, mom, vel, p, t)
    dt = time.perf_counter() - t0
    return {"value": K * cfg["m"] * n / dt, "unit": "particle_point_evals/s", "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"{n} SVGD iterations (iterations 1..{n}) of the same workload, exhaustive FP64 search, "
                      f"{dt:.1f} s", "iters_per_sec": n / dt}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    d, cfg = make_problem(args.workload, 1000)
    import oracle as O
    ref, src = d["ref"], d["src"]
    K = d["particles"].shape[0]
    p = O.Params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0)
    th = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    t0 = time.perf_counter()
    O.step(ref, src, th, mom, vel, p, 0)
    first = time.perf_counter() - t0
    per_step = max(1, min(cfg["T"], int(150.0 / max(args.steps + args.warmup, 1) / max(first, 1e-6))))
    t = 1
    for _ in range(args.warmup):
        for _ in range(per_step):
            O.step(ref, src, th, mom, vel, p, t % cfg["T"])
            t += 1
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            O.step(ref, src, th, mom, vel, p, t % cfg["T"])
            t += 1
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = K * cfg["m"] * per_step / (ms / 1e3)
    sample = f"{per_step} SVGD iterations per step of the {args.workload} workload, exhaustive FP64 search"
    line = {"impl": "reference", "metric": "particle_point_evals_per_sec", "value": value,
            "unit": "particle_point_evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config(args.workload, d, cfg, "exhaustive"),
            "iters_per_sec": per_step / (ms / 1e3),
            "cpu_baseline": {"value": value, "unit": "particle_point_evals/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle_point_evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2106_03287_gb300 as S
    from paper_2106_03287_gb300 import build
    if not os.path.exists(S.LIB_PATH):
        build.build()
    d, cfg = make_problem(args.workload, 1000 + rank)
    K = int(d["particles"].shape[0])
    M, N = int(d["ref"].shape[0]), int(d["src"].shape[0])
    nn_mode = S.SICP_NN_GRID if args.workload != "box" else S.SICP_NN_BRUTE_FP32
    mode_name = {S.SICP_NN_GRID: "voxel grid (exact)", S.SICP_NN_BRUTE_FP32: "exhaustive fp32"}[nn_mode]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = S.sicp_create(local, stream)
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=nn_mode)
    ref_d = torch.from_numpy(d["ref"]).cuda()
    src_d = torch.from_numpy(d["src"]).cuda()
    par_d = torch.from_numpy(d["particles"]).cuda()
    torch.cuda.synchronize()

    def step():
        S.sicp_set_reference(ctx, ref_d)
        return S.sicp_register(ctx, src_d, par_d, p)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # work counters of one (untimed) step: algorithmic bytes of the gradient kernel
    S.sicp_stats(ctx, True)
    step()
    st = S.sicp_stats(ctx, False).astype(np.float64)
    queries = st[0]
    rows_q, segs_q, pts_q = st[1] / queries, st[2] / queries, st[3] / queries
    coarse_frac, exhaustive_frac = st[4] / queries, st[5] / queries
    bytes_per_query = 16 + 4 + 8 * rows_q + 8 * segs_q + 16 * pts_q
    if args.profile_stride > 0:
        S.sicp_profile(ctx, args.profile_stride)
        step()   # capture the profiling graphs outside the timed region
        step()
        S.sicp_profile(ctx, args.profile_stride)   # reset totals

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    prof = S.sicp_profile(ctx, 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    evals = K * cfg["m"] * cfg["T"]
    value = world * evals / (ms_max / 1e3)

    grad_ms = prof[0] / prof[1] if prof[1] else None
    peak, peak_kind = measured_peak()
    queries_per_launch = K * cfg["m"]
    alg_bytes = bytes_per_query * queries_per_launch
    achieved = alg_bytes / (grad_ms * 1e-3) / 1e9 if grad_ms else None
    tpq = ncu_traffic_per_query()
    roofline = {"kernel": "k_grad_grid (transform + grid NN + gradient, one iteration)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "peak_kind": f"{peak_kind} copy bandwidth",
                "frac": achieved / peak if achieved else None,
                "traffic": tpq * queries_per_launch if tpq else None,
                "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_us": grad_ms * 1e3 if grad_ms else None,
                "launches_timed": int(prof[1]),
                "per_query": {"rows": rows_q, "segments": segs_q, "candidates": pts_q, "bytes": bytes_per_query,
                              "far_frac": coarse_frac, "exhaustive_frac": exhaustive_frac},
                "stein_adam_avg_launch_us": 1e3 * prof[2] / prof[3] if prof[3] else None}

    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        ref_h, src_h, par_h = pin(d["ref"]), pin(d["src"]), pin(d["particles"])
        for _ in range(2):
            S.sicp_set_reference(ctx, ref_h)
            S.sicp_register(ctx, src_h, par_h, p)
        wall = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S.sicp_set_reference(ctx, ref_h)
            out = S.sicp_register(ctx, src_h, par_h, p)
            wall.append(time.perf_counter() - t0)
        e2e = {"value": world * evals / statistics.mean(wall), "unit": "particle_point_evals/s",
               "h2d_bytes_per_step": 12 * M + 12 * N + 24 * K, "d2h_bytes_per_step": 24 * K + 8 * 42,
               "ms_per_step": 1e3 * statistics.mean(wall)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, cfg)
    S.sicp_destroy(ctx)
    launches_per_step = 9 + 4 + 2 * cfg["T"]
    if rank == 0:
        line = {"metric": "particle_point_evals_per_sec", "value": value, "unit": "particle_point_evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded generators; no dataset)",
                "config": {**workload_config(args.workload, d, cfg, mode_name),
                           "l2": "256 MB buffer written between timed steps (outside the events)",
                           "parallelism": f"independent problem per rank x{world}"},
                "iters_per_sec": world * cfg["T"] / (ms_max / 1e3),
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_ours_batched(args):
    """The serving-style workload: 256 problems in one persistent launch per step."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2106_03287_gb300 as S
    from paper_2106_03287_gb300 import build
    if not os.path.exists(S.LIB_PATH):
        build.build()
    raw, cfg = make_problem("batched", 1000 + rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = S.sicp_create(local, stream)
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=S.SICP_NN_GRID)
    dev = S.pack_batch([tuple(torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], d["particles"])) for d in raw])
    torch.cuda.synchronize()
    tuned = S.sicp_autotune_batched(ctx, dev, p, trial_iters=3,
                                    cache_path=os.path.join(tempfile.gettempdir(), "sicp_tune.json"))
    Ks = [d["particles"].shape[0] for d in raw]
    evals = sum(Ks) * cfg["m"] * cfg["T"]
    for _ in range(max(args.warmup, 3)):
        S.sicp_register_batched(ctx, dev, p)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        S.sicp_register_batched(ctx, dev, p)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    host = S.pack_batch([(d["ref"], d["src"], d["particles"]) for d in raw])
    for key in ("ref", "src", "par"):
        host[key] = torch.from_numpy(host[key]).pin_memory().numpy()   # pinned staging of the packed inputs
    S.sicp_register_batched(ctx, host, p)
    wall = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sicp_register_batched(ctx, host, p)
        wall.append(time.perf_counter() - t0)
    Mtot = sum(d["ref"].shape[0] for d in raw)
    Ntot = sum(d["src"].shape[0] for d in raw)
    e2e = {"value": world * evals / statistics.mean(wall), "unit": "particle_point_evals/s",
           "h2d_bytes_per_step": 12 * (Mtot + Ntot) + 24 * sum(Ks), "d2h_bytes_per_step": 24 * sum(Ks) + 8 * 42 * len(raw),
           "ms_per_step": 1e3 * statistics.mean(wall)}
    S.sicp_destroy(ctx)
    if rank == 0:
        line = {"metric": "particle_point_evals_per_sec", "value": world * evals / (ms_max / 1e3),
                "unit": "particle_point_evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded generators; no dataset)",
                "config": {"workload": "batched", "problems": len(raw), "reference_points_total": Mtot,
                           "source_points_total": Ntot, "particles_total": sum(Ks), "minibatch": cfg["m"],
                           "iterations": cfg["T"], "nn": "voxel grid (exact), one persistent launch per step",
                           "autotuned": {"cell_factor": tuned[0], "points_per_item": tuned[1]},
                           "l2": "256 MB buffer written between timed steps (outside the events)"},
                "iters_per_sec": world * cfg["T"] / (ms_max / 1e3),
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "clocks": clocks, "e2e": e2e, "gpu_launches": (2 + 2 * 9 + 3 + 4) * args.steps,
                "roofline": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_ours_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
