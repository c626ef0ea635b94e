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
SURR_QUERIES, SURR_EPOCHS = 1 << 21, 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kinect", choices=["kinect", "box", "lidar", "batched", "surrogate", "mc"])
    ap.add_argument("--nn", default=None, choices=["grid", "bf16", "fp32", "surrogate"],
                    help="search of the registration loop (default: per workload)")
    ap.add_argument("--profile-stride", type=int, default=5,
                    help="after the timed steps, time the gradient and Stein kernels of every s-th iteration "
                         "with CUDA events in a separate pass (0: skip)")
    ap.add_argument("--metric", default="point", choices=["point", "plane"],
                    help="ICP error metric: point-to-point (the paper's Stein ICP) or point-to-plane")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-single", action="store_true",
                    help="batched workload: skip the single-problem-path comparison")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched workload: only the first P problems (a small case, for profiling)")
    ap.add_argument("--iters", type=int, default=0,
                    help="batched workload: T iterations instead of the workload's (a small case, for profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: the library's default tuning, no trial launches")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Each rank registers its own problem: the workload generator's seed for `rank`."""
    return 1000 + rank


def slowest_rank_ms(ms: float, world: int, device: str) -> float:
    """The step time of the slowest rank (the job's time): a MAX all-reduce
    over the process group (nccl on GPUs, gloo on CPU)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(evals_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * evals_per_rank / (ms_max / 1e3)


def make_problem(workload: str, seed: int):
    from paper_2106_03287_gb300 import synth
    if workload == "batched":
        return synth.make_batched_problems(seed), dict(synth.WORKLOADS["batched"])
    if workload == "mc":
        return synth.make_kinect_problem(seed, K=synth.WORKLOADS["mc"]["runs"]), dict(synth.WORKLOADS["mc"])
    if workload in ("kinect", "surrogate"):
        d = synth.make_kinect_problem(seed)
    elif workload == "box":
        d = synth.make_box_problem(seed)
    else:
        d = synth.make_lidar_problem(seed)
    return d, dict(synth.WORKLOADS[workload])


NORMAL_K = 10   # neighbours of the reference normals of the point-to-plane metric
# kernels of one sicp_set_reference per workload, counted in ncu launch lists: pack, bbox, the fine
# level (cell assignment, 3-kernel scan, scatter, cell sort, seed init, seed-flooding steps) and the
# coarse level, plus the seed points; the number of flooding steps follows the grid's size
SETREF_LAUNCHES = {"kinect": 23, "box": 22, "lidar": 25, "mc": 23, "surrogate": 23}


def metric_name(metric):
    return "point-to-point" if metric == "point" else f"point-to-plane (normals from {NORMAL_K} nearest neighbours)"


def workload_config(workload, d, cfg, nn_mode_name, metric="point"):
    return {"workload": workload, "reference_points": int(d["ref"].shape[0]),
            "source_points": int(d["src"].shape[0]), "particles": int(d["particles"].shape[0]),
            "minibatch": cfg["m"], "iterations": cfg["T"], "adam_lr": cfg["lr"], "nn": nn_mode_name,
            "metric": metric_name(metric)}


FALLBACK_BF16_TFLOPS = 1900.0
# fp32 FMA lanes: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (nominal unit counts and clock)
ALU_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peak(key="hbm_gbs"):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)[key]), "measured"
    return (FALLBACK_HBM_GBS if key == "hbm_gbs" else FALLBACK_BF16_TFLOPS), "fallback"


DEFAULT_NN = {"kinect": "grid", "box": "bf16", "lidar": "bf16", "surrogate": "surrogate"}


class _Nvml:
    """The few NVML reads the clock record needs, through ctypes (public nvml.h
    API; read-only: nothing here changes a GPU setting)."""

    CLOCK_SM = 1
    # clock-event reason bits (nvmlClocksEventReason*)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str | None, index: int, lib=None):
        import ctypes
        self.c = ctypes
        self.lib = lib if lib is not None else ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        rc = 1
        if uuid:
            rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            self.lib.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = reasons or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def max_sm(self) -> int | None:
        v = self.c.c_uint()
        return v.value if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.CLOCK_SM, self.c.byref(v)) == 0 else None

    def sample(self):
        v, r = self.c.c_uint(), self.c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, self.c.byref(v)) != 0:
            return None
        bits = r.value if self.reasons_fn(self.h, self.c.byref(r)) == 0 else 0
        return v.value, [n for b, n in self.REASONS.items() if bits & b]

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons of the bench's GPU during
    the timed region.  NVML is polled every 2 ms from a thread, so a region of
    a few tens of milliseconds still gets many samples.  nvidia-smi runs
    beside it at its 200 ms interval and is waited for (its first line)
    before start() returns.  The median SM clock is over the NVML samples
    (nvidia-smi's where NVML cannot be loaded); the reasons are those either
    source saw active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.uuid = None
        try:
            import torch
            u = str(torch.cuda.get_device_properties(gpu).uuid)
            self.uuid = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            self.uuid = None
        self.nvml, self.thread, self.samples = None, None, []
        self.stop_flag = False

    def _poll(self):
        while not self.stop_flag:
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)
            time.sleep(0.002)

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.uuid or str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5 and os.path.getsize(self.tmp.name) == 0 and self.proc.poll() is None:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        try:
            self.nvml = _Nvml(self.uuid, self.gpu)
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
        except (OSError, AttributeError):
            self.nvml = None

    def _smi(self) -> str:
        if self.proc is None:
            return ""
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        return self.tmp.read()

    def stop(self):
        nv_max = None
        if self.nvml is not None:
            self.stop_flag = True
            self.thread.join(timeout=5)
            nv_max = self.nvml.max_sm()
            self.nvml.close()
        text = self._smi()
        os.unlink(self.tmp.name)
        return clock_summary(self.samples, nv_max, text)


def clock_summary(nvml_samples, nvml_max, smi_text: str) -> dict:
    """The clock record: NVML samples [(sm MHz, [reasons])], NVML's maximum SM
    clock and nvidia-smi's CSV lines (FIELDS order, no header, no units)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in smi_text.splitlines():
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
    nv_sm = [float(c) for c, _ in nvml_samples]
    for _, rs in nvml_samples:
        reasons.update(rs)
    if not nv_sm and not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi and NVML unavailable"]}
    mxs = ([float(nvml_max)] if nvml_max else []) + mx
    use = nv_sm or sm
    return {"sm_mhz": statistics.median(use), "sm_min_mhz": min(use), "sm_max_mhz": max(mxs) if mxs else None,
            "reasons": sorted(reasons), "samples": len(use),
            "source": "nvml, 2 ms" if nv_sm else "nvidia-smi, 200 ms", "nvidia_smi_samples": len(sm)}


def grad_kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_grid.cu", "grid_search.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2106_03287_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_grad_record():
    """The committed ncu summary of the gradient kernel (DRAM and L2 bytes of
    one launch), if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "k_grad_grid_kinect.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("source_hash") != grad_kernel_source_hash():
        return None
    return rec


def measure_l2_gbs(torch, sizes_mb=(4, 8, 16, 24), reps=50):
    """Bandwidth of a copy whose source and destination stay in the 129 MB
    L2: bytes read plus written per second, CUDA events around one graph of
    `reps` back-to-back copies after a warm-up; the best over buffer sizes
    (MB per buffer).  Returns (GB/s, size in MB)."""
    best = (0.0, 0)
    for mb in sizes_mb:
        n = mb * (1 << 20) // 4
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        for _ in range(10):
            b.copy_(a)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()   # one graph of `reps` copies: no host launch gaps between them
        with torch.cuda.graph(g):
            for _ in range(reps):
                b.copy_(a)
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        gbs = 2.0 * n * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
        best = max(best, (gbs, mb))
        del g, a, b
    return best


def cpu_baseline(d, cfg, budget_s=10.0, metric="point", single_budget_s=5.0):
    """The oracle as it stands, on a bounded number of iterations of the same workload
    (point-to-plane: the reference normals are computed before the timed sample): on all
    host threads, then the same iterations again on one thread."""
    import oracle as O
    ref, src = d["ref"], d["src"]
    normals = O.normals(ref, NORMAL_K)[0] if metric == "plane" else None
    t0 = time.perf_counter()
    tree = O.KDTree(ref)
    build_s = time.perf_counter() - t0
    p = O.Params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, normals=normals, tree=tree)
    K = d["particles"].shape[0]

    def sample(budget, first):
        th = d["particles"].astype(np.float64).copy()
        mom, vel = np.zeros_like(th), np.zeros_like(th)
        O.step(ref, src, th, mom, vel, p, 0)   # untimed first iteration
        t0 = time.perf_counter()
        n = 0
        while n < min(cfg["T"] - 1, first) and (n == 0 or time.perf_counter() - t0 < budget):
            n += 1
            O.step(ref, src, th, mom, vel, p, n)
        return n, time.perf_counter() - t0

    cores = O.num_threads()
    n, dt = sample(budget_s, cfg["T"])
    out = {"value": K * cfg["m"] * n / dt, "unit": "particle_point_evals/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{n} SVGD iterations (iterations 1..{n}) of the same workload, FP64, exact k-d tree search "
                     f"(tree built once in {build_s * 1e3:.0f} ms, not timed), {dt:.1f} s", "iters_per_sec": n / dt}
    O.set_threads(1)
    try:
        n1, dt1 = sample(single_budget_s, n)
    finally:
        O.set_threads(cores)
    out["single_thread"] = {"value": K * cfg["m"] * n1 / dt1, "cores": 1,
                            "sample": f"{n1} SVGD iterations (iterations 1..{n1}) on one thread, {dt1:.1f} s"}
    return out


def pose_gate(name, d, mean, cov, metric="point"):
    """The run's final pose mean and spread against the FP64 oracle run of the
    same inputs stored by tests/golden/make_pose_gate.py ("at fixed pose
    error": within 1 mm and 0.05 deg), with the oracle's own spread under a
    one-ulp change of its initial particles beside it."""
    from paper_2106_03287_gb300 import gate
    path = os.path.join(ROOT, "tests", "golden", "pose_gate.json")
    if metric != "point" or not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f).get(name)
    if g is None:
        return None
    same = g["inputs_sha256_16"] == gate.inputs_hash(d)
    err = gate.pose_errors(mean, cov, np.array(g["mean"]), np.array(g["cov"]).reshape(6, 6))
    fl = g["floor"]
    return {"reference": f"FP64 oracle run {name}, tests/golden/pose_gate.json", "same_inputs": same, **err,
            "gate_mm": gate.GATE_MM, "gate_deg": gate.GATE_DEG, "met": bool(same and gate.within(err)),
            "oracle_ulp_floor": fl,
            "within_2x_floor": bool(same and gate.within(err, max(gate.GATE_MM, 2 * max(fl["dmean_mm"], fl["dsd_mm"])),
                                                        max(gate.GATE_DEG, 2 * max(fl["dmean_deg"], fl["dsd_deg"]))))}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    d, cfg = make_problem(args.workload, 1000)
    if args.workload == "batched":
        d = d[0]              # the oracle takes the batch's first problem (its runs are independent)
    import oracle as O
    ref, src = d["ref"], d["src"]
    parts = d["particles"][:100] if args.workload == "mc" else d["particles"]   # mc: 100 of the independent runs
    K = parts.shape[0]
    normals = O.normals(ref, NORMAL_K)[0] if args.metric == "plane" else None
    p = O.Params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, normals=normals, independent=args.workload == "mc",
                 tree=O.KDTree(ref))
    th = parts.astype(np.float64).copy()
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
    sample = (f"{per_step} SVGD iterations per step of the {args.workload} workload"
              + (" (problem 0 of the batch)" if args.workload == "batched" else "")
              + (" (100 of the independent runs)" if args.workload == "mc" else "") + ", FP64, exact k-d tree search")
    line = {"impl": "reference", "metric": "particle_point_evals_per_sec", "value": value,
            "unit": "particle_point_evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, d, cfg, "exact k-d tree (FP64)", args.metric),
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
    d, cfg = make_problem(args.workload, rank_seed(rank))
    K = int(d["particles"].shape[0])
    M, N = int(d["ref"].shape[0]), int(d["src"].shape[0])
    nn = args.nn or DEFAULT_NN[args.workload]
    modes = {"grid": S.SICP_NN_GRID, "bf16": S.SICP_NN_BRUTE_BF16, "fp32": S.SICP_NN_BRUTE_FP32,
             "surrogate": S.SICP_NN_SURROGATE}
    names = {"grid": "voxel grid (exact)", "bf16": "exhaustive, bf16 tensor-core tiles + exact fp32 re-check",
             "fp32": "exhaustive fp32",
             "surrogate": "learned closest-point field for the first iterations, exact voxel grid after and as fallback"}
    nn_mode, mode_name = modes[nn], names[nn]
    plane = args.metric == "plane"
    if plane:
        if nn == "surrogate":
            raise SystemExit("the point-to-plane metric runs with the exact searches (--nn grid, fp32 or bf16)")
        nn_mode |= S.SICP_POINT_TO_PLANE
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = S.sicp_create(local, stream)
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=nn_mode,
                              surrogate_iters=cfg.get("surrogate_iters", 0))
    ref_d = torch.from_numpy(d["ref"]).cuda()
    src_d = torch.from_numpy(d["src"]).cuda()
    par_d = torch.from_numpy(d["particles"]).cuda()
    torch.cuda.synchronize()
    training = None
    if nn == "surrogate":
        # the learned field belongs to the reference: trained once, timed apart from the loop
        S.sicp_set_reference(ctx, ref_d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = S.sicp_surrogate_train(ctx, SURR_QUERIES, seed=3, epochs=SURR_EPOCHS, batch=4096, lr=1e-3)
        training = {"queries": SURR_QUERIES, "epochs": SURR_EPOCHS, "batch": 4096, "seconds": time.perf_counter() - t0,
                    "final_loss": loss}

    def set_ref(ref):
        S.sicp_set_reference(ctx, ref)
        if plane:
            S.sicp_reference_normals(ctx, NORMAL_K, want=False)

    def step():
        if nn != "surrogate":
            set_ref(ref_d)
        return S.sicp_register(ctx, src_d, par_d, p)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # work counters of one (untimed) step: algorithmic bytes of the gradient kernel
    S.sicp_stats(ctx, True)
    step()
    st = S.sicp_stats(ctx, False).astype(np.float64)
    queries = max(st[0], 1.0)   # grid-search counters (zero in the exhaustive modes)
    rows_q, segs_q, pts_q = st[1] / queries, st[2] / queries, st[3] / queries
    coarse_frac, exhaustive_frac = st[4] / queries, st[5] / queries
    bytes_per_query = 16 + 4 + 8 * rows_q + 8 * segs_q + 16 * pts_q + (16 if plane else 0)   # + the normal
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
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # kernel durations for the roofline: a separate, untimed pass with CUDA events
    # recorded around the kernels of every s-th iteration (they would slow the timed steps)
    prof = kernel_profile(S, ctx, step, args.profile_stride)
    ms = statistics.mean(step_ms)
    ms_max = slowest_rank_ms(ms, world, "cuda")
    evals = K * cfg["m"] * cfg["T"]
    value = job_value(evals, world, ms_max)

    grad_ms = prof[0] / prof[1] if prof[1] else None
    queries_per_launch = K * cfg["m"]
    stein_us = 1e3 * prof[2] / prof[3] if prof[3] else None
    if nn == "grid":
        peak, peak_kind = measured_peak()
        alg_bytes = bytes_per_query * queries_per_launch
        achieved = alg_bytes / (grad_ms * 1e-3) / 1e9 if grad_ms else None
        rec = ncu_grad_record()
        tpq = rec["dram_bytes"] / rec["queries"] if rec else None
        l2pq = rec["lts_bytes"] / rec["queries"] if rec and "lts_bytes" in rec else None
        l2_gbs, l2_mb = measure_l2_gbs(torch)
        l2_achieved = l2pq * queries_per_launch / (grad_ms * 1e-3) / 1e9 if l2pq and grad_ms else None
        roofline = {"kernel": "k_grad_grid (transform + grid NN + gradient, one iteration)"
                              + (", point-to-plane" if plane else ""), "bound": "hbm",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "peak_kind": f"{peak_kind} copy bandwidth",
                    "frac": achieved / peak if achieved else None,
                    "traffic": tpq * queries_per_launch if tpq else None,
                    "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_us": grad_ms * 1e3 if grad_ms else None,
                    "launches_timed": int(prof[1]),
                    "per_query": {"rows": rows_q, "segments": segs_q, "candidates": pts_q, "bytes": bytes_per_query,
                                  "far_frac": coarse_frac, "exhaustive_frac": exhaustive_frac},
                    "l2": {"bytes_per_launch": l2pq * queries_per_launch if l2pq else None,
                           "achieved": l2_achieved, "peak": l2_gbs, "unit": "GB/s",
                           "peak_kind": f"measured L2-resident copy (2 x {l2_mb} MB, read + write; "
                                        "best of 4-24 MB buffers)",
                           "frac": l2_achieved / l2_gbs if l2_achieved else None,
                           "bytes_source": "lts__t_sectors.sum x 32 B of the committed ncu capture"},
                    "stein_adam_avg_launch_us": stein_us}
    elif nn == "bf16":
        peak, peak_kind = measured_peak("bf16_tflops")
        R = (M + 255) // 256
        qtiles, rtiles = float(st[8]), float(st[9])   # query tiles and reference tiles swept over the step
        swept = rtiles / qtiles if qtiles else float(R)
        # executed: 128 x 256 x 16 MMAs over the reference tiles the query tiles swept
        mma_flops = 2.0 * 16 * 128 * 256 * (rtiles / cfg["T"]) if qtiles else 2.0 * 16 * queries_per_launch * 256 * R
        alg_flops = 2.0 * 4 * queries_per_launch * M
        achieved = alg_flops / (grad_ms * 1e-3) / 1e12 if grad_ms else None
        roofline = {"kernel": "k_nn_bf16 (tensor-core distance tiles + fp32 re-check + gradient terms), the "
                              "three launches that put the queries in key order (from 32 reference tiles) and the "
                              "per-particle reduction, one iteration", "bound": "tensor",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "peak_kind": f"{peak_kind} dense bf16 (burst)",
                    "frac": achieved / peak if achieved else None, "traffic": None,
                    "algorithmic_flops_per_launch": alg_flops,
                    "executed_mma_flops_per_launch": mma_flops,
                    "executed_tflops": mma_flops / (grad_ms * 1e-3) / 1e12 if grad_ms else None,
                    "reference_tiles": R, "reference_tiles_swept_per_query_tile": swept,
                    "avg_launch_us": grad_ms * 1e3 if grad_ms else None, "launches_timed": int(prof[1]),
                    "stein_adam_avg_launch_us": stein_us}
    elif nn == "fp32":
        achieved = 8.0 * queries_per_launch * M / (grad_ms * 1e-3) / 1e12 if grad_ms else None
        roofline = {"kernel": "k_grad_brute (transform + fp32 exhaustive search + gradient, one iteration)",
                    "bound": "alu", "achieved": achieved, "peak": ALU_FP32_TFLOPS, "unit": "TFLOP/s",
                    "peak_kind": "nominal fp32 FMA rate (152 SMs x 128 lanes x 2 x 2.07 GHz)",
                    "frac": achieved / ALU_FP32_TFLOPS if achieved else None, "traffic": None,
                    "flops_per_pair": 8, "avg_launch_us": grad_ms * 1e3 if grad_ms else None,
                    "launches_timed": int(prof[1]), "stein_adam_avg_launch_us": stein_us}
    else:
        roofline = surrogate_roofline(S, ctx, p, src_d, par_d, queries_per_launch, cfg)
        roofline["stein_adam_avg_launch_us"] = stein_us

    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        ref_h, src_h, par_h = pin(d["ref"]), pin(d["src"]), pin(d["particles"])
        with_ref = nn != "surrogate"   # the learned field stays with the reference it was trained on
        for _ in range(2):
            if with_ref:
                set_ref(ref_h)
            S.sicp_register(ctx, src_h, par_h, p)
        wall = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if with_ref:
                set_ref(ref_h)
            out = S.sicp_register(ctx, src_h, par_h, p)
            wall.append(time.perf_counter() - t0)
        e2e = {"value": world * evals / statistics.mean(wall), "unit": "particle_point_evals/s",
               "h2d_bytes_per_step": (12 * M if with_ref else 0) + 12 * N + 24 * K,
               "d2h_bytes_per_step": 24 * K + 8 * 42, "ms_per_step": 1e3 * statistics.mean(wall)}

    gate_rec = None
    if rank == 0 and nn != "surrogate" and args.workload != "mc":
        _, mean_f, cov_f = step()
        gate_rec = pose_gate(args.workload, d, np.asarray(mean_f.cpu()), np.asarray(cov_f.cpu()), args.metric)

    comparison = None
    if nn in ("bf16", "surrogate"):
        comparison = compare_paths(S, ctx, nn, p, lambda: set_ref(ref_d), src_d, par_d, cfg, K, flush, stream,
                                   args.steps)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, cfg, metric=args.metric)
    S.sicp_destroy(ctx)
    # the bf16 search puts each launch's queries in key order (3 launches) from 32 reference tiles on
    bf_order = nn == "bf16" and (int(d["ref"].shape[0]) + 255) // 256 >= 32
    per_iter = {"grid": 3, "fp32": 2, "bf16": 6 if bf_order else 3}.get(nn)
    if per_iter is not None:
        # reference build (pack, bbox, two grid levels, seed map: 23 launches on the kinect grid, counted
        # in an ncu launch list), the run's pack / finite check / minibatch / moments, and per iteration
        # the gradient kernel(s) and the Stein kernel; point-to-plane adds the normals kernel; each new
        # reference's bf16 build: brick order (cell offsets, a 3-kernel scan, the scatter), tiles, boxes
        launches_per_step = (SETREF_LAUNCHES[args.workload] + 4 + per_iter * cfg["T"] + (1 if plane else 0)
                             + (7 if nn == "bf16" else 0))
    else:   # surrogate, fallback, reduction and Stein for the surrogate iterations; grid, reduction and Stein after
        si = min(cfg.get("surrogate_iters", 0), cfg["T"])
        launches_per_step = 4 + 4 * si + 3 * (cfg["T"] - si)
    if rank == 0:
        line = {"metric": "particle_point_evals_per_sec", "value": value, "unit": "particle_point_evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded generators; no dataset)",
                "config": {**workload_config(args.workload, d, cfg, mode_name, args.metric),
                           "l2": "256 MB buffer written between timed steps (outside the events)",
                           "parallelism": f"independent problem per rank x{world}"},
                "iters_per_sec": world * cfg["T"] / (ms_max / 1e3),
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline, "cpu_baseline": cpu}
        if gate_rec:
            line["pose_gate"] = gate_rec
        if training:
            line["surrogate_training"] = training
        if comparison:
            line["comparison"] = comparison
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def single_problem_path(S, torch, raw, p, evals, stream, flush, passes=2):
    """The batch's problems through the single-problem path, outside the timed
    region: one context per problem (each keeps its captured registration
    graph), and every pass rebuilds each problem's reference and registers it,
    as a batched step rebuilds every grid.  Device inputs, CUDA events around
    each pass after two untimed passes."""
    dev = [tuple(torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], d["particles"])) for d in raw]
    ctxs = [S.sicp_create(torch.cuda.current_device(), stream) for _ in dev]
    try:
        def run():
            for c, (r, src, par) in zip(ctxs, dev):
                S.sicp_set_reference(c, r)
                S.sicp_register(c, src, par, p)
        run()
        run()
        ms = []
        for _ in range(passes):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    finally:
        for c in ctxs:
            S.sicp_destroy(c)
    t = statistics.mean(ms)
    return {"value": evals / (t * 1e-3), "unit": "particle_point_evals/s", "ms_per_pass": t,
            "how": f"{len(raw)} contexts, one per problem: reference build + one captured registration each, "
                   f"the same problems and parameters; mean of {passes} passes after 2 untimed ones"}


def kernel_profile(S, ctx, step, stride, runs=3):
    """Average kernel durations over `runs` untimed steps with profiling on
    (the first captures the profiling graphs and is discarded)."""
    if stride <= 0:
        return [0.0, 0.0, 0.0, 0.0]
    S.sicp_profile(ctx, stride)
    step()
    S.sicp_profile(ctx, stride)   # drop the capture run's totals
    for _ in range(runs):
        step()
    prof = S.sicp_profile(ctx, 0)
    step()                        # leave the context's unprofiled graph captured again
    return prof


def timed_runs(fn, flush, stream, steps):
    import torch
    fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def compare_paths(S, ctx, nn, p, set_ref, src_d, par_d, cfg, K, flush, stream, steps):
    """bf16: the same run with the fp32 exhaustive search (the precision
    comparison; same metric).  surrogate: the all-exact run (the ablation) and
    the final pose mean / spread of the surrogate run against it.  set_ref()
    sets the reference (and its normals for the point-to-plane metric)."""
    import ctypes
    q = S.sicp_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
    if nn == "bf16":
        q.nn_mode = S.SICP_NN_BRUTE_FP32 | (p.nn_mode & S.SICP_POINT_TO_PLANE)
        run = lambda: (set_ref(), S.sicp_register(ctx, src_d, par_d, q))[1]
        name = "exhaustive fp32 search"
    else:
        q.nn_mode = S.SICP_NN_GRID
        run = lambda: S.sicp_register(ctx, src_d, par_d, q)
        name = "all-exact run (voxel grid every iteration)"
    ms = timed_runs(run, flush, stream, steps)
    th_o, mean_o, cov_o = [np.asarray(x.cpu() if hasattr(x, "cpu") else x) for x in run()]
    if nn != "surrogate":
        set_ref()
    th_s, mean_s, cov_s = [np.asarray(x.cpu() if hasattr(x, "cpu") else x) for x in S.sicp_register(ctx, src_d, par_d, p)]
    sd_o, sd_s = np.sqrt(np.diag(cov_o)), np.sqrt(np.diag(cov_s))
    return {"other": name, "other_value": K * cfg["m"] * cfg["T"] / (ms / 1e3),
            "other_iters_per_sec": cfg["T"] / (ms / 1e3), "other_ms_per_step": ms,
            "particles_max_abs_diff": float(np.abs(th_s - th_o).max()),
            "mean_diff_mm": (1e3 * np.abs(mean_s[:3] - mean_o[:3])).tolist(),
            "mean_diff_deg": np.degrees(np.abs(mean_s[3:] - mean_o[3:])).tolist(),
            "sd_diff_mm": (1e3 * np.abs(sd_s[:3] - sd_o[:3])).tolist(),
            "sd_diff_deg": np.degrees(np.abs(sd_s[3:] - sd_o[3:])).tolist(),
            "gate_1mm_0.05deg": bool(np.all(1e3 * np.abs(mean_s[:3] - mean_o[:3]) <= 1.0) and
                                     np.all(np.degrees(np.abs(mean_s[3:] - mean_o[3:])) <= 0.05) and
                                     np.all(1e3 * np.abs(sd_s[:3] - sd_o[:3]) <= 1.0) and
                                     np.all(np.degrees(np.abs(sd_s[3:] - sd_o[3:])) <= 0.05))}


def surrogate_roofline(S, ctx, p, src_d, par_d, queries, cfg):
    """The surrogate's gradient kernels timed on a run that uses the surrogate in
    every iteration (untimed for the metric), against the dense bf16 peak:
    three layers, 2 (112 x 128 + 128 x 128 + 128 x 16) flops per query."""
    import ctypes
    q = S.sicp_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
    q.surrogate_iters = q.T
    S.sicp_profile(ctx, 1)
    S.sicp_register(ctx, src_d, par_d, q)
    S.sicp_stats(ctx, True)
    S.sicp_register(ctx, src_d, par_d, q)
    st = S.sicp_stats(ctx, False)
    prof = S.sicp_profile(ctx, 0)
    grad_ms = prof[0] / prof[1] if prof[1] else None
    flops = 2.0 * (112 * 128 + 128 * 128 + 128 * 16) * queries
    peak, peak_kind = measured_peak("bf16_tflops")
    achieved = flops / (grad_ms * 1e-3) / 1e12 if grad_ms else None
    return {"kernel": "k_grad_surrogate + exact fallback + reduction (one surrogate iteration)", "bound": "tensor",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "peak_kind": f"{peak_kind} dense bf16 (burst)",
            "frac": achieved / peak if achieved else None, "traffic": None, "flops_per_launch": flops,
            "avg_launch_us": grad_ms * 1e3 if grad_ms else None, "launches_timed": int(prof[1]),
            "fallback_fraction": float(st[7] / st[6]) if st[6] else None}


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
    raw, cfg = make_problem("batched", rank_seed(rank))
    if args.problems:   # a smaller case of the same workload (profiling): the first P problems, T iterations
        raw = raw[:args.problems]
    if args.iters:
        cfg["T"] = args.iters
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = S.sicp_create(local, stream)
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=S.SICP_NN_GRID)
    dev = S.pack_batch([tuple(torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], d["particles"])) for d in raw])
    torch.cuda.synchronize()
    if args.no_autotune:   # the library's defaults; no trial launches before the measured ones
        tuned = (None, None, None)
    else:
        tuned = S.sicp_autotune_batched(ctx, dev, p, trial_iters=3,
                                        cache_path=os.path.join(tempfile.gettempdir(), "sicp_tune.json"))
    Ks = [d["particles"].shape[0] for d in raw]
    evals = sum(Ks) * cfg["m"] * cfg["T"]
    for _ in range(max(args.warmup, 3)):
        S.sicp_register_batched(ctx, dev, p)
    # work counters of one (untimed) step: algorithmic bytes of the searches
    S.sicp_stats(ctx, True)
    S.sicp_register_batched(ctx, dev, p)
    st = S.sicp_stats(ctx, False).astype(np.float64)
    queries = st[0]
    rows_q, segs_q, pts_q = st[1] / queries, st[2] / queries, st[3] / queries
    bytes_per_query = 16 + 4 + 8 * rows_q + 8 * segs_q + 16 * pts_q
    S.sicp_profile(ctx, 1)   # the persistent launch of each timed step joins the totals
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
    prof = S.sicp_profile(ctx, 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    ms_max = slowest_rank_ms(ms, world, "cuda")
    kernel_ms = prof[0] / prof[1] if prof[1] else None
    peak, peak_kind = measured_peak()
    alg_bytes = bytes_per_query * queries
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9 if kernel_ms else None
    roofline = {"kernel": "kb_persistent (all T iterations of all problems: transform + grid NN + gradient, "
                          "then the Stein/Adam phase, grid barriers between)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "peak_kind": f"{peak_kind} copy bandwidth",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "algorithmic_bytes_per_launch": alg_bytes, "queries_per_launch": queries,
                "avg_launch_us": kernel_ms * 1e3 if kernel_ms else None, "launches_timed": int(prof[1]),
                "per_query": {"rows": rows_q, "segments": segs_q, "candidates": pts_q, "bytes": bytes_per_query,
                              "far_frac": st[4] / queries, "exhaustive_frac": st[5] / queries}}
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
    single = single_problem_path(S, torch, raw, p, evals, stream, flush) if not args.no_single else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(raw[0], cfg, budget_s=10.0)
        cpu["sample"] = "problem 0 of the batch: " + cpu["sample"]
    if rank == 0:
        line = {"metric": "particle_point_evals_per_sec", "value": world * evals / (ms_max / 1e3),
                "unit": "particle_point_evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded generators; no dataset)",
                "config": {"workload": "batched", "problems": len(raw), "reference_points_total": Mtot,
                           "source_points_total": Ntot, "particles_total": sum(Ks), "minibatch": cfg["m"],
                           "iterations": cfg["T"], "nn": "voxel grid (exact), one persistent launch per step",
                           "autotuned": {"cell_factor": tuned[0], "points_per_item": tuned[1], "cta_threads": tuned[2]},
                           "l2": "256 MB buffer written between timed steps (outside the events)"},
                "iters_per_sec": world * cfg["T"] / (ms_max / 1e3),
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "clocks": clocks, "e2e": e2e, "gpu_launches": (2 + 2 * 9 + 3 + 4) * args.steps,
                "roofline": roofline, "vs_single_problem_path": single, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_ours_mc(args):
    """The experiments' distribution-quality protocol on the kinect scene: a
    Monte Carlo reference of 1000 independent SGD-ICP runs (each its own
    minibatch stream) in one registration call, timed as the step; then Stein
    ICP with 100 of the same initial poses, and the KL divergence and
    overlapping coefficient between the two Gaussians."""
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
    d, cfg = make_problem("mc", rank_seed(rank))
    R, Ks = cfg["runs"], cfg["stein_K"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = S.sicp_create(local, stream)
    p_mc = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0,
                                 nn_mode=S.SICP_NN_GRID | S.SICP_INDEPENDENT)
    p_st = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=S.SICP_NN_GRID)
    ref_d = torch.from_numpy(d["ref"]).cuda()
    src_d = torch.from_numpy(d["src"]).cuda()
    par_d = torch.from_numpy(d["particles"]).cuda()

    def step():
        S.sicp_set_reference(ctx, ref_d)
        return S.sicp_register(ctx, src_d, par_d, p_mc)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 3)):
        step()
    S.sicp_stats(ctx, True)
    step()
    st = S.sicp_stats(ctx, False).astype(np.float64)
    queries = max(st[0], 1.0)
    bytes_per_query = 16 + 4 + 8 * st[1] / queries + 8 * st[2] / queries + 16 * st[3] / queries
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    out = None
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        out = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_max = slowest_rank_ms(statistics.mean(step_ms), world, "cuda")
    prof = kernel_profile(S, ctx, step, 5)
    evals = R * cfg["m"] * cfg["T"]
    grad_ms = prof[0] / prof[1] if prof[1] else None
    peak, peak_kind = measured_peak()
    alg_bytes = bytes_per_query * R * cfg["m"]
    achieved = alg_bytes / (grad_ms * 1e-3) / 1e9 if grad_ms else None
    roofline = {"kernel": "k_grad_grid over 1000 independent runs, each with its own minibatch (one iteration)",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "peak_kind": f"{peak_kind} copy bandwidth", "frac": achieved / peak if achieved else None,
                "traffic": None, "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_us": grad_ms * 1e3 if grad_ms else None, "launches_timed": int(prof[1]),
                "update_avg_launch_us": 1e3 * prof[2] / prof[3] if prof[3] else None}
    # end to end: pinned host inputs, copies and the reference build inside the timed region
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    ref_h, src_h, par_h = pin(d["ref"]), pin(d["src"]), pin(d["particles"])
    for _ in range(2):
        S.sicp_set_reference(ctx, ref_h)
        S.sicp_register(ctx, src_h, par_h, p_mc)
    wall = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sicp_set_reference(ctx, ref_h)
        S.sicp_register(ctx, src_h, par_h, p_mc)
        wall.append(time.perf_counter() - t0)
    e2e = {"value": world * evals / statistics.mean(wall), "unit": "particle_point_evals/s",
           "h2d_bytes_per_step": 12 * int(d["ref"].shape[0]) + 12 * int(d["src"].shape[0]) + 24 * R,
           "d2h_bytes_per_step": 24 * R + 8 * 42, "ms_per_step": 1e3 * statistics.mean(wall)}
    # quality: Stein ICP from the first stein_K initial poses against the Monte Carlo reference
    S.sicp_set_reference(ctx, ref_d)
    _, m_mc, c_mc = [np.asarray(x.cpu()) for x in out]
    _, m_st, c_st = [np.asarray(x.cpu()) for x in S.sicp_register(ctx, src_d, par_d[:Ks].contiguous(), p_st)]
    reg = 1e-12 * np.eye(6)
    quality = {"reference": f"{R} independent SGD-ICP runs", "estimate": f"Stein ICP, {Ks} particles",
               "kl_reference_to_estimate": S.sicp_gaussian_kl(m_mc, c_mc + reg, m_st, c_st + reg),
               "kl_estimate_to_reference": S.sicp_gaussian_kl(m_st, c_st + reg, m_mc, c_mc + reg),
               "ovl": S.sicp_gaussian_ovl(m_mc, c_mc + reg, m_st, c_st + reg, n=200_000, seed=0),
               "sd_reference_mm_deg": (1e3 * np.sqrt(np.diag(c_mc)[:3])).tolist()
               + np.degrees(np.sqrt(np.diag(c_mc)[3:])).tolist(),
               "sd_estimate_mm_deg": (1e3 * np.sqrt(np.diag(c_st)[:3])).tolist()
               + np.degrees(np.sqrt(np.diag(c_st)[3:])).tolist(),
               "mean_diff_mm": (1e3 * np.abs(m_mc[:3] - m_st[:3])).tolist()}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        sub = 100   # a bounded sample: 100 of the runs, as many iterations as fit in about 10 s
        th = d["particles"][:sub].astype(np.float64).copy()
        mom, vel = np.zeros_like(th), np.zeros_like(th)
        po = O.Params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, independent=True, tree=O.KDTree(d["ref"]))
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < 10.0 and n < cfg["T"]:
            O.step(d["ref"], d["src"], th, mom, vel, po, n)
            n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": sub * cfg["m"] * n / dt, "unit": "particle_point_evals/s", "cores": O.num_threads(),
               "kind": "oracle", "sample": f"{sub} of the {R} runs, {n} iterations, FP64, exact k-d tree search, {dt:.1f} s"}
    S.sicp_destroy(ctx)
    if rank == 0:
        line = {"metric": "particle_point_evals_per_sec", "value": job_value(evals, world, ms_max),
                "unit": "particle_point_evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded generators; no dataset)",
                "config": {"workload": "mc", "reference_points": int(d["ref"].shape[0]),
                           "source_points": int(d["src"].shape[0]), "runs": R, "minibatch": cfg["m"],
                           "iterations": cfg["T"], "adam_lr": cfg["lr"], "nn": "voxel grid (exact)",
                           "l2": "256 MB buffer written between timed steps (outside the events)",
                           "parallelism": f"independent problem per rank x{world}"},
                "iters_per_sec": world * cfg["T"] / (ms_max / 1e3),
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "clocks": clocks, "e2e": e2e, "gpu_launches": (SETREF_LAUNCHES["mc"] + 4 + 3 * cfg["T"]) * args.steps,
                "roofline": roofline, "cpu_baseline": cpu, "quality": quality}
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
    if args.workload == "mc":
        return run_ours_mc(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
