"""Write pose_gate.json: FP64 oracle runs of the benchmark workloads, the
reference that the benchmark's "at fixed pose error" gate compares with.

For each workload (the generator seed the benchmark uses on rank 0, 1000;
minibatch seed 0) this runs the oracle once on the workload's inputs and four
more times with every initial particle component moved by one float32 ulp
(up, down, and two seeded random +-1 ulp patterns).  The spread of those four
runs around the first is the method's own sensitivity to float32 rounding of
its inputs: a float32 run cannot be expected to land closer to the FP64 run
than that.  The file stores the reference run's mean and covariance, that
floor, and a hash of the inputs so that a reader can tell whether a machine
generated the same clouds.

It calls only the oracle (and the input generators):
    python tests/golden/make_pose_gate.py [workload ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2106_03287_gb300 import gate, synth  # noqa: E402

OUT = os.path.join(HERE, "pose_gate.json")
PROBLEM_SEED = 1000
F32 = lambda x: float(np.float32(x))  # noqa: E731  (the library takes its parameters as float32)


def problems(workload):
    """(name, inputs, run parameters) of the workload's gated runs."""
    if workload == "batched":
        probs = synth.make_batched_problems(PROBLEM_SEED)
        cfg = synth.WORKLOADS["batched"]
        # problem p of a batch draws its minibatches with seed (run seed 0) + p
        return [(f"batched[{p}]", probs[p], dict(cfg, seed=p)) for p in (0, 1, 2)]
    make = {"kinect": synth.make_kinect_problem, "box": synth.make_box_problem,
            "lidar": synth.make_lidar_problem}[workload]
    return [(workload, make(PROBLEM_SEED), dict(synth.WORKLOADS[workload], seed=0))]


def ulp_variants(parts):
    rng = np.random.default_rng(12345)
    up = np.nextafter(parts, np.float32(np.inf))
    down = np.nextafter(parts, np.float32(-np.inf))
    out = [up, down]
    for _ in range(2):
        pick = rng.integers(0, 2, parts.shape).astype(bool)
        out.append(np.where(pick, up, down).astype(np.float32))
    return out


def run(name, d, cfg):
    tree = O.KDTree(d["ref"])
    p = O.Params(T=cfg["T"], m=cfg["m"], lr=F32(cfg["lr"]), beta1=F32(0.9), beta2=F32(0.999), eps=F32(1e-8),
                 seed=cfg["seed"], tree=tree)
    t0 = time.perf_counter()
    th, mean, cov = O.register(d["ref"], d["src"], d["particles"], p)
    secs = time.perf_counter() - t0
    floor_runs = []
    for v in ulp_variants(d["particles"]):
        _, m2, c2 = O.register(d["ref"], d["src"], v, p)
        floor_runs.append(gate.pose_errors(m2, c2, mean, cov))
    rec = {"inputs_sha256_16": gate.inputs_hash(d), "reference_points": int(d["ref"].shape[0]),
           "source_points": int(d["src"].shape[0]), "particles": int(d["particles"].shape[0]),
           "T": cfg["T"], "m": cfg["m"], "lr": cfg["lr"], "minibatch_seed": cfg["seed"],
           "mean": mean.tolist(), "cov": cov.ravel().tolist(),
           "floor": gate.worst(floor_runs), "floor_runs": floor_runs,
           "oracle_seconds": secs, "oracle_threads": O.num_threads()}
    print(f"{name}: {secs:.1f} s, floor {rec['floor']}", flush=True)
    return rec


def main(argv):
    wanted = argv or ["box", "kinect", "lidar", "batched"]
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["_about"] = ("FP64 oracle runs (k-d tree search) of the benchmark workloads, generator seed 1000, "
                      "and the spread of four runs whose initial particles moved by one float32 ulp; "
                      "written by tests/golden/make_pose_gate.py")
    for w in wanted:
        for name, d, cfg in problems(w):
            data[name] = run(name, d, cfg)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
