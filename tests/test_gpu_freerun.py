"""Whole-run parity: free GPU runs against free FP64 oracle runs on the same
seeded inputs (the Stein ICP loop of Sec. IV, summary paragraph).

Protocol.  Both runs are advanced in lockstep: the GPU one iteration per
sicp_register_continue call (a split run is bit-identical to one call; the
test checks that the chain ends where one sicp_register call ends), the
oracle by its own step.  At every iteration:
  * the correspondences of the two runs are compared, the GPU's on its own
    particles, the oracle's on its own;
  * until the first iteration with a differing correspondence the particles
    must agree within 1e-4 relative per particle (max-norm over the six
    components, relative to max(|theta|, 1e-2));
  * every differing correspondence must be explained by the distance between
    the two runs' query points q_g (GPU particles) and q_o (oracle's):
    |r_gpu - q_o| <= |r_oracle - q_o| + 2 |q_g - q_o| + the float32 rounding
    floor (the triangle inequality, since r_gpu is the nearest point of q_g).
    The first such iteration is logged ("diverged at tie t = ...").
After the first differing correspondence the runs are separate samples of the
same stochastic method and are judged by the pose gate: mean and standard
deviation within 1 mm and 0.05 deg of the oracle run.  On workloads where the
oracle itself moves by more than that when its initial particles move by one
float32 ulp (the floor stored in tests/golden/pose_gate.json, recomputed
here), a float32 run cannot do better, and the bound is twice that floor.
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import gate, synth  # noqa: E402

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
F32 = lambda x: float(np.float32(x))  # noqa: E731
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pose_gate.json")


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _oracle_params(cfg, seed, tree):
    return O.Params(T=cfg["T"], m=cfg["m"], lr=F32(cfg["lr"]), beta1=F32(0.9), beta2=F32(0.999), eps=F32(1e-8),
                    seed=seed, tree=tree)


def _floor(d, cfg, seed, tree, mean_o, cov_o):
    """The oracle's own spread when its initial particles move by one float32 ulp."""
    p = _oracle_params(cfg, seed, tree)
    parts = d["particles"]
    errs = []
    for v in (np.nextafter(parts, np.float32(np.inf)), np.nextafter(parts, np.float32(-np.inf))):
        _, m2, c2 = O.register(d["ref"], d["src"], v, p)
        errs.append(gate.pose_errors(m2, c2, mean_o, cov_o))
    return gate.worst(errs)


def _lockstep(ctx, d, cfg, seed, mode):
    ref, src = d["ref"], d["src"]
    N, K, m, T = src.shape[0], d["particles"].shape[0], cfg["m"], cfg["T"]
    tree = O.KDTree(ref)
    po = _oracle_params(cfg, seed, tree)
    th_o = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th_o), np.zeros_like(th_o)
    p1 = S.sicp_default_params(T=1, m=m, lr=cfg["lr"], seed=seed, nn_mode=mode)
    state = np.zeros((3, K, 6), np.float32)
    state[0] = d["particles"]
    X = float(max(np.abs(ref).max(), np.abs(src).max()) + 1.0)
    floor = 16 * U32 * X * (1 + X)
    log = {"first_flip_t": None, "flips_at_first": 0, "rel_before_first_flip": 0.0, "worst_explained_gap": 0.0,
           "iterations_with_flips": 0}
    for t in range(T):
        mb = O.minibatch(seed, t, N, m)
        _, nn_g = S.sicp_icp_grad(ctx, src, mb, state[0], mode)
        _, nn_o, _ = tree.icp_grad(src, mb, th_o)
        rel = float((np.abs(state[0] - th_o).max(1) / np.maximum(np.abs(th_o).max(1), 1e-2)).max())
        diff = nn_g != nn_o
        if diff.any():
            log["iterations_with_flips"] += 1
            j, k = np.nonzero(diff)
            s = src[mb[k]].astype(np.float64)
            q_o = np.stack([O.transform(th_o[jj], s[i:i + 1])[0] for i, jj in enumerate(j)])
            q_g = np.stack([O.transform(state[0][jj].astype(np.float64), s[i:i + 1])[0] for i, jj in enumerate(j)])
            d_g = np.linalg.norm(ref[nn_g[j, k]].astype(np.float64) - q_o, axis=1)
            d_o = np.linalg.norm(ref[nn_o[j, k]].astype(np.float64) - q_o, axis=1)
            slack = 2 * np.linalg.norm(q_g - q_o, axis=1) + 8 * floor
            assert np.all(d_g <= d_o + slack), (t, (d_g - d_o - slack).max())
            log["worst_explained_gap"] = max(log["worst_explained_gap"], float((d_g - d_o).max()))
            if log["first_flip_t"] is None:
                log["first_flip_t"], log["flips_at_first"] = t, int(diff.sum())
        if log["first_flip_t"] is None:
            assert rel <= 1e-4, (t, rel)
            log["rel_before_first_flip"] = max(log["rel_before_first_flip"], rel)
        S.sicp_register_continue(ctx, src, state, t, p1)
        O.step(ref, src, th_o, mom, vel, po, t)
    return state, th_o, log, tree


def _free_run_case(ctx, d, cfg, seed, mode, name, strict):
    S.sicp_set_reference(ctx, d["ref"])
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=seed, nn_mode=mode)
    th_g, mean_g, cov_g = S.sicp_register(ctx, d["src"], d["particles"], p)
    state, th_o, log, tree = _lockstep(ctx, d, cfg, seed, mode)
    assert np.array_equal(state[0], th_g)                 # the split run ends where one call ends
    mean_o, cov_o = O.moments(th_o)
    err = gate.pose_errors(mean_g, cov_g, mean_o, cov_o)
    rel = float((np.abs(th_g - th_o).max(1) / np.maximum(np.abs(th_o).max(1), 1e-2)).max())
    if log["first_flip_t"] is None:
        assert rel <= 1e-4, rel                            # no tie ever differed: the particles agree
    fl = _floor(d, cfg, seed, tree, mean_o, cov_o)
    tag = "no differing correspondence" if log["first_flip_t"] is None else f"diverged at tie t = {log['first_flip_t']}"
    print(f"{name} mode={mode}: {tag} ({log['flips_at_first']} correspondences; "
          f"{log['iterations_with_flips']} iterations with any); particles before it within "
          f"{log['rel_before_first_flip']:.1e}; final particle rel {rel:.1e}; pose errors {err}; "
          f"oracle ulp floor {fl}")
    if strict:
        assert gate.within(err), err
    else:
        assert gate.within(err, max(gate.GATE_MM, 2 * max(fl["dmean_mm"], fl["dsd_mm"])),
                           max(gate.GATE_DEG, 2 * max(fl["dmean_deg"], fl["dsd_deg"]))), (err, fl)
    return err, fl, log


@pytest.mark.parametrize("mode", [S.SICP_NN_BRUTE_FP32, S.SICP_NN_GRID, S.SICP_NN_BRUTE_BF16])
def test_free_run_box_against_oracle(ctx, mode):
    """C1 (2,000-point box, 500 source points, 32 particles, m = 100, T = 100):
    the pose gate is met outright."""
    d = synth.make_box_problem(0)
    _free_run_case(ctx, d, dict(T=100, m=100, lr=0.01), 7, mode, "box", strict=True)


def test_free_run_kinect_bench_config_against_oracle(ctx):
    """C2 exactly as the benchmark runs it (generator seed 1000, minibatch
    seed 0, 50,000-point reference, 10,000 source points, 100 particles,
    m = 300, T = 150, lr 0.03, grid search).  The benchmark's pose gate reads
    its oracle run from tests/golden/pose_gate.json (tests/golden/make_pose_gate.py):
    where this machine generates the same inputs, the stored run must be the
    oracle run recomputed here."""
    d = synth.make_kinect_problem(1000)
    cfg = dict(synth.WORKLOADS["kinect"])
    _free_run_case(ctx, d, cfg, 0, S.SICP_NN_GRID, "kinect", strict=False)
    with open(GOLDEN) as f:
        g = json.load(f)["kinect"]
    if g["inputs_sha256_16"] == gate.inputs_hash(d):
        tree = O.KDTree(d["ref"])
        _, mean_o, cov_o = O.register(d["ref"], d["src"], d["particles"], _oracle_params(cfg, 0, tree))
        e = gate.pose_errors(mean_o, cov_o, np.array(g["mean"]), np.array(g["cov"]).reshape(6, 6))
        print(f"stored oracle run against the one recomputed here: {e}")
        assert gate.within(e, 2 * max(g["floor"]["dmean_mm"], g["floor"]["dsd_mm"]),
                           2 * max(g["floor"]["dmean_deg"], g["floor"]["dsd_deg"]))


def test_free_run_batched_problems_single_path_against_oracle(ctx):
    """Three problems of the C4 serving batch (generator seed 1000), each run
    alone through sicp_register with the batch's seed rule (seed + p):
    the pose gate is met outright."""
    probs = synth.make_batched_problems(1000)
    cfg = dict(synth.WORKLOADS["batched"])
    for pidx in (0, 1, 2):
        _free_run_case(ctx, probs[pidx], cfg, pidx, S.SICP_NN_GRID, f"batched[{pidx}]", strict=True)


@pytest.mark.parametrize("mode", [S.SICP_NN_BRUTE_BF16, S.SICP_NN_GRID])
def test_lidar_run_against_stored_oracle_run(ctx, mode):
    """C3 at full size (a ~112k-point scan, 200 particles, m = 500, T = 200,
    lr 0.01; generator seed 1000, minibatch seed 0) with the tensor-core
    exhaustive search and with the grid search, against the FP64 oracle run of
    the same inputs stored by tests/golden/make_pose_gate.py (the oracle is
    bit-reproducible across machines: the stored run was checked against a
    run on the GPU host).  Judged by the pose gate, against twice the
    oracle's own one-ulp floor where that floor is above it."""
    d = synth.make_lidar_problem(1000)
    with open(GOLDEN) as f:
        g = json.load(f)["lidar"]
    if g["inputs_sha256_16"] != gate.inputs_hash(d):
        pytest.skip("this machine generates other lidar clouds than the stored run's")
    cfg = dict(synth.WORKLOADS["lidar"])
    S.sicp_set_reference(ctx, d["ref"])
    p = S.sicp_default_params(T=cfg["T"], m=cfg["m"], lr=cfg["lr"], seed=0, nn_mode=mode)
    _, mean_g, cov_g = S.sicp_register(ctx, d["src"], d["particles"], p)
    err = gate.pose_errors(mean_g, cov_g, np.array(g["mean"]), np.array(g["cov"]).reshape(6, 6))
    fl = g["floor"]
    print(f"lidar mode={mode}: pose errors {err}; oracle ulp floor {fl}; strict gate met: {gate.within(err)}")
    assert gate.within(err, max(gate.GATE_MM, 2 * max(fl["dmean_mm"], fl["dsd_mm"])),
                       max(gate.GATE_DEG, 2 * max(fl["dmean_deg"], fl["dsd_deg"]))), (err, fl)
