"""The batched persistent path (sicp_register_batched) against the FP64 oracle.

Each problem p of a batch is an independent Stein ICP run with minibatch
seed `seed + p`.  One batched iteration is compared with one oracle step
from the same initial particles: the Stein direction is checked through the
Adam step it produces (Adam moves a component by lr * sign(phi) on its
first step, so components whose phi is within the FP32 tolerance of zero
may go either way; every other component must match).
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _mixed_problems():
    probs = []
    for i, (M, N, K) in enumerate([(2000, 500, 32), (5000, 1000, 7), (3000, 800, 1), (4000, 900, 60)]):
        d = synth.make_box_problem(100 + i, M=M, N=N, K=K)
        probs.append((d["ref"], d["src"], d["particles"]))
    for i, (M, N, K) in enumerate([(12000, 2500, 40), (6000, 1200, 17)]):
        d = synth.make_kinect_problem(200 + i, M=M, N=N, K=K, width=320, height=240)
        probs.append((d["ref"], d["src"], d["particles"]))
    return probs


def _one_step_matches_oracle(parts, probs, m, seed, lr):
    lr32 = float(np.float32(lr))
    for p, (ref, src, th0) in enumerate(probs):
        th = th0.astype(np.float64).copy()
        mom, vel = np.zeros_like(th), np.zeros_like(th)
        out = O.step(ref, src, th, mom, vel, O.Params(T=1, m=m, lr=lr32, seed=seed + p), 0)
        phi = out["phi"]
        tol_phi = 1e-4 * np.abs(phi).max(1, keepdims=True) + 1e-5 * np.abs(out["G"]).max()
        sure = np.abs(phi) > tol_phi                    # sign of phi fixed beyond the FP32 tolerance
        diff = np.abs(np.asarray(parts[p], np.float64) - th)
        assert np.all(diff[sure] <= 1e-4 * lr32 + 4 * 2.0 ** -24 * np.abs(th[sure])), (p, diff[sure].max())
        assert np.all(diff <= 2 * lr32 + 1e-6)


@pytest.mark.parametrize("on_device", [False, True])
def test_batched_one_iteration_matches_oracle(ctx, on_device):
    probs = _mixed_problems()
    if on_device:
        probs = [tuple(torch.from_numpy(a).cuda() for a in pr) for pr in probs]
    params = S.sicp_default_params(T=1, m=100, lr=0.01, seed=40, nn_mode=S.SICP_NN_GRID)
    parts, mean, cov = S.sicp_register_batched(ctx, probs, params)
    if on_device:
        parts = [x.cpu().numpy() for x in parts]
        mean, cov = mean.cpu().numpy(), cov.cpu().numpy()
        probs = [tuple(a.cpu().numpy() for a in pr) for pr in probs]
    _one_step_matches_oracle(parts, probs, 100, 40, 0.01)
    for p, th in enumerate(parts):
        mo, co = O.moments(np.asarray(th, np.float64))
        assert np.allclose(mean[p], mo, atol=1e-12) and np.allclose(cov[p], co, atol=1e-12)


def test_batched_matches_single_problem_path(ctx):
    """A batched run equals the single-problem runs it contains over a few
    iterations (same search, same kernels; only the summation order of the
    gradient chunks differs)."""
    probs = _mixed_problems()[:4]
    params = S.sicp_default_params(T=4, m=100, lr=0.01, seed=7, nn_mode=S.SICP_NN_GRID)
    parts, mean, _ = S.sicp_register_batched(ctx, probs, params)
    for p, (ref, src, th0) in enumerate(probs):
        S.sicp_set_reference(ctx, ref)
        single, m1, _ = S.sicp_register(ctx, src, th0, S.sicp_default_params(T=4, m=100, lr=0.01, seed=7 + p,
                                                                             nn_mode=S.SICP_NN_GRID))
        d = np.abs(parts[p] - single)
        assert np.mean(d <= 1e-5) > 0.97 and d.max() <= 8 * 0.01, (p, d.max())


def test_batched_autotune_and_cache(ctx, tmp_path):
    probs = _mixed_problems()
    params = S.sicp_default_params(T=3, m=100, lr=0.01, seed=1, nn_mode=S.SICP_NN_GRID)
    cache = str(tmp_path / "tune.json")
    f, k = S.sicp_autotune_batched(ctx, probs, params, trial_iters=2, cache_path=cache)
    assert any(abs(f - c) < 1e-6 for c in (0.35, 0.5, 0.7, 1.0)) and k in (2, 4, 8)
    text = open(cache).read()
    json.loads(text)
    f2, k2 = S.sicp_autotune_batched(ctx, probs, params, trial_iters=2, cache_path=cache)   # read back
    assert abs(f2 - f) < 1e-3 and k2 == k
    parts, _, _ = S.sicp_register_batched(ctx, probs, S.sicp_default_params(T=1, m=100, lr=0.01, seed=40,
                                                                            nn_mode=S.SICP_NN_GRID))
    _one_step_matches_oracle(parts, probs, 100, 40, 0.01)          # still exact with the tuned layout


def test_batched_errors(ctx):
    probs = _mixed_problems()[:2]
    with pytest.raises(S.SicpError) as e:
        S.sicp_register_batched(ctx, probs, S.sicp_default_params(T=1, m=100, nn_mode=S.SICP_NN_BRUTE_FP32))
    assert e.value.code == S.SICP_EINVAL
    with pytest.raises(S.SicpError) as e:
        S.sicp_register_batched(ctx, probs, S.sicp_default_params(T=1, m=600, nn_mode=S.SICP_NN_GRID))  # N < m
    assert e.value.code == S.SICP_EINVAL
    bad = [(probs[0][0], probs[0][1], np.full((3, 6), np.nan, np.float32))]
    with pytest.raises(S.SicpError):
        S.sicp_register_batched(ctx, bad, S.sicp_default_params(T=1, m=100, nn_mode=S.SICP_NN_GRID))


def test_batched_serving_workload_sampled(ctx):
    """32 problems of the serving-style generator (log-uniform 5k-80k points,
    20% sources, 50-200 particles) for 100 iterations: finite, moments
    consistent; the first iteration of sampled problems teacher-forced."""
    raw = synth.make_batched_problems(5, P=32)
    probs = [(d["ref"], d["src"], d["particles"]) for d in raw]
    params = S.sicp_default_params(T=100, m=300, lr=0.01, seed=3, nn_mode=S.SICP_NN_GRID)
    parts, mean, cov = S.sicp_register_batched(ctx, probs, params)
    for p in range(32):
        assert np.all(np.isfinite(parts[p]))
        mo, co = O.moments(parts[p].astype(np.float64))
        assert np.allclose(mean[p], mo, atol=1e-12) and np.allclose(cov[p], co, atol=1e-12)
    sample = [probs[i] for i in (0, 1, 13)]
    one, _, _ = S.sicp_register_batched(ctx, sample, S.sicp_default_params(T=1, m=300, lr=0.01, seed=3,
                                                                           nn_mode=S.SICP_NN_GRID))
    _one_step_matches_oracle(one, sample, 300, 3, 0.01)
