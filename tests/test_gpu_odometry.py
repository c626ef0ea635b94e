"""Odometry chaining through the C ABI against the oracle (reading R18):
particle sets to pose distributions (mean pose, se(3) covariance) and their
second- / fourth-order compounding.

Tolerances: both sides are float64; compounding is a fixed formula (1e-12
relative); a pose distribution comes from an iteration and closed-form
exp/log on one side, scipy's matrix exp/log on the other (1e-9).
"""
import math

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


def _spd(rng, scale):
    A = rng.normal(size=(6, 6))
    return scale * (A @ A.T / 6 + 0.1 * np.eye(6))


@pytest.mark.parametrize("order", [2, 4])
def test_compound_matches_oracle(order):
    rng = np.random.default_rng(order)
    for _ in range(10):
        T1 = O.pose_matrix(np.r_[rng.normal(0, 2, 3), rng.uniform(-math.pi, math.pi, 3)])
        T2 = O.pose_matrix(np.r_[rng.normal(0, 2, 3), rng.uniform(-math.pi, math.pi, 3)])
        S1, S2 = _spd(rng, 0.01), _spd(rng, 0.02)
        T, C = S.sicp_compound(T1, S1, T2, S2, order)
        To, Co = O.compound(T1, S1, T2, S2, order)
        assert np.allclose(T, To, atol=1e-12)
        assert np.abs(C - Co).max() <= 1e-12 * np.abs(Co).max()


def test_pose_distribution_matches_oracle():
    rng = np.random.default_rng(5)
    for K, yaw in ((1, 0.3), (2, 1.0), (100, 3.1), (500, -2.0)):
        th = np.c_[rng.normal(0, 0.05, (K, 3)), rng.normal(0, 0.03, (K, 3))]
        th[:, 5] += yaw                    # 3.1: the particles straddle +-pi in yaw
        th = th.astype(np.float32)
        T, C = S.sicp_pose_distribution(th)
        To, Co = O.pose_distribution(th)
        assert np.allclose(T, To, atol=1e-9)
        assert np.abs(C - Co).max() <= 1e-9 * max(np.abs(Co).max(), 1e-12)
        if K == 1:
            assert np.all(C == 0) and np.allclose(T, O.pose_matrix(th[0].astype(np.float64)), atol=1e-7)


def test_chain_matches_oracle():
    rng = np.random.default_rng(7)
    dists = [(O.pose_matrix(np.r_[rng.normal(0, 1, 3), rng.uniform(-1, 1, 3)]), _spd(rng, 0.001)) for _ in range(6)]
    chain = S.chain_odometry(dists, order=4)
    T, C = dists[0]
    for (T2, C2), (Tg, Cg) in zip(dists[1:], chain[1:]):
        T, C = O.compound(T, C, T2, C2, 4)
        assert np.allclose(Tg, T, atol=1e-11) and np.abs(Cg - C).max() <= 1e-11 * np.abs(C).max()


def test_odometry_errors():
    I, Z = np.eye(4), np.eye(6) * 1e-4
    with pytest.raises(S.SicpError):
        S.sicp_compound(I, Z, I, Z, order=3)
    bad = np.eye(4)
    bad[0, 0] = 2.0                        # not a rotation
    with pytest.raises(S.SicpError):
        S.sicp_compound(bad, Z, I, Z)
    with pytest.raises(S.SicpError):
        S.sicp_compound(I, np.full((6, 6), np.nan), I, Z)
    with pytest.raises(S.SicpError):
        S.sicp_pose_distribution(np.full((3, 6), np.inf, np.float32))


def test_stein_icp_odometry_chain(ctx):
    """Three kinect-scene scan pairs, each registered by Stein ICP (100
    particles, 150 iterations), chained: each pair's mean pose is near its
    true transform, the accumulated mean is the product of the pairs' mean
    poses, its error against the product of the true transforms is what the
    pairs' own errors compose to, and the accumulated covariance is at least
    the first pair's.  (The box is no test bed here: its half-turn symmetries
    make the posterior multimodal, and the particles spread over the copies.)"""
    dists, truth, errs = [], np.eye(4), []
    for seed in range(3):
        d = synth.make_kinect_problem(seed)
        S.sicp_set_reference(ctx, d["ref"])
        th, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                                   S.sicp_default_params(T=150, m=300, lr=0.03, seed=seed, nn_mode=S.SICP_NN_GRID))
        T, C = S.sicp_pose_distribution(th)
        Tt = O.pose_matrix(d["theta_true"])
        e = O.se3_log(T @ np.linalg.inv(Tt))
        errs.append(e)
        print(f"pair {seed}: translation error {1e3 * np.linalg.norm(T[:3, 3] - Tt[:3, 3]):.1f} mm, "
              f"rotation error {np.degrees(np.linalg.norm(e[3:])):.3f} deg")
        assert np.linalg.norm(T[:3, 3] - Tt[:3, 3]) < 0.05 and np.degrees(np.linalg.norm(e[3:])) < 1.0
        dists.append((T, C))
        truth = truth @ Tt
    T, C = S.chain_odometry(dists)[-1]
    prod = dists[0][0] @ dists[1][0] @ dists[2][0]
    assert np.allclose(T, prod, atol=1e-12)
    # each estimate is exp(e_i^) truth_i, so the chain is their product exactly
    composed = np.eye(4)
    for seed, e in enumerate(errs):
        composed = composed @ O.se3_exp(e) @ O.pose_matrix(synth.make_kinect_problem(seed)["theta_true"])
    assert np.allclose(T, composed, atol=1e-9)
    assert np.trace(C) >= np.trace(dists[0][1]) - 1e-15
