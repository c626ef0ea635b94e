"""The experiments' distribution-quality protocol through the C ABI: the Monte
Carlo reference (SICP_INDEPENDENT: many SGD-ICP runs from spread initial
poses in one sicp_register call) and the KL divergence / overlapping
coefficient between Gaussians (reading R17 of oracle.c).

Tolerances: independent runs are bit-identical to the K = 1 runs they stand
for (same kernels, same arithmetic); KL and OVL are float64 on both sides with
the same draws, so they agree to 1e-10 relative.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
IND = S.SICP_INDEPENDENT


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


@pytest.mark.parametrize("mode", [S.SICP_NN_GRID, S.SICP_NN_BRUTE_FP32, S.SICP_NN_BRUTE_BF16])
def test_independent_runs_are_single_particle_runs(ctx, mode):
    d = synth.make_box_problem(4, K=6)
    S.sicp_set_reference(ctx, d["ref"])
    p = S.sicp_default_params(T=40, m=100, lr=0.01, seed=5, nn_mode=mode | IND)
    th, mean, cov = S.sicp_register(ctx, d["src"], d["particles"], p)
    for j in range(6):      # run j is the single-particle run with seed + j
        one, _, _ = S.sicp_register(ctx, d["src"], d["particles"][j:j + 1],
                                    S.sicp_default_params(T=40, m=100, lr=0.01, seed=5 + j, nn_mode=mode))
        assert np.array_equal(th[j], one[0]), j
    coupled, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                                    S.sicp_default_params(T=40, m=100, lr=0.01, seed=5, nn_mode=mode))
    assert not np.array_equal(coupled, th)
    mo, co = O.moments(th.astype(np.float64))
    assert np.allclose(mean, mo, atol=1e-12) and np.allclose(cov, co, atol=1e-12)


def test_independent_runs_with_priors_and_point_to_plane(ctx):
    d = synth.make_box_problem(5, K=4)
    S.sicp_set_reference(ctx, d["ref"])
    S.sicp_reference_normals(ctx, 10, want=False)
    extra = dict(prior=1, prior_mu=(0, 0, 0, 0, 0, 0), prior_sigma=(0.01,) * 3, prior_kappa=(5.0,) * 3)
    flags = S.SICP_NN_GRID | S.SICP_POINT_TO_PLANE
    th, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                               S.sicp_default_params(T=30, m=100, seed=2, nn_mode=flags | IND, **extra))
    for j in range(4):
        one, _, _ = S.sicp_register(ctx, d["src"], d["particles"][j:j + 1],
                                    S.sicp_default_params(T=30, m=100, seed=2 + j, nn_mode=flags, **extra))
        assert np.array_equal(th[j], one[0]), j


def test_independent_free_run_against_oracle(ctx):
    """Noise-free box, eight runs from spread poses: the GPU's runs and the
    oracle's independent runs all land on the generating pose (1 mm, 0.05 deg)."""
    d = synth.make_box_problem(0, K=8, noise=0.0)
    S.sicp_set_reference(ctx, d["ref"])
    th, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                               S.sicp_default_params(T=300, m=100, lr=0.01, seed=7, nn_mode=S.SICP_NN_GRID | IND))
    th_o, _, _ = O.register(d["ref"], d["src"], d["particles"],
                            O.Params(T=300, m=100, lr=float(np.float32(0.01)), seed=7, independent=True))
    for x in (th.astype(np.float64), th_o):
        err = x - d["theta_true"]
        assert np.abs(err[:, :3]).max() < 1e-3 and np.abs(err[:, 3:]).max() < math.radians(0.05)


def test_independent_runs_resume(ctx):
    """An independent run split by sicp_register_continue equals one call."""
    d = synth.make_box_problem(6, K=5)
    S.sicp_set_reference(ctx, d["ref"])
    full, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                                 S.sicp_default_params(T=30, m=100, seed=4, nn_mode=S.SICP_NN_GRID | IND))
    state = np.zeros((3, 5, 6), np.float32)
    state[0] = d["particles"]
    S.sicp_register_continue(ctx, d["src"], state, 0, S.sicp_default_params(T=12, m=100, seed=4,
                                                                           nn_mode=S.SICP_NN_GRID | IND))
    S.sicp_register_continue(ctx, d["src"], state, 12, S.sicp_default_params(T=18, m=100, seed=4,
                                                                            nn_mode=S.SICP_NN_GRID | IND))
    assert np.array_equal(state[0], full)


def test_flags_are_checked(ctx):
    d = synth.make_box_problem(1)
    S.sicp_set_reference(ctx, d["ref"])
    mb = O.minibatch(1, 0, d["src"].shape[0], 20)
    with pytest.raises(S.SicpError) as e:              # a gradient call has no update to make independent
        S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_GRID | IND)
    assert e.value.code == S.SICP_EINVAL
    with pytest.raises(S.SicpError) as e:              # nor a plain search a metric
        S.sicp_nn(ctx, d["src"], S.SICP_NN_GRID | S.SICP_POINT_TO_PLANE)
    assert e.value.code == S.SICP_EINVAL
    with pytest.raises(S.SicpError) as e:
        S.sicp_register(ctx, d["src"], d["particles"], S.sicp_default_params(T=2, m=20, nn_mode=S.SICP_NN_GRID | 0x400))
    assert e.value.code == S.SICP_EINVAL
    S.sicp_surrogate_train(ctx, 50_000, seed=1, epochs=1)
    with pytest.raises(S.SicpError) as e:              # the learned field is not an exact search
        S.sicp_register(ctx, d["src"], d["particles"],
                        S.sicp_default_params(T=2, m=20, nn_mode=S.SICP_NN_SURROGATE | IND, surrogate_iters=2))
    assert e.value.code == S.SICP_EINVAL


def _spd(rng, d, scale):
    A = rng.normal(size=(d, d))
    return scale * (A @ A.T / d + 0.2 * np.eye(d))


@pytest.mark.parametrize("d", [1, 3, 6])
def test_kl_and_ovl_match_oracle(d):
    rng = np.random.default_rng(d)
    for trial in range(5):
        m0, m1 = rng.normal(size=d), rng.normal(size=d) * 0.5
        S0, S1 = _spd(rng, d, 0.4), _spd(rng, d, 0.7)
        kl = S.sicp_gaussian_kl(m0, S0, m1, S1)
        kl_o = O.gaussian_kl(m0, S0, m1, S1)
        assert abs(kl - kl_o) <= 1e-10 * max(1.0, abs(kl_o))
        z0, z1 = rng.standard_normal((20_000, d)), rng.standard_normal((20_000, d))
        ovl = S.sicp_gaussian_ovl(m0, S0, m1, S1, z0=z0, z1=z1)
        assert abs(ovl - O.gaussian_ovl(m0, S0, m1, S1, z0, z1)) <= 1e-10
        assert 0.0 <= ovl <= 1.0
    assert S.sicp_gaussian_ovl(m0, S0, m0, S0, n=1000) == 1.0
    assert abs(S.sicp_gaussian_kl(m0, S0, m0, S0)) < 1e-12


def test_kl_and_ovl_errors():
    m, I = np.zeros(3), np.eye(3)
    bad = np.diag([1.0, -1.0, 1.0])
    for args in ((m, bad, m, I), (m, I, m, bad), (m, I, np.full(3, np.nan), I)):
        with pytest.raises(S.SicpError) as e:
            S.sicp_gaussian_kl(*args)
        assert e.value.code == S.SICP_EINVAL
        with pytest.raises(S.SicpError) as e:
            S.sicp_gaussian_ovl(*args, n=10)
        assert e.value.code == S.SICP_EINVAL


def test_monte_carlo_reference_protocol(ctx):
    """The protocol end to end on the box: a Monte Carlo reference of 1000
    independent runs from initial poses spread like Stein ICP's particles,
    Stein ICP with 100 particles, then KL and OVL between their Gaussians.
    The library's numbers equal the oracle's on the same moments and draws."""
    d = synth.make_box_problem(3, K=1000)
    S.sicp_set_reference(ctx, d["ref"])
    base = dict(T=150, m=100, lr=0.01, seed=9)
    th_mc, m_mc, c_mc = S.sicp_register(ctx, d["src"], d["particles"],
                                        S.sicp_default_params(nn_mode=S.SICP_NN_GRID | IND, **base))
    th_s, m_s, c_s = S.sicp_register(ctx, d["src"], d["particles"][:100],
                                     S.sicp_default_params(nn_mode=S.SICP_NN_GRID, **base))
    reg = 1e-12 * np.eye(6)
    kl = S.sicp_gaussian_kl(m_mc, c_mc + reg, m_s, c_s + reg)
    rng = np.random.default_rng(0)
    z0, z1 = rng.standard_normal((50_000, 6)), rng.standard_normal((50_000, 6))
    ovl = S.sicp_gaussian_ovl(m_mc, c_mc + reg, m_s, c_s + reg, z0=z0, z1=z1)
    assert np.isfinite(kl) and kl >= 0.0 and 0.0 <= ovl <= 1.0
    assert abs(kl - O.gaussian_kl(m_mc, c_mc + reg, m_s, c_s + reg)) <= 1e-8 * max(1.0, kl)
    assert abs(ovl - O.gaussian_ovl(m_mc, c_mc + reg, m_s, c_s + reg, z0, z1)) <= 1e-10
    print(f"box: KL(MC || Stein) = {kl:.3g}, OVL = {ovl:.3f}")
