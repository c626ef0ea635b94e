"""The prior path (Eqs. trans_prior, rot_prior: Gaussian priors on the
translation, von Mises priors on the angles) and circular moments for
rotation blocks, through the C ABI against the oracle.

Tolerances: the Stein direction and the Adam step as in the uniform-prior
parity tests (1e-4 relative, with a floor of 1e-5 max|G|); circular moments
are float64 on both sides, so they agree to 1e-12 (libm and CUDA's sin, cos
and atan2 differ by an ulp or two).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
MU = (0.02, -0.03, 0.01, 3.0, -0.4, 0.2)        # one angle's mean next to +-pi
SIGMA = (0.0025, 0.01, 0.0004)                  # variances (the paper's sigma)
KAPPA = (20.0, 50.0, 8.0)


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _prior_params(**kw):
    return S.sicp_default_params(prior=1, prior_mu=MU, prior_sigma=SIGMA, prior_kappa=KAPPA, **kw)


def _oracle_G(th64, gbar64, N):
    return O.log_post_grad(th64, gbar64, N, 1, MU, SIGMA, KAPPA)


def _wrapped(a):
    return np.angle(np.exp(1j * np.asarray(a)))


@pytest.mark.parametrize("K", [1, 2, 100, 200])
@pytest.mark.parametrize("t", [1, 7])
def test_stein_adam_with_priors_matches_oracle(ctx, K, t):
    rng = np.random.default_rng(K * 100 + t)
    th = np.c_[rng.uniform(-0.15, 0.15, (K, 3)), rng.uniform(-0.35, 0.35, (K, 3))].astype(np.float32)
    th[:, 3] += 2.9                                 # angles around the prior's mean at 3.0, across +-pi
    gbar = rng.normal(0, 1e-5, (K, 6)).astype(np.float32)
    am = np.zeros((K, 6), np.float32) if t == 1 else rng.normal(0, 1.0, (K, 6)).astype(np.float32)
    av = np.zeros((K, 6), np.float32) if t == 1 else rng.uniform(0.5, 4.0, (K, 6)).astype(np.float32)
    p = _prior_params(lr=0.01)
    N = 1000
    th_g, am_g, av_g = th.copy(), am.copy(), av.copy()
    phi, h = S.sicp_stein_adam(ctx, th_g, am_g, av_g, gbar, N, t, p)
    th64 = th.astype(np.float64)
    G = _oracle_G(th64, gbar.astype(np.float64), N)
    # the prior term must matter here: it is of the size of the data term
    assert np.abs(G - (-N * gbar.astype(np.float64))).max() > 0.1 * np.abs(G).max()
    h_t, h_r = O.bandwidths(th64)
    assert abs(h[0] - h_t) <= 1e-5 * h_t and abs(h[1] - h_r) <= 1e-5 * h_r
    phi_ref = O.stein_phi(th64, G, h_t, h_r)
    err = np.abs(phi - phi_ref).max(1)
    assert np.all(err <= np.maximum(1e-4 * np.abs(phi_ref).max(1), 1e-5 * np.abs(G).max())), err.max()
    x, mo, ve = th64.copy(), am.astype(np.float64), av.astype(np.float64)
    O.adam(x, mo, ve, -phi_ref, t, float(np.float32(p.lr)), float(np.float32(p.beta1)),
           float(np.float32(p.beta2)), float(np.float32(p.eps)))
    dg = np.abs(phi - phi_ref)
    lr = float(np.float32(p.lr))
    bound = 2 * lr * np.minimum(1.0, 2 * dg / (np.abs(phi_ref) + 1e-8)) + 1e-4 * lr + 4 * U32 * np.abs(x)
    assert np.all(np.abs(th_g - x) <= bound)


def test_svgd_with_the_priors_reaches_the_prior_on_the_gpu(ctx):
    """No data (gbar = 0): the GPU's Stein + Adam steps must carry the
    particles to the prior itself, N(mu, sigma) per translation axis and von
    Mises(mu, kappa) per angle (mean resultant length I1(kappa)/I0(kappa)),
    with one angle's particles straddling +-pi."""
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    K = 200
    th = rng.uniform(-0.5, 0.5, (K, 6)).astype(np.float32)
    th[:, 3] += 3.0
    am, av = np.zeros((K, 6), np.float32), np.zeros((K, 6), np.float32)
    gbar = np.zeros((K, 6), np.float32)
    p = _prior_params(lr=0.01)
    for t in range(1, 1201):
        S.sicp_stein_adam(ctx, th, am, av, gbar, 1000, t, p)
    mu, sd = np.array(MU), np.sqrt(np.array(SIGMA))
    assert np.all(np.abs(th[:, :3].mean(0) - mu[:3]) < 2 * sd / math.sqrt(K))
    ratio = th[:, :3].astype(np.float64).std(0, ddof=1) / sd
    assert np.all((ratio > 0.9) & (ratio < 1.1)), ratio
    mean_c, cov_c = S.sicp_moments_circular(ctx, th)
    kappa = np.array(KAPPA)
    assert np.all(np.abs(_wrapped(mean_c[3:] - mu[3:])) < 2 / np.sqrt(kappa) / math.sqrt(K))
    R = np.abs(np.mean(np.exp(1j * th[:, 3:].astype(np.float64)), axis=0))
    A = special.i1(kappa) / special.i0(kappa)
    spread = np.sqrt(-2 * np.log(R)) / np.sqrt(-2 * np.log(A))
    assert np.all((spread > 0.9) & (spread < 1.1)), spread
    # and the library's circular moments of these particles are the oracle's
    mo, co = O.moments_circular(th.astype(np.float64))
    assert np.all(np.abs(_wrapped(mean_c - mo)) < 1e-12) and np.allclose(cov_c, co, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("K", [1, 2, 100, 2048])
def test_moments_circular_match_oracle(ctx, K):
    rng = np.random.default_rng(K)
    th = np.c_[rng.normal(0, 0.2, (K, 3)), rng.uniform(-0.6, 0.6, (K, 3))]
    th[:, 3] += math.pi                              # straddles the cut
    th[:, 5] += 2 * math.pi * rng.integers(-2, 3, K)  # whole turns change nothing
    th = th.astype(np.float32)
    mean, cov = S.sicp_moments_circular(ctx, th)
    mo, co = O.moments_circular(th.astype(np.float64))
    assert np.all(np.abs(_wrapped(mean - mo)) < 1e-12), np.abs(_wrapped(mean - mo)).max()
    assert np.allclose(cov, co, rtol=1e-12, atol=1e-14)
    # device tensors in, device tensors out
    m_d, c_d = S.sicp_moments_circular(ctx, torch.from_numpy(th).cuda())
    assert np.array_equal(m_d.cpu().numpy(), mean) and np.array_equal(c_d.cpu().numpy(), cov)


def test_moments_circular_errors(ctx):
    with pytest.raises(S.SicpError) as e:
        S.sicp_moments_circular(ctx, np.zeros((0, 6), np.float32))
    assert e.value.code == S.SICP_EINVAL


def test_teacher_forced_box_run_with_priors(ctx):
    """Whole iterations under the priors: at each step the oracle's state
    feeds one GPU gradient and one GPU Stein + Adam step, compared with the
    oracle's own step (same priors), which then advances."""
    d = synth.make_box_problem(0)
    ref, src = d["ref"], d["src"]
    S.sicp_set_reference(ctx, ref)
    T, m, seed = 30, 100, 7
    params = O.Params(T=T, m=m, lr=float(np.float32(0.01)), seed=seed, prior=1, mu=MU, sigma=SIGMA, kappa=KAPPA)
    p = _prior_params(T=T, m=m, lr=0.01, seed=seed, nn_mode=S.SICP_NN_GRID)
    th = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    N = src.shape[0]
    worst = 0.0
    for t in range(T):
        mb = O.minibatch(seed, t, N, m)
        th32 = th.astype(np.float32)
        g_gpu, _ = S.sicp_icp_grad(ctx, src, mb, th32, S.SICP_NN_GRID, want_nn=False)
        tg, mg, vg = th32.copy(), mom.astype(np.float32), vel.astype(np.float32)
        phi, _ = S.sicp_stein_adam(ctx, tg, mg, vg, g_gpu, N, t + 1, p)
        th_in = th32.astype(np.float64)
        G = _oracle_G(th_in, g_gpu.astype(np.float64), N)
        phi_ref = O.stein_phi(th_in, G, *O.bandwidths(th_in))
        e = np.abs(phi - phi_ref).max(1) / np.maximum(np.abs(phi_ref).max(1), 1e-5 * np.abs(G).max())
        worst = max(worst, e.max())
        O.step(ref, src, th, mom, vel, params, t)
    print(f"box with priors: worst phi rel err {worst:.2e}")
    assert worst <= 1e-4


def test_register_with_priors_uses_them(ctx):
    """The captured loop passes the priors to every Stein step: a run whose
    priors are centred away from the data's pose ends nearer the prior mean
    than the uniform-prior run, and both return the moments of the particles
    they return."""
    d = synth.make_box_problem(0)
    S.sicp_set_reference(ctx, d["ref"])
    base = dict(T=100, m=100, lr=0.01, seed=7, nn_mode=S.SICP_NN_GRID)
    th_u, mean_u, _ = S.sicp_register(ctx, d["src"], d["particles"], S.sicp_default_params(**base))
    far = (0.2, 0.2, 0.2, 0.0, 0.0, 0.0)
    p = S.sicp_default_params(prior=1, prior_mu=far, prior_sigma=(1e-6,) * 3, prior_kappa=(1e-3,) * 3, **base)
    th_p, mean_p, cov_p = S.sicp_register(ctx, d["src"], d["particles"], p)
    assert np.linalg.norm(mean_p[:3] - far[:3]) < np.linalg.norm(mean_u[:3] - far[:3])
    mo, co = O.moments(th_p.astype(np.float64))
    assert np.allclose(mean_p, mo, atol=1e-12) and np.allclose(cov_p, co, atol=1e-12)
