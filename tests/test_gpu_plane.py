"""The point-to-plane metric (SICP_POINT_TO_PLANE) and the reference normals
it uses, through the C ABI against the oracle (reading R16 of oracle.c).

Tolerances:
- normals: the oracle ranks the neighbours by their exact fp64 distance, the
  GPU by its fp32 distance; the two sets are the same wherever the k-th and
  (k+1)-th fp64 distances are more than 1e-6 apart (relative), and there
  the float64 covariances agree and the eigenvectors (Jacobi on the GPU,
  LAPACK in the oracle) agree to float32 rounding, |n_gpu . n_oracle| >=
  1 - 1e-6, wherever the two smallest eigenvalues are apart (gap above 1e-3
  of the largest).  Where the neighbourhood is a near-tie, or the two
  smallest eigenvalues are not apart, the normal is not unique and only its
  length is checked;
- gradient: teacher-forced on the GPU's correspondences and normals, 1e-4
  relative per particle with the fp32 rounding floor of the point-to-point
  tests.
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
PL = S.SICP_POINT_TO_PLANE
MODES = [S.SICP_NN_GRID, S.SICP_NN_BRUTE_FP32, S.SICP_NN_BRUTE_BF16]


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _clouds():
    rng = np.random.default_rng(11)
    xy = rng.uniform(-1, 1, (3000, 2))
    return {
        "box": synth.make_box_problem(1)["ref"],
        "kinect": synth.make_kinect_problem(2, M=12_000, N=100, K=1)["ref"],
        "uniform": rng.uniform(-1, 1, (4000, 3)).astype(np.float32),
        "plane": np.c_[xy, 0.3 * xy[:, 0] - 0.2 * xy[:, 1] + 0.5].astype(np.float32),
        "far": (1000.0 + rng.uniform(-0.5, 0.5, (2000, 3))).astype(np.float32),
    }


@pytest.mark.parametrize("name", ["box", "kinect", "uniform", "plane", "far"])
@pytest.mark.parametrize("k", [3, 10, 32])
def test_normals_match_oracle(ctx, name, k):
    ref = _clouds()[name]
    S.sicp_set_reference(ctx, ref)
    n_g = S.sicp_reference_normals(ctx, k).astype(np.float64)
    assert np.all(np.isfinite(n_g)) and np.allclose(np.linalg.norm(n_g, axis=1), 1.0, atol=1e-6)
    n_o, w = O.normals(ref, k)
    defined = (w[:, 1] - w[:, 0]) > 1e-3 * np.maximum(w[:, 2], 1e-300)
    if k < ref.shape[0]:
        _, d2 = O.knn(ref, k + 1, with_d2=True)
        defined &= d2[:, k] > d2[:, k - 1] * (1 + 1e-6)      # the k-neighbourhood is unique
    dots = np.abs(np.einsum("ij,ij->i", n_g, n_o))
    assert np.all(dots[defined] >= 1 - 1e-6), dots[defined].min()
    if k >= 10 and name != "uniform":
        assert defined.mean() > 0.9
    if name == "plane" and k >= 10:
        # (three neighbours can be nearly collinear, and then the fp32 rounding of the
        # coordinates tilts their plane; both sides see the same rounding)
        true = np.array([0.3, -0.2, -1.0]) / np.linalg.norm([0.3, -0.2, -1.0])
        assert np.all(np.abs(n_g @ true) >= 1 - 1e-6)


def test_normals_device_output_and_degenerate_clouds(ctx):
    ref = _clouds()["box"]
    S.sicp_set_reference(ctx, ref)
    host = S.sicp_reference_normals(ctx, 10)
    dev = S.sicp_reference_normals(ctx, 10, device=True)
    assert np.array_equal(dev.cpu().numpy(), host)
    assert S.sicp_reference_normals(ctx, 10, want=False) is None
    # every point equal, or on one line: the normal is not defined, but it is finite and unit
    rng = np.random.default_rng(1)
    for cloud in (np.tile(np.float32([1, 2, 3]), (50, 1)),
                  np.c_[rng.uniform(-1, 1, 200), np.zeros(200), np.zeros(200)].astype(np.float32)):
        S.sicp_set_reference(ctx, cloud)
        n = S.sicp_reference_normals(ctx, 8).astype(np.float64)
        assert np.all(np.isfinite(n)) and np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)


def _check_plane_grad(ctx, ref, src, theta, mb, mode, normals):
    g, nn = S.sicp_icp_grad(ctx, src, mb, theta, mode | PL)
    th64 = theta.astype(np.float64)
    g_ref = O.icp_grad_given_nn(ref, src, mb, th64, nn, normals=normals.astype(np.float64))
    X = float(max(np.abs(ref).max(), np.abs(src).max()) + np.abs(theta[:, :3]).max())
    floor = 16 * U32 * X * (1 + X)
    err = np.abs(g - g_ref).max(1)
    assert np.all(err <= np.maximum(1e-4 * np.abs(g_ref).max(1), floor)), (err / np.abs(g_ref).max(1)).max()
    # the metric changes the residual, not the correspondences
    _, nn_pp = S.sicp_icp_grad(ctx, src, mb, theta, mode)
    assert np.array_equal(nn, nn_pp)
    return g


@pytest.mark.parametrize("mode", MODES)
def test_plane_gradient_box(ctx, mode):
    d = synth.make_box_problem(3)
    S.sicp_set_reference(ctx, d["ref"])
    nrm = S.sicp_reference_normals(ctx, 10)
    mb = O.minibatch(5, 0, d["src"].shape[0], 100)
    g = _check_plane_grad(ctx, d["ref"], d["src"], d["particles"], mb, mode, nrm)
    g_pp, _ = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode)
    assert np.abs(g - g_pp).max() > 1e-3 * np.abs(g_pp).max()     # it is another metric


@pytest.mark.parametrize("mode", MODES)
def test_plane_gradient_kinect_ragged(ctx, mode):
    d = synth.make_kinect_problem(4, M=20_000, N=4000, K=24)
    S.sicp_set_reference(ctx, d["ref"])
    nrm = S.sicp_reference_normals(ctx, 12)
    for m in (1, 33, 300):
        mb = O.minibatch(6, 3, d["src"].shape[0], m)
        _check_plane_grad(ctx, d["ref"], d["src"], d["particles"], mb, mode, nrm)


def test_plane_gradient_full_size_kinect(ctx):
    """Kinect sizes (50k reference, 30,000 queries): one iteration, every particle."""
    d = synth.make_kinect_problem(0)
    S.sicp_set_reference(ctx, d["ref"])
    nrm = S.sicp_reference_normals(ctx, 10)
    mb = O.minibatch(1, 0, d["src"].shape[0], 300)
    _check_plane_grad(ctx, d["ref"], d["src"], d["particles"], mb, S.SICP_NN_GRID, nrm)


def test_plane_bf16_equals_fp32_and_lidar_full_size(ctx):
    """The tensor-core search finds the fp32 search's correspondences, so with
    the point-to-plane metric the two gradients are sums of the same terms in
    another order (1e-5 relative); at LiDAR sizes (100,000 queries against the
    ~112,000-point scan) as well."""
    d = synth.make_lidar_problem(1)
    S.sicp_set_reference(ctx, d["ref"])
    S.sicp_reference_normals(ctx, 10, want=False)
    mb = O.minibatch(7, 0, d["src"].shape[0], 500)
    g_bf, nn_bf = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_BRUTE_BF16 | PL)
    g_fp, nn_fp = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_BRUTE_FP32 | PL)
    assert np.array_equal(nn_bf, nn_fp)
    assert np.all(np.abs(g_bf - g_fp) <= 1e-5 * np.abs(g_fp).max(1, keepdims=True))


def test_plane_run_recovers_known_pose(ctx):
    """K = 1 with the point-to-plane metric on a noise-free box lands on the
    generating pose (1 mm, 0.05 deg), as the oracle does."""
    d = synth.make_box_problem(0, K=1, noise=0.0)
    S.sicp_set_reference(ctx, d["ref"])
    S.sicp_reference_normals(ctx, 10, want=False)
    p = S.sicp_default_params(T=300, m=100, lr=0.01, seed=7, nn_mode=S.SICP_NN_GRID | PL)
    th, _, _ = S.sicp_register(ctx, d["src"], d["particles"], p)
    err = th[0].astype(np.float64) - d["theta_true"]
    assert np.abs(err[:3]).max() < 1e-3 and np.abs(err[3:]).max() < math.radians(0.05)


def test_plane_teacher_forced_box_run(ctx):
    """Every iteration: the oracle's state into one GPU gradient (point-to-plane)
    and one GPU Stein + Adam step, compared with the oracle's step on the GPU's
    normals, which then advances."""
    d = synth.make_box_problem(0)
    ref, src = d["ref"], d["src"]
    S.sicp_set_reference(ctx, ref)
    nrm = S.sicp_reference_normals(ctx, 10).astype(np.float64)
    T, m, seed = 40, 100, 7
    params = O.Params(T=T, m=m, lr=float(np.float32(0.01)), seed=seed, normals=nrm)
    p = S.sicp_default_params(T=T, m=m, lr=0.01, seed=seed, nn_mode=S.SICP_NN_GRID | PL)
    th = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    N = src.shape[0]
    worst = 0.0
    for t in range(T):
        mb = O.minibatch(seed, t, N, m)
        th32 = th.astype(np.float32)
        g_gpu = _check_plane_grad(ctx, ref, src, th32, mb, S.SICP_NN_GRID, nrm)
        tg, mg, vg = th32.copy(), mom.astype(np.float32), vel.astype(np.float32)
        phi, _ = S.sicp_stein_adam(ctx, tg, mg, vg, g_gpu, N, t + 1, p)
        th_in = th32.astype(np.float64)
        G = O.log_post_grad(th_in, g_gpu.astype(np.float64), N)
        phi_ref = O.stein_phi(th_in, G, *O.bandwidths(th_in))
        e = np.abs(phi - phi_ref).max(1) / np.maximum(np.abs(phi_ref).max(1), 1e-5 * np.abs(G).max())
        worst = max(worst, e.max())
        O.step(ref, src, th, mom, vel, params, t)
    print(f"box point-to-plane: worst phi rel err {worst:.2e}")
    assert worst <= 1e-4


def test_plane_errors(ctx):
    d = synth.make_box_problem(2)
    S.sicp_set_reference(ctx, d["ref"])
    mb = O.minibatch(1, 0, d["src"].shape[0], 50)
    with pytest.raises(S.SicpError) as e:                    # no normals yet
        S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_GRID | PL)
    assert e.value.code == S.SICP_ENOREF
    for k in (2, 33, d["ref"].shape[0] + 1):
        with pytest.raises(S.SicpError) as e:
            S.sicp_reference_normals(ctx, k)
        assert e.value.code == S.SICP_EINVAL
    S.sicp_reference_normals(ctx, 10, want=False)
    with pytest.raises(S.SicpError) as e:                    # the learned field has no reference point
        S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_SURROGATE | PL)
    assert e.value.code == S.SICP_EINVAL
    S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_GRID | PL)
    S.sicp_set_reference(ctx, d["ref"])                         # a new reference drops the normals
    with pytest.raises(S.SicpError) as e:
        S.sicp_register(ctx, d["src"], d["particles"],
                        S.sicp_default_params(T=3, m=50, nn_mode=S.SICP_NN_GRID | PL))
    assert e.value.code == S.SICP_ENOREF
