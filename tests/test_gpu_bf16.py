"""The exhaustive search with tensor-core (bf16) distance tiles and an exact
fp32 re-check, through the C ABI.

It must return exactly what the fp32 exhaustive search returns: the same
indices (ties to the lowest index) and bit-identical float32 squared
distances, because the bf16 tiles only rule points out and every surviving
candidate is compared with the fp32 distance itself.  The gradients it feeds
are sums of the same per-query terms in another order: 1e-5 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
BF, FP = S.SICP_NN_BRUTE_BF16, S.SICP_NN_BRUTE_FP32


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _queries(ref, n_near, n_far, seed):
    rng = np.random.default_rng(seed)
    ext = float((ref.max(0) - ref.min(0)).max())
    near = ref[rng.integers(0, ref.shape[0], n_near)] + rng.normal(0, 0.01 * ext, (n_near, 3))
    far = ref.min(0) + rng.uniform(-1.0, 2.0, (n_far, 3)) * ext
    on = ref[rng.integers(0, ref.shape[0], 100)]
    return np.concatenate([near, far, on]).astype(np.float32)


@pytest.mark.parametrize("name", ["box", "kinect", "lidar", "uniform", "tiny"])
def test_bf16_search_equals_fp32_search(ctx, name):
    rng = np.random.default_rng(3)
    ref = {"box": lambda: synth.make_box_problem(1)["ref"],
           "kinect": lambda: synth.make_kinect_problem(1, M=20_001, N=100, K=1)["ref"],
           "lidar": lambda: synth.make_lidar_problem(1, K=1, az_step=0.8)["ref"],
           "uniform": lambda: rng.uniform(-2, 2, (3001, 3)).astype(np.float32),
           "tiny": lambda: rng.uniform(-1, 1, (5, 3)).astype(np.float32)}[name]()
    q = _queries(ref, 3001, 500, 4)
    S.sicp_set_reference(ctx, ref)
    i_bf, d_bf = S.sicp_nn(ctx, q, BF)
    i_fp, d_fp = S.sicp_nn(ctx, q, FP)
    assert np.array_equal(i_bf, i_fp)
    assert np.array_equal(d_bf.view(np.uint32), d_fp.view(np.uint32))
    if ref.shape[0] <= 20_001:   # and both are the oracle's answer up to fp64 near-ties
        idx_o, d2_o = O.nn(ref, q.astype(np.float64))
        bad = np.flatnonzero(i_bf != idx_o)
        d2g = ((ref[i_bf[bad]].astype(np.float64) - q[bad]) ** 2).sum(1)
        assert np.all(d2g <= d2_o[bad] * (1 + 1e-6) + 1e-300)


def test_bf16_ties_and_degenerate_clouds(ctx):
    rng = np.random.default_rng(5)
    base = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    ref = np.concatenate([base, base[:100], base[:50]])[rng.permutation(450)]
    S.sicp_set_reference(ctx, ref)
    idx, d2 = S.sicp_nn(ctx, ref, BF)
    for r in range(450):
        same = np.flatnonzero(np.all(ref == ref[r], axis=1))
        assert idx[r] == same.min() and d2[r] == 0.0
    for cloud in (np.array([[0.5, -0.25, 2.0]], np.float32), np.tile(np.float32([1, 2, 3]), (300, 1)),
                  np.c_[rng.uniform(-1, 1, (700, 2)), np.zeros(700)].astype(np.float32),
                  (1000.0 + rng.uniform(-0.01, 0.01, (900, 3))).astype(np.float32)):   # far from the origin
        S.sicp_set_reference(ctx, cloud)
        for n in (1, 127, 128, 129, 1000):
            q = (cloud.mean(0) + rng.uniform(-2, 2, (n, 3)) * (cloud.std(0).max() + 1e-3)).astype(np.float32)
            a = S.sicp_nn(ctx, q, BF)
            b = S.sicp_nn(ctx, q, FP)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_bf16_device_tensors(ctx):
    ref = synth.make_box_problem(2)["ref"]
    S.sicp_set_reference(ctx, ref)
    q = _queries(ref, 1000, 100, 6)
    a = S.sicp_nn(ctx, q, BF)
    b = S.sicp_nn(ctx, torch.from_numpy(q).cuda(), BF)
    assert np.array_equal(a[0], b[0].cpu().numpy()) and np.array_equal(a[1], b[1].cpu().numpy())


@pytest.mark.parametrize("K,m", [(1, 1), (3, 100), (32, 100), (200, 500)])
def test_bf16_gradient_matches_fp32(ctx, K, m):
    d = synth.make_kinect_problem(6, M=20_000, N=3000, K=K)
    S.sicp_set_reference(ctx, d["ref"])
    mb = O.minibatch(2, 0, d["src"].shape[0], m).astype(np.int32)
    g_bf, nn_bf = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=BF)
    g_fp, nn_fp = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=FP)
    assert np.array_equal(nn_bf, nn_fp)
    scale = np.abs(g_fp).max(1, keepdims=True)
    assert np.all(np.abs(g_bf - g_fp) <= 1e-5 * scale), np.abs(g_bf - g_fp).max()
    # and the oracle's gradient given those correspondences
    g_o = O.icp_grad_given_nn(d["ref"], d["src"], mb, d["particles"].astype(np.float64), nn_bf)
    assert np.all(np.abs(g_bf - g_o) <= 1e-4 * np.abs(g_o).max(1, keepdims=True) + 1e-12)


def test_bf16_registration_matches_fp32(ctx):
    """C1 (box, brute-force search): the whole run with either search."""
    d = synth.make_box_problem(0)
    S.sicp_set_reference(ctx, d["ref"])
    res = {}
    for mode in (BF, FP):
        p = S.sicp_default_params(T=100, m=100, lr=0.01, nn_mode=mode, seed=3)
        res[mode] = S.sicp_register(ctx, d["src"], d["particles"], p)
    m_bf, m_fp = res[BF][1], res[FP][1]
    assert np.all(np.abs(m_bf[:3] - m_fp[:3]) <= 1e-3)
    assert np.all(np.degrees(np.abs(m_bf[3:] - m_fp[3:])) <= 0.05)


def test_bf16_lidar_iteration_full_size(ctx):
    """C3 sizes: one iteration's 100,000 queries (K = 200, m = 500) against the
    ~112,000-point scan; every correspondence equals the fp32 search's."""
    d = synth.make_lidar_problem(1)
    S.sicp_set_reference(ctx, d["ref"])
    mb = O.minibatch(7, 0, d["src"].shape[0], 500).astype(np.int32)
    g_bf, nn_bf = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=BF)
    g_fp, nn_fp = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=FP)
    assert np.array_equal(nn_bf, nn_fp)
    assert np.all(np.abs(g_bf - g_fp) <= 1e-5 * np.abs(g_fp).max(1, keepdims=True))
