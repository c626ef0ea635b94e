"""The grid search's gradient kernel against the exhaustive fp32 search on
the same GPU-transformed queries.

Both return the exact nearest point under the fp32 squared distance with
ties to the lowest index, so their correspondences must be equal bit for
bit, for particles near the answer (queries near the surface), spread as
initialised, far outside the reference's grid, with K = 200,
K = 1, and on a cloud with duplicated points; the mean gradients sum the
same terms in another order (1e-5 relative).
"""
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


def _particles_near(d, K, spread_t, spread_r, seed):
    rng = np.random.default_rng(seed)
    th = np.asarray(d.get("theta_true", np.zeros(6)), np.float64)
    out = th + np.c_[rng.normal(0, spread_t, (K, 3)), rng.normal(0, spread_r, (K, 3))]
    return out.astype(np.float32)


def _cases():
    kin = synth.make_kinect_problem(31, M=20_000, N=4000, K=100)
    box = synth.make_box_problem(32, K=48)
    rng = np.random.default_rng(33)
    base = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    dup = dict(ref=np.concatenate([base, base[:500], base[:100]]), src=base[rng.permutation(3000)[:800]],
               particles=(rng.normal(0, 0.02, (40, 6))).astype(np.float32))
    return [
        ("kinect converged", kin, _particles_near(kin, 100, 0.01, 0.005, 1)),     # mostly certified
        ("kinect spread", kin, kin["particles"]),                                 # many queued
        ("kinect far", kin, _particles_near(kin, 100, 1.5, 0.6, 2)),              # far outside the grid
        ("kinect K=200", kin, _particles_near(kin, 200, 0.03, 0.01, 3)),          # no pose table
        ("kinect K=1", kin, _particles_near(kin, 1, 0.01, 0.005, 4)),
        ("box", box, box["particles"]),
        ("duplicates", dup, dup["particles"]),
    ]


def test_grid_gradient_correspondences_equal_exhaustive_search(ctx):
    for name, d, parts in _cases():
        S.sicp_set_reference(ctx, d["ref"])
        N = d["src"].shape[0]
        for m in (1, 97, 300):
            mb = O.minibatch(5, m, N, min(m, N))
            g_grid, nn_grid = S.sicp_icp_grad(ctx, d["src"], mb, parts, S.SICP_NN_GRID)
            g_fp32, nn_fp32 = S.sicp_icp_grad(ctx, d["src"], mb, parts, S.SICP_NN_BRUTE_FP32)
            assert np.array_equal(nn_grid, nn_fp32), (name, m, np.sum(nn_grid != nn_fp32))
            scale = max(np.abs(g_fp32).max(), 1e-30)
            assert np.abs(g_grid - g_fp32).max() <= 1e-5 * scale + 1e-30, name   # same terms, other order


def test_half_warp_search_of_independent_runs_equals_warp_search(ctx):
    """Independent runs search with half-warps (two queries per warp), a
    single-particle run with whole warps.  Both are exact with the same tie
    rule, so run j of an independent registration equals the K = 1 run with
    seed + j bit for bit: on the kinect scene with spread, converged and far
    initial poses (far: the coarse level), and an odd K (the last warp has an
    idle half)."""
    kin = synth.make_kinect_problem(31, M=20_000, N=4000, K=100)
    S.sicp_set_reference(ctx, kin["ref"])
    parts = np.concatenate([kin["particles"][:6], _particles_near(kin, 6, 0.01, 0.005, 5),
                            _particles_near(kin, 5, 1.5, 0.6, 6)])
    kw = dict(T=15, m=150, lr=0.03)
    th, _, _ = S.sicp_register(ctx, kin["src"], parts,
                               S.sicp_default_params(seed=11, nn_mode=S.SICP_NN_GRID | S.SICP_INDEPENDENT, **kw))
    S.sicp_stats(ctx, True)
    S.sicp_register(ctx, kin["src"], parts,
                    S.sicp_default_params(seed=11, nn_mode=S.SICP_NN_GRID | S.SICP_INDEPENDENT, **kw))
    st = S.sicp_stats(ctx, False)
    assert st[4] > 0                       # some queries took the coarse level
    for j in range(parts.shape[0]):
        one, _, _ = S.sicp_register(ctx, kin["src"], parts[j:j + 1],
                                    S.sicp_default_params(seed=11 + j, nn_mode=S.SICP_NN_GRID, **kw))
        assert np.array_equal(th[j], one[0]), j
