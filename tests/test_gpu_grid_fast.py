"""The grid search's lane-per-query gradient kernel (neighbourhood lists of
the fine cells, certified answers, a work queue for the rest) against the
exact searches.

Both grid gradient kernels return the exact nearest point under the fp32
squared distance with ties to the lowest index, the same as the exhaustive
fp32 search, and compute the same per-query gradient terms: the
correspondences must equal the exhaustive search's bit for bit, and a whole
registration must equal the warp-per-query kernel's (selected in a child
process by SICP_GRID_WARP_SEARCH) bit for bit.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_fast_kernel_correspondences_equal_exhaustive_search(ctx):
    for name, d, parts in _cases():
        S.sicp_set_reference(ctx, d["ref"])
        N = d["src"].shape[0]
        for m in (1, 97, 300):
            mb = O.minibatch(5, m, N, min(m, N))
            S.sicp_stats(ctx, True)
            g_grid, nn_grid = S.sicp_icp_grad(ctx, d["src"], mb, parts, S.SICP_NN_GRID)
            st = S.sicp_stats(ctx, False)
            g_fp32, nn_fp32 = S.sicp_icp_grad(ctx, d["src"], mb, parts, S.SICP_NN_BRUTE_FP32)
            assert np.array_equal(nn_grid, nn_fp32), (name, m, np.sum(nn_grid != nn_fp32))
            scale = max(np.abs(g_fp32).max(), 1e-30)
            assert np.abs(g_grid - g_fp32).max() <= 1e-5 * scale + 1e-30, name   # same terms, other order
            print(f"{name} m={m}: {int(st[10])} of {int(st[0])} queries queued for the warp search")


_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_2106_03287_gb300 as S
from paper_2106_03287_gb300 import synth
d = synth.make_kinect_problem(34, M=20_000, N=4000, K=100)
c = S.sicp_create(0)
S.sicp_set_reference(c, d["ref"])
out = {{}}
for name, mode, T in (("stein", S.SICP_NN_GRID, 40), ("independent", S.SICP_NN_GRID | S.SICP_INDEPENDENT, 25)):
    p = S.sicp_default_params(T=T, m=150, lr=0.03, seed=9, nn_mode=mode)
    th, mean, cov = S.sicp_register(c, d["src"], d["particles"], p)
    out[name] = th.tobytes().hex()
S.sicp_destroy(c)
print(json.dumps(out))
"""


def _run_child(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_registration_equals_warp_search_kernel_bit_for_bit():
    fast = _run_child({})
    warp = _run_child({"SICP_GRID_WARP_SEARCH": "1"})
    for k in fast:
        assert fast[k] == warp[k], k
