"""Per-iteration telemetry of registration runs (sicp_set_telemetry) against
independent computations on the same states.

Row t describes iteration t.  Its particle mean and standard deviation must
equal the float64 moments of the particles the iteration started from: the
result of the same run stopped after t iterations, which equals the first t
iterations of the longer run bit for bit.  Its mean correspondence distance
must equal the FP64 oracle's nearest-neighbour distances of the same
queries, which are those particles applied to the minibatch row of
iteration t.  The telemetry kernels write nothing the run reads, so results
with telemetry on and off must be bit-identical.  In a run on the learned
field, the learned share of each iteration must account for exactly the
fallback queries that sicp_stats counts.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kin():
    from paper_2106_03287_gb300 import build
    build.build()
    d = synth.make_kinect_problem(41, M=20_000, N=4000, K=100)
    c = S.sicp_create(0)
    S.sicp_set_reference(c, d["ref"])
    yield c, d, O.KDTree(d["ref"])
    S.sicp_destroy(c)


def _run(ctx, d, parts, p, tel):
    S.sicp_set_telemetry(ctx, tel)
    try:
        out = S.sicp_register(ctx, d["src"], parts, p)
        rows = S.sicp_read_telemetry(ctx)
    finally:
        S.sicp_set_telemetry(ctx, False)
    return out, rows


def _check_rows(ctx, d, tree, parts, kw, seed, mode, rows, ts, indep):
    N, m, K = d["src"].shape[0], kw["m"], parts.shape[0]
    for t in ts:
        p_t = S.sicp_default_params(T=t, seed=seed, nn_mode=mode, **kw)
        x = (S.sicp_register(ctx, d["src"], parts, p_t)[0] if t > 0 else parts).astype(np.float64)
        np.testing.assert_allclose(rows[t, :6], x.mean(0), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(rows[t, 6:12], x.std(0, ddof=1), rtol=1e-5, atol=1e-7)
        assert rows[t, 14] == t and rows[t, 15] == 1.0 and rows[t, 13] == 0.0
        dist = []
        for j in range(K):
            mb = O.minibatch(seed + j if indep else seed, t, N, m)
            _, d2 = tree.nn(O.transform(x[j], d["src"][mb]))
            dist.append(np.sqrt(d2))
        want = np.mean(np.concatenate(dist))
        assert abs(rows[t, 12] - want) <= 1e-5 * want, (t, rows[t, 12], want)


@pytest.mark.parametrize("mode", [S.SICP_NN_GRID, S.SICP_NN_BRUTE_FP32, S.SICP_NN_BRUTE_BF16])
def test_rows_match_the_states_and_the_oracle(kin, mode):
    ctx, d, tree = kin
    parts = d["particles"][:40]
    kw = dict(m=150, lr=0.03)
    T, seed = 8, 13
    p = S.sicp_default_params(T=T, seed=seed, nn_mode=mode, **kw)
    off, rows0 = _run(ctx, d, parts, p, False)
    on, rows = _run(ctx, d, parts, p, True)
    assert rows0.shape == (0, 16) and rows.shape == (T, 16)
    for a, b in zip(on, off):
        assert np.array_equal(a, b)
    _check_rows(ctx, d, tree, parts, kw, seed, mode, rows, (0, 3, T - 1), indep=False)


def test_independent_runs_rows(kin):
    ctx, d, tree = kin
    parts = d["particles"][:6]
    kw = dict(m=120, lr=0.03)
    mode = S.SICP_NN_GRID | S.SICP_INDEPENDENT
    p = S.sicp_default_params(T=6, seed=21, nn_mode=mode, **kw)
    off, _ = _run(ctx, d, parts, p, False)
    on, rows = _run(ctx, d, parts, p, True)
    assert np.array_equal(on[0], off[0])
    _check_rows(ctx, d, tree, parts, kw, 21, mode, rows, (0, 5), indep=True)


def test_continued_run_numbers_its_rows_from_t0(kin):
    ctx, d, _ = kin
    parts = d["particles"][:20]
    p = S.sicp_default_params(T=5, m=100, lr=0.03, seed=4, nn_mode=S.SICP_NN_GRID)
    _, whole = _run(ctx, d, parts, S.sicp_default_params(T=10, m=100, lr=0.03, seed=4, nn_mode=S.SICP_NN_GRID), True)
    S.sicp_register(ctx, d["src"], parts, p)
    state = S.sicp_export_state(ctx)
    S.sicp_set_telemetry(ctx, True)
    try:
        S.sicp_import_state(ctx, state)
        S.sicp_resume(ctx, d["src"], p)
        rows = S.sicp_read_telemetry(ctx)
    finally:
        S.sicp_set_telemetry(ctx, False)
    assert np.array_equal(rows[:, 14], np.arange(5, 10, dtype=np.float32))
    assert np.array_equal(rows, whole[5:])   # the same iterations, the same rows


def test_learned_share_accounts_for_the_fallback_queries(kin):
    ctx, d, _ = kin
    S.sicp_surrogate_train(ctx, 1 << 21, seed=3, epochs=10, batch=4096, lr=1e-3)
    parts = d["particles"][:40]
    m, T, Ts = 150, 10, 6
    p = S.sicp_default_params(T=T, m=m, lr=0.03, seed=2, nn_mode=S.SICP_NN_SURROGATE, surrogate_iters=Ts)
    off, _ = _run(ctx, d, parts, p, False)
    S.sicp_stats(ctx, True)
    on, rows = _run(ctx, d, parts, p, True)
    st = S.sicp_stats(ctx, False)
    for a, b in zip(on, off):
        assert np.array_equal(a, b)
    q = parts.shape[0] * m
    fallback = np.rint((1.0 - rows[:Ts, 13].astype(np.float64)) * q).sum()
    assert st[6] == Ts * q and fallback == st[7], (st[6], st[7], fallback, rows[:Ts, 13])
    assert np.all((rows[:Ts, 13] >= 0) & (rows[:Ts, 13] <= 1)) and np.all(rows[Ts:, 13] == 0)
    assert rows[:Ts, 13].max() > 0          # the trained field answers some queries
    assert np.all(np.isfinite(rows)) and np.all(rows[:, 12] > 0)


def test_read_without_rows_and_bad_arguments(kin):
    ctx, d, _ = kin
    S.sicp_register(ctx, d["src"], d["particles"][:8], S.sicp_default_params(T=3, m=50, seed=1))
    assert S.sicp_read_telemetry(ctx).shape == (0, 16)
    n = ctypes.c_int32(-1)
    assert S.lib().sicp_read_telemetry(ctx, None, 0, ctypes.byref(n)) == S.SICP_OK and n.value == 0
    assert S.lib().sicp_read_telemetry(ctx, None, -1, None) == S.SICP_EINVAL
    assert S.lib().sicp_read_telemetry(ctx, None, 4, None) == S.SICP_EINVAL


def test_single_particle_and_empty_run(kin):
    """K = 1: the spread columns are 0 (divisor K - 1 undefined), the mean is
    the particle itself and the distance that of its own queries; T = 0
    records no rows and leaves the particles as they came in."""
    ctx, d, tree = kin
    parts = d["particles"][:1]
    N, m, seed = d["src"].shape[0], 64, 8
    p = S.sicp_default_params(T=4, m=m, lr=0.03, seed=seed, nn_mode=S.SICP_NN_GRID)
    _, rows = _run(ctx, d, parts, p, True)
    assert rows.shape == (4, 16) and np.all(rows[:, 6:12] == 0) and np.all(rows[:, 15] == 1.0)
    np.testing.assert_allclose(rows[0, :6], parts[0], rtol=1e-6, atol=1e-7)
    _, d2 = tree.nn(O.transform(parts[0].astype(np.float64), d["src"][O.minibatch(seed, 0, N, m)]))
    want = np.sqrt(d2).mean()
    assert abs(rows[0, 12] - want) <= 1e-5 * want
    p0 = S.sicp_default_params(T=0, m=m, lr=0.03, seed=seed, nn_mode=S.SICP_NN_GRID)
    (th, _, _), rows0 = _run(ctx, d, parts, p0, True)
    assert np.array_equal(th, parts) and rows0.shape == (0, 16)
