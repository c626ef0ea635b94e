"""Failure detection without a GPU fault.

Bounded device waits: with sicp_set_wait_check every bounded wait of the
context's kernels waits for an event that never happens (the Stein update's
arrival counter one short, the persistent kernel's grid barrier one CTA
short, an mbarrier nothing arrives on in the tensor-core search) and gives up
after a few thousand polls.  Each call must return SICP_ETIMEOUT, write none
of its outputs, and leave the context usable: with the check off the same
call gives the result of a fresh context, bit for bit.

Memory budget: with sicp_set_memory_limit below what a call needs, the call
returns SICP_ENOMEM before it launches anything, its outputs untouched; with
the budget lifted the context works again.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
POLLS = 4096


@pytest.fixture(scope="module")
def kin():
    from paper_2106_03287_gb300 import build
    build.build()
    return synth.make_kinect_problem(21, M=20_000, N=4000, K=100)


def _fresh_register(d, p):
    c = S.sicp_create(0)
    try:
        S.sicp_set_reference(c, d["ref"])
        return S.sicp_register(c, d["src"], d["particles"], p)
    finally:
        S.sicp_destroy(c)


def _raw_register(ctx, d, p, sentinel):
    """sicp_register through the C ABI with output buffers preset to `sentinel`."""
    src, parts = np.ascontiguousarray(d["src"]), np.ascontiguousarray(d["particles"])
    K = parts.shape[0]
    out = np.full((K, 6), sentinel, np.float32)
    mean = np.full(6, sentinel, np.float64)
    cov = np.full(36, sentinel, np.float64)
    rc = S.lib().sicp_register(ctx, src.ctypes.data_as(ctypes.c_void_p), src.shape[0],
                               parts.ctypes.data_as(ctypes.c_void_p), K, ctypes.byref(p),
                               out.ctypes.data_as(ctypes.c_void_p), mean.ctypes.data_as(ctypes.c_void_p),
                               cov.ctypes.data_as(ctypes.c_void_p), 0)
    return rc, out, mean, cov


@pytest.mark.parametrize("mode", [S.SICP_NN_GRID, S.SICP_NN_BRUTE_BF16])
def test_registration_wait_gives_up_and_context_recovers(kin, mode):
    p = S.sicp_default_params(T=12, m=120, lr=0.03, seed=2, nn_mode=mode)
    want = _fresh_register(kin, p)
    ctx = S.sicp_create(0)
    try:
        S.sicp_set_reference(ctx, kin["ref"])
        S.sicp_set_wait_check(ctx, True, POLLS)
        rc, out, mean, cov = _raw_register(ctx, kin, p, 7.0)
        assert rc == S.SICP_ETIMEOUT, (rc, S.sicp_last_error(ctx))
        assert "gave up" in S.sicp_last_error(ctx)
        assert np.all(out == 7.0) and np.all(mean == 7.0) and np.all(cov == 7.0)
        S.sicp_set_wait_check(ctx, False, 0)
        got = S.sicp_register(ctx, kin["src"], kin["particles"], p)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
    finally:
        S.sicp_destroy(ctx)


def test_stein_update_wait_gives_up(kin):
    """K = 100: each block's update is split over four CTAs that wait for one
    another; with the check on every one of them gives up."""
    rng = np.random.default_rng(3)
    th = rng.normal(0, 0.1, (100, 6)).astype(np.float32)
    gbar = rng.normal(0, 1e-3, (100, 6)).astype(np.float32)
    p = S.sicp_default_params(lr=0.01)
    ctx = S.sicp_create(0)
    try:
        S.sicp_set_wait_check(ctx, True, POLLS)
        t1, m1, v1 = th.copy(), np.zeros_like(th), np.zeros_like(th)
        with pytest.raises(S.SicpError) as e:
            S.sicp_stein_adam(ctx, t1, m1, v1, gbar, 4000, 1, p)
        assert e.value.code == S.SICP_ETIMEOUT
        assert np.array_equal(t1, th) and not m1.any() and not v1.any()    # nothing written
        S.sicp_set_wait_check(ctx, False, 0)
        phi, h = S.sicp_stein_adam(ctx, t1, m1, v1, gbar, 4000, 1, p)
        th64 = th.astype(np.float64)
        G = O.log_post_grad(th64, gbar.astype(np.float64), 4000)
        phi_ref = O.stein_phi(th64, G, *O.bandwidths(th64))
        assert np.all(np.abs(phi - phi_ref).max(1) <= np.maximum(1e-4 * np.abs(phi_ref).max(1),
                                                                 1e-5 * np.abs(G).max()))
    finally:
        S.sicp_destroy(ctx)


def test_tensor_core_search_wait_gives_up(kin):
    q = (kin["ref"][:3000] + np.float32(0.004)).astype(np.float32)
    ctx = S.sicp_create(0)
    try:
        S.sicp_set_reference(ctx, kin["ref"])
        i32, d32 = S.sicp_nn(ctx, q, S.SICP_NN_BRUTE_FP32)
        S.sicp_set_wait_check(ctx, True, POLLS)
        with pytest.raises(S.SicpError) as e:
            S.sicp_nn(ctx, q, S.SICP_NN_BRUTE_BF16)
        assert e.value.code == S.SICP_ETIMEOUT
        # the exhaustive fp32 and grid searches have no device wait: unaffected
        assert np.array_equal(S.sicp_nn(ctx, q, S.SICP_NN_GRID)[0], i32)
        S.sicp_set_wait_check(ctx, False, 0)
        i16, d16 = S.sicp_nn(ctx, q, S.SICP_NN_BRUTE_BF16)
        assert np.array_equal(i16, i32) and np.array_equal(d16, d32)
    finally:
        S.sicp_destroy(ctx)


def test_batched_grid_barrier_gives_up():
    probs = synth.make_batched_problems(5, P=6, M_lo=3000, M_hi=9000)
    problems = [(d["ref"], d["src"], d["particles"]) for d in probs]
    p = S.sicp_default_params(T=6, m=100, lr=0.01, seed=0, nn_mode=S.SICP_NN_GRID)
    ctx = S.sicp_create(0)
    try:
        want = S.sicp_register_batched(ctx, problems, p)
        S.sicp_set_wait_check(ctx, True, POLLS)
        with pytest.raises(S.SicpError) as e:
            S.sicp_register_batched(ctx, problems, p)
        assert e.value.code == S.SICP_ETIMEOUT
        S.sicp_set_wait_check(ctx, False, 0)
        got = S.sicp_register_batched(ctx, problems, p)
        assert np.array_equal(np.concatenate(got[0]), np.concatenate(want[0]))
        assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])
    finally:
        S.sicp_destroy(ctx)


def test_memory_budget_gives_enomem_with_outputs_untouched(kin):
    p = S.sicp_default_params(T=5, m=100, lr=0.03, seed=1, nn_mode=S.SICP_NN_GRID)
    want = _fresh_register(kin, p)
    ctx = S.sicp_create(0)
    try:
        held = S.sicp_set_memory_limit(ctx, 0)
        S.sicp_set_reference(ctx, kin["ref"])
        held_ref = S.sicp_set_memory_limit(ctx, 0)
        assert held_ref > held
        # a run needs its source, minibatches, particles and scratch: more than 1 KB on top
        S.sicp_set_memory_limit(ctx, held_ref + 1024)
        rc, out, mean, cov = _raw_register(ctx, kin, p, -3.0)
        assert rc == S.SICP_ENOMEM, (rc, S.sicp_last_error(ctx))
        assert "budget" in S.sicp_last_error(ctx)
        assert np.all(out == -3.0) and np.all(mean == -3.0) and np.all(cov == -3.0)
        S.sicp_set_memory_limit(ctx, 0)
        got = S.sicp_register(ctx, kin["src"], kin["particles"], p)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        # a reference larger than the budget allows: ENOMEM; once the budget is lifted and the
        # reference set again, the context gives the fresh context's result
        big = np.concatenate([kin["ref"]] * 8)
        S.sicp_set_memory_limit(ctx, S.sicp_set_memory_limit(ctx, 0) + 4096)
        with pytest.raises(S.SicpError) as e:
            S.sicp_set_reference(ctx, big)
        assert e.value.code == S.SICP_ENOMEM
        S.sicp_set_memory_limit(ctx, 0)
        S.sicp_set_reference(ctx, kin["ref"])
        got = S.sicp_register(ctx, kin["src"], kin["particles"], p)
        assert np.array_equal(got[0], want[0])
    finally:
        S.sicp_destroy(ctx)
