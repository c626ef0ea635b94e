"""The grid search reads its description from a constant-memory slot of the
context (32 slots), or, for contexts beyond them, from device memory.  Both
give the same answers, and contexts that interleave reference changes each
keep their own description.  Comparisons are exact (same kernels, same
arithmetic).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _grad_and_run(ctx, d):
    """Gradient, correspondences and a short registration on ctx's current reference."""
    mb = O.minibatch(3, 0, d["src"].shape[0], 100)
    g, nn = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_GRID)
    th, _, _ = S.sicp_register(ctx, d["src"], d["particles"],
                               S.sicp_default_params(T=20, m=100, lr=0.01, seed=2, nn_mode=S.SICP_NN_GRID))
    return g, nn, th


def test_constant_slots_and_device_fallback_agree():
    from paper_2106_03287_gb300 import build
    build.build()
    d = synth.make_box_problem(7, K=40)
    ctxs = [S.sicp_create(0) for _ in range(34)]
    try:
        for c in ctxs:   # every context takes a slot at its first reference build, while they last
            S.sicp_set_reference(c, d["ref"])
        first = _grad_and_run(ctxs[0], d)    # a constant-memory slot
        last = _grad_and_run(ctxs[-1], d)    # past the 32 slots: the device-memory copy
        for a, b in zip(first, last):
            assert np.array_equal(a, b)
    finally:
        for c in ctxs:
            S.sicp_destroy(c)


def test_interleaved_references_keep_their_own_description():
    from paper_2106_03287_gb300 import build
    build.build()
    d1, d2 = synth.make_box_problem(8, K=20), synth.make_kinect_problem(2, K=20)
    a, b, ref = S.sicp_create(0), S.sicp_create(0), S.sicp_create(0)
    try:
        S.sicp_set_reference(ref, d1["ref"])
        want1 = _grad_and_run(ref, d1)
        S.sicp_set_reference(ref, d2["ref"])
        want2 = _grad_and_run(ref, d2)
        S.sicp_set_reference(a, d1["ref"])
        S.sicp_set_reference(b, d2["ref"])   # after a's build: a must still search d1's cloud
        got1 = _grad_and_run(a, d1)
        got2 = _grad_and_run(b, d2)
        for x, y in zip(got1 + got2, want1 + want2):
            assert np.array_equal(x, y)
    finally:
        for c in (a, b, ref):
            S.sicp_destroy(c)
