"""The allocation-free gradient entry point (sicp_icp_grad_noalloc) against
the context path (sicp_icp_grad with the exhaustive FP32 search).

The allocation-free variant serves callers that cannot allocate device
memory: its scratch is a fixed device array inside the library, so two calls
in a row reuse the same memory.  Its arithmetic is that of the context path
(same chunks, distance, tie rule, in-CTA reduction order and chunk fold), so
both calls must give the context path's gradients bit for bit, from one
chunk (m <= 256) to the four chunks and 256 particles that fill the scratch.
This file is collected last so that a run that stops at the first failure
has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2106_03287_gb300 import build
    build.build()


def _within(g, g_ref, ref, src, theta):
    X = float(max(np.abs(ref).max(), np.abs(src).max()) + np.abs(theta[:, :3]).max())
    floor = 16 * U32 * X * (1 + X)
    err = np.abs(g - g_ref).max(1)
    return np.all(err <= np.maximum(1e-4 * np.abs(g_ref).max(1), floor))


def test_noalloc_matches_context_path_twice():
    from paper_2106_03287_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    ctx = S.sicp_create(0)
    try:
        cases = [(synth.make_box_problem(11, K=32), (100, 300)),
                 (synth.make_kinect_problem(12, M=8000, N=3000, K=40), (100, 300, 700)),
                 (synth.make_kinect_problem(14, M=5000, N=2000, K=256), (1024, 513))]
        for d, ms in cases:
            N = d["src"].shape[0]
            S.sicp_set_reference(ctx, d["ref"])
            for t, m in enumerate(ms):
                mb = O.minibatch(9, t, N, m)
                g_ctx, _ = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], S.SICP_NN_BRUTE_FP32, want_nn=False)
                dev = [torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], mb, d["particles"])]
                out1 = S.sicp_icp_grad_noalloc(*dev).cpu().numpy()
                out2 = S.sicp_icp_grad_noalloc(*dev).cpu().numpy()   # second call, same scratch
                np.testing.assert_array_equal(out1, g_ctx)
                np.testing.assert_array_equal(out2, g_ctx)
                assert _within(out1, g_ctx, d["ref"], d["src"], d["particles"])
    finally:
        S.sicp_destroy(ctx)


def test_noalloc_out_of_range_minibatch_entries_add_nothing():
    """An index outside [0, N) in the device minibatch reads nothing: the sum
    is over the valid entries, still divided by m (checked against the FP64
    oracle on the valid entries)."""
    d = synth.make_box_problem(15, K=8)
    N, m = d["src"].shape[0], 100
    mb = O.minibatch(3, 0, N, m).copy()
    mb[[5, 50]] = [N, -7]
    keep = np.ones(m, bool)
    keep[[5, 50]] = False
    g_o, _, _ = O.icp_grad(d["ref"], d["src"], mb[keep], d["particles"].astype(np.float64))
    want = g_o * keep.sum() / m
    dev = [torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], mb, d["particles"])]
    got = S.sicp_icp_grad_noalloc(*dev).cpu().numpy()
    assert _within(got, want, d["ref"], d["src"], d["particles"])


def test_noalloc_rejects_sizes_beyond_its_limits():
    d = synth.make_box_problem(13, K=300)
    dev = [torch.from_numpy(a).cuda() for a in (d["ref"], d["src"], O.minibatch(1, 0, 500, 50), d["particles"])]
    with pytest.raises(S.SicpError) as e:
        S.sicp_icp_grad_noalloc(*dev)                      # K = 300 > 256
    assert e.value.code == S.SICP_EINVAL
    big_mb = torch.zeros(2000, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SicpError):
        S.sicp_icp_grad_noalloc(dev[0], dev[1], big_mb, dev[3][:8])   # m = 2000 > 1024
