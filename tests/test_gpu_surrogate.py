"""The learned closest-point field on the GPU (through the C ABI) against the
oracle's FP64 network.

Tolerances.  The kernels round features, weights, activations and the
backward deltas to bf16 and accumulate in fp32; the oracle's bf16ops mode
rounds at the same points, so the two differ only by fp32 accumulation order
and by the rare bf16 rounding decision that an fp32 and an fp64 value take
differently (one bf16 ulp, 2^-8 relative, of one activation).  Measured on a
GB300: gradient relative L2 error 1.4e-3 against the bf16 oracle and 6.5e-3
against the plain FP64 one; the bounds below (5e-3 and 2e-2) leave a factor
of about 3.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

NP = 33040
oW2 = 128 * 112 + 128
ob2 = oW2 + 128 * 128
oW3 = ob2 + 128
ob3 = oW3 + 16 * 128
BLOCKS = {"W1": (0, 128 * 112), "b1": (128 * 112, oW2), "W2": (oW2, ob2), "b2": (ob2, oW3), "W3": (oW3, ob3),
          "b3": (ob3, NP)}


@pytest.fixture(scope="module")
def ctx():
    from paper_2106_03287_gb300 import build
    build.build()
    c = S.sicp_create(0)
    yield c
    S.sicp_destroy(c)


def _random_params(seed):
    rng = np.random.default_rng(seed)
    W = np.zeros(NP)
    W[:128 * 112] = rng.normal(0, math.sqrt(2 / 112), 128 * 112)
    W[128 * 112:oW2] = rng.normal(0, 0.05, 128)
    W[oW2:ob2] = rng.normal(0, math.sqrt(2 / 128), 128 * 128)
    W[ob2:oW3] = rng.normal(0, 0.05, 128)
    W[oW3:oW3 + 4 * 128] = rng.normal(0, 0.1, 4 * 128)
    W[ob3:ob3 + 4] = rng.normal(0, 0.1, 4)
    return W.astype(np.float32)


@pytest.mark.parametrize("n,seed", [(128, 1), (384, 2), (1024, 3)])
def test_loss_grad_matches_bf16_oracle(ctx, n, seed):
    rng = np.random.default_rng(seed)
    W = _random_params(seed)
    qn = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    ds = rng.normal(0, 0.05, (n, 3)).astype(np.float32)
    lg, gg = S.sicp_surrogate_loss_grad(ctx, W, qn, ds, 0.1, 0.02)
    l16, g16 = O.mlp_loss_grad(W, qn, ds, lam=0.1, delta=0.02, bf16ops=True)
    l64, g64 = O.mlp_loss_grad(W, qn, ds, lam=0.1, delta=0.02)
    assert abs(lg - l16) <= 1e-3 * abs(l16)
    e16 = np.linalg.norm(gg - g16) / np.linalg.norm(g16)
    e64 = np.linalg.norm(gg - g64) / np.linalg.norm(g64)
    assert e16 <= 5e-3, e16
    assert e16 < 0.5 * e64, (e16, e64)     # the kernels round where the bf16 oracle rounds
    # against the plain FP64 network, an absolute bound: bf16 keeps 8 significant bits (relative
    # rounding 2^-9 per value), and the features, weights, two activations and the deltas are each
    # rounded once on the way to a weight gradient; measured 6.5e-3, bound 2e-2
    assert e64 <= 2e-2, e64
    assert abs(lg - l64) <= 2e-2 * abs(l64), (lg, l64)
    for name, (a, b) in BLOCKS.items():
        ref = g16[a:b]
        if name in ("W3", "b3"):
            ref, got = ref.reshape(16, -1)[:4], gg[a:b].reshape(16, -1)[:4]   # rows 4..15 are dead outputs
            assert np.all(gg[a:b].reshape(16, -1)[4:] == 0.0)
        else:
            got = gg[a:b]
        assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref), name


def test_loss_grad_leaves_context_surrogate(ctx):
    W = _random_params(7)
    norm4 = np.array([0.0, 0.0, 1.0, 2.0], np.float32)
    S.sicp_surrogate_params(ctx, W, norm4)
    rng = np.random.default_rng(8)
    S.sicp_surrogate_loss_grad(ctx, _random_params(9), rng.uniform(-1, 1, (256, 3)), rng.normal(0, .1, (256, 3)))
    p, n = S.sicp_surrogate_params(ctx)
    assert np.array_equal(p, W) and np.array_equal(n, norm4)


@pytest.mark.parametrize("n", [1, 255, 256, 1000])
def test_infer_matches_oracle_forward(ctx, n):
    W = _random_params(11)
    norm4 = np.array([0.1, -0.2, 0.3, 1.7], np.float32)
    S.sicp_surrogate_params(ctx, W, norm4)
    rng = np.random.default_rng(n)
    q = rng.uniform(-1.5, 1.5, (n, 3)).astype(np.float32)
    d, c = S.sicp_surrogate_infer(ctx, q)
    qn = ((q - norm4[:3]) / norm4[3]).astype(np.float32)     # the kernel's fp32 normalisation
    out = O.mlp_forward(W, qn, bf16ops=True)
    dref = norm4[3] * out[:, :3]
    cref = 1.0 / (1.0 + np.exp(-out[:, 3]))
    assert np.abs(d - dref).max() <= 1e-2 * max(1.0, np.abs(dref).max())
    assert np.abs(c - cref).max() <= 5e-3
    # device tensors give the same answer
    dd, cd = S.sicp_surrogate_infer(ctx, torch.from_numpy(q).cuda())
    assert np.array_equal(dd.cpu().numpy(), d) and np.array_equal(cd.cpu().numpy(), c)


def test_empty_infer(ctx):
    S.sicp_surrogate_params(ctx, _random_params(1), np.array([0, 0, 0, 1], np.float32))
    d, c = S.sicp_surrogate_infer(ctx, np.zeros((0, 3), np.float32))
    assert d.shape == (0, 3) and c.shape == (0,)


def _constant_field(b, conf_logit, centre=(0.0, 0.0, 0.0), s=1.5):
    """Parameters whose output is exactly (b, conf_logit) for every query:
    W3 = 0, so o = b3 whatever the hidden layers compute."""
    W = _random_params(3)
    W[oW3:ob3] = 0.0
    W[ob3:] = 0.0
    W[ob3:ob3 + 3] = b
    W[ob3 + 3] = conf_logit
    return W, np.array(list(centre) + [s], np.float32)


def test_icp_grad_constant_field_matches_oracle(ctx):
    """A field whose prediction is the constant displacement s*b: the
    gradient of every query is that of the residual e = -s*b."""
    d = synth.make_box_problem(3, M=2000, N=500, K=16)
    S.sicp_set_reference(ctx, d["ref"])
    b = np.array([0.01, -0.02, 0.005], np.float32)
    W, norm4 = _constant_field(b, 30.0)
    S.sicp_surrogate_params(ctx, W, norm4)
    mb = O.minibatch(4, 0, d["src"].shape[0], 100).astype(np.int32)
    th = d["particles"]
    g, _ = S.sicp_icp_grad(ctx, d["src"], mb, th, mode=S.SICP_NN_SURROGATE, want_nn=False)
    e = -(norm4[3].astype(np.float64) * b.astype(np.float64))
    want = np.zeros((th.shape[0], 6))
    src = d["src"][mb].astype(np.float64)
    for j in range(th.shape[0]):
        R, dR = O.rotation(th[j])
        want[j, :3] = e
        for a in range(3):
            want[j, 3 + a] = np.mean((src @ dR[a].T) @ e)
    scale = np.abs(want).max(1, keepdims=True)
    assert np.all(np.abs(g - want) <= 1e-5 * scale + 1e-7), np.abs(g - want).max()


def test_icp_grad_unconfident_field_is_the_exact_search(ctx):
    """With confidence ~0 everywhere every query falls back to the exact grid
    search, so the surrogate mode gives the grid mode's gradient."""
    d = synth.make_kinect_problem(5, M=20_000, N=3000, K=24)
    S.sicp_set_reference(ctx, d["ref"])
    W, norm4 = _constant_field(np.zeros(3, np.float32), -30.0, centre=(0.0, 0.0, 2.0), s=2.0)
    S.sicp_surrogate_params(ctx, W, norm4)
    mb = O.minibatch(6, 2, d["src"].shape[0], 300).astype(np.int32)
    S.sicp_stats(ctx, True)
    g_s, _ = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=S.SICP_NN_SURROGATE, want_nn=False)
    st = S.sicp_stats(ctx, False)
    g_e, _ = S.sicp_icp_grad(ctx, d["src"], mb, d["particles"], mode=S.SICP_NN_GRID, want_nn=False)
    assert st[6] == 24 * 300 and st[7] == 24 * 300
    scale = np.abs(g_e).max(1, keepdims=True)
    assert np.all(np.abs(g_s - g_e) <= 1e-5 * scale), np.abs(g_s - g_e).max()


def test_errors(ctx):
    c = S.sicp_create(0)
    try:
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_params(c)
        assert e.value.code == S.SICP_ENOSURROGATE
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_infer(c, np.zeros((4, 3), np.float32))
        assert e.value.code == S.SICP_ENOSURROGATE
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_train(c, 4096)
        assert e.value.code == S.SICP_ENOREF
        d = synth.make_box_problem(1)
        S.sicp_set_reference(c, d["ref"])
        p = S.sicp_default_params(T=5, m=50, nn_mode=S.SICP_NN_SURROGATE, surrogate_iters=3)
        with pytest.raises(S.SicpError) as e:
            S.sicp_register(c, d["src"], d["particles"], p)
        assert e.value.code == S.SICP_ENOSURROGATE
        for kw in [dict(n_queries=100), dict(n_queries=4096, epochs=0), dict(n_queries=4096, batch=100),
                   dict(n_queries=4096, lr=0.0), dict(n_queries=4096, batch=131072)]:
            with pytest.raises(S.SicpError) as e:
                S.sicp_surrogate_train(c, **kw)
            assert e.value.code == S.SICP_EINVAL, kw
        W = _random_params(1)
        bad = W.copy()
        bad[5] = np.nan
        for params, norm4 in [(bad, [0, 0, 0, 1]), (W, [0, 0, 0, 0]), (W, [np.inf, 0, 0, 1])]:
            with pytest.raises(S.SicpError) as e:
                S.sicp_surrogate_params(c, params, np.array(norm4, np.float32))
            assert e.value.code == S.SICP_EINVAL
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_loss_grad(c, W, np.zeros((100, 3)), np.zeros((100, 3)))
        assert e.value.code == S.SICP_EINVAL
        S.sicp_surrogate_params(c, W, np.array([0, 0, 0, 1], np.float32))
        p.surrogate_min_conf = 1.5
        with pytest.raises(S.SicpError) as e:
            S.sicp_register(c, d["src"], d["particles"], p)
        assert e.value.code == S.SICP_EINVAL
        p.surrogate_min_conf = 0.5
        p.surrogate_iters = -1
        with pytest.raises(S.SicpError) as e:
            S.sicp_register(c, d["src"], d["particles"], p)
        assert e.value.code == S.SICP_EINVAL
        with pytest.raises(S.SicpError) as e:      # surrogate mode keeps no correspondences
            S.sicp_icp_grad(c, d["src"], np.arange(10, dtype=np.int32), d["particles"], mode=S.SICP_NN_SURROGATE)
        assert e.value.code == S.SICP_EINVAL
        # a new reference drops the surrogate trained on the old one
        S.sicp_set_reference(c, d["ref"])
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_infer(c, np.zeros((4, 3), np.float32))
        assert e.value.code == S.SICP_ENOSURROGATE
    finally:
        S.sicp_destroy(c)


@pytest.fixture(scope="module")
def trained():
    """A surrogate trained on the Kinect-like scene (C2 sizes), and the scene."""
    c = S.sicp_create(0)
    d = synth.make_kinect_problem(1)
    S.sicp_set_reference(c, d["ref"])
    loss1 = S.sicp_surrogate_train(c, 1 << 18, seed=3, epochs=1, batch=4096, lr=1e-3)
    loss = S.sicp_surrogate_train(c, 1 << 21, seed=3, epochs=10, batch=4096, lr=1e-3)
    yield c, d, loss1, loss
    S.sicp_destroy(c)


def test_training_learns_the_field(trained):
    c, d, loss1, loss = trained
    assert loss < 0.7 * loss1, (loss1, loss)
    # held-out queries: the source under the initial particles (the early-iteration workload)
    rng = np.random.default_rng(0)
    idx = rng.choice(d["src"].shape[0], 300, replace=False)
    q = np.concatenate([O.transform(th, d["src"][idx]) for th in d["particles"][:20]]).astype(np.float32)
    disp, conf = S.sicp_surrogate_infer(c, q)
    nn, _ = S.sicp_nn(c, q)
    err = np.linalg.norm(q + disp - d["ref"][nn], axis=1)
    dist = np.linalg.norm(d["ref"][nn] - q, axis=1)
    sure = conf >= 0.5
    assert sure.mean() > 0.02
    assert np.median(err) < 0.5 * np.median(dist)               # better than predicting no displacement
    assert np.median(err[sure]) < 0.03                           # confident answers are within 3 cm
    assert np.median(err[sure]) < 0.6 * np.median(err[~sure])    # and the confidence ranks the errors


def test_register_surrogate_matches_exact(trained):
    """C5: 200 iterations, the first 150 on the surrogate; the final particle
    mean and spread against the all-exact run: a sanity bound (5 mm, 0.2
    deg, spread within 1 cm, both runs within 5 cm of the true pose), not the
    1 mm / 0.05 deg gate, which the learned field does not meet (see the
    next test)."""
    c, d, _, _ = trained
    W5 = synth.WORKLOADS["surrogate"]
    res = {}
    for mode in (S.SICP_NN_GRID, S.SICP_NN_SURROGATE):
        p = S.sicp_default_params(T=W5["T"], m=W5["m"], lr=W5["lr"], nn_mode=mode, seed=5,
                                  surrogate_iters=W5["surrogate_iters"])
        S.sicp_stats(c, True)
        res[mode] = S.sicp_register(c, d["src"], d["particles"], p)
        res[mode] += (S.sicp_stats(c, False),)
    _, m_e, c_e, _ = res[S.SICP_NN_GRID]
    _, m_s, c_s, st = res[S.SICP_NN_SURROGATE]
    assert st[6] == 150 * 100 * 300 and 0 < st[7] < st[6]
    assert np.all(np.abs(m_s[:3] - m_e[:3]) <= 5e-3)
    assert np.all(np.degrees(np.abs(m_s[3:] - m_e[3:])) <= 0.2)
    assert np.all(np.abs(np.sqrt(np.diag(c_s))[:3] - np.sqrt(np.diag(c_e))[:3]) <= 1e-2)
    # and both are near the true pose
    assert np.linalg.norm(m_s[:3] - d["theta_true"][:3]) < 0.05


def test_what_the_learned_field_gains_on_the_kinect_scene(trained):
    """What the trained network gains over the method without it, on C5
    (the kinect scene, 200 iterations, the first 150 on the learned field):
    iterations per second and the final pose mean and spread against the
    all-exact run, beside the all-exact run's own sensitivity (its particles
    moved by one float32 ulp), for the field trained on the fixed
    distribution and on the run's own queries (sicp_surrogate_train_run).

    On this scene the field gains nothing: a learned iteration (three layers
    per query plus the fallback queries' exact search) costs more device
    time than an exact grid iteration (measured on a GB300: 0.65-0.67x the
    all-exact speed), and its final pose lies about as far from the
    all-exact run as that run's own one-ulp floor or farther (2.96 / 2.97 mm
    in the mean against a 2.5 mm floor).  The test measures and prints both
    and holds the code to the speed it measured; a change that made the field
    pay would fail it and have to be documented."""
    import time
    c, d, _, _ = trained
    W5 = synth.WORKLOADS["surrogate"]
    from paper_2106_03287_gb300 import gate

    def timed(p, particles, reps=3):
        out = S.sicp_register(c, d["src"], particles, p)
        t0 = time.perf_counter()
        for _ in range(reps):
            out = S.sicp_register(c, d["src"], particles, p)
        return out, (time.perf_counter() - t0) / reps

    pe = S.sicp_default_params(T=W5["T"], m=W5["m"], lr=W5["lr"], nn_mode=S.SICP_NN_GRID, seed=5)
    (_, m_e, c_e), t_e = timed(pe, d["particles"])
    _, m_u, c_u = S.sicp_register(c, d["src"], np.nextafter(d["particles"], np.float32(np.inf)), pe)
    floor = gate.pose_errors(m_u, c_u, m_e, c_e)
    rows = {}
    for name in ("fixed", "run"):
        if name == "run":
            S.sicp_surrogate_train_run(c, d["src"], d["particles"], 1 << 21, seed=3, epochs=10, batch=4096, lr=1e-3)
        ps = S.sicp_default_params(T=W5["T"], m=W5["m"], lr=W5["lr"], nn_mode=S.SICP_NN_SURROGATE, seed=5,
                                   surrogate_iters=W5["surrogate_iters"])
        (_, m_s, c_s), t_s = timed(ps, d["particles"])
        rows[name] = (t_e / t_s, gate.pose_errors(m_s, c_s, m_e, c_e))
    print(f"all-exact run {1e3 * t_e:.2f} ms, its one-ulp floor {floor}")
    for name, (speed, err) in rows.items():
        print(f"learned field trained on {name} queries: speed {speed:.2f}x the all-exact run, pose errors {err}")
        assert 0 < speed < 1.0
        assert np.isfinite(list(err.values())).all()


def test_exact_registration_is_independent_of_context_history(trained):
    """The same registration on a fresh context and on one that has trained,
    inferred and searched before gives bit-identical particles."""
    c, d, _, _ = trained
    p = S.sicp_default_params(T=40, m=300, lr=0.03, nn_mode=S.SICP_NN_GRID, seed=9)
    S.sicp_surrogate_infer(c, d["src"][:5000])
    S.sicp_nn(c, d["src"][:7000] + np.float32(0.01))
    a = S.sicp_register(c, d["src"], d["particles"], p)[0]
    f = S.sicp_create(0)
    try:
        S.sicp_set_reference(f, d["ref"])
        b = S.sicp_register(f, d["src"], d["particles"], p)[0]
    finally:
        S.sicp_destroy(f)
    assert np.array_equal(a, b)


def test_save_load_roundtrip_and_corrupt_files(ctx, tmp_path):
    W = _random_params(21)
    norm4 = np.array([0.5, -1.0, 2.0, 3.0], np.float32)
    S.sicp_surrogate_params(ctx, W, norm4)
    path = str(tmp_path / "field.sicp")
    S.sicp_surrogate_save(ctx, path)
    c = S.sicp_create(0)
    try:
        S.sicp_surrogate_load(c, path)
        p, n = S.sicp_surrogate_params(c)
        assert np.array_equal(p, W) and np.array_equal(n, norm4)
        q = np.random.default_rng(0).uniform(-2, 2, (300, 3)).astype(np.float32)
        a, b = S.sicp_surrogate_infer(ctx, q), S.sicp_surrogate_infer(c, q)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        raw = open(path, "rb").read()
        bad = {"truncated": raw[:-5], "flipped": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
               "magic": b"XICPSURR" + raw[8:], "empty": b""}
        for name, blob in bad.items():
            f = tmp_path / f"{name}.sicp"
            f.write_bytes(blob)
            with pytest.raises(S.SicpError) as e:
                S.sicp_surrogate_load(c, str(f))
            assert e.value.code == S.SICP_EINVAL, name
        with pytest.raises(S.SicpError) as e:
            S.sicp_surrogate_load(c, str(tmp_path / "missing.sicp"))
        assert e.value.code == S.SICP_EINVAL
        p2, _ = S.sicp_surrogate_params(c)         # a failed load leaves the loaded field alone
        assert np.array_equal(p2, W)
    finally:
        S.sicp_destroy(c)
