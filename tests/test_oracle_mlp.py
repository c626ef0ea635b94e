"""Pins of the oracle's learned closest-point field (an MLP): bf16 rounding
against torch, the forward pass against torch's fp64 linear layers, the
gradient against central differences of the loss, feature invariants."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")


def _params(seed=0, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, O.mlp_nparam())


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.normal(0, 3, 2000), rng.uniform(-1e-3, 1e-3, 500),
                         1.0 + np.arange(64) * 2.0 ** -9])          # exact ties between bf16 neighbours
    want = torch.tensor(xs.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.bf16(x) for x in xs.astype(np.float32)])
    assert np.array_equal(got, want)


def test_features_invariants():
    rng = np.random.default_rng(2)
    for q in rng.uniform(-1.2, 1.2, (20, 3)):
        x = O.mlp_features(q)
        assert np.array_equal(x[:3], q)
        s, c = x[3:99:2], x[4:99:2]
        assert np.allclose(s ** 2 + c ** 2, 1.0, atol=1e-15)
        assert np.all(x[99:] == 0.0)
        assert np.allclose(x[3:6:2], np.sin(math.pi * q[:2]), atol=1e-15)      # f = 0: frequency pi
        xm = O.mlp_features(-q)
        assert np.allclose(xm[3:99:2], -s, atol=1e-12) and np.allclose(xm[4:99:2], c, atol=1e-12)


def test_forward_matches_torch_linear_layers():
    p = _params(3)
    W1, b1, W2, b2, W3, b3 = O.mlp_split(p)
    rng = np.random.default_rng(4)
    q = rng.uniform(-1, 1, (50, 3))
    X = torch.tensor(np.stack([O.mlp_features(v) for v in q]))
    h = torch.relu(torch.nn.functional.linear(X, torch.tensor(W1), torch.tensor(b1)))
    h = torch.relu(torch.nn.functional.linear(h, torch.tensor(W2), torch.tensor(b2)))
    out = torch.nn.functional.linear(h, torch.tensor(W3), torch.tensor(b3)).numpy()
    assert np.allclose(O.mlp_forward(p, q), out, rtol=1e-12, atol=1e-12)


def test_gradient_central_differences():
    p = _params(5, 0.2)
    rng = np.random.default_rng(6)
    q = rng.uniform(-1, 1, (12, 3))
    t = rng.normal(0, 0.1, (12, 3))
    out = O.mlp_forward(p, q)
    cstar = np.exp(-((out[:, :3] - t) ** 2).sum(1) / 0.02 ** 2)       # held constant, as in training
    loss, g = O.mlp_loss_grad(p, q, t, lam=0.5, delta=0.02, cstar=cstar)
    idx = np.concatenate([rng.choice(O.mlp_nparam(), 60, replace=False),
                          [128 * 112 + 5, 33040 - 16 + 3, 33040 - 16, 128 * 112 + 128 + 17]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.mlp_loss_grad(pp, q, t, lam=0.5, delta=0.02, cstar=cstar)[0] -
              O.mlp_loss_grad(pm, q, t, lam=0.5, delta=0.02, cstar=cstar)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    assert abs(loss - O.mlp_loss_grad(p, q, t, lam=0.5, delta=0.02, cstar=cstar)[0]) == 0.0


def test_bf16_mode_is_a_small_perturbation():
    p = _params(7)
    rng = np.random.default_rng(8)
    q = rng.uniform(-1, 1, (40, 3))
    t = rng.normal(0, 0.1, (40, 3))
    l64, g64 = O.mlp_loss_grad(p, q, t)
    l16, g16 = O.mlp_loss_grad(p, q, t, bf16ops=True)
    assert abs(l16 - l64) < 2e-2 * abs(l64)
    assert np.linalg.norm(g16 - g64) < 5e-2 * np.linalg.norm(g64)
    assert np.abs(O.mlp_forward(p, q, bf16ops=True) - O.mlp_forward(p, q)).max() < 5e-2
