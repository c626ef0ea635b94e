"""Pins of the FP64 oracle against facts the paper and mathematics fix.

None of these re-types the oracle's formula: each compares it with a library
routine (scipy, numpy), a closed form, an invariant, published generator
outputs, finite differences of an independently computed cost, or recovery
of a known pose.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2106_03287_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- minibatch RNG

def test_splitmix64_published_vectors():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [O.splitmix64_at(1234567, k) for k in range(1, 6)] == vals


def test_mb_key_is_a_stream_of_a_stream():
    for seed, t, i in [(0, 0, 0), (7, 3, 11), (2**63 + 5, 199, 99_999)]:
        base = O.splitmix64_at(seed, t + 1)
        assert O.mb_key(seed, t, i) == O.splitmix64_at(base, i + 1)


@pytest.mark.parametrize("N,m", [(50, 10), (1000, 100), (777, 777), (10, 1)])
def test_minibatch_is_the_m_smallest_keys(N, m):
    for t in (0, 1, 57):
        mb = O.minibatch(11, t, N, m)
        assert mb.shape == (m,)
        assert np.all(np.diff(mb) > 0) and mb.min() >= 0 and mb.max() < N
        keys = np.array([O.mb_key(11, t, i) for i in range(N)], dtype=np.uint64)
        assert len(np.unique(keys)) == N                 # keys of one iteration are distinct
        sel = np.zeros(N, bool)
        sel[mb] = True
        if m < N:
            assert keys[sel].max() < keys[~sel].min()


def test_minibatch_rejects_bad_sizes():
    with pytest.raises(ValueError):
        O.minibatch(0, 0, 10, 11)
    with pytest.raises(ValueError):
        O.minibatch(0, 0, 10, 0)


def test_minibatch_frequencies_are_uniform():
    N, m, T = 40, 8, 3000
    cnt = np.zeros(N)
    for t in range(T):
        cnt[O.minibatch(5, t, N, m)] += 1
    expect = T * m / N
    chi2 = ((cnt - expect) ** 2 / expect).sum()
    assert chi2 < 80.0          # 39 dof: p(chi2 > 80) < 1e-4


# ---------------------------------------------------------------- rotation

def test_rotation_matches_scipy_fixed_axis_angles():
    rng = np.random.default_rng(1)
    for _ in range(50):
        ang = rng.uniform(-math.pi, math.pi, 3)
        R, _ = O.rotation(np.r_[0, 0, 0, ang])
        ref = Rotation.from_euler("xyz", ang).as_matrix()
        assert np.abs(R - ref).max() < 1e-14
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14


def test_rotation_single_axes_are_textbook():
    a = 0.3
    c, s = math.cos(a), math.sin(a)
    Rx, _ = O.rotation([0, 0, 0, a, 0, 0])
    Ry, _ = O.rotation([0, 0, 0, 0, a, 0])
    Rz, _ = O.rotation([0, 0, 0, 0, 0, a])
    assert np.allclose(Rx, [[1, 0, 0], [0, c, -s], [0, s, c]], atol=1e-15)
    assert np.allclose(Ry, [[c, 0, s], [0, 1, 0], [-s, 0, c]], atol=1e-15)
    assert np.allclose(Rz, [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)


def test_rotation_partials_central_differences():
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(20):
        th = np.r_[rng.normal(size=3), rng.uniform(-3, 3, 3)]
        _, dR = O.rotation(th)
        for a in range(3):
            tp, tm = th.copy(), th.copy()
            tp[3 + a] += h
            tm[3 + a] -= h
            fd = (O.rotation(tp)[0] - O.rotation(tm)[0]) / (2 * h)
            assert np.abs(fd - dR[a]).max() < 1e-9


# ---------------------------------------------------------------- correspondences

@pytest.mark.parametrize("kind", ["uniform", "clustered", "box"])
def test_nn_matches_kdtree(kind):
    rng = np.random.default_rng(3)
    if kind == "uniform":
        ref = rng.uniform(-1, 1, (2000, 3))
    elif kind == "clustered":
        c = rng.uniform(-1, 1, (10, 3))
        ref = c[rng.integers(0, 10, 2000)] + rng.normal(0, 0.01, (2000, 3))
    else:
        ref = synth.make_box_problem(3)["ref"]
    ref = ref.astype(np.float32)
    q = rng.uniform(-1.2, 1.2, (500, 3))
    idx, d2 = O.nn(ref, q)
    dd, ii = cKDTree(ref.astype(np.float64)).query(q, k=2)
    unique = dd[:, 1] ** 2 - dd[:, 0] ** 2 > 1e-12
    assert np.array_equal(idx[unique], ii[unique, 0])
    assert np.allclose(d2, dd[:, 0] ** 2, rtol=1e-12, atol=1e-15)


def test_nn_ties_go_to_lowest_index_and_self_queries_are_exact():
    rng = np.random.default_rng(4)
    base = rng.uniform(-1, 1, (100, 3)).astype(np.float32)
    ref = np.concatenate([base, base[:50]])          # duplicates at indices 100..149
    perm = rng.permutation(150)
    ref = ref[perm]
    idx, d2 = O.nn(ref, ref.astype(np.float64))
    assert np.all(d2 == 0.0)
    for r in range(150):
        same = np.flatnonzero(np.all(ref == ref[r], axis=1))
        assert idx[r] == same.min()


def test_nn2_second_distance_matches_kdtree():
    rng = np.random.default_rng(5)
    base = rng.uniform(-1, 1, (1500, 3)).astype(np.float32)
    ref = np.concatenate([base, base[:20]])          # duplicates: their second distance is 0
    q = np.concatenate([rng.uniform(-1.3, 1.3, (600, 3)), base[:20].astype(np.float64)])
    idx, d2, d2b = O.nn2(ref, q)
    dd, ii = cKDTree(ref.astype(np.float64)).query(q, k=2)
    assert np.allclose(d2, dd[:, 0] ** 2, rtol=1e-12, atol=1e-15)
    assert np.allclose(d2b, dd[:, 1] ** 2, rtol=1e-12, atol=1e-15)
    assert np.all(d2b[-20:] == 0.0) and np.all(d2b >= d2)
    i1, _ = O.nn(ref, q)
    assert np.array_equal(idx, i1)


def _kd_clouds():
    rng = np.random.default_rng(21)
    c = rng.uniform(-1, 1, (12, 3))
    lat = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.25
    base = rng.uniform(-1, 1, (700, 3))
    return {
        "uniform": rng.uniform(-1, 1, (5000, 3)),
        "clustered": c[rng.integers(0, 12, 4000)] + rng.normal(0, 1e-3, (4000, 3)),
        "lattice": lat[rng.permutation(lat.shape[0])],                 # many exact ties
        "duplicates": np.concatenate([base, base[:300], base[:300], base[:5]])[rng.permutation(1305)],
        "box": synth.make_box_problem(2)["ref"],
        "planar": np.c_[rng.uniform(-1, 1, (3000, 2)), np.zeros(3000)],
        "one": np.array([[0.1, -0.2, 0.3]]),
        "two": np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]),
    }


@pytest.mark.parametrize("name", ["uniform", "clustered", "lattice", "duplicates", "box", "planar", "one", "two"])
def test_kdtree_equals_exhaustive_search(name):
    """The k-d tree returns exactly the exhaustive argmin, lowest index on ties."""
    ref = _kd_clouds()[name].astype(np.float32)
    rng = np.random.default_rng(len(name))
    ext = float(np.abs(ref).max()) + 1e-3
    q = np.concatenate([
        rng.uniform(-1.2 * ext, 1.2 * ext, (1500, 3)),                        # inside and around
        rng.uniform(-50 * ext, 50 * ext, (200, 3)),                           # far away
        ref[rng.integers(0, ref.shape[0], 300)].astype(np.float64),           # on reference points
        (ref[rng.integers(0, ref.shape[0], 200)] + 0.125).astype(np.float64),  # lattice midpoints: ties
    ])
    i_b, d_b = O.nn(ref, q)
    i_k, d_k = O.KDTree(ref).nn(q)
    assert np.array_equal(i_b, i_k)
    assert np.array_equal(d_b, d_k)
    if name == "lattice":     # the tie rule was exercised: some queries have several nearest points
        dd, _ = cKDTree(ref.astype(np.float64)).query(q, k=2)
        assert np.sum(dd[:, 1] == dd[:, 0]) > 50


def test_kdtree_gradient_and_run_equal_exhaustive():
    d = synth.make_box_problem(4, K=6)
    tree = O.KDTree(d["ref"])
    mb = O.minibatch(3, 0, d["src"].shape[0], 100)
    th = d["particles"].astype(np.float64)
    g_b, nn_b, l_b = O.icp_grad(d["ref"], d["src"], mb, th)
    g_k, nn_k, l_k = tree.icp_grad(d["src"], mb, th)
    assert np.array_equal(nn_b, nn_k) and np.array_equal(g_b, g_k) and np.array_equal(l_b, l_k)
    p = O.Params(T=15, m=60, lr=0.01, seed=5)
    a = O.register(d["ref"], d["src"], d["particles"], p)
    p.tree = tree
    b = O.register(d["ref"], d["src"], d["particles"], p)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    with pytest.raises(ValueError):
        O.register(d["ref"][:-1], d["src"], d["particles"], p)        # a tree of another cloud


# ---------------------------------------------------------------- ICP gradient

def _half_loss(theta, ref, src_mb):
    """L/2 of Eq. (icp-objective1) over a minibatch, with nearest neighbours
    recomputed: scipy rotation + cKDTree, independent of the oracle."""
    R = Rotation.from_euler("xyz", theta[3:]).as_matrix()
    q = src_mb.astype(np.float64) @ R.T + theta[:3]
    d, i = cKDTree(ref.astype(np.float64)).query(q)
    return 0.5 * np.mean(d ** 2), i


def test_icp_gradient_central_differences():
    rng = np.random.default_rng(5)
    ref = rng.uniform(-1, 1, (400, 3)).astype(np.float32)
    src = rng.uniform(-1, 1, (200, 3)).astype(np.float32)
    mb = O.minibatch(3, 0, 200, 60)
    h = 1e-6
    checked = 0
    for trial in range(10):
        th = np.r_[rng.normal(0, 0.1, 3), rng.uniform(-0.5, 0.5, 3)]
        g, nnk, loss = O.icp_grad(ref, src, mb, th[None])
        l0, i0 = _half_loss(th, ref, src[mb])
        assert abs(loss[0] - l0) < 1e-12 * max(1.0, l0)
        assert np.array_equal(nnk[0], i0)
        fd = np.empty(6)
        stable = True
        for a in range(6):
            tp, tm = th.copy(), th.copy()
            tp[a] += h
            tm[a] -= h
            lp, ip = _half_loss(tp, ref, src[mb])
            lm, im = _half_loss(tm, ref, src[mb])
            stable &= np.array_equal(ip, i0) and np.array_equal(im, i0)
            fd[a] = (lp - lm) / (2 * h)
        if not stable:
            continue                     # a correspondence switched inside +-h
        checked += 1
        assert np.abs(fd - g[0]).max() <= 1e-7 * np.abs(g[0]).max() + 1e-12
    assert checked >= 5


# ---------------------------------------------------------------- point-to-plane (reading R16)

def _half_loss_plane(theta, ref, normals, src_mb):
    """Point-to-plane L/2 over a minibatch, nearest neighbours recomputed
    (scipy rotation + cKDTree), normals held fixed; independent of the oracle."""
    R = Rotation.from_euler("xyz", theta[3:]).as_matrix()
    q = src_mb.astype(np.float64) @ R.T + theta[:3]
    _, i = cKDTree(ref.astype(np.float64)).query(q)
    e = np.einsum("ij,ij->i", normals[i], q - ref[i].astype(np.float64))
    return 0.5 * np.mean(e ** 2), i


def test_point_to_plane_gradient_central_differences():
    rng = np.random.default_rng(6)
    ref = rng.uniform(-1, 1, (400, 3)).astype(np.float32)
    nrm = rng.normal(size=(400, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    src = rng.uniform(-1, 1, (200, 3)).astype(np.float32)
    mb = O.minibatch(4, 0, 200, 60)
    h = 1e-6
    checked = 0
    for trial in range(10):
        th = np.r_[rng.normal(0, 0.1, 3), rng.uniform(-0.5, 0.5, 3)]
        g, nnk, loss = O.icp_grad(ref, src, mb, th[None], normals=nrm)
        l0, i0 = _half_loss_plane(th, ref, nrm, src[mb])
        assert abs(loss[0] - l0) < 1e-12 * max(1.0, l0) and np.array_equal(nnk[0], i0)
        fd = np.empty(6)
        stable = True
        for a in range(6):
            tp, tm = th.copy(), th.copy()
            tp[a] += h
            tm[a] -= h
            lp, ip = _half_loss_plane(tp, ref, nrm, src[mb])
            lm, im = _half_loss_plane(tm, ref, nrm, src[mb])
            stable &= np.array_equal(ip, i0) and np.array_equal(im, i0)
            fd[a] = (lp - lm) / (2 * h)
        if not stable:
            continue
        checked += 1
        assert np.abs(fd - g[0]).max() <= 1e-7 * np.abs(g[0]).max() + 1e-12
    assert checked >= 5


def test_point_to_plane_gradient_closed_form():
    """A planar reference z = 0 on a 1 cm lattice; source points over lattice
    points, lifted by delta and slid by eps < half a cell within the plane.
    At the identity pose the point-to-plane residual is delta along z, so
    gbar = (0, 0, delta, delta mean(y), -delta mean(x), 0); point-to-point
    adds the in-plane slide to the translation."""
    xs, ys = np.meshgrid(np.arange(-20, 21) * 0.01, np.arange(-15, 16) * 0.01)
    ref = np.c_[xs.ravel(), ys.ravel(), np.zeros(xs.size)].astype(np.float32)
    nrm = np.tile([0.0, 0.0, -1.0], (ref.shape[0], 1))          # the sign of a normal is irrelevant
    delta, eps = 0.003, 0.002
    pick = np.random.default_rng(2).choice(ref.shape[0], 300, replace=False)
    src = (ref[pick].astype(np.float64) + [eps, 0.0, delta]).astype(np.float32)
    mb = np.arange(300, dtype=np.int32)
    th = np.zeros((1, 6))
    g, nnk, _ = O.icp_grad(ref, src, mb, th, normals=nrm)
    assert np.array_equal(nnk[0], pick)
    s = src.astype(np.float64)
    dz = s[:, 2] - 0.0
    expect = [0.0, 0.0, dz.mean(), np.mean(dz * s[:, 1]), -np.mean(dz * s[:, 0]), 0.0]
    assert np.allclose(g[0], expect, atol=1e-15)
    g_pp, _, _ = O.icp_grad(ref, src, mb, th)
    assert abs(g_pp[0, 0] - np.mean(s[:, 0] - ref[pick, 0])) < 1e-12 and abs(g_pp[0, 0]) > 1e-3


@pytest.mark.parametrize("k", [1, 10, 32])
def test_knn_matches_kdtree(k):
    rng = np.random.default_rng(k)
    ref = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    idx, d2 = O.knn(ref, k, with_d2=True)
    d, i = cKDTree(ref.astype(np.float64)).query(ref.astype(np.float64), k + 1)
    assert np.array_equal(idx[:, 0], np.arange(3000))             # each point is its own nearest
    same = np.array([set(idx[r]) == set(i[r, :k]) for r in range(3000)])
    # ranked by the exact fp64 distance: a set may differ only at an exact tie of the k-th and
    # (k+1)-th distances (to the rounding of scipy's own distance sum)
    near_tie = np.abs(d[:, k] - d[:, k - 1]) <= 1e-12 * d[:, k]
    assert np.all(same | near_tie) and same.mean() > 0.999
    assert np.allclose(d2, d[:, :k] ** 2, rtol=1e-12, atol=1e-15)
    assert np.all(np.diff(d2, axis=1) >= 0)
    exact = ((ref[idx].astype(np.float64) - ref[:, None, :].astype(np.float64)) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-15, atol=0)
    # ties go to the lower index: duplicates of point 7 follow it in index order
    dup = np.concatenate([ref[:100], ref[7:8], ref[7:8]])
    di = O.knn(dup, 3)
    assert list(di[7]) == [7, 100, 101] and list(di[101]) == [7, 100, 101]


def test_neighbourhood_cov_matches_numpy():
    rng = np.random.default_rng(3)
    ref = rng.normal(size=(500, 3)).astype(np.float32)
    idx = rng.integers(0, 500, (50, 12))
    cov = O.neighbourhood_cov(ref, idx)
    for r in range(50):
        assert np.allclose(cov[r], np.cov(ref[idx[r]].astype(np.float64).T, bias=True), atol=1e-14)


def test_normals_of_a_plane_and_a_sphere():
    rng = np.random.default_rng(8)
    xy = rng.uniform(-1, 1, (2000, 2))
    z = 0.3 * xy[:, 0] - 0.2 * xy[:, 1] + 0.5
    plane = np.c_[xy, z].astype(np.float32)
    n, w = O.normals(plane, 12)
    true = np.array([0.3, -0.2, -1.0]) / np.linalg.norm([0.3, -0.2, -1.0])
    assert np.all(np.abs(n @ true) > 1 - 1e-9)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-12)
    # Fibonacci sphere: the normal of a small symmetric patch is radial
    N = 20000
    i = np.arange(N) + 0.5
    phi, cz = np.pi * (1 + 5 ** 0.5) * i, 1 - 2 * i / N
    sph = np.c_[np.sqrt(1 - cz ** 2) * np.cos(phi), np.sqrt(1 - cz ** 2) * np.sin(phi), cz].astype(np.float32)
    n, w = O.normals(sph, 16)
    radial = sph.astype(np.float64) / np.linalg.norm(sph.astype(np.float64), axis=1, keepdims=True)
    assert np.all(np.abs(np.einsum("ij,ij->i", n, radial)) > 0.999)


def test_point_to_plane_run_recovers_known_pose_noise_free():
    """K = 1 with the point-to-plane metric on a noise-free box: the
    generating pose zeroes every residual, and the run lands on it."""
    d = synth.make_box_problem(0, K=1, noise=0.0)
    nrm, _ = O.normals(d["ref"], 10)
    th, _, _ = O.register(d["ref"], d["src"], d["particles"], O.Params(T=300, m=100, seed=7, normals=nrm))
    err = th[0] - d["theta_true"]
    assert np.abs(err[:3]).max() < 1e-3
    assert np.abs(err[3:]).max() < math.radians(0.05)


# ---------------------------------------------------------------- Monte Carlo ground truth, KL, OVL (R17)

def test_independent_runs_are_single_particle_runs():
    """Independent mode: particle j evolves exactly as the separate K = 1 run
    (SGD-ICP with Adam) with seed + j."""
    d = synth.make_box_problem(2, M=600, N=200, K=5)
    p = O.Params(T=20, m=40, seed=3, independent=True)
    th, _, _ = O.register(d["ref"], d["src"], d["particles"], p)
    for j in range(5):
        one, _, _ = O.register(d["ref"], d["src"], d["particles"][j:j + 1], O.Params(T=20, m=40, seed=3 + j))
        assert np.array_equal(th[j], one[0])
    coupled, _, _ = O.register(d["ref"], d["src"], d["particles"], O.Params(T=20, m=40, seed=3))
    assert not np.array_equal(coupled, th)


def _random_spd(rng, d, scale):
    A = rng.normal(size=(d, d))
    return scale * (A @ A.T / d + 0.2 * np.eye(d))


def test_gaussian_kl_closed_forms_and_monte_carlo():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(12)
    m0, m1 = rng.normal(size=6), rng.normal(size=6)
    S0, S1 = _random_spd(rng, 6, 0.5), _random_spd(rng, 6, 0.8)
    assert abs(O.gaussian_kl(m0, S0, m0, S0)) < 1e-12
    # one axis differs, the rest identical: the 1-D formula
    mu0, s0, mu1, s1 = 0.3, 0.7, -0.2, 1.3
    D0, D1 = np.eye(6), np.eye(6)
    D0[2, 2], D1[2, 2] = s0 ** 2, s1 ** 2
    a, b = np.zeros(6), np.zeros(6)
    a[2], b[2] = mu0, mu1
    one_d = math.log(s1 / s0) + (s0 ** 2 + (mu0 - mu1) ** 2) / (2 * s1 ** 2) - 0.5
    assert abs(O.gaussian_kl(a, D0, b, D1) - one_d) < 1e-12
    # E_p0[log p0 - log p1] by Monte Carlo with scipy's densities
    x = stats.multivariate_normal(m0, S0).rvs(400_000, random_state=5)
    diff = stats.multivariate_normal(m0, S0).logpdf(x) - stats.multivariate_normal(m1, S1).logpdf(x)
    assert abs(O.gaussian_kl(m0, S0, m1, S1) - diff.mean()) < 4 * diff.std() / math.sqrt(x.shape[0])


def test_gaussian_ovl_closed_forms():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(13)
    n = 200_000
    z0, z1 = rng.standard_normal((n, 6)), rng.standard_normal((n, 6))
    m0 = rng.normal(size=6)
    S = _random_spd(rng, 6, 0.3)
    assert O.gaussian_ovl(m0, S, m0, S, z0, z1) == 1.0
    # equal covariances: OVL = 2 Phi(-delta / 2), delta the Mahalanobis distance of the means
    for shift in (0.3, 1.0, 2.5):
        m1 = m0 + shift * np.linalg.cholesky(S) @ np.r_[1.0, np.zeros(5)]
        expect = 2 * stats.norm.cdf(-shift / 2)
        assert abs(O.gaussian_ovl(m0, S, m1, S, z0, z1) - expect) < 0.005, shift
    far = m0 + 100.0
    assert O.gaussian_ovl(m0, S, far, S, z0, z1) < 1e-6


# ---------------------------------------------------------------- odometry chaining (R18)

def _so3_exp_batch(phi):
    """Rodrigues' formula, vectorised (independent of the oracle's scipy expm)."""
    th = np.linalg.norm(phi, axis=1)[:, None, None]
    K = np.zeros((phi.shape[0], 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -phi[:, 2], phi[:, 1], -phi[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = phi[:, 2], -phi[:, 1], phi[:, 0]
    a = np.where(th > 1e-9, np.sin(th) / np.maximum(th, 1e-300), 1.0)
    b = np.where(th > 1e-9, (1 - np.cos(th)) / np.maximum(th, 1e-300) ** 2, 0.5)
    c = np.where(th > 1e-9, (th - np.sin(th)) / np.maximum(th, 1e-300) ** 3, 1.0 / 6)
    K2 = K @ K
    return np.eye(3) + a * K + b * K2, np.eye(3) + b * K + c * K2


def _se3_exp_batch(xi):
    C, V = _so3_exp_batch(xi[:, 3:])
    T = np.tile(np.eye(4), (xi.shape[0], 1, 1))
    T[:, :3, :3] = C
    T[:, :3, 3] = np.einsum("nij,nj->ni", V, xi[:, :3])
    return T


def _se3_log_batch(T):
    C = T[:, :3, :3]
    cos = np.clip((np.trace(C, axis1=1, axis2=2) - 1) / 2, -1, 1)
    th = np.arccos(cos)
    w = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], 1)
    s = np.where(th > 1e-9, th / (2 * np.sin(np.maximum(th, 1e-300))), 0.5)
    phi = s[:, None] * w
    _, V = _so3_exp_batch(phi)
    rho = np.linalg.solve(V, T[:, :3, 3][..., None])[..., 0]
    return np.c_[rho, phi]


def test_se3_exp_log_and_adjoint():
    rng = np.random.default_rng(21)
    for _ in range(20):
        xi = np.r_[rng.normal(0, 1, 3), rng.normal(0, 0.8, 3)]
        T = O.se3_exp(xi)
        assert np.allclose(T, _se3_exp_batch(xi[None])[0], atol=1e-12)
        assert np.allclose(O.se3_log(T), xi, atol=1e-10)
        # T exp(xi^) T^-1 = exp((Ad(T) xi)^)
        P = O.pose_matrix(np.r_[rng.normal(0, 1, 3), rng.uniform(-1, 1, 3)])
        eps = xi * 1e-3
        assert np.allclose(P @ O.se3_exp(eps) @ np.linalg.inv(P), O.se3_exp(O.adjoint(P) @ eps), atol=1e-12)
    assert np.allclose(O.pose_matrix([1, 2, 3, 0, 0, 0]), np.r_[np.c_[np.eye(3), [1, 2, 3]], [[0, 0, 0, 1]]])


def test_compounding_against_monte_carlo():
    """Compound two uncertain poses by sampling (own vectorised exp/log) and
    compare: the second-order covariance is good for small uncertainty, and
    the fourth-order terms remove most of its error for large uncertainty."""
    rng = np.random.default_rng(3)
    T1 = O.pose_matrix([0.5, -0.2, 0.3, 0.3, -0.2, 0.5])
    T2 = O.pose_matrix([1.0, 0.4, -0.2, -0.4, 0.1, 0.2])
    n = 200_000
    for sc, tol2, ratio in ((0.05, 0.02, None), (0.5, None, 0.4)):
        S1 = np.diag([1, 2, 1, 1, 0.5, 2.0]) * sc ** 2
        S2 = np.diag([2, 1, 1, 0.5, 1, 1.5]) * sc ** 2
        x1 = rng.standard_normal((n, 6)) @ np.linalg.cholesky(S1).T
        x2 = rng.standard_normal((n, 6)) @ np.linalg.cholesky(S2).T
        Tm = T1 @ T2
        T = _se3_exp_batch(x1) @ T1 @ _se3_exp_batch(x2) @ T2 @ np.linalg.inv(Tm)
        S_mc = np.cov(_se3_log_batch(T).T)
        Tc, S2nd = O.compound(T1, S1, T2, S2, order=2)
        _, S4th = O.compound(T1, S1, T2, S2, order=4)
        assert np.allclose(Tc, Tm, atol=1e-14)
        e2 = np.linalg.norm(S2nd - S_mc) / np.linalg.norm(S_mc)
        e4 = np.linalg.norm(S4th - S_mc) / np.linalg.norm(S_mc)
        if tol2 is not None:
            assert e2 < tol2 and e4 < tol2
        else:
            assert e4 < ratio * e2 and e4 < 0.03, (e2, e4)


def test_pose_distribution_of_particles():
    """Particles drawn as exp(xi^) T_bar around a known pose: the mean pose is
    recovered and the covariance is the sample covariance of the xi."""
    rng = np.random.default_rng(4)
    Tb = O.pose_matrix([0.3, -0.1, 0.2, 0.2, 0.1, 3.0])      # yaw next to pi
    xi = rng.normal(0, 1, (400, 6)) * [0.01, 0.02, 0.01, 0.02, 0.01, 0.03]
    xi -= xi.mean(0)
    Ts = _se3_exp_batch(xi) @ Tb
    from scipy.spatial.transform import Rotation as Rot
    th = np.c_[Ts[:, :3, 3], Rot.from_matrix(Ts[:, :3, :3]).as_euler("xyz")]
    T_hat, S = O.pose_distribution(th)
    assert np.allclose(T_hat, Tb, atol=1e-9)
    assert np.allclose(S, np.cov(xi.T), atol=1e-12)


def test_icp_gradient_single_point_closed_form():
    ref = np.array([[0.3, -0.2, 0.5]], np.float32)
    src = np.array([[0.1, 0.4, -0.2]], np.float32)
    th = np.array([0.05, -0.1, 0.2, 0.3, -0.4, 0.7])
    g, nnk, _ = O.icp_grad(ref, src, np.array([0], np.int32), th[None])
    R = Rotation.from_euler("xyz", th[3:]).as_matrix()
    e = R @ src[0].astype(np.float64) + th[:3] - ref[0]
    assert np.abs(g[0, :3] - e).max() < 1e-15
    assert nnk[0, 0] == 0


def test_icp_gradient_given_nn_matches_search():
    d = synth.make_box_problem(6, K=4)
    mb = O.minibatch(1, 0, d["src"].shape[0], 100)
    th = d["particles"].astype(np.float64)
    g, nnk, _ = O.icp_grad(d["ref"], d["src"], mb, th)
    g2 = O.icp_grad_given_nn(d["ref"], d["src"], mb, th, nnk)
    assert np.array_equal(g, g2)


# ---------------------------------------------------------------- priors

def test_prior_gradients_closed_form():
    th = np.array([[0.1, 0.2, 0.3, 0.5, -0.5, 3.0]])
    mu = np.array([0.0, 0.1, 0.2, 0.4, -0.4, -3.0])
    sigma = np.array([0.5, 0.25, 2.0])
    kappa = np.array([2.0, 3.0, 4.0])
    gb = np.zeros((1, 6))
    G = O.log_post_grad(th, gb, 1000, 1, mu, sigma, kappa)
    assert np.allclose(G[0, :3], -(th[0, :3] - mu[:3]) / sigma, atol=1e-15)
    assert np.allclose(G[0, 3:], -kappa * np.sin(th[0, 3:] - mu[3:]), atol=1e-15)
    G0 = O.log_post_grad(th, np.ones((1, 6)), 1000, 0)
    assert np.all(G0 == -1000.0)


# ---------------------------------------------------------------- bandwidth & Stein

def test_median_matches_numpy():
    rng = np.random.default_rng(7)
    for n in (1, 2, 9, 100, 10_000):
        x = rng.normal(size=n)
        assert O.median(x) == np.median(x)


def _two_particles(d_t, d_r):
    th = np.zeros((2, 6))
    th[0, :3] = [0.1, 0.2, -0.1]
    th[1, :3] = th[0, :3] + d_t
    th[0, 3:] = [3.1, 0.2, -0.3]
    th[1, 3:] = th[0, 3:] + d_r
    return th


def test_two_particle_bandwidth_closed_form():
    # K = 2: the four squared distances are {0, 0, d^2, d^2}: median d^2/2, h = d^2 / (2 ln 3)
    d_t = np.array([0.03, -0.04, 0.12])
    d_r = np.array([0.2, 0.1, -0.05])
    h_t, h_r = O.bandwidths(_two_particles(d_t, d_r))
    assert abs(h_t - (d_t @ d_t) / (2 * math.log(3))) < 1e-15
    assert abs(h_r - (d_r @ d_r) / (2 * math.log(3))) < 1e-15


@pytest.mark.parametrize("cross_pi", [False, True])
def test_two_particle_stein_closed_form(cross_pi):
    d_t = np.array([0.03, -0.04, 0.12])
    d_r = np.array([0.2, 0.1, -0.05])
    th = _two_particles(d_t, d_r)
    if cross_pi:
        th[1, 3] = -3.1           # roll difference 3.1 - (-3.1) wraps to 6.2 - 2 pi
    rng = np.random.default_rng(8)
    G = rng.normal(size=(2, 6))
    h_t, h_r = O.bandwidths(th)
    phi = O.stein_phi(th, G, h_t, h_r)
    # with h = d^2/(2 ln 3) the off-diagonal kernel is exp(-2 ln 3) = 1/9
    dw = th[0, 3:] - th[1, 3:]
    dw = (dw + np.pi) % (2 * np.pi) - np.pi
    d_r_eff = -dw
    assert abs(h_r - (d_r_eff @ d_r_eff) / (2 * math.log(3))) < 1e-14
    for i, j in ((0, 1), (1, 0)):
        dt = th[i, :3] - th[j, :3]
        dr = (th[i, 3:] - th[j, 3:] + np.pi) % (2 * np.pi) - np.pi
        exp_t = 0.5 * (G[i, :3] + G[j, :3] / 9 + (2 / h_t) * dt / 9)
        exp_r = 0.5 * (G[i, 3:] + G[j, 3:] / 9 + (2 / h_r) * dr / 9)
        assert np.abs(phi[i, :3] - exp_t).max() < 1e-12 * max(1, np.abs(exp_t).max())
        assert np.abs(phi[i, 3:] - exp_r).max() < 1e-12 * max(1, np.abs(exp_r).max())


def test_single_particle_stein_is_the_gradient():
    th = np.array([[0.1, 0.2, 0.3, 0.4, 0.5, 0.6]])
    G = np.array([[1.0, -2.0, 3.0, -4.0, 5.0, -6.0]])
    h_t, h_r = O.bandwidths(th)
    assert h_t == 1.0 and h_r == 1.0
    assert np.array_equal(O.stein_phi(th, G, h_t, h_r), G)


def test_svgd_recovers_a_gaussian_target():
    """SVGD with the median heuristic transports particles to a 6-D Gaussian:
    mean within sigma/sqrt(K), per-axis spread within 10%."""
    rng = np.random.default_rng(0)
    K = 200
    mu = np.array([0.3, -0.2, 0.1, 0.2, -0.1, 0.3])
    sig = np.array([0.05, 0.1, 0.02, 0.1, 0.05, 0.2])
    th = np.ascontiguousarray(rng.uniform(-0.5, 0.5, (K, 6)))
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    for t in range(1, 801):
        G = -(th - mu) / sig ** 2
        phi = O.stein_phi(th, G, *O.bandwidths(th))
        O.adam(th, mom, vel, -phi, t, 0.01)
    assert np.all(np.abs(th.mean(0) - mu) < sig / math.sqrt(K))
    ratio = th.std(0, ddof=1) / sig
    assert np.all((ratio > 0.9) & (ratio < 1.1)), ratio


def _circ_mean_resultant(a):
    return abs(np.mean(np.exp(1j * a)))


def test_svgd_with_the_priors_recovers_gaussian_and_von_mises():
    """With no data (gbar = 0) and prior = 1, G is the gradient of the log
    prior alone (Eqs. trans_prior, rot_prior), so SVGD must transport the
    particles to the prior itself: N(mu, sigma) per translation axis (sigma
    read as the variance) and von Mises(mu, kappa) per angle, whose mean
    resultant length is I1(kappa)/I0(kappa).  One angle's mean sits next to
    +-pi, so the particles straddle the cut."""
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    K = 200
    mu = np.array([0.3, -0.2, 0.1, 3.0, -0.4, 0.2])
    var = np.array([0.0025, 0.01, 0.0004])
    kappa = np.array([20.0, 50.0, 8.0])
    th = np.ascontiguousarray(rng.uniform(-0.5, 0.5, (K, 6)))
    th[:, 3] += 3.0
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    for t in range(1, 1201):
        G = O.log_post_grad(th, np.zeros_like(th), 1000, 1, mu, var, kappa)
        phi = O.stein_phi(th, G, *O.bandwidths(th))
        O.adam(th, mom, vel, -phi, t, 0.01)
    sd = np.sqrt(var)
    assert np.all(np.abs(th[:, :3].mean(0) - mu[:3]) < 2 * sd / math.sqrt(K))
    ratio = th[:, :3].std(0, ddof=1) / sd
    assert np.all((ratio > 0.9) & (ratio < 1.1)), ratio
    mean_c, _ = O.moments_circular(th)
    circ_sd = 1.0 / np.sqrt(kappa)
    dmu = np.angle(np.exp(1j * (mean_c[3:] - mu[3:])))
    assert np.all(np.abs(dmu) < 2 * circ_sd / math.sqrt(K)), dmu
    R = np.array([_circ_mean_resultant(th[:, 3 + a]) for a in range(3)])
    A = special.i1(kappa) / special.i0(kappa)
    # circular spread sqrt(-2 ln R) against the target's, within 10%
    spread = np.sqrt(-2 * np.log(R)) / np.sqrt(-2 * np.log(A))
    assert np.all((spread > 0.9) & (spread < 1.1)), spread


# ---------------------------------------------------------------- Adam

def test_adam_constant_gradient_closed_form():
    # bias correction makes mhat = g and vhat = g^2 for a constant g, so each
    # step is lr * g / (|g| + eps)
    g = np.array([3.0, -1e-3, 2e-9, 0.0, -5.0, 1e-7])
    x = np.zeros(6)
    mom, vel = np.zeros(6), np.zeros(6)
    for t in range(1, 11):
        O.adam(x, mom, vel, g, t, 0.01)
        assert np.allclose(x, -t * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_adam_three_steps_varying_gradient_by_hand():
    """beta1 = 1/2, beta2 = 3/4, eps = 0, gradients 1, -1, 2 (worked by hand):
    m = 1/2, -1/4, 7/8 and v = 1/4, 7/16, 85/64; bias corrections 1/2, 3/4, 7/8
    and 1/4, 7/16, 37/64 give mhat = 1, -1/3, 1 and vhat = 1, 1, 85/37, so the
    steps are lr, -lr/3, lr sqrt(37/85).  Swapping the betas gives another
    third step (the second case below), and dropping the bias correction
    another first step (m1 / sqrt(v1) = 1 only with both corrections)."""
    lr = 0.1
    x, mom, vel = np.zeros(1), np.zeros(1), np.zeros(1)
    steps = []
    for t, g in enumerate([1.0, -1.0, 2.0], start=1):
        x0 = x.copy()
        O.adam(x, mom, vel, np.array([g]), t, lr, 0.5, 0.75, 0.0)
        steps.append(float(x0[0] - x[0]))
        if t == 2:
            assert mom[0] == -0.25 and vel[0] == 7.0 / 16.0
    assert steps[0] == pytest.approx(lr, rel=1e-15)
    assert steps[1] == pytest.approx(-lr / 3.0, rel=1e-15)
    assert steps[2] == pytest.approx(lr * math.sqrt(37.0 / 85.0), rel=1e-15)
    assert mom[0] == 0.875 and vel[0] == 85.0 / 64.0
    # betas swapped (beta1 = 3/4, beta2 = 1/2): m = 1/4, -1/16, 29/64; v = 1/2, 3/4, 19/8;
    # corrections 1/4, 7/16, 37/64 and 1/2, 3/4, 7/8: mhat_3 = 29/37, vhat_3 = 19/7
    x, mom, vel = np.zeros(1), np.zeros(1), np.zeros(1)
    for t, g in enumerate([1.0, -1.0, 2.0], start=1):
        x0 = x.copy()
        O.adam(x, mom, vel, np.array([g]), t, lr, 0.75, 0.5, 0.0)
    assert float(x0[0] - x[0]) == pytest.approx(lr * (29.0 / 37.0) / math.sqrt(19.0 / 7.0), rel=1e-14)
    assert mom[0] == 29.0 / 64.0 and vel[0] == 19.0 / 8.0
    # the defaults (0.9, 0.999, eps 1e-8) with gradients 1, 0: mhat_2 = 0.09 / 0.19,
    # vhat_2 = 0.000999 / 0.001999, second step lr * mhat_2 / (sqrt(vhat_2) + 1e-8)
    x, mom, vel = np.zeros(1), np.zeros(1), np.zeros(1)
    O.adam(x, mom, vel, np.array([1.0]), 1, lr)
    x1 = x.copy()
    O.adam(x, mom, vel, np.array([0.0]), 2, lr)
    want = lr * (0.09 / 0.19) / (math.sqrt(0.000999 / 0.001999) + 1e-8)
    assert float(x1[0] - x[0]) == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------- moments & whole run

def test_moments_match_numpy():
    rng = np.random.default_rng(9)
    th = rng.normal(size=(37, 6))
    mean, cov = O.moments(th)
    assert np.allclose(mean, th.mean(0), atol=1e-15)
    assert np.allclose(cov, np.cov(th.T), atol=1e-14)
    m1, c1 = O.moments(th[:1])
    assert np.array_equal(m1, th[0]) and np.all(c1 == 0)


def test_circular_moments_two_angles_across_pi():
    # the circular mean of pi - 0.1 and -pi + 0.1 is pi (the arithmetic mean is 0);
    # the wrapped deviations are -0.1 and +0.1, so the variance is 0.02
    th = np.zeros((2, 6))
    th[:, 4] = [math.pi - 0.1, -math.pi + 0.1]
    mean, cov = O.moments_circular(th)
    assert abs(abs(mean[4]) - math.pi) < 1e-15
    assert abs(cov[4, 4] - 0.02) < 1e-15
    assert np.count_nonzero(cov) == 1 and np.all(mean[[0, 1, 2, 3, 5]] == 0)
    m_lin, c_lin = O.moments(th)
    assert m_lin[4] == 0 and abs(c_lin[4, 4] - (2 * math.pi - 0.2) ** 2 / 2) < 1e-12   # plain: across the circle


@pytest.mark.parametrize("centre", [0.3, math.pi, -2.5])
def test_circular_moments_symmetric_samples(centre):
    """Angles c +- d_i (so their circular mean is c), each shifted by a random
    multiple of 2 pi: the mean is c mod 2 pi, and the covariance is that of
    [t, d] computed directly."""
    rng = np.random.default_rng(4)
    n = 40
    dev = rng.normal(0, 0.3, (n, 3))
    t = rng.normal(0, 0.1, (2 * n, 3))
    rot = np.concatenate([centre + dev, centre - dev])
    rot += 2 * math.pi * rng.integers(-3, 4, rot.shape)
    th = np.concatenate([t, rot], axis=1)
    mean, cov = O.moments_circular(th)
    assert np.allclose(mean[:3], t.mean(0), atol=1e-15)
    assert np.all(np.abs(np.angle(np.exp(1j * (mean[3:] - centre)))) < 1e-13)
    direct = np.cov(np.concatenate([t, np.concatenate([dev, -dev])], axis=1).T)
    assert np.allclose(cov, direct, atol=1e-13)


def test_circular_moments_shift_equivariance_and_single_particle():
    rng = np.random.default_rng(5)
    th = np.c_[rng.normal(0, 0.1, (50, 3)), rng.uniform(-math.pi, math.pi, (50, 3))]
    th[:, 3:] = 0.8 + 0.4 * np.tanh(th[:, 3:])      # a cluster of angles
    mean, cov = O.moments_circular(th)
    sh = th.copy()
    sh[:, 3:] += 2.9                                # moves the cluster across +-pi
    mean2, cov2 = O.moments_circular(sh)
    assert np.all(np.abs(np.angle(np.exp(1j * (mean2[3:] - mean[3:] - 2.9)))) < 1e-13)
    assert np.allclose(cov2, cov, atol=1e-13) and np.allclose(mean2[:3], mean[:3], atol=1e-15)
    one = np.array([[0.1, 0.2, 0.3, 7.0, -4.0, 0.5]])
    m1, c1 = O.moments_circular(one)
    assert np.allclose(m1, [0.1, 0.2, 0.3, 7.0 - 2 * math.pi, -4.0 + 2 * math.pi, 0.5], atol=1e-15)
    assert np.all(c1 == 0)


def test_single_particle_recovers_known_pose_noise_free():
    """K = 1 reduces Stein ICP to SGD-ICP with Adam; on a noise-free box it
    must land on the generating pose (1 mm, 0.05 deg)."""
    d = synth.make_box_problem(0, K=1, noise=0.0)
    th, mean, cov = O.register(d["ref"], d["src"], d["particles"], O.Params(T=300, m=100, seed=7))
    err = th[0] - d["theta_true"]
    assert np.abs(err[:3]).max() < 1e-3
    assert np.abs(err[3:]).max() < math.radians(0.05)


def test_run_is_deterministic_and_T0_returns_input():
    d = synth.make_box_problem(1, M=300, N=100, K=5)
    p = O.Params(T=5, m=20, seed=3)
    a = O.register(d["ref"], d["src"], d["particles"], p)
    b = O.register(d["ref"], d["src"], d["particles"], p)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    th, mean, _ = O.register(d["ref"], d["src"], d["particles"], O.Params(T=0, m=20))
    assert np.array_equal(th, d["particles"].astype(np.float64))


def test_step_loop_equals_register():
    d = synth.make_box_problem(2, M=400, N=120, K=6)
    p = O.Params(T=4, m=30, seed=9)
    th = d["particles"].astype(np.float64).copy()
    mom, vel = np.zeros_like(th), np.zeros_like(th)
    for t in range(p.T):
        O.step(d["ref"], d["src"], th, mom, vel, p, t)
    th2, _, _ = O.register(d["ref"], d["src"], d["particles"], p)
    assert np.array_equal(th, th2)
