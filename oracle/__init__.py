"""Plain FP64 CPU oracle for Stein ICP -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It is the slow, obviously correct
statement of the method (see `oracle.c` for the readings of the paper it
follows) and shares no code with the CUDA library.

Parity status of each function (what pins it in `tests/test_oracle.py`):
  splitmix64_at   published splitmix64 output vectors
  minibatch       selection invariants and per-index frequency
  rotation        scipy's rotation from fixed-axis angles; orthogonality;
                  central differences for the partial derivatives
  nn / nn2        scipy cKDTree (nearest and second-nearest distances);
                  exact duplicates and self-queries
  KDTree          identical indices and distances to the exhaustive nn on
                  random, clustered, lattice (many exact ties) and
                  duplicated clouds, queries near and far
  icp_grad        central differences of L/2; single-point closed form
  bandwidths      numpy.median; two-particle closed form
  stein_phi       two-particle closed form (incl. wrap across +-pi);
                  SVGD on a Gaussian target; K = 1 reduces to G
  adam            closed form under a constant gradient; three steps under a
                  varying gradient worked out by hand (exact fractions)
  register        K = 1 recovery of a known pose on noise-free data
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _setup(_lib)
    return _lib


_p = ctypes.c_void_p
_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


class _Params(ctypes.Structure):
    _fields_ = [("T", _i32), ("m", _i32), ("lr", _f64), ("beta1", _f64), ("beta2", _f64),
                ("eps", _f64), ("seed", _u64), ("prior", _i32), ("mu", _f64 * 6),
                ("sigma", _f64 * 3), ("kappa", _f64 * 3), ("normals", _p), ("independent", _i32),
                ("tree", _p)]


def _setup(L):
    sig = {
        "or_splitmix64_at": (_u64, [_u64, _u64]),
        "or_mb_key": (_u64, [_u64, _i64, _i64]),
        "or_minibatch": (ctypes.c_int, [_u64, _i64, _i64, _i32, _p]),
        "or_rotation": (None, [_p, _p, _p]),
        "or_nn": (None, [_p, _i64, _p, _i64, _p, _p]),
        "or_nn2": (None, [_p, _i64, _p, _i64, _p, _p, _p]),
        "or_icp_grad": (None, [_p, _i64, _p, _p, _i32, _p, _i32, _p, _p, _p, _p]),
        "or_icp_grad_given_nn": (None, [_p, _p, _p, _i32, _p, _i32, _p, _p, _p]),
        "or_knn": (None, [_p, _i64, _i32, _p, _p]),
        "or_kd_build": (_p, [_p, _i64]),
        "or_kd_free": (None, [_p]),
        "or_kd_nn": (None, [_p, _p, _i64, _p, _p]),
        "or_icp_grad_kd": (None, [_p, _p, _p, _i32, _p, _i32, _p, _p, _p, _p]),
        "or_neighbourhood_cov": (None, [_p, _i64, _i32, _p, _p]),
        "or_log_post_grad": (None, [_p, _p, _i32, _f64, _i32, _p, _p, _p, _p]),
        "or_median": (_f64, [_p, _i64]),
        "or_bandwidths": (None, [_p, _i32, _p, _p]),
        "or_stein_phi": (None, [_p, _p, _i32, _f64, _f64, _p]),
        "or_adam": (None, [_p, _p, _p, _p, _i64, _i64, _f64, _f64, _f64, _f64]),
        "or_moments": (None, [_p, _i32, _p, _p]),
        "or_moments_circular": (None, [_p, _i32, _p, _p]),
        "or_step": (None, [_p, _i64, _p, _i64, _p, _p, _p, _i32, _p, _i64, _p, _p, _p, _p]),
        "or_register": (ctypes.c_int, [_p, _i64, _p, _i64, _p, _i32, _p, _p, _p, _p]),
        "or_num_threads": (ctypes.c_int, []),
        "or_set_threads": (None, [ctypes.c_int]),
        "or_mlp_nparam": (ctypes.c_int, []),
        "or_bf16": (_f64, [_f64]),
        "or_mlp_features": (None, [_p, _p]),
        "or_mlp_forward": (None, [_p, _p, _i64, ctypes.c_int, _p]),
        "or_mlp_loss_grad": (_f64, [_p, _p, _p, _i64, _f64, _f64, ctypes.c_int, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64a(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Run parameters (Sec. V: Adam step 0.01-0.03, minibatch 150-300)."""
    T: int = 100
    m: int = 100
    lr: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 0
    prior: int = 0
    mu: tuple = (0.0,) * 6
    sigma: tuple = (1.0,) * 3
    kappa: tuple = (1.0,) * 3
    normals: object = None     # None: point-to-point; M x 3 unit normals: point-to-plane (R16)
    independent: bool = False  # independent SGD-ICP runs, no Stein coupling (R17)
    tree: object = None        # None: exhaustive search; a KDTree of the reference: the same answers, faster

    def c(self) -> _Params:
        p = _Params()
        p.T, p.m, p.lr, p.beta1, p.beta2, p.eps = self.T, self.m, self.lr, self.beta1, self.beta2, self.eps
        p.seed, p.prior = self.seed & ((1 << 64) - 1), self.prior
        p.mu[:] = list(self.mu)
        p.sigma[:] = list(self.sigma)
        p.kappa[:] = list(self.kappa)
        p.independent = 1 if self.independent else 0
        if self.normals is not None:
            self._normals64 = _f64a(self.normals)     # kept alive with the parameters
            p.normals = _ptr(self._normals64)
        if self.tree is not None:
            p.tree = self.tree.handle
        return p


def num_threads() -> int:
    return _L().or_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (timing only; results do not depend on it)."""
    _L().or_set_threads(int(n))


def splitmix64_at(state: int, k: int) -> int:
    return int(_L().or_splitmix64_at(state & ((1 << 64) - 1), k))


def mb_key(seed: int, t: int, i: int) -> int:
    return int(_L().or_mb_key(seed & ((1 << 64) - 1), t, i))


def minibatch(seed: int, t: int, N: int, m: int) -> np.ndarray:
    out = np.empty(m, np.int32)
    rc = _L().or_minibatch(seed & ((1 << 64) - 1), t, N, m, _ptr(out))
    if rc != 0:
        raise ValueError(f"or_minibatch rc={rc}")
    return out


def rotation(theta):
    th = _f64a(theta)
    R = np.empty(9)
    dR = np.empty(27)
    _L().or_rotation(_ptr(th), _ptr(R), _ptr(dR))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def nn(ref, q):
    ref, q = _f32(ref), _f64a(q)
    n = q.shape[0]
    idx = np.empty(n, np.int64)
    d2 = np.empty(n)
    _L().or_nn(_ptr(ref), ref.shape[0], _ptr(q), n, _ptr(idx), _ptr(d2))
    return idx, d2


def nn2(ref, q):
    ref, q = _f32(ref), _f64a(q)
    n = q.shape[0]
    idx = np.empty(n, np.int64)
    d2 = np.empty(n)
    d2b = np.empty(n)
    _L().or_nn2(_ptr(ref), ref.shape[0], _ptr(q), n, _ptr(idx), _ptr(d2), _ptr(d2b))
    return idx, d2, d2b


class KDTree:
    """k-d tree of a reference cloud (oracle.c, or_kd_build): nearest
    neighbours identical to the exhaustive search `nn`, lowest index on ties,
    in far fewer distance evaluations.  Pass it as Params(tree=...) to make
    `step` and `register` search through it."""

    def __init__(self, ref):
        self.ref = _f32(ref).copy()          # the tree points into this array
        self.handle = _L().or_kd_build(_ptr(self.ref), self.ref.shape[0])
        if not self.handle:
            raise ValueError("or_kd_build failed")

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.or_kd_free(h)

    def nn(self, q):
        q = _f64a(q).reshape(-1, 3)
        n = q.shape[0]
        idx = np.empty(n, np.int64)
        d2 = np.empty(n)
        _L().or_kd_nn(self.handle, _ptr(q), n, _ptr(idx), _ptr(d2))
        return idx, d2

    def icp_grad(self, src, mb, theta, normals=None):
        """icp_grad of the tree's reference, searching through the tree."""
        src = _f32(src)
        mb = np.ascontiguousarray(mb, np.int32)
        th = _f64a(theta).reshape(-1, 6)
        K, m = th.shape[0], mb.shape[0]
        g = np.empty((K, 6))
        nnk = np.empty((K, m), np.int64)
        loss = np.empty(K)
        keep, np_ = _normals_ptr(normals, self.ref.shape[0])
        _L().or_icp_grad_kd(self.handle, _ptr(src), _ptr(mb), m, _ptr(th), K, np_, _ptr(g), _ptr(nnk), _ptr(loss))
        return g, nnk, loss


def _check_tree(ref, params):
    if params.tree is not None and not (params.tree.ref.shape == ref.shape and np.array_equal(params.tree.ref, ref)):
        raise ValueError("Params.tree was built on another reference cloud")


def transform(theta, pts):
    """R(theta) p + u for each row of pts (float64 result)."""
    R, _ = rotation(theta)
    return np.asarray(pts, np.float64) @ R.T + np.asarray(theta[:3], np.float64)


def _normals_ptr(normals, M):
    if normals is None:
        return None, None
    n = _f64a(normals).reshape(M, 3)
    return n, _ptr(n)


def icp_grad(ref, src, mb, theta, normals=None):
    """gbar, correspondences and L/2 of each particle; with normals (M x 3)
    the point-to-plane metric (reading R16 of oracle.c)."""
    ref, src = _f32(ref), _f32(src)
    mb = np.ascontiguousarray(mb, np.int32)
    th = _f64a(theta).reshape(-1, 6)
    K, m = th.shape[0], mb.shape[0]
    g = np.empty((K, 6))
    nnk = np.empty((K, m), np.int64)
    loss = np.empty(K)
    keep, np_ = _normals_ptr(normals, ref.shape[0])
    _L().or_icp_grad(_ptr(ref), ref.shape[0], _ptr(src), _ptr(mb), m, _ptr(th), K, np_, _ptr(g),
                     _ptr(nnk), _ptr(loss))
    return g, nnk, loss


def icp_grad_given_nn(ref, src, mb, theta, nnk, normals=None):
    ref, src = _f32(ref), _f32(src)
    mb = np.ascontiguousarray(mb, np.int32)
    th = _f64a(theta).reshape(-1, 6)
    K, m = th.shape[0], mb.shape[0]
    nnk = np.ascontiguousarray(nnk, np.int64).reshape(K, m)
    g = np.empty((K, 6))
    keep, np_ = _normals_ptr(normals, ref.shape[0])
    _L().or_icp_grad_given_nn(_ptr(ref), _ptr(src), _ptr(mb), m, _ptr(th), K, _ptr(nnk), np_, _ptr(g))
    return g


def knn(ref, k: int, with_d2: bool = False):
    """The k nearest reference points of every reference point (itself
    included), nearest first, ranked by exact fp64 squared distance with ties
    to the lower index: M x k indices (and the M x k squared distances)."""
    ref = _f32(ref)
    if not 1 <= k <= min(64, ref.shape[0]):
        raise ValueError("knn needs 1 <= k <= min(64, M)")
    idx = np.empty((ref.shape[0], k), np.int64)
    d2 = np.empty((ref.shape[0], k))
    _L().or_knn(_ptr(ref), ref.shape[0], k, _ptr(idx), _ptr(d2))
    return (idx, d2) if with_d2 else idx


def neighbourhood_cov(ref, idx):
    ref = _f32(ref)
    idx = np.ascontiguousarray(idx, np.int64)
    M, k = idx.shape
    cov = np.empty((M, 9))
    _L().or_neighbourhood_cov(_ptr(ref), M, k, _ptr(idx), _ptr(cov))
    return cov.reshape(M, 3, 3)


def normals(ref, k: int):
    """Unit normal of every reference point (reading R16 of oracle.c): the
    eigenvector of the smallest eigenvalue of the fp64 covariance of its k
    nearest neighbours, from LAPACK (numpy.linalg.eigh).  Returns the
    normals (M x 3) and the ascending eigenvalues (M x 3)."""
    w, v = np.linalg.eigh(neighbourhood_cov(ref, knn(ref, k)))
    return np.ascontiguousarray(v[:, :, 0]), w


def log_post_grad(theta, gbar, N, prior=0, mu=(0,) * 6, sigma=(1,) * 3, kappa=(1,) * 3):
    th = _f64a(theta).reshape(-1, 6)
    gb = _f64a(gbar).reshape(-1, 6)
    K = th.shape[0]
    G = np.empty((K, 6))
    _L().or_log_post_grad(_ptr(th), _ptr(gb), K, float(N), prior, _ptr(_f64a(mu)),
                          _ptr(_f64a(sigma)), _ptr(_f64a(kappa)), _ptr(G))
    return G


def median(x) -> float:
    x = _f64a(x).ravel()
    return float(_L().or_median(_ptr(x), x.size))


def bandwidths(theta):
    th = _f64a(theta).reshape(-1, 6)
    ht, hr = _f64(), _f64()
    _L().or_bandwidths(_ptr(th), th.shape[0], ctypes.byref(ht), ctypes.byref(hr))
    return ht.value, hr.value


def stein_phi(theta, G, h_t, h_r):
    th = _f64a(theta).reshape(-1, 6)
    G = _f64a(G).reshape(-1, 6)
    phi = np.empty_like(th)
    _L().or_stein_phi(_ptr(th), _ptr(G), th.shape[0], float(h_t), float(h_r), _ptr(phi))
    return phi


def adam(x, mom, vel, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays x, mom, vel."""
    for a in (x, mom, vel):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64a(g)
    _L().or_adam(_ptr(x), _ptr(mom), _ptr(vel), _ptr(g), x.size, t, lr, beta1, beta2, eps)


def moments(theta):
    th = _f64a(theta).reshape(-1, 6)
    mean = np.empty(6)
    cov = np.empty(36)
    _L().or_moments(_ptr(th), th.shape[0], _ptr(mean), _ptr(cov))
    return mean, cov.reshape(6, 6)


def moments_circular(theta):
    """Mean and covariance with circular statistics for the three angles
    (reading R15 of oracle.c)."""
    th = _f64a(theta).reshape(-1, 6)
    mean = np.empty(6)
    cov = np.empty(36)
    _L().or_moments_circular(_ptr(th), th.shape[0], _ptr(mean), _ptr(cov))
    return mean, cov.reshape(6, 6)


def step(ref, src, th, mom, vel, params: Params, t: int):
    """Iteration t in place on th, mom, vel (float64 K x 6); returns the
    iteration's gbar, G, phi and (h_t, h_r)."""
    ref, src = _f32(ref), _f32(src)
    _check_tree(ref, params)
    for a in (th, mom, vel):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    K = th.shape[0]
    gbar, G, phi, h = np.empty((K, 6)), np.empty((K, 6)), np.empty((K, 6)), np.empty(2)
    p = params.c()
    _L().or_step(_ptr(ref), ref.shape[0], _ptr(src), src.shape[0], _ptr(th), _ptr(mom), _ptr(vel),
                 K, ctypes.byref(p), t, _ptr(gbar), _ptr(G), _ptr(phi), _ptr(h))
    return dict(gbar=gbar, G=G, phi=phi, h=(h[0], h[1]))


def register(ref, src, theta0, params: Params):
    ref, src, th0 = _f32(ref), _f32(src), _f32(theta0).reshape(-1, 6)
    _check_tree(ref, params)
    K = th0.shape[0]
    th = np.empty((K, 6))
    mean = np.empty(6)
    cov = np.empty(36)
    p = params.c()
    rc = _L().or_register(_ptr(ref), ref.shape[0], _ptr(src), src.shape[0], _ptr(th0), K,
                          ctypes.byref(p), _ptr(th), _ptr(mean), _ptr(cov))
    if rc != 0:
        raise ValueError(f"or_register rc={rc}")
    return th, mean, cov.reshape(6, 6)


# ---------------------------------------------------------------- learned closest-point field

MLP_D_IN, MLP_H, MLP_D_OUT = 112, 128, 16


def mlp_nparam() -> int:
    return _L().or_mlp_nparam()


def bf16(x: float) -> float:
    return float(_L().or_bf16(float(x)))


def mlp_features(qn):
    qn = _f64a(qn).reshape(3)
    x = np.empty(MLP_D_IN)
    _L().or_mlp_features(_ptr(qn), _ptr(x))
    return x


def mlp_forward(params, qn, bf16ops=False):
    params, qn = _f64a(params), _f64a(qn).reshape(-1, 3)
    out = np.empty((qn.shape[0], MLP_D_OUT))
    _L().or_mlp_forward(_ptr(params), _ptr(qn), qn.shape[0], int(bf16ops), _ptr(out))
    return out


def mlp_loss_grad(params, qn, dstar, lam=0.1, delta=0.02, bf16ops=False, cstar=None):
    params, qn, dstar = _f64a(params), _f64a(qn).reshape(-1, 3), _f64a(dstar).reshape(-1, 3)
    grad = np.empty(mlp_nparam())
    cs = None if cstar is None else _f64a(cstar)
    loss = _L().or_mlp_loss_grad(_ptr(params), _ptr(qn), _ptr(dstar), qn.shape[0], lam, delta, int(bf16ops),
                                 None if cs is None else _ptr(cs), _ptr(grad))
    return float(loss), grad


def mlp_split(params):
    """Views W1, b1, W2, b2, W3, b3 of a flat parameter vector."""
    p = np.asarray(params)
    sizes = [(MLP_H, MLP_D_IN), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_D_OUT, MLP_H), (MLP_D_OUT,)]
    out, o = [], 0
    for sh in sizes:
        n = int(np.prod(sh))
        out.append(p[o:o + n].reshape(sh))
        o += n
    return out


# ---------------------------------------------------------------- distribution quality (reading R17)

def gaussian_kl(m0, S0, m1, S1):
    """KL(N(m0, S0) || N(m1, S1)) in closed form (float64):
    1/2 [tr(S1^-1 S0) + (m1 - m0)^T S1^-1 (m1 - m0) - d + ln det S1 - ln det S0]."""
    m0, m1 = np.asarray(m0, np.float64), np.asarray(m1, np.float64)
    S0, S1 = np.asarray(S0, np.float64), np.asarray(S1, np.float64)
    d = m0.shape[0]
    S1i = np.linalg.inv(S1)
    dm = m1 - m0
    _, ld0 = np.linalg.slogdet(S0)
    _, ld1 = np.linalg.slogdet(S1)
    return 0.5 * (np.trace(S1i @ S0) + dm @ S1i @ dm - d + ld1 - ld0)


def _gauss_logpdf(x, m, S):
    d = m.shape[0]
    L = np.linalg.cholesky(S)
    y = np.linalg.solve(L, (x - m).T)
    return -0.5 * np.sum(y * y, axis=0) - np.log(np.diag(L)).sum() - 0.5 * d * np.log(2 * np.pi)


def gaussian_ovl(m0, S0, m1, S1, z0, z1):
    """Overlapping coefficient, integral of min(p0, p1), of two Gaussians by
    Monte Carlo on given standard-normal draws z0, z1 ([n][d] each):
    1/2 [mean over x = m0 + L0 z0 of min(1, p1/p0) + mean over x = m1 + L1 z1
    of min(1, p0/p1)], L the Cholesky factors."""
    m0, m1 = np.asarray(m0, np.float64), np.asarray(m1, np.float64)
    S0, S1 = np.asarray(S0, np.float64), np.asarray(S1, np.float64)
    x0 = m0 + np.asarray(z0, np.float64) @ np.linalg.cholesky(S0).T
    x1 = m1 + np.asarray(z1, np.float64) @ np.linalg.cholesky(S1).T
    a = np.minimum(1.0, np.exp(_gauss_logpdf(x0, m1, S1) - _gauss_logpdf(x0, m0, S0)))
    b = np.minimum(1.0, np.exp(_gauss_logpdf(x1, m0, S0) - _gauss_logpdf(x1, m1, S1)))
    return 0.5 * (a.mean() + b.mean())


# ---------------------------------------------------------------- odometry chaining (reading R18)
#
# R18: the odometry experiment chains scan-to-scan estimates as
# T_E = T^1_0 T^2_1 ... T^l_(l-1) of the mean transforms and combines their
# covariances to fourth order (an approximation it cites, not prints).  Read
# here: each scan pair's distribution is its particles' mean pose (where
# their left perturbations average to zero) with the sample covariance of
# those perturbations; two independent distributions compound to the mean
# T1 T2 with S1 + Ad(T1) S2 Ad(T1)^T plus the published fourth-order terms.
#
# A pose is T = [[C, r], [0, 1]] with C = R(theta) and r = theta[:3]; a pose
# distribution is a mean pose T_bar and the covariance of the left
# perturbation xi = [rho; phi] in T = exp(xi^) T_bar.  Matrix exponential and
# logarithm come from scipy.linalg (expm, logm), not from closed forms.

def _hat(xi):
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    X[:3, 3] = rho
    return X


def se3_exp(xi):
    import scipy.linalg
    return scipy.linalg.expm(_hat(xi))


def se3_log(T):
    import scipy.linalg
    X = np.real(scipy.linalg.logm(np.asarray(T, np.float64)))
    return np.r_[X[:3, 3], X[2, 1], X[0, 2], X[1, 0]]


def pose_matrix(theta):
    R, _ = rotation(theta)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(theta[:3], np.float64)
    return T


def adjoint(T):
    C, r = T[:3, :3], T[:3, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = C
    A[3:, 3:] = C
    A[:3, 3:] = _hat(np.r_[0, 0, 0, r])[:3, :3] @ C
    return A


def pose_distribution(particles, iters=50):
    """Mean pose (the point where the left perturbations of the particles
    average to zero, found by fixed-point iteration from the pose of the mean
    parameters) and the covariance of those perturbations (divisor K - 1)."""
    th = np.asarray(particles, np.float64).reshape(-1, 6)
    Ts = [pose_matrix(t) for t in th]
    Tb = pose_matrix(moments_circular(th)[0])
    for _ in range(iters):
        xis = np.array([se3_log(T @ np.linalg.inv(Tb)) for T in Ts])
        step = xis.mean(0)
        Tb = se3_exp(step) @ Tb
        if np.abs(step).max() < 1e-15:
            break
    xis = np.array([se3_log(T @ np.linalg.inv(Tb)) for T in Ts])
    K = th.shape[0]
    cov = xis.T @ xis / (K - 1) if K > 1 else np.zeros((6, 6))
    return Tb, cov


def _angle3(M):
    return -np.trace(M) * np.eye(3) + M


def _angle6(S):
    Spp, Spf = S[3:, 3:], S[:3, 3:]
    A = np.zeros((6, 6))
    A[:3, :3] = _angle3(Spp)
    A[:3, 3:] = _angle3(Spf + Spf.T)
    A[3:, 3:] = _angle3(Spp)
    return A


def _bb(A, B):
    return _angle3(A) @ _angle3(B) + _angle3(B @ A)


def compound(T1, S1, T2, S2, order=4):
    """The distribution of T1 T2 for independent T1 = exp(xi1^) T1_bar,
    T2 = exp(xi2^) T2_bar: mean T1_bar T2_bar and covariance to second order,
    S1 + Ad(T1_bar) S2 Ad(T1_bar)^T, or with the fourth-order terms."""
    T1, T2 = np.asarray(T1, np.float64), np.asarray(T2, np.float64)
    S1, S2 = np.asarray(S1, np.float64), np.asarray(S2, np.float64)
    A = adjoint(T1)
    S2p = A @ S2 @ A.T
    S = S1 + S2p
    if order == 4:
        a1, a2 = _angle6(S1), _angle6(S2p)
        S = S + (a1 @ S2p + S2p @ a1.T + a2 @ S1 + S1 @ a2.T) / 12.0
        s1rr, s1rp, s1pp = S1[:3, :3], S1[:3, 3:], S1[3:, 3:]
        s2rr, s2rp, s2pp = S2p[:3, :3], S2p[:3, 3:], S2p[3:, 3:]
        B = np.zeros((6, 6))
        B[:3, :3] = _bb(s1pp, s2rr) + _bb(s1rp.T, s2rp) + _bb(s1rp, s2rp.T) + _bb(s1rr, s2pp)
        B[:3, 3:] = _bb(s1pp, s2rp.T) + _bb(s1rp.T, s2pp)
        B[3:, :3] = B[:3, 3:].T
        B[3:, 3:] = _bb(s1pp, s2pp)
        S = S + B / 4.0
    return T1 @ T2, S
