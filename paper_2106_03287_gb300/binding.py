"""ctypes binding of libsteinicp (include/steinicp.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks shapes and dtypes, allocates outputs next
to the inputs (numpy arrays for host calls, torch CUDA tensors for device
calls) and passes raw pointers.  Host inputs are numpy arrays (on_device = 0);
device inputs are torch CUDA tensors (on_device = 1).  A call whose C code
returns an error raises SicpError with the library's message.

There is no fallback: if the shared library is missing the import of this
module still works, but the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SICP_CHECKED=1: the bounds-checked build (build.build(checked=True)) instead of the normal one
LIB_PATH = os.path.join(_HERE, "libsteinicp_checked.so" if os.environ.get("SICP_CHECKED") == "1"
                        else "libsteinicp.so")

SICP_OK = 0
SICP_EINVAL = -1
SICP_ENOREF = -2
SICP_ENOMEM = -3
SICP_ECUDA = -4
SICP_ETIMEOUT = -5
SICP_ENOSURROGATE = -6

SICP_NN_BRUTE_FP32 = 0
SICP_NN_BRUTE_BF16 = 1
SICP_NN_GRID = 2
SICP_NN_SURROGATE = 3
SICP_POINT_TO_PLANE = 0x100   # metric flag, OR-ed into nn_mode / mode (with the grid, fp32 or bf16 search)
SICP_INDEPENDENT = 0x200      # sicp_register flag: independent SGD-ICP runs (the Monte Carlo reference)

_CODES = {-1: "EINVAL", -2: "ENOREF", -3: "ENOMEM", -4: "ECUDA", -5: "ETIMEOUT", -6: "ENOSURROGATE"}

# Every C entry point declared in include/steinicp.h.
EXPORTS = (
    "sicp_default_params", "sicp_create", "sicp_destroy", "sicp_last_error", "sicp_set_reference",
    "sicp_register", "sicp_minibatch", "sicp_nn", "sicp_icp_grad", "sicp_stein_adam", "sicp_moments",
    "sicp_moments_circular", "sicp_reference_normals", "sicp_gaussian_kl", "sicp_gaussian_ovl",
    "sicp_pose_distribution", "sicp_compound", "sicp_stats", "sicp_profile", "sicp_icp_grad_noalloc", "sicp_register_batched", "sicp_autotune_batched",
    "sicp_surrogate_train", "sicp_surrogate_params", "sicp_surrogate_loss_grad", "sicp_surrogate_infer",
    "sicp_register_continue", "sicp_surrogate_save", "sicp_surrogate_load",
    "sicp_export_state", "sicp_import_state", "sicp_resume", "sicp_set_memory_limit", "sicp_set_wait_check",
    "sicp_trace_batched", "sicp_read_batched_trace", "sicp_surrogate_train_run", "sicp_set_telemetry",
    "sicp_read_telemetry", "sicp_check_status",
)

SURROGATE_NPARAM = 33040


class SicpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class sicp_params(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_int32), ("m", ctypes.c_int32),
        ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("nn_mode", ctypes.c_int32), ("surrogate_iters", ctypes.c_int32), ("prior", ctypes.c_int32),
        ("prior_mu", ctypes.c_float * 6), ("prior_sigma", ctypes.c_float * 3), ("prior_kappa", ctypes.c_float * 3),
        ("surrogate_min_conf", ctypes.c_float),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2106_03287_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U64, F32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
        pp = ctypes.POINTER(sicp_params)
        sig = {
            "sicp_default_params": (None, [pp]),
            "sicp_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P]),
            "sicp_destroy": (None, [P]),
            "sicp_last_error": (ctypes.c_char_p, [P]),
            "sicp_set_reference": (ctypes.c_int, [P, P, I64, F32, ctypes.c_int]),
            "sicp_register": (ctypes.c_int, [P, P, I64, P, I32, pp, P, P, P, ctypes.c_int]),
            "sicp_minibatch": (ctypes.c_int, [P, U64, I64, I32, I64, I32, P, ctypes.c_int]),
            "sicp_nn": (ctypes.c_int, [P, P, I64, I32, P, P, ctypes.c_int]),
            "sicp_icp_grad": (ctypes.c_int, [P, P, I64, P, I32, P, I32, I32, P, P, ctypes.c_int]),
            "sicp_stein_adam": (ctypes.c_int, [P, P, P, P, P, I32, I64, I64, pp, P, P, ctypes.c_int]),
            "sicp_moments": (ctypes.c_int, [P, P, I32, P, P, ctypes.c_int]),
            "sicp_moments_circular": (ctypes.c_int, [P, P, I32, P, P, ctypes.c_int]),
            "sicp_stats": (ctypes.c_int, [P, ctypes.c_int, P]),
            "sicp_profile": (ctypes.c_int, [P, ctypes.c_int, P]),
            "sicp_icp_grad_noalloc": (ctypes.c_int, [P, I64, P, I64, P, I32, P, I32, P, P]),
            "sicp_register_batched": (ctypes.c_int, [P, I32, P, P, P, P, P, P, pp, P, P, P, ctypes.c_int]),
            "sicp_autotune_batched": (ctypes.c_int, [P, I32, P, P, P, P, P, P, pp, I32, ctypes.c_char_p, P, P, P,
                                                     ctypes.c_int]),
            "sicp_surrogate_train": (ctypes.c_int, [P, I64, U64, I32, I32, F32, P]),
            "sicp_surrogate_params": (ctypes.c_int, [P, ctypes.c_int, P, P]),
            "sicp_surrogate_loss_grad": (ctypes.c_int, [P, P, P, P, I64, F32, F32, P, P]),
            "sicp_surrogate_infer": (ctypes.c_int, [P, P, I64, P, P, ctypes.c_int]),
            "sicp_register_continue": (ctypes.c_int, [P, P, I64, P, I32, I64, pp, P, P, ctypes.c_int]),
            "sicp_export_state": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
            "sicp_import_state": (ctypes.c_int, [P, P, ctypes.c_size_t]),
            "sicp_resume": (ctypes.c_int, [P, P, I64, pp, P, P, P, ctypes.c_int]),
            "sicp_surrogate_save": (ctypes.c_int, [P, ctypes.c_char_p]),
            "sicp_surrogate_load": (ctypes.c_int, [P, ctypes.c_char_p]),
            "sicp_reference_normals": (ctypes.c_int, [P, I32, P, ctypes.c_int]),
            "sicp_gaussian_kl": (ctypes.c_int, [P, P, P, P, I32, P]),
            "sicp_gaussian_ovl": (ctypes.c_int, [P, P, P, P, I32, P, P, ctypes.c_int64, P]),
            "sicp_pose_distribution": (ctypes.c_int, [P, I32, P, P]),
            "sicp_compound": (ctypes.c_int, [P, P, P, P, I32, P, P]),
            "sicp_set_memory_limit": (ctypes.c_int, [P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "sicp_set_wait_check": (ctypes.c_int, [P, ctypes.c_int, I64]),
            "sicp_trace_batched": (ctypes.c_int, [P, I32]),
            "sicp_surrogate_train_run": (ctypes.c_int, [P, P, I64, P, I32, I64, U64, I32, I32, F32, P, ctypes.c_int]),
            "sicp_read_batched_trace": (ctypes.c_int, [P, P, P, P, P, P, P]),
            "sicp_set_telemetry": (ctypes.c_int, [P, ctypes.c_int]),
            "sicp_read_telemetry": (ctypes.c_int, [P, P, I32, ctypes.POINTER(I32)]),
            "sicp_check_status": (ctypes.c_int, [ctypes.POINTER(I32), ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- marshalling helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _on_device(*arrays) -> int:
    dev = [_is_torch(a) and a.is_cuda for a in arrays if a is not None]
    if any(dev) and not all(dev):
        raise ValueError("mix of device tensors and host arrays in one call")
    return int(bool(dev) and dev[0])


def _ptr(a, dtype):
    if a is None:
        return None
    if _is_torch(a):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise ValueError(f"tensor must be contiguous {tdt}, got {a.dtype}")
        return ctypes.c_void_p(a.data_ptr())
    if a.dtype != dtype or not a.flags.c_contiguous:
        raise ValueError(f"array must be C-contiguous {np.dtype(dtype)}, got {a.dtype}")
    return a.ctypes.data_as(ctypes.c_void_p)


def _empty(like, shape, dtype):
    if _is_torch(like) and like.is_cuda:
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=like.device)
    return np.empty(shape, dtype=dtype)


def _host(a, dtype):
    if _is_torch(a):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _check(ctx, rc: int):
    if rc != SICP_OK:
        raise SicpError(rc, lib().sicp_last_error(ctx).decode())


# ---------------------------------------------------------------- entry points

def sicp_default_params(**overrides) -> sicp_params:
    p = sicp_params()
    lib().sicp_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k in ("prior_mu", "prior_sigma", "prior_kappa"):
            getattr(p, k)[:] = [float(x) for x in v]
        else:
            setattr(p, k, v)
    return p


def sicp_create(device: int = 0, stream=None):
    """Context on CUDA `device`; `stream` is a torch.cuda.Stream or raw handle (None: own stream)."""
    h = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib().sicp_create(ctypes.byref(h), device, s)
    if rc != SICP_OK:
        raise SicpError(rc, f"sicp_create(device={device}) failed")
    return h


def sicp_destroy(ctx) -> None:
    lib().sicp_destroy(ctx)


def sicp_last_error(ctx) -> str:
    return lib().sicp_last_error(ctx).decode()


_REF_SIZE = {}   # reference size of each context, as set through this binding


def ctx_reference_size(ctx) -> int:
    """M of the reference last set on `ctx` through sicp_set_reference."""
    if ctx.value not in _REF_SIZE:
        raise SicpError(SICP_ENOREF, "no reference cloud set through this binding")
    return _REF_SIZE[ctx.value]


def sicp_set_reference(ctx, xyz, cell_size: float = 0.0) -> None:
    xyz = _host(xyz, np.float32)
    _REF_SIZE.pop(ctx.value, None)
    _check(ctx, lib().sicp_set_reference(ctx, _ptr(xyz, np.float32), xyz.shape[0], float(cell_size),
                                         _on_device(xyz)))
    _REF_SIZE[ctx.value] = int(xyz.shape[0])


def sicp_register(ctx, src_xyz, particles, params: sicp_params):
    """Returns (particles_out [K][6] float32, mean [6] float64, cov [6][6] float64)."""
    src_xyz, particles = _host(src_xyz, np.float32), _host(particles, np.float32)
    K = particles.shape[0]
    out = _empty(particles, (K, 6), np.float32)
    mean = _empty(particles, (6,), np.float64)
    cov = _empty(particles, (6, 6), np.float64)
    _check(ctx, lib().sicp_register(ctx, _ptr(src_xyz, np.float32), src_xyz.shape[0],
                                    _ptr(particles, np.float32), K, ctypes.byref(params),
                                    _ptr(out, np.float32), _ptr(mean, np.float64), _ptr(cov, np.float64),
                                    _on_device(src_xyz, particles)))
    return out, mean, cov


def sicp_register_continue(ctx, src_xyz, state, t0: int, params: sicp_params):
    """T = params.T more iterations of a run that has done t0; state [3][K][6]
    float32 (particles, Adam m, Adam v) is updated in place.  Returns (mean [6], cov [6][6])."""
    src_xyz = _host(src_xyz, np.float32)
    if state.shape[0] != 3 or state.shape[2] != 6:
        raise ValueError("state must be [3][K][6]")
    K = state.shape[1]
    mean = _empty(state, (6,), np.float64)
    cov = _empty(state, (6, 6), np.float64)
    _check(ctx, lib().sicp_register_continue(ctx, _ptr(src_xyz, np.float32), src_xyz.shape[0], _ptr(state, np.float32),
                                             K, int(t0), ctypes.byref(params), _ptr(mean, np.float64),
                                             _ptr(cov, np.float64), _on_device(src_xyz, state)))
    return mean, cov


def sicp_export_state(ctx) -> bytes:
    """The context's run state (K, iterations done, seed, particles and Adam
    moments, checksummed) as bytes."""
    n = ctypes.c_size_t(0)
    _check(ctx, lib().sicp_export_state(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib().sicp_export_state(ctx, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def sicp_import_state(ctx, data: bytes):
    """Make bytes from sicp_export_state the context's run state."""
    data = bytes(data)
    buf = ctypes.create_string_buffer(data, len(data))
    _check(ctx, lib().sicp_import_state(ctx, buf, len(data)))


def sicp_resume(ctx, src_xyz, params: sicp_params):
    """params.T more iterations of the context's run state.  Returns
    (particles [K][6], mean [6], cov [6][6])."""
    n = ctypes.c_size_t(0)
    _check(ctx, lib().sicp_export_state(ctx, None, ctypes.byref(n)))   # 36 + 72 K bytes
    K = (n.value - 36) // 72
    src_xyz = _host(src_xyz, np.float32)
    out = _empty(src_xyz, (K, 6), np.float32)
    mean = _empty(src_xyz, (6,), np.float64)
    cov = _empty(src_xyz, (6, 6), np.float64)
    _check(ctx, lib().sicp_resume(ctx, _ptr(src_xyz, np.float32), src_xyz.shape[0], ctypes.byref(params),
                                  _ptr(out, np.float32), _ptr(mean, np.float64), _ptr(cov, np.float64),
                                  _on_device(src_xyz)))
    return out, mean, cov


def sicp_minibatch(ctx, seed: int, t0: int, T: int, N: int, m: int, device=None):
    """Minibatch indices [T][m] int32 (host array, or a tensor on `device`)."""
    if device is not None:
        import torch
        out = torch.empty((T, m), dtype=torch.int32, device=device)
        on = 1
    else:
        out = np.empty((T, m), np.int32)
        on = 0
    _check(ctx, lib().sicp_minibatch(ctx, seed & ((1 << 64) - 1), t0, T, N, m, _ptr(out, np.int32), on))
    return out


def sicp_nn(ctx, q, mode: int = SICP_NN_GRID):
    """Nearest reference index [n] int32 and squared distance [n] float32 per query [n][3]."""
    q = _host(q, np.float32)
    n = q.shape[0]
    idx = _empty(q, (n,), np.int32)
    d2 = _empty(q, (n,), np.float32)
    _check(ctx, lib().sicp_nn(ctx, _ptr(q, np.float32), n, mode, _ptr(idx, np.int32), _ptr(d2, np.float32),
                              _on_device(q)))
    return idx, d2


def sicp_icp_grad(ctx, src_xyz, mb, particles, mode: int = SICP_NN_GRID, want_nn: bool = True):
    """Mean gradients [K][6] float32 and correspondences [K][m] int32 (or None)."""
    src_xyz, mb, particles = _host(src_xyz, np.float32), _host(mb, np.int32), _host(particles, np.float32)
    K, m = particles.shape[0], mb.shape[0]
    g = _empty(particles, (K, 6), np.float32)
    nn = _empty(particles, (K, m), np.int32) if want_nn else None
    _check(ctx, lib().sicp_icp_grad(ctx, _ptr(src_xyz, np.float32), src_xyz.shape[0], _ptr(mb, np.int32), m,
                                    _ptr(particles, np.float32), K, mode, _ptr(g, np.float32),
                                    _ptr(nn, np.int32), _on_device(src_xyz, mb, particles)))
    return g, nn


def sicp_stein_adam(ctx, particles, adam_m, adam_v, gbar, N: int, t: int, params: sicp_params):
    """In-place update of particles, adam_m, adam_v ([K][6] float32); returns (phi [K][6], h [2])."""
    K = particles.shape[0]
    phi = _empty(particles, (K, 6), np.float32)
    h = _empty(particles, (2,), np.float32)
    _check(ctx, lib().sicp_stein_adam(ctx, _ptr(particles, np.float32), _ptr(adam_m, np.float32),
                                      _ptr(adam_v, np.float32), _ptr(gbar, np.float32), K, N, t,
                                      ctypes.byref(params), _ptr(phi, np.float32), _ptr(h, np.float32),
                                      _on_device(particles, adam_m, adam_v, gbar)))
    return phi, h


def sicp_moments(ctx, particles):
    particles = _host(particles, np.float32)
    mean = _empty(particles, (6,), np.float64)
    cov = _empty(particles, (6, 6), np.float64)
    _check(ctx, lib().sicp_moments(ctx, _ptr(particles, np.float32), particles.shape[0], _ptr(mean, np.float64),
                                   _ptr(cov, np.float64), _on_device(particles)))
    return mean, cov


def sicp_reference_normals(ctx, k: int = 10, want: bool = True, device: bool = False):
    """Compute (and keep on the context, for SICP_POINT_TO_PLANE) the unit
    normals of the current reference from k nearest neighbours; returns them
    as [M][3] float32 (a numpy array, or a CUDA tensor with device=True), or
    None with want=False."""
    out = None
    if want:
        M = int(ctx_reference_size(ctx))
        if device:
            import torch
            out = torch.empty((M, 3), dtype=torch.float32, device="cuda")
        else:
            out = np.empty((M, 3), np.float32)
    _check(ctx, lib().sicp_reference_normals(ctx, int(k), _ptr(out, np.float32) if out is not None else None,
                                             1 if device else 0))
    return out


def _gauss_args(m0, S0, m1, S1):
    m0, m1 = np.ascontiguousarray(m0, np.float64).ravel(), np.ascontiguousarray(m1, np.float64).ravel()
    d = m0.shape[0]
    S0 = np.ascontiguousarray(S0, np.float64).reshape(d, d)
    S1 = np.ascontiguousarray(S1, np.float64).reshape(d, d)
    return m0, S0, m1, S1, d


def _plain_check(rc, what):
    if rc != SICP_OK:
        raise SicpError(rc, what)


def sicp_gaussian_kl(m0, S0, m1, S1) -> float:
    """KL(N(m0, S0) || N(m1, S1))."""
    m0, S0, m1, S1, d = _gauss_args(m0, S0, m1, S1)
    out = ctypes.c_double()
    _plain_check(lib().sicp_gaussian_kl(_ptr(m0, np.float64), _ptr(S0, np.float64), _ptr(m1, np.float64),
                                        _ptr(S1, np.float64), d, ctypes.byref(out)),
                 "sicp_gaussian_kl: bad sizes, non-finite values or a covariance that is not positive definite")
    return out.value


def sicp_gaussian_ovl(m0, S0, m1, S1, n: int = 100_000, seed: int = 0, z0=None, z1=None) -> float:
    """Overlapping coefficient of N(m0, S0) and N(m1, S1) by Monte Carlo; the
    standard-normal draws z0, z1 ([n][d]) come from numpy's generator seeded
    with `seed` unless given."""
    m0, S0, m1, S1, d = _gauss_args(m0, S0, m1, S1)
    if z0 is None or z1 is None:
        rng = np.random.default_rng(seed)
        z0, z1 = rng.standard_normal((n, d)), rng.standard_normal((n, d))
    z0 = np.ascontiguousarray(z0, np.float64).reshape(-1, d)
    z1 = np.ascontiguousarray(z1, np.float64).reshape(-1, d)
    if z0.shape != z1.shape:
        raise ValueError("z0 and z1 must have the same shape")
    out = ctypes.c_double()
    _plain_check(lib().sicp_gaussian_ovl(_ptr(m0, np.float64), _ptr(S0, np.float64), _ptr(m1, np.float64),
                                         _ptr(S1, np.float64), d, _ptr(z0, np.float64), _ptr(z1, np.float64),
                                         z0.shape[0], ctypes.byref(out)),
                 "sicp_gaussian_ovl: bad sizes, non-finite values or a covariance that is not positive definite")
    return out.value


def sicp_pose_distribution(particles):
    """(mean pose 4 x 4, se(3) covariance 6 x 6) of particles [K][6] (host data)."""
    th = np.ascontiguousarray(particles.cpu().numpy() if _is_torch(particles) else particles, np.float32).reshape(-1, 6)
    T = np.empty((4, 4))
    S = np.empty((6, 6))
    _plain_check(lib().sicp_pose_distribution(_ptr(th, np.float32), th.shape[0], _ptr(T, np.float64),
                                              _ptr(S, np.float64)),
                 "sicp_pose_distribution: bad size or a non-finite value")
    return T, S


def sicp_compound(T1, S1, T2, S2, order: int = 4):
    """(T1 T2, covariance) of two independent pose distributions."""
    a = [np.ascontiguousarray(x, np.float64) for x in (T1, S1, T2, S2)]
    T = np.empty((4, 4))
    S = np.empty((6, 6))
    _plain_check(lib().sicp_compound(*[_ptr(x, np.float64) for x in a], int(order), _ptr(T, np.float64),
                                     _ptr(S, np.float64)),
                 "sicp_compound: order must be 2 or 4, the poses rigid transforms, the values finite")
    return T, S


def chain_odometry(distributions, order: int = 4):
    """Compound a sequence of scan-to-scan distributions (T, S) in order:
    returns the list of accumulated (T_E, S_E) after each pair."""
    out = []
    T, S = distributions[0]
    out.append((np.asarray(T, np.float64), np.asarray(S, np.float64)))
    for T2, S2 in distributions[1:]:
        T, S = sicp_compound(T, S, T2, S2, order)
        out.append((T, S))
    return out


def sicp_moments_circular(ctx, particles):
    """Mean [6] and covariance [6][6] with circular statistics for the angles."""
    particles = _host(particles, np.float32)
    mean = _empty(particles, (6,), np.float64)
    cov = _empty(particles, (6, 6), np.float64)
    _check(ctx, lib().sicp_moments_circular(ctx, _ptr(particles, np.float32), particles.shape[0],
                                            _ptr(mean, np.float64), _ptr(cov, np.float64), _on_device(particles)))
    return mean, cov


def sicp_stats(ctx, enable: bool = True):
    """Search counters since the last call (queries, rows, segments, points,
    coarse-level queries, exhaustive-scan queries, surrogate queries,
    surrogate queries sent to the exact search, tensor-core query tiles,
    reference tiles they swept) as a uint64 array; then resets them and sets
    counting on/off."""
    out = np.zeros(10, np.uint64)
    _check(ctx, lib().sicp_stats(ctx, int(enable), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def sicp_set_memory_limit(ctx, nbytes: int) -> int:
    """Cap the context's device memory at nbytes (0: no cap); returns the bytes it holds now."""
    held = ctypes.c_size_t(0)
    _check(ctx, lib().sicp_set_memory_limit(ctx, int(nbytes), ctypes.byref(held)))
    return int(held.value)


def sicp_set_wait_check(ctx, on: bool, polls: int = 0):
    """Make every bounded device wait of later calls wait for an event that never comes (on = True),
    giving up after `polls` polls (0: the defaults)."""
    _check(ctx, lib().sicp_set_wait_check(ctx, int(bool(on)), int(polls)))


TELEMETRY_FIELDS = ("mean_x", "mean_y", "mean_z", "mean_roll", "mean_pitch", "mean_yaw",
                    "sd_x", "sd_y", "sd_z", "sd_roll", "sd_pitch", "sd_yaw",
                    "nn_mean_dist", "learned_share", "t", "found_share")


def sicp_set_telemetry(ctx, on: bool = True):
    """Record one telemetry row per iteration of later registration runs (TELEMETRY_FIELDS)."""
    _check(ctx, lib().sicp_set_telemetry(ctx, int(bool(on))))


def sicp_read_telemetry(ctx, max_rows: int = 1 << 20):
    """The last run's telemetry rows, float32 [T][16] (columns TELEMETRY_FIELDS)."""
    n = ctypes.c_int32(0)
    _check(ctx, lib().sicp_read_telemetry(ctx, None, 0, ctypes.byref(n)))
    rows = min(int(n.value), int(max_rows))
    out = np.zeros((rows, 16), np.float32)
    if rows:
        _check(ctx, lib().sicp_read_telemetry(ctx, out.ctypes.data_as(ctypes.c_void_p), rows, ctypes.byref(n)))
    return out


def sicp_check_status():
    """(checked, first, count): whether the loaded library is the bounds-checked build, the first
    index check that failed since the last call (0: none; else bit 63 | site << 40 | index) and
    how many failed; then clears them.  Synchronises the device."""
    c, f, n = ctypes.c_int32(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib().sicp_check_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(n))
    if rc != SICP_OK:
        raise SicpError(rc, "sicp_check_status failed")
    return bool(c.value), int(f.value), int(n.value)


def sicp_profile(ctx, stride: int = 0):
    """Kernel times since the last call: (gradient ms, gradient launches,
    Stein ms, Stein launches); then resets them and sets the stride."""
    out = np.zeros(4, np.float64)
    _check(ctx, lib().sicp_profile(ctx, int(stride), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def sicp_surrogate_train_run(ctx, src_xyz, particles, n_queries: int, seed: int = 0, epochs: int = 10,
                             batch: int = 4096, lr: float = 1e-3) -> float:
    """Train the learned field on a run's own queries (source points under poses from the box of the
    initial particles); returns the mean batch loss of the last epoch."""
    src_xyz, particles = _host(src_xyz, np.float32), _host(particles, np.float32)
    loss = ctypes.c_float(0.0)
    _check(ctx, lib().sicp_surrogate_train_run(ctx, _ptr(src_xyz, np.float32), src_xyz.shape[0],
                                               _ptr(particles, np.float32), particles.shape[0], int(n_queries),
                                               seed & ((1 << 64) - 1), int(epochs), int(batch), float(lr),
                                               ctypes.byref(loss), _on_device(src_xyz, particles)))
    return float(loss.value)


def sicp_surrogate_train(ctx, n_queries: int, seed: int = 0, epochs: int = 10, batch: int = 4096,
                         lr: float = 1e-3) -> float:
    """Train the context's learned closest-point field; returns the mean batch loss of the last epoch."""
    loss = ctypes.c_float(0.0)
    _check(ctx, lib().sicp_surrogate_train(ctx, int(n_queries), seed & ((1 << 64) - 1), int(epochs), int(batch),
                                           float(lr), ctypes.byref(loss)))
    return float(loss.value)


def sicp_surrogate_params(ctx, params=None, norm4=None):
    """With params/norm4 None: returns (params [33040] float32, norm4 [4] float32).
    Otherwise sets them (host arrays) and returns None."""
    if params is None:
        p = np.empty(SURROGATE_NPARAM, np.float32)
        n = np.empty(4, np.float32)
        _check(ctx, lib().sicp_surrogate_params(ctx, 0, _ptr(p, np.float32), _ptr(n, np.float32)))
        return p, n
    p = np.ascontiguousarray(params, np.float32)
    n = np.ascontiguousarray(norm4, np.float32)
    if p.shape != (SURROGATE_NPARAM,) or n.shape != (4,):
        raise ValueError("params must have 33040 values and norm4 four")
    _check(ctx, lib().sicp_surrogate_params(ctx, 1, _ptr(p, np.float32), _ptr(n, np.float32)))
    return None


def sicp_surrogate_loss_grad(ctx, params, qn, dstar, lam: float = 0.1, delta: float = 0.02):
    """Loss and gradient [33040] of the training kernels (host arrays)."""
    p = np.ascontiguousarray(params, np.float32)
    qn = np.ascontiguousarray(qn, np.float32)
    dstar = np.ascontiguousarray(dstar, np.float32)
    if p.shape != (SURROGATE_NPARAM,) or qn.shape != dstar.shape or qn.ndim != 2 or qn.shape[1] != 3:
        raise ValueError("params [33040], qn and dstar [n][3]")
    g = np.empty(SURROGATE_NPARAM, np.float32)
    loss = ctypes.c_float(0.0)
    _check(ctx, lib().sicp_surrogate_loss_grad(ctx, _ptr(p, np.float32), _ptr(qn, np.float32),
                                               _ptr(dstar, np.float32), qn.shape[0], float(lam), float(delta),
                                               ctypes.byref(loss), _ptr(g, np.float32)))
    return float(loss.value), g


def sicp_surrogate_save(ctx, path: str) -> None:
    _check(ctx, lib().sicp_surrogate_save(ctx, os.fsencode(path)))


def sicp_surrogate_load(ctx, path: str) -> None:
    _check(ctx, lib().sicp_surrogate_load(ctx, os.fsencode(path)))


def sicp_surrogate_infer(ctx, q):
    """Predicted displacement [n][3] (metres) and confidence [n] per query [n][3]."""
    q = _host(q, np.float32)
    n = q.shape[0]
    d = _empty(q, (n, 3), np.float32)
    c = _empty(q, (n,), np.float32)
    _check(ctx, lib().sicp_surrogate_infer(ctx, _ptr(q, np.float32), n, _ptr(d, np.float32), _ptr(c, np.float32),
                                           _on_device(q)))
    return d, c


def sicp_icp_grad_noalloc(ref_xyz, src_xyz, mb, particles, out_gbar=None, stream=None):
    """Allocation-free mean gradient (exhaustive FP32 search) on torch CUDA
    tensors; returns out_gbar [K][6].  Raises SicpError on a bad size.  The
    call only queues work on `stream` (default: torch's current stream)."""
    import torch
    for t in (ref_xyz, src_xyz, mb, particles):
        if not (_is_torch(t) and t.is_cuda):
            raise ValueError("sicp_icp_grad_noalloc takes CUDA tensors only")
    K = particles.shape[0]
    if out_gbar is None:
        out_gbar = torch.empty((K, 6), dtype=torch.float32, device=particles.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sicp_icp_grad_noalloc(_ptr(ref_xyz, np.float32), ref_xyz.shape[0], _ptr(src_xyz, np.float32),
                                     src_xyz.shape[0], _ptr(mb, np.int32), mb.shape[0], _ptr(particles, np.float32),
                                     K, _ptr(out_gbar, np.float32), ctypes.c_void_p(s.cuda_stream))
    if rc != SICP_OK:
        raise SicpError(rc, "sicp_icp_grad_noalloc: bad size or pointer (K <= 256, m <= 1024) or CUDA failure")
    return out_gbar


def _batch_args(problems):
    """Pack a list of (ref [M][3], src [N][3], particles [K][6]) into CSR arrays."""
    refs = [_host(p[0], np.float32) for p in problems]
    srcs = [_host(p[1], np.float32) for p in problems]
    pars = [_host(p[2], np.float32) for p in problems]
    dev = _is_torch(refs[0]) and refs[0].is_cuda
    ref_off = np.zeros(len(problems) + 1, np.int64)
    src_off = np.zeros(len(problems) + 1, np.int64)
    part_off = np.zeros(len(problems) + 1, np.int32)
    ref_off[1:] = np.cumsum([r.shape[0] for r in refs])
    src_off[1:] = np.cumsum([s.shape[0] for s in srcs])
    part_off[1:] = np.cumsum([q.shape[0] for q in pars])
    if dev:
        import torch
        cat = lambda xs: torch.cat(xs).contiguous()
    else:
        cat = lambda xs: np.ascontiguousarray(np.concatenate(xs))
    return cat(refs), cat(srcs), cat(pars), ref_off, src_off, part_off, int(dev)


def pack_batch(problems):
    """Pack a list of (ref, src, particles) once, for repeated batched calls."""
    ref, src, par, ref_off, src_off, part_off, dev = _batch_args(problems)
    return dict(ref=ref, src=src, par=par, ref_off=ref_off, src_off=src_off, part_off=part_off, dev=dev)


def sicp_register_batched(ctx, problems, params: sicp_params):
    """Run the registrations of `problems` (a list of (ref, src, particles), or
    the result of pack_batch) in one launch.  Returns (particles list,
    mean [P][6], cov [P][6][6])."""
    b = problems if isinstance(problems, dict) else pack_batch(problems)
    ref, src, par, ref_off, src_off, part_off, dev = (b["ref"], b["src"], b["par"], b["ref_off"], b["src_off"],
                                                      b["part_off"], b["dev"])
    P = len(ref_off) - 1
    out = _empty(par, tuple(par.shape), np.float32)
    mean = _empty(par, (P, 6), np.float64)
    cov = _empty(par, (P, 6, 6), np.float64)
    _check(ctx, lib().sicp_register_batched(ctx, P, ref_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(ref, np.float32), src_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(src, np.float32), part_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(par, np.float32), ctypes.byref(params), _ptr(out, np.float32),
                                            _ptr(mean, np.float64), _ptr(cov, np.float64), dev))
    parts = [out[part_off[i]:part_off[i + 1]] for i in range(P)]
    return parts, mean, cov


def sicp_trace_batched(ctx, t: int):
    """Record iteration t of the next sicp_register_batched call (t < 0: none)."""
    _check(ctx, lib().sicp_trace_batched(ctx, int(t)))


def sicp_read_batched_trace(ctx, Ktot: int, m: int):
    """The recorded iteration: dict of theta, adam_m, adam_v, gbar, phi [sum K][6] and nn [sum K][m]."""
    out = {k: np.empty((Ktot, 6), np.float32) for k in ("theta", "adam_m", "adam_v", "gbar", "phi")}
    out["nn"] = np.empty((Ktot, m), np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(ctx, lib().sicp_read_batched_trace(ctx, ptr(out["theta"]), ptr(out["adam_m"]), ptr(out["adam_v"]),
                                              ptr(out["nn"]), ptr(out["gbar"]), ptr(out["phi"])))
    return out


def sicp_autotune_batched(ctx, problems, params: sicp_params, trial_iters: int = 5, cache_path=None):
    """Pick and keep the fastest (cell-size factor, minibatch entries per work item, CTA threads)."""
    b = problems if isinstance(problems, dict) else pack_batch(problems)
    ref, src, par, ref_off, src_off, part_off, dev = (b["ref"], b["src"], b["par"], b["ref_off"], b["src_off"],
                                                      b["part_off"], b["dev"])
    f = ctypes.c_float()
    k = ctypes.c_int32()
    t = ctypes.c_int32()
    _check(ctx, lib().sicp_autotune_batched(ctx, len(ref_off) - 1, ref_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(ref, np.float32), src_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(src, np.float32), part_off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(par, np.float32), ctypes.byref(params), trial_iters,
                                            cache_path.encode() if cache_path else None, ctypes.byref(f),
                                            ctypes.byref(k), ctypes.byref(t), dev))
    return f.value, k.value, t.value
