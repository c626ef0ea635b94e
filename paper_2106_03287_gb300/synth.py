"""Seeded synthetic inputs shaped like the Stein ICP workloads.

This module makes point clouds, ground-truth poses and initial particle sets.
It holds none of the method's arithmetic (no correspondence search, no
gradient, no Stein step): the CUDA path and the CPU oracle both take their
inputs from here and nothing else is shared between them.

Randomness: every draw comes from a counter-based splitmix64 stream
(output k of the generator seeded with s is mix64(s + k*gamma)), mapped to
uniform doubles in [0, 1) by the top 53 bits and to normals by Box-Muller, so
a seed gives the same cloud on any machine and numpy version.

Rotations used to place sensors and to move clouds are built by
scipy.spatial.transform.Rotation from three angles about the fixed x, y and z
axes (roll, pitch, yaw), i.e. R = Rz(yaw) Ry(pitch) Rx(roll).

Workloads (sizes follow the method's RGB-D and laser experiments):
  box      -- points on the surface of a 0.20 x 0.10 x 0.05 m box
  kinect   -- analytic ray cast of a 640x480 pinhole depth camera into a room
              corner (floor, back wall, side wall) with a 0.07 m-radius,
              0.25 m-tall cylinder; depth noise N(0, 0.001 z^2)
  lidar    -- 64-beam spinning scanner (-25..+3 deg, 0.2 deg azimuth step)
              over a ground plane, 40 boxes and 20 poles; range noise 0.02 m
  batched  -- 256 problems mixing the box and kinect generators
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.transform import Rotation

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based splitmix64 stream used for synthetic data only."""

    def __init__(self, seed: int, salt: int = 0):
        base = np.array([(seed * 0x100000001B3 + salt) & _MASK], dtype=np.uint64)
        self.seed = _mix64(base)[0]
        self.k = 0

    def u64(self, n: int) -> np.ndarray:
        ks = np.arange(self.k + 1, self.k + 1 + n, dtype=np.uint64)
        self.k += n
        with np.errstate(over="ignore"):
            return _mix64(self.seed + ks * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        x = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * x

    def normal(self, n: int, sigma=1.0) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        return sigma * r * np.cos(2.0 * np.pi * u2)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)


def rotation(roll: float, pitch: float, yaw: float) -> np.ndarray:
    return Rotation.from_euler("xyz", [roll, pitch, yaw]).as_matrix()


def euler_of(R: np.ndarray) -> np.ndarray:
    """(roll, pitch, yaw) with R = Rz(yaw) Ry(pitch) Rx(roll)."""
    return Rotation.from_matrix(R).as_euler("xyz")


def random_pose(st: Stream, t_max: float, ang_max_deg: float):
    """Translation uniform in direction with |t| <= t_max; each angle U(+-ang)."""
    d = st.normal(3)
    d /= np.linalg.norm(d)
    t = d * st.uniform(1, 0.0, t_max)[0]
    ang = np.deg2rad(st.uniform(3, -ang_max_deg, ang_max_deg))
    return rotation(*ang), t


def init_particles(st: Stream, K: int, t_half: float, ang_half_deg: float) -> np.ndarray:
    """K x 6 particles, each component uniform in +-half around identity."""
    th = np.empty((K, 6))
    th[:, :3] = st.uniform(3 * K, -t_half, t_half).reshape(K, 3)
    a = np.deg2rad(ang_half_deg)
    th[:, 3:] = st.uniform(3 * K, -a, a).reshape(K, 3)
    return th.astype(np.float32)


# ----------------------------------------------------------------------------
# box surface
# ----------------------------------------------------------------------------

def box_surface(st: Stream, M: int, size=(0.20, 0.10, 0.05)) -> np.ndarray:
    a, b, c = size
    # faces: +-z (a*b), +-y (a*c), +-x (b*c); chosen with probability ~ area
    areas = np.array([a * b, a * b, a * c, a * c, b * c, b * c])
    cdf = np.cumsum(areas) / areas.sum()
    f = np.searchsorted(cdf, st.uniform(M), side="right")
    u = st.uniform(M) - 0.5
    v = st.uniform(M) - 0.5
    p = np.empty((M, 3))
    sgn = np.where(f % 2 == 0, 0.5, -0.5)
    z_face = f < 2
    y_face = (f >= 2) & (f < 4)
    x_face = f >= 4
    p[z_face] = np.stack([u[z_face] * a, v[z_face] * b, sgn[z_face] * c], 1)
    p[y_face] = np.stack([u[y_face] * a, sgn[y_face] * b, v[y_face] * c], 1)
    p[x_face] = np.stack([sgn[x_face] * a, u[x_face] * b, v[x_face] * c], 1)
    return p


def make_box_problem(seed: int, M=2000, N=500, K=32, noise=0.002, t_max=0.05,
                     ang_max_deg=10.0, init_t=0.1, init_ang_deg=15.0,
                     size=(0.20, 0.10, 0.05)):
    """Reference on a box surface; source = subset moved by a seeded pose."""
    st = Stream(seed, 1)
    ref = box_surface(st, M, size)
    sub = ref[st.permutation(M)[:N]]
    R_gt, t_gt = random_pose(st, t_max, ang_max_deg)
    src = sub @ R_gt.T + t_gt
    if noise > 0:
        src = src + st.normal(3 * N, noise).reshape(N, 3)
    # theta maps source into the reference frame: R = R_gt^T, u = -R_gt^T t_gt
    theta_true = np.concatenate([-R_gt.T @ t_gt, euler_of(R_gt.T)])
    particles = init_particles(st, K, init_t, init_ang_deg)
    return dict(ref=ref.astype(np.float32), src=src.astype(np.float32),
                particles=particles, theta_true=theta_true)


# ----------------------------------------------------------------------------
# Kinect-like depth render of a room corner with a cylinder
# ----------------------------------------------------------------------------

_FLOOR_Y = 1.0      # camera frame: +z forward, +y down
_BACK_Z = 3.0
_SIDE_X = -1.2
_CYL_C = (0.2, 1.8)  # (x, z)
_CYL_R = 0.07
_CYL_H = 0.25


def _render_kinect(st: Stream, R_cam, t_cam, width=640, height=480, f=525.0, return_depth=False):
    """Depth-render the scene from a camera at (R_cam, t_cam) in the reference
    camera frame. Returns valid points in the rendering camera's frame (and,
    with return_depth, the noisy depth image, inf where a ray hits nothing)."""
    scale = width / 640.0
    fx = fy = f * scale
    cx, cy = (width - 1) / 2.0, (height - 1) / 2.0
    vv, uu = np.mgrid[0:height, 0:width]
    dc = np.stack([(uu.ravel() - cx) / fx, (vv.ravel() - cy) / fy,
                   np.ones(width * height)], 1)          # camera-frame rays, z = 1
    d = dc @ np.asarray(R_cam).T
    o = np.asarray(t_cam, dtype=np.float64)
    inf = np.full(d.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        # floor y = 1
        t = (_FLOOR_Y - o[1]) / d[:, 1]
        h = o + t[:, None] * d
        ok = (d[:, 1] > 0) & (t > 0) & (h[:, 0] >= _SIDE_X) & (h[:, 2] <= _BACK_Z)
        best = np.where(ok, t, inf)
        # back wall z = 3
        t = (_BACK_Z - o[2]) / d[:, 2]
        h = o + t[:, None] * d
        ok = (d[:, 2] > 0) & (t > 0) & (h[:, 0] >= _SIDE_X) & (h[:, 1] <= _FLOOR_Y)
        best = np.where(ok & (t < best), t, best)
        # side wall x = -1.2
        t = (_SIDE_X - o[0]) / d[:, 0]
        h = o + t[:, None] * d
        ok = (d[:, 0] < 0) & (t > 0) & (h[:, 2] <= _BACK_Z) & (h[:, 1] <= _FLOOR_Y)
        best = np.where(ok & (t < best), t, best)
        # cylinder side (axis along y), closed top cap at y = 1 - H
        ox, oz = o[0] - _CYL_C[0], o[2] - _CYL_C[1]
        a = d[:, 0] ** 2 + d[:, 2] ** 2
        b = 2 * (ox * d[:, 0] + oz * d[:, 2])
        c = ox * ox + oz * oz - _CYL_R ** 2
        disc = b * b - 4 * a * c
        t = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
        hy = o[1] + t * d[:, 1]
        ok = (disc > 0) & (t > 0) & (hy >= _FLOOR_Y - _CYL_H) & (hy <= _FLOOR_Y)
        best = np.where(ok & (t < best), t, best)
        t = (_FLOOR_Y - _CYL_H - o[1]) / d[:, 1]
        hx = o[0] + t * d[:, 0] - _CYL_C[0]
        hz = o[2] + t * d[:, 2] - _CYL_C[1]
        ok = (d[:, 1] > 0) & (t > 0) & (hx * hx + hz * hz <= _CYL_R ** 2)
        best = np.where(ok & (t < best), t, best)
    valid = np.isfinite(best)
    depth = best[valid]                      # rays have camera z = 1: t is depth
    depth = depth + st.normal(depth.size, 0.001 * depth ** 2)
    pts = dc[valid] * depth[:, None]
    if not return_depth:
        return pts
    image = np.full(width * height, np.inf)
    image[valid] = depth
    return pts, image.reshape(height, width)


def _seen_by(image, p, f=525.0):
    """Which points p [n][3] (camera frame of the view that rendered `image`)
    that view also sees: they project inside the image onto a pixel whose
    depth agrees within 2 cm + 1 %."""
    height, width = image.shape
    fx = fy = f * width / 640.0
    cx, cy = (width - 1) / 2.0, (height - 1) / 2.0
    z = p[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.rint(fx * p[:, 0] / z + cx)
        v = np.rint(fy * p[:, 1] / z + cy)
    inside = (z > 0) & (u >= 0) & (u < width) & (v >= 0) & (v < height)
    ok = np.zeros(p.shape[0], bool)
    ui, vi = u[inside].astype(np.int64), v[inside].astype(np.int64)
    ok[inside] = np.abs(image[vi, ui] - z[inside]) <= 0.02 + 0.01 * z[inside]
    return ok


def make_kinect_problem(seed: int, M=50_000, N=10_000, K=100, t_max=0.1,
                        ang_max_deg=20.0, init_t=0.15, init_ang_deg=20.0,
                        width=640, height=480):
    """Reference: M points of a render from the identity view. Source: N points
    of a render from a view offset by a seeded pose, drawn from the part of
    that render the reference view also sees (without this overlap crop the
    point-to-point cost of a 20-degree offset is lowest far from the true pose,
    pulled by source points that have no counterpart in the reference)."""
    st = Stream(seed, 2)
    ref_all, ref_depth = _render_kinect(st, np.eye(3), np.zeros(3), width, height, return_depth=True)
    ref = ref_all[st.permutation(ref_all.shape[0])[:M]]
    R_gt, t_gt = random_pose(st, t_max, ang_max_deg)
    src_all = _render_kinect(st, R_gt, t_gt, width, height)
    src_all = src_all[_seen_by(ref_depth, src_all @ R_gt.T + t_gt)]
    src = src_all[st.permutation(src_all.shape[0])[:N]]
    # a source point s (camera frame of the moved view) is R_gt s + t_gt in the reference frame
    theta_true = np.concatenate([t_gt, euler_of(R_gt)])
    particles = init_particles(st, K, init_t, init_ang_deg)
    return dict(ref=ref.astype(np.float32), src=src.astype(np.float32),
                particles=particles, theta_true=theta_true)


# ----------------------------------------------------------------------------
# spinning 64-beam LiDAR over ground, boxes and poles
# ----------------------------------------------------------------------------

def _lidar_scene(st: Stream, n_boxes=40, n_poles=20, half=50.0, keep_out=3.0,
                 sensors=((0.0, 0.0),)):
    def far(x, y, rad):
        return all(math.hypot(x - sx, y - sy) > keep_out + rad for sx, sy in sensors)
    boxes = []
    while len(boxes) < n_boxes:
        sx, sy, sz = st.uniform(3, 1.0, 10.0)
        cx, cy = st.uniform(2, -half, half)
        if far(cx, cy, 0.5 * math.hypot(sx, sy)):
            boxes.append((cx - sx / 2, cy - sy / 2, 0.0, cx + sx / 2, cy + sy / 2, sz))
    poles = []
    while len(poles) < n_poles:
        r = st.uniform(1, 0.1, 0.3)[0]
        h = st.uniform(1, 3.0, 8.0)[0]
        cx, cy = st.uniform(2, -half, half)
        if far(cx, cy, r):
            poles.append((cx, cy, r, h))
    return np.array(boxes), np.array(poles)


def _cast_scene(boxes, poles, o, d):
    """Distance along unit rays d [n][3] from o to the first surface (inf: none)."""
    best = np.full(d.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = -o[2] / d[:, 2]
        best = np.where((d[:, 2] < 0) & (t > 0), t, best)
        inv = 1.0 / d
        for x0, y0, z0, x1, y1, z1 in boxes:
            ta = (np.array([x0, y0, z0]) - o) * inv
            tb = (np.array([x1, y1, z1]) - o) * inv
            tmin = np.nanmax(np.minimum(ta, tb), axis=1)
            tmax = np.nanmin(np.maximum(ta, tb), axis=1)
            hit = (tmax >= np.maximum(tmin, 0)) & (tmin > 0)
            best = np.where(hit & (tmin < best), tmin, best)
        for cx, cy, r, h in poles:
            ox, oy = o[0] - cx, o[1] - cy
            a = d[:, 0] ** 2 + d[:, 1] ** 2
            b = 2 * (ox * d[:, 0] + oy * d[:, 1])
            c = ox * ox + oy * oy - r * r
            disc = b * b - 4 * a * c
            t = (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a)
            hz = o[2] + t * d[:, 2]
            hit = (disc > 0) & (t > 0) & (hz >= 0) & (hz <= h)
            best = np.where(hit & (t < best), t, best)
    return best


def _scan_lidar(st: Stream, boxes, poles, sensor_xyz, yaw, beams=64,
                el_lo=-25.0, el_hi=3.0, az_step=0.2, max_range=120.0, noise=0.02):
    el = np.deg2rad(np.linspace(el_lo, el_hi, beams))
    az = np.deg2rad(np.arange(0.0, 360.0, az_step))
    E, A = np.meshgrid(el, az, indexing="ij")
    dl = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    Rz = rotation(0.0, 0.0, yaw)
    o = np.asarray(sensor_xyz, dtype=np.float64)
    best = _cast_scene(boxes, poles, o, dl @ Rz.T)
    valid = best <= max_range
    rng_ = best[valid] + st.normal(int(valid.sum()), noise)
    return dl[valid] * rng_[:, None]          # sensor frame (yawed with the sensor)


def _lidar_seen_by(boxes, poles, o, p, max_range, el_lo=-25.0, el_hi=3.0):
    """Which world points p [n][3] a scanner at o sees: inside its range and
    elevation span, and the first surface along the ray is p itself."""
    v = p - o
    r = np.linalg.norm(v, axis=1)
    d = v / np.maximum(r, 1e-12)[:, None]
    el = np.degrees(np.arcsin(np.clip(d[:, 2], -1.0, 1.0)))
    ok = (r <= max_range) & (el >= el_lo - 0.2) & (el <= el_hi + 0.2)
    hit = _cast_scene(boxes, poles, o, d[ok])
    ok[ok] = np.abs(hit - r[ok]) <= 0.1 + 0.002 * r[ok]
    return ok


def make_lidar_problem(seed: int, K=200, t_max_xy=2.0, yaw_max_deg=10.0,
                       init_t=1.5, init_ang_deg=15.0, sensor_height=1.73,
                       az_step=0.2, max_range=120.0):
    """Reference: scan from the origin. Source: scan from a pose offset by up to
    t_max_xy in the ground plane and yaw_max_deg in yaw, keeping the points the
    reference scanner also sees (the overlap)."""
    st = Stream(seed, 3)
    ang = st.uniform(1, 0, 2 * np.pi)[0]
    rad = st.uniform(1, 0, t_max_xy)[0]
    t_gt = np.array([rad * np.cos(ang), rad * np.sin(ang), 0.0])
    yaw = np.deg2rad(st.uniform(1, -yaw_max_deg, yaw_max_deg)[0])
    boxes, poles = _lidar_scene(st, sensors=((0.0, 0.0), (t_gt[0], t_gt[1])))
    ref = _scan_lidar(st, boxes, poles, (0, 0, sensor_height), 0.0, az_step=az_step, max_range=max_range)
    src = _scan_lidar(st, boxes, poles, (t_gt[0], t_gt[1], sensor_height), yaw, az_step=az_step,
                      max_range=max_range)
    # a source point s (sensor frame, yawed) is Rz(yaw) s + t_gt in the reference frame
    o_ref = np.array([0.0, 0.0, sensor_height])
    world = src @ rotation(0.0, 0.0, yaw).T + t_gt + o_ref
    src = src[_lidar_seen_by(boxes, poles, o_ref, world, max_range)]
    theta_true = np.array([t_gt[0], t_gt[1], 0.0, 0.0, 0.0, yaw])
    particles = init_particles(st, K, init_t, init_ang_deg)
    return dict(ref=ref.astype(np.float32), src=src.astype(np.float32),
                particles=particles, theta_true=theta_true)


# ----------------------------------------------------------------------------
# batched serving-style workload
# ----------------------------------------------------------------------------

def make_batched_problems(seed: int, P=256, M_lo=5_000, M_hi=80_000, src_frac=0.2,
                          K_lo=50, K_hi=200, render=(320, 240)):
    """P independent problems; reference sizes log-uniform in [M_lo, M_hi],
    alternating the box and kinect generators, source = src_frac * M points,
    particle counts uniform in [K_lo, K_hi]."""
    st = Stream(seed, 4)
    Ms = np.exp(st.uniform(P, math.log(M_lo), math.log(M_hi))).astype(np.int64)
    Ks = st.integers(P, K_lo, K_hi)
    kin_ref = _render_kinect(st, np.eye(3), np.zeros(3), 640, 480)
    probs = []
    for p in range(P):
        M, K = int(Ms[p]), int(Ks[p])
        N = max(1, int(src_frac * M))
        if p % 2 == 0:
            d = make_box_problem(seed * 1000 + p, M=M, N=N, K=K)
        else:
            sp = Stream(seed * 1000 + p, 5)
            ref = kin_ref[sp.permutation(kin_ref.shape[0])[:M]]
            R_gt, t_gt = random_pose(sp, 0.1, 20.0)
            src_all = _render_kinect(sp, R_gt, t_gt, *render, f=525.0)
            src = src_all[sp.permutation(src_all.shape[0])[:N]]
            d = dict(ref=ref.astype(np.float32), src=src.astype(np.float32),
                     particles=init_particles(sp, K, 0.15, 20.0),
                     theta_true=np.concatenate([t_gt, euler_of(R_gt)]))
        probs.append(d)
    return probs


# parameters of each workload's run (iterations T, minibatch m, Adam step)
WORKLOADS = {
    "box": dict(T=100, m=100, lr=0.01),
    "kinect": dict(T=150, m=300, lr=0.03),
    "lidar": dict(T=200, m=500, lr=0.01),
    "batched": dict(T=100, m=300, lr=0.01),
    "surrogate": dict(T=200, m=300, lr=0.03, surrogate_iters=150),
    # the experiments' quality protocol on the kinect scene: a Monte Carlo reference of
    # `runs` independent SGD-ICP runs, and Stein ICP with the first `stein_K` of the
    # same initial poses
    "mc": dict(T=150, m=300, lr=0.03, runs=1000, stein_K=100),
}
