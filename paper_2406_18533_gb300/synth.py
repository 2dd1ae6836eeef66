"""Seeded synthetic inputs for the 3DGS training hot path.

This module only draws random numbers and lays them out.  It holds none of the
method's arithmetic (no projection, colour, blending, loss or optimiser step), so
both the FP64 oracle and the CUDA path may take their inputs from it.

The paper trains on Rubble, MatrixCity, Mip-NeRF 360, Tanks&Temples and
DeepBlending (Sec. 5.1, Table "scenes-main").  None of those datasets or the
paper's trained checkpoints are available here, so every workload below is a
synthetic stand-in with the shape of the paper's: an aerial scene made of
Gaussian clusters, posed 1080p / 4K cameras, and a target image.

Parameter layout (one Gaussian = 60 float32, four float4 structure-of-arrays
planes; 59 are parameters, ``ls[:, 3]`` is padding):

* ``mo[N,4]``  = (x, y, z, opacity logit)
* ``ls[N,4]``  = (log sx, log sy, log sz, 0)
* ``q[N,4]``   = (w, x, y, z) rotation quaternion, not necessarily unit
* ``sh[12,N,4]`` = 48 SH coefficients, flat index ``3*k + ch`` for coefficient k
  (0..15) and colour channel ch; flat index j lives in plane ``j // 4`` lane
  ``j % 4``.

Draw order (fixed, seed 0 unless stated): cluster centres, then per chunk of
2**20 Gaussians: means (cluster id, offsets), log-scales, quaternions, opacity
logits, SH DC, SH rest; then cameras; then targets / upstream gradients; then
request arrivals.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CHUNK = 1 << 20


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    ``R`` maps world to camera (rows = right, down, forward), ``t = -R @ C``.
    Every float is already rounded to float32 so that the oracle (FP64) and
    the CUDA path (FP32) start from identical values.
    """
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    near: float = 0.01

    @property
    def center(self) -> np.ndarray:
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclasses.dataclass
class Scene:
    mo: np.ndarray
    ls: np.ndarray
    q: np.ndarray
    sh: np.ndarray
    sh_degree: int = 3

    @property
    def N(self) -> int:
        return int(self.mo.shape[0])

    def flat(self) -> np.ndarray:
        """[N, 60] view in the (mo, ls, q, sh0..sh11) order, a copy."""
        N = self.N
        out = np.empty((N, 60), np.float32)
        out[:, 0:4] = self.mo
        out[:, 4:8] = self.ls
        out[:, 8:12] = self.q
        out[:, 12:60] = self.sh.transpose(1, 0, 2).reshape(N, 48)
        return out

    def copy(self) -> "Scene":
        return Scene(self.mo.copy(), self.ls.copy(), self.q.copy(), self.sh.copy(), self.sh_degree)


def _f32(x) -> float:
    return float(np.float32(x))


def camera_look_at(pos, target, up, W, H, fovy_deg, near=0.01) -> Camera:
    """Camera at ``pos`` aimed at ``target``; ``up`` is the world up vector."""
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return _camera_from_axes(pos, right, down, fwd, W, H, fovy_deg, near)


def camera_yaw_pitch(pos, yaw, pitch, W, H, fovy_deg, near=0.01) -> Camera:
    """Aerial camera (world +z up) from yaw and downward pitch, no nadir singularity."""
    cp, sp, cy, sy = math.cos(pitch), math.sin(pitch), math.cos(yaw), math.sin(yaw)
    fwd = np.array([cp * cy, cp * sy, -sp])
    right = np.array([-sy, cy, 0.0])
    down = np.cross(fwd, right)
    return _camera_from_axes(np.asarray(pos, np.float64), right, down, fwd, W, H, fovy_deg, near)


def _camera_from_axes(pos, right, down, fwd, W, H, fovy_deg, near) -> Camera:
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-(R.astype(np.float64) @ pos)).astype(np.float32)
    f = (H / 2.0) / math.tan(math.radians(fovy_deg) / 2.0)
    return Camera(R=R, t=t, fx=_f32(f), fy=_f32(f), cx=_f32(W / 2.0), cy=_f32(H / 2.0),
                  W=int(W), H=int(H), near=_f32(near))


def _aim_at(pos, target, W, H, fovy_deg, near=0.01) -> Camera:
    d = np.asarray(target, np.float64) - np.asarray(pos, np.float64)
    d /= np.linalg.norm(d)
    yaw = math.atan2(d[1], d[0])
    pitch = math.asin(-d[2])
    return camera_yaw_pitch(pos, yaw, pitch, W, H, fovy_deg, near)


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------

def _empty_scene(N: int) -> Scene:
    return Scene(mo=np.empty((N, 4), np.float32), ls=np.zeros((N, 4), np.float32),
                 q=np.empty((N, 4), np.float32), sh=np.empty((12, N, 4), np.float32))


def _fill_attrs(rng, sc: Scene, lo: int, hi: int, log_s, logit, dc=(0.5, 0.2), rest=0.05):
    n = hi - lo
    sc.ls[lo:hi, 0:3] = rng.standard_normal((n, 3), dtype=np.float32) * np.float32(log_s[1]) + np.float32(log_s[0])
    qq = rng.standard_normal((n, 4), dtype=np.float32)
    qq /= np.linalg.norm(qq, axis=1, keepdims=True)
    sc.q[lo:hi] = qq
    sc.mo[lo:hi, 3] = rng.standard_normal(n, dtype=np.float32) * np.float32(logit[1]) + np.float32(logit[0])
    flat = np.empty((n, 48), np.float32)
    flat[:, 0:3] = rng.standard_normal((n, 3), dtype=np.float32) * np.float32(dc[1]) + np.float32(dc[0])
    flat[:, 3:48] = rng.standard_normal((n, 45), dtype=np.float32) * np.float32(rest)
    sc.sh[:, lo:hi, :] = flat.reshape(n, 12, 4).transpose(1, 0, 2)


def cube_scene(N: int, seed: int = 0, half=1.0, log_s=(-4.0, 0.5), logit=(0.0, 1.0)) -> Scene:
    """Means uniform in [-half, half]^3 (the 10k-Gaussian plain fwd+bwd workload)."""
    rng = np.random.default_rng(seed)
    sc = _empty_scene(N)
    for lo in range(0, N, CHUNK):
        hi = min(N, lo + CHUNK)
        sc.mo[lo:hi, 0:3] = (rng.random((hi - lo, 3), dtype=np.float32) * 2 - 1) * np.float32(half)
        _fill_attrs(rng, sc, lo, hi, log_s, logit)
    return sc


def cluster_scene(N: int, n_clusters: int, sigma: float, box, log_s, logit, seed: int = 0):
    """Mixture of isotropic clusters in an axis-aligned box centred at the origin in x, y
    with z in [0, box_z]; members are clipped to the box.  Returns (scene, rng) so the
    caller keeps drawing cameras from the same stream."""
    rng = np.random.default_rng(seed)
    bx, by, bz = (float(b) for b in box)
    lo_b = np.array([-bx / 2, -by / 2, 0.0], np.float32)
    hi_b = np.array([bx / 2, by / 2, bz], np.float32)
    centres = lo_b + rng.random((n_clusters, 3), dtype=np.float32) * (hi_b - lo_b)
    sc = _empty_scene(N)
    for lo in range(0, N, CHUNK):
        hi = min(N, lo + CHUNK)
        cid = rng.integers(0, n_clusters, hi - lo)
        pts = centres[cid] + rng.standard_normal((hi - lo, 3), dtype=np.float32) * np.float32(sigma)
        sc.mo[lo:hi, 0:3] = np.clip(pts, lo_b, hi_b)
        _fill_attrs(rng, sc, lo, hi, log_s, logit)
    return sc, rng


# --------------------------------------------------------------------------
# Named workloads (the five configurations of the hot path)
# --------------------------------------------------------------------------

WORKLOADS = {
    "c0_plain_10k_256": dict(N=10_000, B=1, W=256, H=256),
    "c1_train_1m_1080p": dict(N=1_000_000, B=1, W=1920, H=1080),
    "c2_batch16_4m_1080p": dict(N=4_000_000, B=16, W=1920, H=1080),
    "c3_batch4_40m_4k": dict(N=40_000_000, B=4, W=3840, H=2160),
    "c4_serve_10m": dict(N=10_000_000, B=0, W=0, H=0),
}


def workload_c0(seed=0, N=10_000):
    sc = cube_scene(N, seed, half=1.0, log_s=(-4.0, 0.5), logit=(0.0, 1.0))
    rng = np.random.default_rng(seed + 1)
    cam = camera_look_at((0, 0, 4), (0, 0, 0), (0, 1, 0), 256, 256, 60.0, 0.01)
    d_img = rng.standard_normal((3, 256, 256), dtype=np.float32)
    return sc, [cam], d_img


def aerial_scene(N, n_clusters=64, seed=0, box=(100, 100, 20), sigma=2.0, log_s=(-2.5, 0.7), logit=(-1.0, 1.0)):
    return cluster_scene(N, n_clusters, sigma, box, log_s, logit, seed)


def ring_cameras(rng, B, alt, ring=40.0, target=(0, 0, 10), W=1920, H=1080, fovy=50.0):
    cams = []
    for _ in range(B):
        yaw = rng.random() * 2 * math.pi
        a = alt[0] + rng.random() * (alt[1] - alt[0]) if alt[1] > alt[0] else alt[0]
        pos = (ring * math.cos(yaw), ring * math.sin(yaw), a)
        cams.append(_aim_at(pos, target, W, H, fovy))
    return cams


def blurred_noise_target(rng, H, W):
    """Uniform noise per channel, 9x9 box blur with clamp-to-edge borders."""
    from scipy.ndimage import uniform_filter
    x = rng.random((3, H, W), dtype=np.float32)
    return uniform_filter(x, size=(1, 9, 9), mode="nearest").astype(np.float32)


def workload_c1(seed=0, N=1_000_000, W=1920, H=1080):
    sc, rng = aerial_scene(N, 64, seed)
    cams = ring_cameras(rng, 1, (60.0, 60.0), W=W, H=H)
    tgt = blurred_noise_target(rng, H, W)[None]
    return sc, cams, tgt


def workload_c2(seed=0, N=4_000_000, B=16, W=1920, H=1080):
    sc, rng = aerial_scene(N, 256, seed)
    cams = ring_cameras(rng, B, (20.0, 120.0), W=W, H=H)
    tgt = np.stack([blurred_noise_target(rng, H, W) for _ in range(B)])
    return sc, cams, tgt


def large_scene(N, seed=0):
    return cluster_scene(N, 4096, 4.0, (1000, 1000, 100), (-1.5, 0.8), (-1.0, 1.0), seed)


def oblique_cameras(rng, B, W=3840, H=2160, fovy=50.0):
    cams = []
    for _ in range(B):
        x, y = (rng.random(2) - 0.5) * 800.0
        alt = 100.0 + rng.random() * 100.0
        pitch = math.radians(45.0 + rng.random() * 45.0)
        yaw = rng.random() * 2 * math.pi
        cams.append(camera_yaw_pitch((x, y, alt), yaw, pitch, W, H, fovy))
    return cams


def workload_c3(seed=0, N=40_000_000, B=4, W=3840, H=2160):
    sc, rng = large_scene(N, seed)
    cams = oblique_cameras(rng, B, W, H)
    tgt = np.stack([blurred_noise_target(rng, H, W) for _ in range(B)])
    return sc, cams, tgt


SERVE_RES = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))
SERVE_P = (0.4, 0.3, 0.2, 0.1)


def serve_requests(rng, n, rate=200.0, radius=150.0, centre=(0, 0, 50)):
    """Poisson arrivals (seconds), resolution mix and hemisphere poses."""
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps)
    res = rng.choice(len(SERVE_RES), size=n, p=SERVE_P)
    reqs = []
    for i in range(n):
        az = rng.random() * 2 * math.pi
        el = math.radians(15.0 + rng.random() * 70.0)
        pos = (centre[0] + radius * math.cos(el) * math.cos(az),
               centre[1] + radius * math.cos(el) * math.sin(az),
               centre[2] + radius * math.sin(el))
        W, H = SERVE_RES[res[i]]
        reqs.append((float(t[i]), _aim_at(pos, centre, W, H, 50.0)))
    return reqs


# --------------------------------------------------------------------------
# Small cases for tests
# --------------------------------------------------------------------------

def tiny_scene(N, seed=0, spread=0.6, depth=(2.5, 4.5), log_s=(-3.0, 0.4), logit=(0.0, 1.2)) -> Scene:
    """N Gaussians in front of the default test camera (at origin looking +z)."""
    rng = np.random.default_rng(seed)
    sc = _empty_scene(N)
    sc.mo[:, 0:2] = (rng.random((N, 2), dtype=np.float32) * 2 - 1) * np.float32(spread)
    sc.mo[:, 2] = np.float32(depth[0]) + rng.random(N, dtype=np.float32) * np.float32(depth[1] - depth[0])
    _fill_attrs(rng, sc, 0, N, log_s, logit)
    return sc


def test_camera(W=64, H=48, fovy=60.0, pos=(0, 0, 0), target=(0, 0, 1)) -> Camera:
    return camera_look_at(pos, target, (0, -1, 0), W, H, fovy, 0.01)


def synthetic_proj(n, W, H, seed=0, tile=16, max_sigma=6.0, ties=0):
    """Random per-Gaussian screen-space features for stage tests of binning and
    blending: centre (u, v), an SPD conic drawn from random axes, opacity, rgb,
    depth, and an integer footprint radius.  ``ties`` Gaussians copy the depth of
    another one so equal-depth ordering is exercised."""
    rng = np.random.default_rng(seed)
    u = (rng.random(n) * (W + 40) - 20).astype(np.float32)
    v = (rng.random(n) * (H + 40) - 20).astype(np.float32)
    s1 = 0.5 + rng.random(n) * max_sigma
    s2 = 0.5 + rng.random(n) * max_sigma
    th = rng.random(n) * math.pi
    c, s = np.cos(th), np.sin(th)
    a = c * c / s1 ** 2 + s * s / s2 ** 2
    b = c * s * (1 / s1 ** 2 - 1 / s2 ** 2)
    cc = s * s / s1 ** 2 + c * c / s2 ** 2
    opac = (0.05 + 0.95 * rng.random(n)).astype(np.float32)
    rgb = rng.random((n, 3)).astype(np.float32)
    depth = (1.0 + rng.random(n) * 50.0).astype(np.float32)
    if ties:
        src = rng.integers(0, n, ties)
        dst = rng.integers(0, n, ties)
        depth[dst] = depth[src]
    radius = np.ceil(3.0 * np.maximum(s1, s2)).astype(np.int32)
    radius[rng.random(n) < 0.05] = 0
    xy = np.stack([u, v], 1).astype(np.float32)
    conic_o = np.stack([a, b, cc, opac], 1).astype(np.float32)
    rgb_d = np.concatenate([rgb, depth[:, None]], 1).astype(np.float32)
    return dict(xy=xy, conic_o=conic_o, rgb_d=rgb_d, radius=radius)
