"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no rendering arithmetic: it only draws Gaussians, feature
tables, query vectors and pinhole cameras with numpy's PCG64 generator
(``numpy.random.default_rng(seed)``).  Everything the renderer computes from
them lives elsewhere.

Workload shapes (the paper's data is ScanNet / LeRF; these synthetic scenes
stand in for them with the same structure):

* ``tiny_scene``  -- 2,000 Gaussians, means U[-1,1]^3, log-scales N(-3.5,0.5),
  uniform unit quaternions, opacity sigmoid(N(0,1)), 16-D N(0,1) features;
  camera 128x128, fx=fy=128, at (0,0,3) looking at the origin.
* ``room_scene``  -- an indoor room [-3,3]x[-3,3]x[0,3] m: 60 % of the
  Gaussians lie within 2 cm of the floor or one of the four walls (plane
  chosen in proportion to its area), 40 % uniform in the box; log-scales
  N(-4,0.6), opacity sigmoid(N(0.5,1.5)), C-D N(0,1) features normalised to
  unit L2 norm per Gaussian (CLIP-like embeddings).
* ``room_camera`` -- 60 degree horizontal field of view at the room centre.

Conventions (Sec. 3 of the paper leaves them open): quaternions are (w,x,y,z);
``opacity`` is already activated; the camera maps a world point x to camera
space as R x + t with x right, y down, z forward; the principal point is the
image centre and pixel (x, y) is sampled at (x+0.5, y+0.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Gaussians:
    mean: np.ndarray        # [N,3] float32, world space
    log_scale: np.ndarray   # [N,3] float32, natural log of the per-axis std-dev
    quat: np.ndarray        # [N,4] float32, (w,x,y,z), not necessarily exactly unit
    opacity: np.ndarray     # [N]   float32, in (0,1)

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])


@dataclasses.dataclass
class Camera:
    R: np.ndarray           # [3,3] float32, world -> camera rotation (rows = camera axes)
    t: np.ndarray           # [3]   float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    def as_array(self) -> np.ndarray:
        """[R(9), t(3), fx, fy, cx, cy, near] as float32 (the exact values both sides use)."""
        return np.concatenate([
            self.R.reshape(-1).astype(np.float32), self.t.astype(np.float32),
            np.array([self.fx, self.fy, self.cx, self.cy, self.near], np.float32)])


def _sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def tiny_scene(seed: int = 0, n: int = 2000, channels: int = 16):
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    log_scale = rng.normal(-3.5, 0.5, size=(n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, size=n)).astype(np.float32)
    feat = rng.normal(0.0, 1.0, size=(n, channels)).astype(np.float32)
    return Gaussians(mean, log_scale, quat, opacity), feat


ROOM_LO = np.array([-3.0, -3.0, 0.0])
ROOM_HI = np.array([3.0, 3.0, 3.0])


def room_gaussians(rng: np.random.Generator, n: int) -> Gaussians:
    """Room distribution: 60 % near the floor/walls, 40 % uniform in the box."""
    n_plane = int(round(0.6 * n))
    n_free = n - n_plane
    # planes: floor z=0 (36 m^2) and walls x=+-3, y=+-3 (18 m^2 each)
    areas = np.array([36.0, 18.0, 18.0, 18.0, 18.0])
    which = rng.choice(5, size=n_plane, p=areas / areas.sum())
    u = rng.uniform(0.0, 1.0, size=(n_plane, 2))
    off = rng.uniform(0.0, 0.02, size=n_plane)
    pts = np.empty((n_plane, 3))
    # floor
    m = which == 0
    pts[m, 0] = -3 + 6 * u[m, 0]
    pts[m, 1] = -3 + 6 * u[m, 1]
    pts[m, 2] = off[m]
    # wall x = -3 / +3
    for w, sgn in ((1, -1.0), (2, 1.0)):
        m = which == w
        pts[m, 0] = sgn * (3.0 - off[m])
        pts[m, 1] = -3 + 6 * u[m, 0]
        pts[m, 2] = 3 * u[m, 1]
    # wall y = -3 / +3
    for w, sgn in ((3, -1.0), (4, 1.0)):
        m = which == w
        pts[m, 0] = -3 + 6 * u[m, 0]
        pts[m, 1] = sgn * (3.0 - off[m])
        pts[m, 2] = 3 * u[m, 1]
    free = rng.uniform(ROOM_LO, ROOM_HI, size=(n_free, 3))
    mean = np.concatenate([pts, free]).astype(np.float32)
    perm = rng.permutation(n)
    mean = mean[perm]
    log_scale = rng.normal(-4.0, 0.6, size=(n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.5, 1.5, size=n)).astype(np.float32)
    return Gaussians(mean, log_scale, quat, opacity)


def unit_features(rng: np.random.Generator, n: int, channels: int,
                  chunk: int = 65536) -> np.ndarray:
    """N(0,1) rows normalised to unit L2 norm, drawn in row chunks (the same
    values as one draw of the whole [n, channels] array, without its float64
    copy)."""
    out = np.empty((n, channels), np.float32)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        f = rng.normal(0.0, 1.0, size=(b - a, channels))
        f /= np.linalg.norm(f, axis=1, keepdims=True)
        out[a:b] = f
    return out


def room_scene(seed: int = 0, n: int = 500_000, channels: int = 512):
    rng = np.random.default_rng(seed)
    g = room_gaussians(rng, n)
    feat = unit_features(rng, n, channels)
    return g, feat


def look_camera(eye, forward, up, width: int, height: int, fx: float, fy: float,
                near: float = 0.2) -> Camera:
    """Pinhole camera at ``eye`` looking along ``forward`` (x right, y down, z forward)."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    upv = np.asarray(up, np.float64)
    right = np.cross(f, upv)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f]).astype(np.float32)
    t = (-R.astype(np.float64) @ np.asarray(eye, np.float64)).astype(np.float32)
    return Camera(R=R, t=t, fx=float(np.float32(fx)), fy=float(np.float32(fy)),
                  cx=width / 2.0, cy=height / 2.0, width=width, height=height, near=near)


def tiny_camera(width: int = 128, height: int = 128) -> Camera:
    R = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float32)
    t = np.array([0, 0, 3], np.float32)
    return Camera(R=R, t=t, fx=128.0, fy=128.0, cx=width / 2.0, cy=height / 2.0,
                  width=width, height=height, near=0.2)


def hfov_focal(width: int, hfov_deg: float = 60.0) -> float:
    return float(np.float32((width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)))


def room_camera(width: int = 640, height: int = 480, eye=(0.0, 0.0, 1.5),
                yaw: float = 0.0, pitch: float = 0.0, hfov_deg: float = 60.0) -> Camera:
    """Camera inside the room; yaw about +z from +x, pitch up from horizontal (radians)."""
    fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
    f = hfov_focal(width, hfov_deg)
    return look_camera(eye, fwd, (0.0, 0.0, 1.0), width, height, f, f)


def batched_views(seed: int = 0, n_views: int = 32, scenes: int = 4):
    """Per-view (scene index, Camera) for the many-views workload.

    s ~ U[0,1], W = round(320 + 976 s), H = round(240 + 728 s); eye uniform in
    [-2,2]^2 x [1,2]; yaw U[0,2pi); pitch U[-15,15] degrees; 60 degree HFOV.
    """
    rng = np.random.default_rng(seed)
    per = n_views // scenes
    views = []
    for v in range(n_views):
        s = rng.uniform()
        w = int(round(320 + 976 * s))
        h = int(round(240 + 728 * s))
        eye = (rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(1, 2))
        yaw = rng.uniform(0, 2 * math.pi)
        pitch = math.radians(rng.uniform(-15, 15))
        views.append((min(v // per, scenes - 1), room_camera(w, h, eye, yaw, pitch)))
    return views


def unit_queries(seed: int = 7, q: int = 64, channels: int = 512) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return unit_features(rng, q, channels)


def random_selection(seed: int, pixels: int, k: int, n: int, sparsity: float = 0.25):
    """Seeded (ids, weights, counts) for testing the blend on its own.

    ids [P,K] int32 (-1 padded), weights [P,K] float32 (>=0, summing to 1 per
    pixel with count>0), counts [P] uint8.
    """
    rng = np.random.default_rng(seed)
    cnt = rng.integers(0, k + 1, size=pixels)
    cnt[rng.uniform(size=pixels) < sparsity * 0.2] = 0
    mask = np.arange(k)[None, :] < cnt[:, None]
    ids = np.where(mask, rng.integers(0, n, size=(pixels, k)), -1).astype(np.int32)
    x = np.where(mask, rng.uniform(0.05, 1.0, size=(pixels, k)), 0.0)
    s = x.sum(axis=1, keepdims=True)
    w = np.where(s > 0, x / np.where(s > 0, s, 1.0), 0.0).astype(np.float32)
    return ids, w, cnt.astype(np.uint8)


def patch_masks(width: int, height: int, m: int, seed: int = 0, unlabeled: float = 0.1) -> np.ndarray:
    """Synthetic image patches (the masks of Sec. 4.3): a Voronoi partition of
    the image into m regions around random sites; a fraction `unlabeled` of
    the pixels (random) belongs to no patch (-1).  Returns mask_id [H*W] int32."""
    rng = np.random.default_rng(seed)
    sites = np.stack([rng.uniform(0, width, m), rng.uniform(0, height, m)], 1)
    ys, xs = np.mgrid[0:height, 0:width]
    px, py = xs.ravel() + 0.5, ys.ravel() + 0.5
    best = np.full(px.size, np.inf)
    mid = np.zeros(px.size, np.int32)
    for j in range(m):
        d2 = (px - sites[j, 0]) ** 2 + (py - sites[j, 1]) ** 2
        closer = d2 < best
        best[closer] = d2[closer]
        mid[closer] = j
    mid[rng.uniform(size=mid.size) < unlabeled] = -1
    return mid


def patch_targets(m: int, channels: int = 512, seed: int = 3) -> np.ndarray:
    """One CLIP-like embedding per patch: m unit vectors normalise(N(0, I))."""
    return unit_queries(seed, m, channels)


def object_scene(seed: int = 0, n: int = 500_000, channels: int = 512):
    """An object-centric scene (the object workloads of the paper's LeRF /
    MipNeRF360 scenes, stood in for by a synthetic object): 70 % of the
    Gaussians within 1 cm of a unit sphere's surface, 30 % uniform inside it,
    log-scales N(-4.5, 0.5), opacity sigmoid(N(0.5, 1.5)), C-D unit features.
    Seen from outside (object_camera), every pixel's Gaussians come from its
    own patch of the surface, so a frame gathers many distinct feature rows."""
    rng = np.random.default_rng(seed)
    n_s = int(round(0.7 * n))
    d = rng.normal(size=(n_s, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    surf = d * (1.0 + rng.uniform(-0.01, 0.01, size=(n_s, 1)))
    v = rng.normal(size=(n - n_s, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inner = v * rng.uniform(0.0, 1.0, size=(n - n_s, 1)) ** (1.0 / 3.0)
    mean = np.concatenate([surf, inner])[rng.permutation(n)].astype(np.float32)
    log_scale = rng.normal(-4.5, 0.5, size=(n, 3)).astype(np.float32)
    quat = _unit_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.5, 1.5, size=n)).astype(np.float32)
    feat = unit_features(rng, n, channels)
    return Gaussians(mean, log_scale, quat, opacity), feat


def object_camera(width: int = 640, height: int = 480, distance: float = 2.6,
                  hfov_deg: float = 60.0) -> Camera:
    """Camera at `distance` from the object's centre on -y, looking at it, +z up."""
    f = hfov_focal(width, hfov_deg)
    return look_camera((0.0, -distance, 0.3), (0.0, distance, -0.3), (0.0, 0.0, 1.0), width,
                       height, f, f)
