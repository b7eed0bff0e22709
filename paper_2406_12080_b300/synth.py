"""Seeded synthetic inputs shaped like the paper's street-level captures.

This module only draws random inputs: leaf Gaussians (position, scale,
rotation, opacity, SH coefficients) and pinhole cameras placed in the scene.
It holds none of the hierarchical method's arithmetic (no merge, no cut test,
no interpolation, no projection), so that both the CUDA path and the CPU
oracle can consume exactly the same arrays.

Attribute distributions (identical for every scene):
  * log-scale per axis ~ N(-3, 0.5), scale = exp(log-scale)   [metres]
  * rotation: unit quaternion (w, x, y, z) uniform on S^3 (Shoemake 1992)
  * opacity = sigmoid(N(0, 1))
  * SH degree 3: 48 coefficients ~ N(0, 0.3), laid out [k*3 + channel]

Scene shapes follow the paper's capture description: a helmet rig at about
1.7 m (Sec. 7.2), chunks of 50 x 50 m (Sec. 6), 2-8M leaves per chunk (Sec. 8.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_COEFFS = 48
ZNEAR = 0.2


@dataclass
class Leaves:
    """Leaf Gaussians, one row per primitive (float32, C-contiguous)."""
    mean: np.ndarray      # [L, 3]
    scale: np.ndarray     # [L, 3]  (activated, > 0)
    rot: np.ndarray       # [L, 4]  (w, x, y, z), unit norm
    opacity: np.ndarray   # [L]     (activated, in (0, 1))
    sh: np.ndarray        # [L, 48]

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])


@dataclass
class Camera:
    """Pinhole camera. World->camera: x_c = R x_w + T; x right, y down, z forward.

    Pixel (i, j) covers [i, i+1) x [j, j+1) and is sampled at its centre.
    """
    R: np.ndarray         # [3, 3] float32, row-major
    T: np.ndarray         # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tau: float
    znear: float = ZNEAR

    @property
    def center(self) -> np.ndarray:
        return -(self.R.astype(np.float64).T @ self.T.astype(np.float64))


@dataclass
class Scene:
    name: str
    leaves: Leaves
    cameras: list = field(default_factory=list)
    # for chunked scenes: leaf index ranges, one per chunk (each chunk gets its own tree)
    chunk_offsets: np.ndarray | None = None


# --------------------------------------------------------------------------- attributes

def _attributes(rng: np.random.Generator, n: int):
    log_scale = rng.normal(-3.0, 0.5, size=(n, 3))
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    logit = rng.normal(0.0, 1.0, size=n)
    sh = rng.normal(0.0, 0.3, size=(n, SH_COEFFS))
    return (np.exp(log_scale).astype(np.float32), q.astype(np.float32),
            (1.0 / (1.0 + np.exp(-logit))).astype(np.float32), sh.astype(np.float32))


def _leaves(mean: np.ndarray, rng: np.random.Generator) -> Leaves:
    scale, rot, opacity, sh = _attributes(rng, mean.shape[0])
    return Leaves(np.ascontiguousarray(mean, dtype=np.float32), scale, rot, opacity, sh)


def concat_leaves(parts) -> Leaves:
    parts = list(parts)
    return Leaves(*[np.ascontiguousarray(np.concatenate([getattr(p, k) for p in parts]))
                    for k in ("mean", "scale", "rot", "opacity", "sh")])


# --------------------------------------------------------------------------- cameras

def look_camera(pos, forward, up, width, height, hfov_deg, tau) -> Camera:
    """Camera at `pos` looking along `forward`; image y points along -up."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    u = np.asarray(up, np.float64)
    r = np.cross(f, u)
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    T = -R @ np.asarray(pos, np.float64)
    fx = (0.5 * width) / math.tan(math.radians(0.5 * hfov_deg))
    return Camera(R.astype(np.float32), T.astype(np.float32), float(np.float32(fx)),
                  float(np.float32(fx)), 0.5 * width, 0.5 * height, int(width), int(height),
                  float(tau))


def orbit_views(center, radius: float, n_views: int, width: int, height: int, hfov_deg: float = 60.0,
                tau: float = 6.0, elevation: float = 0.3, seed: int = 0):
    """n_views cameras on a ring around `center` (z up), each looking at it; a seeded jitter of the
    ring angle and radius keeps the views distinct."""
    rng = np.random.default_rng([seed, 7])
    c = np.asarray(center, np.float64)
    cams = []
    for i in range(n_views):
        a = 2 * math.pi * (i + rng.uniform(-0.3, 0.3)) / n_views
        r = radius * rng.uniform(0.6, 1.4)
        pos = c + np.array([r * math.cos(a), r * math.sin(a), elevation * r])
        cams.append(look_camera(pos, c - pos, [0, 0, 1], width, height, hfov_deg, tau))
    return cams


def with_tau(cam: Camera, tau: float) -> Camera:
    return Camera(cam.R, cam.T, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                  float(tau), cam.znear)


# --------------------------------------------------------------------------- corridor

@dataclass
class Polyline:
    vertices: np.ndarray   # [S+1, 2]
    seg_len: float

    @property
    def length(self) -> float:
        return self.seg_len * (self.vertices.shape[0] - 1)

    def at(self, s):
        s = np.clip(np.asarray(s, np.float64), 0.0, self.length * (1 - 1e-12))
        seg = np.floor(s / self.seg_len).astype(np.int64)
        d = self.vertices[seg + 1] - self.vertices[seg]
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        p = self.vertices[seg] + (s - seg * self.seg_len)[..., None] * d
        return p, d


def corridor_polyline(seed: int, n_seg: int = 10, seg_len: float = 100.0,
                      max_turn_deg: float = 30.0) -> Polyline:
    rng = np.random.default_rng([seed, 1])
    heading = np.concatenate([[0.0], rng.uniform(-max_turn_deg, max_turn_deg, n_seg - 1)])
    heading = np.radians(np.cumsum(heading))
    steps = seg_len * np.stack([np.cos(heading), np.sin(heading)], axis=1)
    return Polyline(np.concatenate([[[0.0, 0.0]], np.cumsum(steps, axis=0)]), seg_len)


def corridor_leaves(n: int, seed: int, line: Polyline, half_width: float = 10.0,
                    height_scale: float = 5.0) -> Leaves:
    rng = np.random.default_rng([seed, 2])
    s = rng.uniform(0.0, line.length, n)
    lateral = rng.uniform(-half_width, half_width, n)
    h = rng.exponential(height_scale, n)
    p, d = line.at(s)
    normal = np.stack([-d[:, 1], d[:, 0]], axis=1)
    xy = p + lateral[:, None] * normal
    return _leaves(np.column_stack([xy, h]), rng)


def corridor_camera(line: Polyline, s: float, width: int, height: int, tau: float,
                    hfov_deg: float = 60.0, eye_height: float = 1.7) -> Camera:
    p, d = line.at(s)
    pos = [p[0], p[1], eye_height]
    return look_camera(pos, [d[0], d[1], 0.0], [0, 0, 1], width, height, hfov_deg, tau)


# --------------------------------------------------------------------------- scenes

def tiny_scene(seed: int = 0, n_leaves: int = 4096, res: int = 256, tau: float = 6.0) -> Scene:
    """4,096 leaves uniform in a 10 m cube, one 256^2 camera with a 60 deg FOV."""
    rng = np.random.default_rng([seed, 0])
    mean = rng.uniform(0.0, 10.0, size=(n_leaves, 3))
    leaves = _leaves(mean, rng)
    cam = look_camera([5.0, 5.0, -10.0], [0, 0, 1], [0, -1, 0], res, res, 60.0, tau)
    return Scene("tiny", leaves, [cam])


def corridor_scene(seed: int = 1, n_leaves: int = 1_000_000, width: int = 1920,
                   height: int = 1080, tau: float = 6.0, s_cam: float = 300.0) -> Scene:
    """Street corridor: leaves along a 1 km polyline, 20 m wide, heights ~ Exp(5 m)."""
    line = corridor_polyline(seed)
    leaves = corridor_leaves(n_leaves, seed, line)
    return Scene("corridor", leaves, [corridor_camera(line, s_cam, width, height, tau)])


def corridor_views(seed: int = 1, n_views: int = 32,
                   resolutions=((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)),
                   taus=(3.0, 6.0, 15.0), hfov_deg: float = 60.0):
    """Views along the corridor polyline: resolutions in equal groups, tau cycling over `taus`."""
    line = corridor_polyline(seed)
    rng = np.random.default_rng([seed, 6])
    s = np.sort(rng.uniform(50.0, line.length - 50.0, n_views))
    per = max(1, n_views // len(resolutions))
    cams = []
    for i, si in enumerate(s):
        w, h = resolutions[min(i // per, len(resolutions) - 1)]
        cams.append(corridor_camera(line, si, w, h, taus[i % len(taus)], hfov_deg))
    return cams


def optimisation_views(seed: int = 3, n_views: int = 8, width: int = 1280, height: int = 720,
                       tau_min: float = 3.0, tau_max: float = 640.0):
    """Views for the hierarchy-optimisation workload on the corridor.

    Target granularities follow the paper's log-uniform sampling of tau in
    [tau_min, tau_max) (Sec. 5.1); tau_max is half the image width (Sec. 5.2).
    """
    line = corridor_polyline(seed)
    rng = np.random.default_rng([seed, 3])
    s = rng.uniform(50.0, line.length - 50.0, n_views)
    xi = rng.random(n_views)
    taus = tau_max ** xi * tau_min ** (1.0 - xi)
    return line, [corridor_camera(line, si, width, height, ti) for si, ti in zip(s, taus)]


def city_chunk_leaves(seed: int, cx: int, cy: int, per_chunk: int, chunk: float = 50.0,
                      height_scale: float = 5.0) -> Leaves:
    rng = np.random.default_rng([seed, 4, cx, cy])
    xy = rng.uniform(0.0, chunk, size=(per_chunk, 2)) + np.array([cx * chunk, cy * chunk])
    h = rng.exponential(height_scale, per_chunk)
    return _leaves(np.column_stack([xy, h]), rng)


def city_poses(seed: int, n_poses: int, extent: float = 1000.0):
    """Closed loop of (position, forward) pairs at eye height over the city grid."""
    rng = np.random.default_rng([seed, 5])
    k = np.arange(n_poses) / n_poses * 2 * np.pi
    wob = rng.uniform(-0.08, 0.08, size=4)
    rad = 0.32 * extent * (1 + wob[0] * np.sin(2 * k + wob[1] * 10) + wob[2] * np.cos(3 * k))
    cx = cy = 0.5 * extent
    pts = np.stack([cx + rad * np.cos(k), cy + rad * np.sin(k)], axis=1)
    nxt = np.roll(pts, -1, axis=0)
    return [([p[0], p[1], 1.7], [q[0] - p[0], q[1] - p[1], 0.0]) for p, q in zip(pts, nxt)]


def city_path(seed: int, n_poses: int, extent: float = 1000.0, width: int = 1920,
              height: int = 1080, tau: float = 6.0):
    """Closed loop of camera poses at eye height over the city grid."""
    return [look_camera(pos, fwd, [0, 0, 1], width, height, 60.0, tau)
            for pos, fwd in city_poses(seed, n_poses, extent)]


def city_views(seed: int = 2, n_views: int = 32,
               resolutions=((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)),
               taus=(3.0, 6.0, 15.0), extent: float = 1000.0):
    """Views on the city loop: resolutions in equal groups, tau cycling over `taus`."""
    per = max(1, n_views // len(resolutions))
    cams = []
    for i, (pos, fwd) in enumerate(city_poses(seed, n_views, extent)):
        w, h = resolutions[min(i // per, len(resolutions) - 1)]
        cams.append(look_camera(pos, fwd, [0, 0, 1], w, h, 60.0, taus[i % len(taus)]))
    return cams


def city_chunks(seed: int = 2, grid: int = 20, per_chunk: int = 125_000, chunk: float = 50.0):
    """The large-scene workload chunk by chunk: grid x grid chunks of chunk x chunk metres, each drawn
    like the corridor (uniform in the chunk's xy, heights ~ Exp(5 m)).  Yields (index, Leaves)."""
    for c in range(grid * grid):
        yield c, city_chunk_leaves(seed, c % grid, c // grid, per_chunk, chunk)
