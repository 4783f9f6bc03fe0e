"""Seeded synthetic scenes and cameras shaped like the paper's workloads.

This module holds input generation only: no projection, window, compositing or colour
arithmetic of the renderer lives here. It is the one module both the CUDA path's tests
and the FP64 oracle's tests draw inputs from.

The paper trains on Mip-NeRF360 / Tanks&Temples captures initialised from SfM points
(Sec. 3.3, "Optimization"); none is available, so these generators stand in for them:
points are sampled on synthetic surfaces and each becomes a triangle by the paper's
initialisation rule v_i = q + k d u_i, with d the mean distance to the 3 nearest
neighbours, u_i uniform on the unit sphere and k = 2.2 (Sec. 3.3; Supp.
"Initialization").

Cameras use OpenCV axes (+x right, +y down, +z forward), R world->camera, and
fx = fy = 0.9375 W, cx = W/2, cy = H/2 unless a workload fixes them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

INIT_K = 2.2  # Supp. "Initialization": scaling constant k of the initial triangles


@dataclass
class Scene:
    verts: np.ndarray          # [N, 3, 3] float32, world space
    sh: np.ndarray             # [N, (deg+1)^2, 3] float32
    opacity: np.ndarray        # [N] float32 in (0, 1]
    sigma: np.ndarray          # [N] float32 > 0
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.verts.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.verts[idx]), np.ascontiguousarray(self.sh[idx]),
                     np.ascontiguousarray(self.opacity[idx]), np.ascontiguousarray(self.sigma[idx]),
                     self.sh_degree)

    def permuted(self, perm) -> "Scene":
        return self.subset(perm)


@dataclass
class Camera:
    R: np.ndarray              # [3, 3] float32, world -> camera rotation
    t: np.ndarray              # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))

    def position(self) -> np.ndarray:
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


def _f32(x) -> float:
    return float(np.float32(x))


def camera_identity(W: int, H: int, fx: float | None = None, fy: float | None = None,
                    cx: float | None = None, cy: float | None = None) -> Camera:
    fx = 0.9375 * W if fx is None else fx
    fy = fx if fy is None else fy
    return Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), _f32(fx), _f32(fy),
                  _f32(W / 2 if cx is None else cx), _f32(H / 2 if cy is None else cy), int(W), int(H))


def camera_look_at(eye, target, W: int, H: int, up=(0.0, -1.0, 0.0), fx: float | None = None) -> Camera:
    """World->camera pose looking from ``eye`` at ``target``; ``up`` is the world
    direction that appears upward in the image (image +y points down)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    fx = 0.9375 * W if fx is None else fx
    return Camera(R, t, _f32(fx), _f32(fx), _f32(W / 2), _f32(H / 2), int(W), int(H))


def crop_camera(cam: Camera, x0: int, y0: int, W: int, H: int) -> Camera:
    """The window [x0, x0+W) x [y0, y0+H) of ``cam`` as a camera of its own."""
    return Camera(cam.R.copy(), cam.t.copy(), cam.fx, cam.fy, _f32(cam.cx - x0), _f32(cam.cy - y0),
                  int(W), int(H), cam.bg.copy())


def _unit(rng, n):
    u = rng.standard_normal((n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def _knn_mean_dist(points: np.ndarray, k: int = 3) -> np.ndarray:
    from scipy.spatial import cKDTree
    tree = cKDTree(points)
    d, _ = tree.query(points, k=k + 1, workers=-1)
    return d[:, 1:].mean(axis=1)


def triangles_from_points(rng, points: np.ndarray) -> np.ndarray:
    """Paper initialisation (Sec. 3.3): v_i = q + k d u_i."""
    d = _knn_mean_dist(points)
    u = np.stack([_unit(rng, len(points)) for _ in range(3)], axis=1)       # [N,3,3]
    v = points[:, None, :] + INIT_K * d[:, None, None] * u
    return v.astype(np.float32)


def _sh_normal(rng, n, deg, std=0.2):
    return (rng.standard_normal((n, (deg + 1) ** 2, 3)) * std).astype(np.float32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


# --------------------------------------------------------------------------------------
# Workload 1: 5,000 triangles, SH degree 0, 160x120, fx = fy = 150
# --------------------------------------------------------------------------------------
def scene_small(n: int = 5000, seed: int = 1001) -> Scene:
    """Centroids uniform in x in [-1.5,1.5], y in [-1.1,1.1], z in [2,6]; equilateral
    frames with random orientation, edge ~ log-normal (mean 0.05, shape 0.5), each
    vertex radius jittered by 10 %; colour SH degree 0 with c_00 uniform in
    [-sqrt(pi), sqrt(pi)] (the colour range [0, 1] under the +0.5 offset); opacity
    U[0.1, 0.9]; sigma U[0.5, 2]."""
    rng = np.random.default_rng(seed)
    c = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.1, 1.1, n), rng.uniform(2, 6, n)], 1)
    s = 0.5
    base = rng.lognormal(np.log(0.05) - s * s / 2, s, n)
    a = _unit(rng, n)
    b = np.cross(a, _unit(rng, n))
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    e2 = np.cross(a, b)
    ang = np.array([0.0, 2 * np.pi / 3, 4 * np.pi / 3])
    rad = base[:, None] / np.sqrt(3.0) * (1.0 + 0.1 * rng.standard_normal((n, 3)))
    v = c[:, None, :] + rad[..., None] * (np.cos(ang)[None, :, None] * b[:, None, :] +
                                          np.sin(ang)[None, :, None] * e2[:, None, :])
    sh = rng.uniform(-np.sqrt(np.pi), np.sqrt(np.pi), (n, 1, 3)).astype(np.float32)
    opac = rng.uniform(0.1, 0.9, n).astype(np.float32)
    sig = rng.uniform(0.5, 2.0, n).astype(np.float32)
    return Scene(v.astype(np.float32), sh, opac, sig, 0)


def camera_small() -> Camera:
    return camera_identity(160, 120, fx=150.0, fy=150.0, cx=80.0, cy=60.0)


# --------------------------------------------------------------------------------------
# Workload 2: 500k triangles in 200 planar patches, SH degree 3, 1297x840
# --------------------------------------------------------------------------------------
def patch_points(n: int, n_patch: int, rng, radius=0.3, noise=0.02):
    centres = np.stack([rng.uniform(-1.5, 1.5, n_patch), rng.uniform(-1.1, 1.1, n_patch),
                        rng.uniform(2, 6, n_patch)], 1)
    normals = _unit(rng, n_patch)
    which = rng.integers(0, n_patch, n)
    nv = normals[which]
    a = np.cross(nv, _unit(rng, n))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(nv, a)
    rr = radius * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    p = centres[which] + rr[:, None] * (np.cos(th)[:, None] * a + np.sin(th)[:, None] * b)
    p += noise * rng.standard_normal((n, 3))
    return p, centres, which


def scene_patches(n: int = 500_000, n_patch: int = 200, seed: int = 1002, deg: int = 3):
    """Returns (scene, patch centres, patch index per triangle)."""
    rng = np.random.default_rng(seed)
    pts, centres, which = patch_points(n, n_patch, rng)
    v = triangles_from_points(rng, pts)
    sh = _sh_normal(rng, n, deg)
    opac = _sigmoid(rng.standard_normal(n)).astype(np.float32)
    sig = _log_uniform(rng, 0.3, 3.0, n).astype(np.float32)
    return Scene(v, sh, opac, sig, deg), centres, which


def camera_patches(W: int = 1297, H: int = 840) -> Camera:
    return camera_identity(W, H)


def target_image(H: int, W: int, seed: int = 2002) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0, 1, (3, H, W)).astype(np.float32)


def crop_around(scene: Scene, cam: Camera, centre, n_keep=2000, size=128):
    """The ``n_keep`` triangles nearest ``centre`` and a size x size window of ``cam``
    centred on the projection of ``centre``."""
    cen = scene.verts.astype(np.float64).mean(axis=1)
    idx = np.argsort(np.linalg.norm(cen - np.asarray(centre)[None], axis=1), kind="stable")[:n_keep]
    idx = np.sort(idx)
    pc = cam.R.astype(np.float64) @ np.asarray(centre, np.float64) + cam.t
    u = cam.fx * pc[0] / pc[2] + cam.cx
    v = cam.fy * pc[1] / pc[2] + cam.cy
    x0, y0 = int(round(u - size / 2)), int(round(v - size / 2))
    return scene.subset(idx), crop_camera(cam, x0, y0, size, size), idx


# --------------------------------------------------------------------------------------
# Workload 3-5: nested spherical shells (indoor-like), SH degree 3
# --------------------------------------------------------------------------------------
def scene_shells(n: int = 3_000_000, seed: int = 1003, n_shell: int = 16, deg: int = 3,
                 r_lo: float = 1.0, r_hi: float = 10.0) -> Scene:
    rng = np.random.default_rng(seed)
    radii = np.linspace(r_lo, r_hi, n_shell)
    w = radii ** 2 / np.sum(radii ** 2)
    counts = np.floor(w * n).astype(np.int64)
    counts[-1] += n - counts.sum()
    shell = np.repeat(np.arange(n_shell), counts)
    r = radii[shell] * (1.0 + 0.01 * rng.standard_normal(n))
    pts = _unit(rng, n) * r[:, None]
    v = triangles_from_points(rng, pts)
    sh = _sh_normal(rng, n, deg)
    opac = _sigmoid(rng.standard_normal(n)).astype(np.float32)
    sig = _log_uniform(rng, 0.3, 3.0, n).astype(np.float32)
    return Scene(v, sh, opac, sig, deg)


def ring_cameras(n_views: int = 16, radius: float = 4.0, W: int = 1558, H: int = 1038,
                 offset: float = 0.0):
    cams = []
    for k in range(n_views):
        a = offset + 2 * np.pi * k / n_views
        eye = (radius * np.cos(a), 0.0, radius * np.sin(a))
        cams.append(camera_look_at(eye, (0, 0, 0), W, H))
    return cams


SERVE_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080))


def serve_requests(n_req: int = 4096, seed: int = 1004, rate_hz: float = 2000.0,
                   mix=(2, 2, 1), n_scenes: int = 1):
    """Open-loop request trace: Poisson arrivals, mixed resolutions, poses uniform on a
    sphere of radius U[3, 5] looking at the origin. Returns a list of
    (arrival_s, scene_id, Camera)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_req)
    t = np.cumsum(gaps) - gaps[0]
    p = np.asarray(mix, np.float64) / np.sum(mix)
    res = rng.choice(len(SERVE_RESOLUTIONS), n_req, p=p)
    out = []
    for i in range(n_req):
        while True:
            d = _unit(rng, 1)[0]
            if abs(d[1]) < 0.95:
                break
        eye = d * rng.uniform(3.0, 5.0)
        W, H = SERVE_RESOLUTIONS[res[i]]
        out.append((float(t[i]), int(rng.integers(0, n_scenes)), camera_look_at(eye, (0, 0, 0), W, H)))
    return out


def scene_sizes_multi(n_scenes: int = 8, seed: int = 1005, lo: int = 200_000, hi: int = 2_000_000):
    rng = np.random.default_rng(seed)
    return [int(x) for x in _log_uniform(rng, lo, hi, n_scenes)]


# --------------------------------------------------------------------------------------
# small helpers for tests
# --------------------------------------------------------------------------------------
def random_scene(n: int, seed: int, deg: int = 3, box=((-1, 1), (-0.8, 0.8), (2.5, 5.0)),
                 size=(0.05, 0.4), sigma=(0.5, 2.0), opacity=(0.2, 0.95), sh_std=0.3) -> Scene:
    """A small scene of random triangles in front of the identity camera."""
    rng = np.random.default_rng(seed)
    c = np.stack([rng.uniform(*box[0], n), rng.uniform(*box[1], n), rng.uniform(*box[2], n)], 1)
    sz = rng.uniform(*size, n)
    v = c[:, None, :] + sz[:, None, None] * _unit(rng, 3 * n).reshape(n, 3, 3)
    sh = (rng.standard_normal((n, (deg + 1) ** 2, 3)) * sh_std).astype(np.float32)
    opac = rng.uniform(*opacity, n).astype(np.float32)
    sig = rng.uniform(*sigma, n).astype(np.float32)
    return Scene(v.astype(np.float32), sh, opac, sig, deg)
