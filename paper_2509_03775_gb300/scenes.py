"""Seeded synthetic scenes and cameras for the codebook Gaussian rasterizer.

This module only draws inputs: Gaussian records g_i = {p_i, o_i, g2sr_i, g2sh_i}
and the two codebooks C = {SR, SH} of the codebook-compressed state S = {G, C}
(ContraGS, Sec. 4.1), plus pinhole cameras.  It holds none of the rendering
arithmetic, so the CPU oracle and the CUDA path can both consume it.

The paper trains on Tanks&Temples, MipNeRF360, Deep Blending and Blender
(Sec. 5.1).  Those datasets are not used; these scenes stand in for them with
the sizes and value distributions of the five workloads listed below.  Every
array is produced by ``numpy.random.default_rng(1000 + config_index)``.

Layouts (all C-contiguous):
  pos            float32 [N, 3]
  opacity_logit  float32 [N]             (o_i = sigmoid(logit))
  g2sr, g2sh     uint16  [N]
  sr_rows        float32 [K_sr, 8]       (3 log-scales, quaternion w x y z, pad 0)
  sh_rows        float32 [K_sh, (d+1)^2, 3]
Camera: OpenCV axes (x right, y down, z forward); world_to_cam is the 3x4
row-major [R | t]; campos is the eye point the camera was built from.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SR_WIDTH = 8


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # float32 [3, 4]
    campos: np.ndarray        # float32 [3]
    near: float = 0.2


@dataclasses.dataclass
class Scene:
    pos: np.ndarray
    opacity_logit: np.ndarray
    g2sr: np.ndarray
    g2sh: np.ndarray
    sr_rows: np.ndarray
    sh_rows: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def k_sr(self) -> int:
        return int(self.sr_rows.shape[0])

    @property
    def k_sh(self) -> int:
        return int(self.sh_rows.shape[0])

    def copy(self) -> "Scene":
        return Scene(self.pos.copy(), self.opacity_logit.copy(), self.g2sr.copy(),
                     self.g2sh.copy(), self.sr_rows.copy(), self.sh_rows.copy(),
                     self.sh_degree)


def look_at(eye, width: int, height: int, fov_x_deg: float = 60.0,
            target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), near: float = 0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; focal length from the
    horizontal field of view, square pixels, principal point at the centre."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    upv = np.asarray(up, dtype=np.float64)
    if abs(float(f @ upv)) > 0.99:
        raise ValueError("camera direction too close to the up axis")
    right = np.cross(f, upv)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    rot = np.stack([right, down, f])          # rows: camera axes in world frame
    t = -rot @ eye
    w2c = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(width, height, float(np.float32(fx)), float(np.float32(fx)),
                  float(np.float32(0.5 * width)), float(np.float32(0.5 * height)),
                  w2c, eye.astype(np.float32), near)


def fibonacci_dirs(count: int, rng: np.random.Generator) -> np.ndarray:
    """Unit directions on a Fibonacci sphere, rotated by a seeded rotation and
    kept away from the +-y poles (the look-at up axis)."""
    out = []
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                    [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                    [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    golden = math.pi * (3.0 - math.sqrt(5.0))
    i = 0
    while len(out) < count:
        k = len(out) + i
        yy = 1.0 - 2.0 * (k + 0.5) / (count + 4)
        r = math.sqrt(max(0.0, 1.0 - yy * yy))
        d = rot @ np.array([math.cos(golden * k) * r, yy, math.sin(golden * k) * r])
        if abs(d[1]) < 0.9:
            out.append(d)
        else:
            i += 1
    return np.asarray(out)


def _unit_quats(rng: np.random.Generator, k: int) -> np.ndarray:
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sr_rows(rng: np.random.Generator, k: int, ls_mean: float, ls_std: float) -> np.ndarray:
    rows = np.zeros((k, SR_WIDTH), dtype=np.float64)
    rows[:, 0:3] = rng.normal(ls_mean, ls_std, size=(k, 3))
    rows[:, 3:7] = _unit_quats(rng, k)
    return rows.astype(np.float32)


def _sh_rows(rng: np.random.Generator, k: int, degree: int) -> np.ndarray:
    nb = (degree + 1) ** 2
    rows = np.empty((k, nb, 3), dtype=np.float64)
    rows[:, 0, :] = rng.normal(0.0, 0.5, size=(k, 3))
    if nb > 1:
        rows[:, 1:, :] = rng.normal(0.0, 0.1, size=(k, nb - 1, 3))
    return rows.astype(np.float32)


def _zipf_indices(rng: np.random.Generator, n: int, k: int, s: float = 1.1) -> np.ndarray:
    """Row usage P(rank r) proportional to (r + 1)^-s, ranks mapped to rows by a
    seeded permutation."""
    p = (np.arange(k, dtype=np.float64) + 1.0) ** (-s)
    p /= p.sum()
    ranks = rng.choice(k, size=n, p=p)
    perm = rng.permutation(k)
    return perm[ranks].astype(np.uint16)


def _random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    q = _unit_quats(rng, k)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], axis=1)


def _aniso_mixture(rng: np.random.Generator, n: int, clusters: int) -> np.ndarray:
    centres = rng.uniform(-1.0, 1.0, size=(clusters, 3))
    rots = _random_rotations(rng, clusters)
    sig = rng.uniform(0.05, 0.5, size=(clusters, 3))
    lab = rng.integers(0, clusters, size=n)
    z = rng.normal(size=(n, 3)) * sig[lab]
    return centres[lab] + np.einsum("nij,nj->ni", rots[lab], z)


# --------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------

def config_tiny(seed_offset: int = 0):
    """1,024 Gaussians, 4-cluster isotropic mixture (sigma 0.3) clipped to
    [-1,1]^3; K_sr = K_sh = 64 uniform indices; SH degree 1; one 128x128
    camera at radius 3, FOV 60 deg.  Also returns the jittered-position
    target scene (positions + N(0, 0.01))."""
    rng = np.random.default_rng(1001 + seed_offset)
    n, k = 1024, 64
    centres = rng.uniform(-1.0, 1.0, size=(4, 3))
    lab = rng.integers(0, 4, size=n)
    pos = np.clip(centres[lab] + rng.normal(0.0, 0.3, size=(n, 3)), -1.0, 1.0)
    scene = Scene(pos=pos.astype(np.float32),
                  opacity_logit=rng.normal(0.0, 1.0, size=n).astype(np.float32),
                  g2sr=rng.integers(0, k, size=n).astype(np.uint16),
                  g2sh=rng.integers(0, k, size=n).astype(np.uint16),
                  sr_rows=_sr_rows(rng, k, -3.0, 0.5),
                  sh_rows=_sh_rows(rng, k, 1), sh_degree=1)
    cam = look_at(3.0 * np.array([0.35, -0.30, -0.89]) / np.linalg.norm([0.35, -0.30, -0.89]),
                  128, 128)
    target = scene.copy()
    target.pos = (scene.pos + rng.normal(0.0, 0.01, size=(n, 3))).astype(np.float32)
    return scene, [cam], target


def config_single(n: int = 200_000, k: int = 4096, width: int = 800, height: int = 800,
                  seed_offset: int = 0):
    """200k Gaussians: 8-cluster isotropic mixture with per-cluster sigma
    U[0.1, 0.4] plus 10 % uniform background in [-1,1]^3; SH degree 3;
    K_sr = K_sh = 4096 with Zipf(1.1) row usage; 800x800 camera, radius 3."""
    rng = np.random.default_rng(1002 + seed_offset)
    n_bg = n // 10
    n_cl = n - n_bg
    centres = rng.uniform(-1.0, 1.0, size=(8, 3))
    sig = rng.uniform(0.1, 0.4, size=8)
    lab = rng.integers(0, 8, size=n_cl)
    pos = np.concatenate([centres[lab] + rng.normal(size=(n_cl, 3)) * sig[lab, None],
                          rng.uniform(-1.0, 1.0, size=(n_bg, 3))])
    scene = Scene(pos=pos.astype(np.float32),
                  opacity_logit=rng.normal(0.0, 1.0, size=n).astype(np.float32),
                  g2sr=_zipf_indices(rng, n, k), g2sh=_zipf_indices(rng, n, k),
                  sr_rows=_sr_rows(rng, k, -3.0, 0.5), sh_rows=_sh_rows(rng, k, 3),
                  sh_degree=3)
    cam = look_at(3.0 * np.array([-0.42, -0.25, -0.87]) / np.linalg.norm([-0.42, -0.25, -0.87]),
                  width, height)
    return scene, [cam]


def scene_truck(n: int = 1_500_000, k: int = 8192, clusters: int = 64, seed: int = 1003,
                sh_degree: int = 3) -> Scene:
    """Truck-shaped scene: anisotropic mixture (per-cluster covariance =
    random rotation * diag(U[0.05, 0.5])^2), log-scales N(-4, 0.5), random unit
    quaternions, SH degree 3, Zipf(1.1) row usage of both codebooks."""
    rng = np.random.default_rng(seed)
    pos = _aniso_mixture(rng, n, clusters)
    return Scene(pos=pos.astype(np.float32),
                 opacity_logit=rng.normal(0.0, 1.0, size=n).astype(np.float32),
                 g2sr=_zipf_indices(rng, n, k), g2sh=_zipf_indices(rng, n, k),
                 sr_rows=_sr_rows(rng, k, -4.0, 0.5), sh_rows=_sh_rows(rng, k, sh_degree),
                 sh_degree=sh_degree)


TRUCK_EYE_DIR = np.array([0.48, -0.22, -0.85])


def config_truck(scale: float = 1.0):
    """1.5M-Gaussian truck-shaped scene and one 1957x1091 camera at radius 4.
    ``scale`` < 1 shrinks the image (same FOV) for oracle-sized runs."""
    scene = scene_truck()
    w, h = max(16, int(round(1957 * scale))), max(16, int(round(1091 * scale)))
    cam = look_at(4.0 * TRUCK_EYE_DIR / np.linalg.norm(TRUCK_EYE_DIR), w, h)
    return scene, [cam]


BATCHED_RES = [(1957, 1091)] * 4 + [(1280, 720)] * 2 + [(800, 800)] * 2


def config_batched(scale: float = 1.0):
    """The truck-shaped scene seen by 8 cameras on a radius-4 sphere
    (Fibonacci directions, seeded rotation): 4 x 1957x1091, 2 x 1280x720,
    2 x 800x800."""
    scene = scene_truck()
    rng = np.random.default_rng(1004)
    dirs = fibonacci_dirs(len(BATCHED_RES), rng)
    cams = [look_at(4.0 * d, max(16, int(round(w * scale))), max(16, int(round(h * scale))))
            for d, (w, h) in zip(dirs, BATCHED_RES)]
    return scene, cams


def config_large(n: int = 4_000_000, views: int = 16, scale: float = 1.0):
    """4M Gaussians from a 128-cluster mixture, SH degree 3, 16384 rows per
    codebook (stored as BF16 by the caller), 16 cameras at 1957x1091."""
    scene = scene_truck(n=n, k=16384, clusters=128, seed=1005)
    rng = np.random.default_rng(1005 + 7)
    dirs = fibonacci_dirs(views, rng)
    cams = [look_at(4.0 * d, max(16, int(round(1957 * scale))), max(16, int(round(1091 * scale))))
            for d in dirs]
    return scene, cams


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even) and return
    them as float32; also the bit pattern the BF16 codebook storage holds."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of ``bf16_round(a)``."""
    return (bf16_round(a).view(np.uint32) >> 16).astype(np.uint16)
