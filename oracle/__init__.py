"""FP64 CPU oracle of the codebook Gaussian rasterizer -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library and its Python binding never import it; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over independent
tiles).  This module compiles it with gcc (contraction off, so the FP32
decision arithmetic is one IEEE operation per written operation), loads it
with ctypes and strings the steps together in the order of the method:

  Eq. 2 per SR row -> EWA projection and SH colour per (view, Gaussian)
  -> tile lists ordered by FP32 depth -> Eq. 3 per pixel
  -> exact backward of Eq. 3 -> backward of projection / colour / opacity
  -> codebook rows as sums over the Gaussians that index them (Sec. 4.1).

Integer outcomes (culling, tile rectangles, depth keys, skip / clamp /
termination of an evaluation, colour clamp) are decided in FP32 with the
written operation order; continuous values are FP64 under those decisions.
``replay`` evaluates the FP64 forward of a perturbed scene under the
decisions of the unperturbed one (what finite differences differentiate).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mcmc32.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
          "-D_DEFAULT_SOURCE"]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``mcmc32.c`` into ``liboracle.so`` (gcc, no CUDA)."""
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("k_sr", ctypes.c_int), ("k_sh", ctypes.c_int),
                ("sh_degree", ctypes.c_int), ("pos", ctypes.c_void_p), ("logit", ctypes.c_void_p),
                ("g2sr", ctypes.c_void_p), ("g2sh", ctypes.c_void_p), ("sr", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("w2c", ctypes.c_double * 12), ("campos", ctypes.c_double * 3),
                ("near", ctypes.c_double)]


REC64 = np.dtype([("t", "f8", 3), ("mean", "f8", 2), ("cov", "f8", 3), ("conic", "f8", 3),
                  ("opacity", "f8"), ("rgb", "f8", 3), ("dir", "f8", 3), ("dist", "f8"),
                  ("sigma3", "f8", 6)])
REC32 = np.dtype([("mx", "f4"), ("my", "f4"), ("h0", "f4"), ("h1", "f4"), ("h2", "f4"), ("o", "f4"),
                  ("x0", "i4"), ("y0", "i4"), ("x1", "i4"), ("y1", "i4"), ("depth_bits", "u4"),
                  ("rgb_clamped", "u4"), ("visible", "i4"), ("pad", "i4")])

_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_e32.argtypes = [ctypes.c_float]
            L.or_e32.restype = ctypes.c_float
            L.or_normals32.argtypes = [ctypes.c_int64, _P, _P]
            L.or_log32_batch.argtypes = [ctypes.c_int64, _P, _P]
            L.or_sincos2pi32_batch.argtypes = [ctypes.c_int64, _P, _P, _P]
            L.or_e32_batch.argtypes = [ctypes.c_int64, _P, _P]
            L.or_sh_consts32.argtypes = [_P]
            L.or_sh_basis.argtypes = [ctypes.c_int, _P, _P, _P]
            L.or_sr_sigma.argtypes = [_P, _P]
            L.or_sr_sigma32.argtypes = [_P, _P]
            L.or_sr_sigma_backward.argtypes = [_P, _P, _P]
            L.or_shadow32.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P]
            L.or_preprocess64.argtypes = [_P, _P, ctypes.c_int, _P, _P]
            L.or_count_pairs.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, _P]
            L.or_count_pairs.restype = ctypes.c_int64
            L.or_build_lists.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
            L.or_tile_keep32.argtypes = [ctypes.c_float] * 6 + [ctypes.c_int] * 3
            L.or_tile_keep32.restype = ctypes.c_int
            L.or_blend_forward.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P,
                                           _P, _P, _P, _P, _P, _P]
            L.or_blend_backward.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                            _P, _P, _P, _P, _P]
            L.or_pair_sum.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int64, _P]
            L.or_preprocess_backward.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
            L.or_codebook_reduce.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# small helpers used by the pins
# ----------------------------------------------------------------------------

def e32(x) -> np.ndarray:
    """FP32 exp of the decision arithmetic, elementwise."""
    L = lib()
    x = np.asarray(x, dtype=np.float32).ravel()
    return np.array([L.or_e32(float(v)) for v in x], dtype=np.float32)


def sh_basis(degree: int, direction) -> tuple[np.ndarray, np.ndarray]:
    """FP64 real SH basis Y_k(dir) and dY_k/d(x, y, z)."""
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().or_sh_basis(degree, _ptr(d), _ptr(Y), _ptr(dY))
    nb = (degree + 1) ** 2
    return Y[:nb], dY[:nb]


def tile_keep32(mx, my, h0, h1, h2, o, tx, ty, tile) -> bool:
    """The FP32 tile test of the lists."""
    return bool(lib().or_tile_keep32(mx, my, h0, h1, h2, o, tx, ty, tile))


def sh_consts32() -> np.ndarray:
    out = np.zeros(16, dtype=np.float32)
    lib().or_sh_consts32(_ptr(out))
    return out


def sr_sigma(row) -> np.ndarray:
    """Eq. 2 in FP64 for one SR row: Sigma's unique entries 00 01 02 11 12 22."""
    r = np.zeros(8)
    r[:len(row)] = row
    out = np.zeros(6)
    lib().or_sr_sigma(_ptr(r), _ptr(out))
    return out


def sr_sigma32(row) -> np.ndarray:
    r = np.zeros(8, dtype=np.float32)
    r[:len(row)] = row
    out = np.zeros(6, dtype=np.float32)
    lib().or_sr_sigma32(_ptr(r), _ptr(out))
    return out


def sr_sigma_backward(row, g) -> np.ndarray:
    r = np.zeros(8)
    r[:len(row)] = row
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(8)
    lib().or_sr_sigma_backward(_ptr(r), _ptr(gg), _ptr(out))
    return out


def sym6(m: np.ndarray) -> np.ndarray:
    return np.array([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


def full3(s6) -> np.ndarray:
    a = np.asarray(s6, dtype=np.float64)
    return np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])


# ----------------------------------------------------------------------------
# the full render
# ----------------------------------------------------------------------------

class _SceneBuf:
    """FP64 copies of a scene's arrays and the ctypes struct pointing at them."""

    def __init__(self, scene, sr_rows=None, sh_rows=None):
        self.pos = np.ascontiguousarray(scene.pos, dtype=np.float64)
        self.logit = np.ascontiguousarray(scene.opacity_logit, dtype=np.float64)
        self.g2sr = np.ascontiguousarray(scene.g2sr, dtype=np.uint16)
        self.g2sh = np.ascontiguousarray(scene.g2sh, dtype=np.uint16)
        self.sr = np.ascontiguousarray(scene.sr_rows if sr_rows is None else sr_rows, dtype=np.float64)
        self.sh = np.ascontiguousarray(scene.sh_rows if sh_rows is None else sh_rows, dtype=np.float64)
        self.s = _Scene(self.pos.shape[0], self.sr.shape[0], self.sh.shape[0], scene.sh_degree,
                        self.pos.ctypes.data, self.logit.ctypes.data, self.g2sr.ctypes.data,
                        self.g2sh.ctypes.data, self.sr.ctypes.data, self.sh.ctypes.data)
        self.n = self.pos.shape[0]
        self.sh_degree = scene.sh_degree


def _cams(cams):
    arr = (_Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width, arr[i].height = int(c.width), int(c.height)
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        w = np.asarray(c.world_to_cam, dtype=np.float64).ravel()
        for j in range(12):
            arr[i].w2c[j] = float(w[j])
        for j in range(3):
            arr[i].campos[j] = float(c.campos[j])
        arr[i].near = float(c.near)
    return arr


class Render:
    """Oracle render of ``scene`` from ``cams``.

    mode 0: rasterizer rules (alpha skip below 1/255, clamp at 0.99,
    termination below transmittance 1e-4, decided in FP32); mode 1: Eq. 3 as
    printed.  ``tile_mask`` (uint8 per global tile) restricts the per-pixel
    work to a subset of tiles (for sampled checks of large workloads).
    ``cull`` lists a record only in the tiles of its rectangle that pass the
    FP32 tile test (or_tile_keep32); without it, in every tile of it.  The
    default culls under the rasterizer rules (mode 0) and not for Eq. 3 as
    printed (mode 1), where every listed Gaussian contributes.
    ``lists_in_mask`` also restricts the tile lists to the masked tiles (the
    other tiles' lists stay empty), which bounds the work on large scenes.
    """

    def __init__(self, scene, cams, tile: int = 16, bg=(0.0, 0.0, 0.0), mode: int = 0,
                 tile_mask: np.ndarray | None = None, cull: bool | None = None, lists_in_mask: bool = False):
        if len(cams) > 64:
            raise ValueError("the oracle handles at most 64 views")
        L = lib()
        self.scene = scene
        self.cams = list(cams)
        self.tile = int(tile)
        self.bg = np.ascontiguousarray(bg, dtype=np.float64)
        self.mode = int(mode)
        self.V = len(cams)
        self._c = _cams(cams)
        self.sb = _SceneBuf(scene)
        n = self.sb.n
        self.n = n
        self.tiles_x = np.array([-(-c.width // tile) for c in cams], dtype=np.int32)
        self.tiles_y = np.array([-(-c.height // tile) for c in cams], dtype=np.int32)
        ntile_v = self.tiles_x.astype(np.int64) * self.tiles_y
        self.tile_base = np.concatenate([[0], np.cumsum(ntile_v)[:-1]]).astype(np.int64)
        self.n_tiles = int(ntile_v.sum())
        self.pix_counts = np.array([c.width * c.height for c in cams], dtype=np.int64)
        self.pix_base = np.concatenate([[0], np.cumsum(self.pix_counts)[:-1]]).astype(np.int64)
        self.P = int(self.pix_counts.sum())
        self.tile_mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
        # wall time of each step (seconds), for the CPU baseline
        self.timing = {}
        t0 = time.perf_counter()
        # decisions (FP32) and tile lists
        self.rec32 = np.zeros(self.V * n, dtype=REC32)
        L.or_shadow32(ctypes.byref(self.sb.s), self._c, self.V, self.tile, _ptr(self.rec32))
        t1 = time.perf_counter()
        self.timing["shadow"] = t1 - t0
        self.cull = (self.mode == 0) if cull is None else bool(cull)
        lmask = _ptr(self.tile_mask) if (lists_in_mask and self.tile_mask is not None) else None
        self.k_pairs = int(L.or_count_pairs(_ptr(self.rec32), n, self.V, _ptr(self.tiles_x), _ptr(self.tile_base),
                                            self.tile, int(self.cull), lmask))
        if self.k_pairs >= 2 ** 32:
            raise ValueError("pair count exceeds 32-bit indexing")
        self.list = np.zeros(max(self.k_pairs, 1), dtype=np.uint32)
        self.keys = np.zeros(max(self.k_pairs, 1), dtype=np.uint64)
        self.ranges = np.zeros((self.n_tiles, 2), dtype=np.uint32)
        L.or_build_lists(_ptr(self.rec32), n, self.V, _ptr(self.tiles_x), _ptr(self.tile_base),
                         self.n_tiles, self.k_pairs, self.tile, int(self.cull), lmask, _ptr(self.list),
                         _ptr(self.keys), _ptr(self.ranges))
        self.list = self.list[:self.k_pairs]
        self.keys = self.keys[:self.k_pairs]
        t2 = time.perf_counter()
        self.timing["lists"] = t2 - t1
        self.rec64 = self._preprocess(self.sb)
        t3 = time.perf_counter()
        self.timing["preprocess"] = t3 - t2
        self.image, self.t_final, self.n_contrib, self.term_pos = self._forward(self.rec64)
        self.timing["blend_fwd"] = time.perf_counter() - t3

    # -- steps ---------------------------------------------------------------
    def _preprocess(self, sb: _SceneBuf) -> np.ndarray:
        rec64 = np.zeros(self.V * self.n, dtype=REC64)
        lib().or_preprocess64(ctypes.byref(sb.s), self._c, self.V, _ptr(self.rec32), _ptr(rec64))
        return rec64

    def _forward(self, rec64):
        image = np.zeros(3 * self.P)
        t_final = np.zeros(self.P)
        n_contrib = np.zeros(self.P, dtype=np.int32)
        term_pos = np.full(self.P, -1, dtype=np.int32)
        mask = _ptr(self.tile_mask) if self.tile_mask is not None else None
        lib().or_blend_forward(self._c, self.V, self.tile, _ptr(self.bg), self.mode, _ptr(self.rec32),
                               _ptr(rec64), _ptr(self.list), _ptr(self.ranges), mask, _ptr(image),
                               _ptr(t_final), _ptr(n_contrib), _ptr(term_pos))
        return image, t_final, n_contrib, term_pos

    def replay(self, scene, sr_rows=None, sh_rows=None) -> np.ndarray:
        """FP64 image of a (perturbed) scene under this render's decisions."""
        sb = _SceneBuf(scene, sr_rows, sh_rows)
        rec64 = self._preprocess(sb)
        return self._forward(rec64)[0]

    def backward(self, d_image: np.ndarray) -> dict:
        """Exact FP64 gradient of sum(d_image * image) under this render's
        decisions."""
        L = lib()
        d_image = np.ascontiguousarray(d_image, dtype=np.float64).ravel()
        assert d_image.size == 3 * self.P
        n_rec = self.V * self.n
        grad9 = np.zeros((n_rec, 9))
        mask = _ptr(self.tile_mask) if self.tile_mask is not None else None
        pair = np.zeros((max(self.k_pairs, 1), 9))
        t0 = time.perf_counter()
        L.or_blend_backward(self._c, self.V, self.tile, _ptr(self.bg), self.mode, _ptr(self.rec32),
                            _ptr(self.rec64), _ptr(self.list), _ptr(self.ranges), mask, _ptr(d_image),
                            _ptr(pair))
        t1 = time.perf_counter()
        L.or_pair_sum(_ptr(self.list), self.k_pairs, _ptr(pair), n_rec, _ptr(grad9))
        t2 = time.perf_counter()
        del pair
        self.timing["blend_bwd"] = t1 - t0
        self.timing["pair_sum"] = t2 - t1
        t1 = t2
        dpos = np.zeros((self.n, 3))
        dlogit = np.zeros(self.n)
        dsigma = np.zeros((self.n, 6))
        drgb = np.zeros((n_rec, 3))
        L.or_preprocess_backward(ctypes.byref(self.sb.s), self._c, self.V, _ptr(self.rec32),
                                 _ptr(self.rec64), _ptr(grad9), _ptr(dpos), _ptr(dlogit), _ptr(dsigma),
                                 _ptr(drgb))
        nb = (self.scene.sh_degree + 1) ** 2
        d_sr = np.zeros((self.sb.sr.shape[0], 8))
        d_sh = np.zeros((self.sb.sh.shape[0], nb, 3))
        L.or_codebook_reduce(ctypes.byref(self.sb.s), self.V, _ptr(self.rec64), _ptr(dsigma), _ptr(drgb),
                             _ptr(d_sr), _ptr(d_sh))
        self.timing["gaussian_bwd_reduce"] = time.perf_counter() - t1
        return {"grad9": grad9, "dpos": dpos, "dlogit": dlogit, "dsigma": dsigma, "drgb": drgb,
                "d_sr": d_sr, "d_sh": d_sh}

    # -- views of the outputs ----------------------------------------------------
    def view_image(self, v: int) -> np.ndarray:
        c = self.cams[v]
        b = 3 * self.pix_base[v]
        return self.image[b:b + 3 * c.width * c.height].reshape(3, c.height, c.width)

    def view_pixels(self, arr: np.ndarray, v: int) -> np.ndarray:
        c = self.cams[v]
        b = self.pix_base[v]
        return arr[b:b + c.width * c.height].reshape(c.height, c.width)

    def tile_list(self, gt: int) -> np.ndarray:
        b, e = self.ranges[gt]
        return self.list[b:e]


def codebook_reduce(scene, rec64, dsigma, drgb, n_views: int):
    """The codebook-row sums alone, from per-Gaussian terms (FP64)."""
    L = lib()
    sb = _SceneBuf(scene)
    nb = (scene.sh_degree + 1) ** 2
    d_sr = np.zeros((sb.sr.shape[0], 8))
    d_sh = np.zeros((sb.sh.shape[0], nb, 3))
    L.or_codebook_reduce(ctypes.byref(sb.s), n_views, _ptr(np.ascontiguousarray(rec64)),
                         _ptr(np.ascontiguousarray(dsigma, dtype=np.float64)),
                         _ptr(np.ascontiguousarray(drgb, dtype=np.float64)), _ptr(d_sr), _ptr(d_sh))
    return d_sr, d_sh
