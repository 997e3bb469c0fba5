"""Oracle of the reconstruction loss of Eq. 4 -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and bench.py's CPU legs may
import this module; the CUDA library never does.

L_recon = (1 - lambda) L_1 + lambda L_SSIM (Eq. 4, Sec. 2.1), both averaged
over every value of every rendered view.  The paper names SSIM without its
parameters; the reading here is the usual one of the 3DGS training lineage
the paper builds on: SSIM of Wang et al. (2004) per colour channel with an
11 x 11 Gaussian window of standard deviation 1.5 (normalised to sum 1),
zero padding outside the image (one value per pixel), C1 = 0.01^2,
C2 = 0.03^2, L_SSIM = 1 - mean SSIM, and lambda = 0.2.

Everything is FP64 and follows the definition directly: each windowed mean
is the explicit sum over the 121 offsets of the window.
"""
from __future__ import annotations

import numpy as np

RADIUS = 5
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA_SSIM = 0.2


def window1d() -> np.ndarray:
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-(k * k) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def window2d() -> np.ndarray:
    g = window1d()
    return np.outer(g, g)


def windowed(x: np.ndarray) -> np.ndarray:
    """sum_q w(q) x(p + q) for every pixel p of an [H, W] array, with x = 0
    outside the image."""
    h, w = x.shape
    pad = np.zeros((h + 2 * RADIUS, w + 2 * RADIUS), dtype=np.float64)
    pad[RADIUS:RADIUS + h, RADIUS:RADIUS + w] = x
    win = window2d()
    out = np.zeros((h, w), dtype=np.float64)
    for dy in range(2 * RADIUS + 1):
        for dx in range(2 * RADIUS + 1):
            out += win[dy, dx] * pad[dy:dy + h, dx:dx + w]
    return out


def ssim_maps(x: np.ndarray, y: np.ndarray) -> dict:
    """Per-pixel SSIM of one channel and the partial derivatives of S with
    respect to the windowed moments mu_x, E[x^2], E[xy] (what the gradient
    with respect to x needs)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    mx, my = windowed(x), windowed(y)
    exx, eyy, exy = windowed(x * x), windowed(y * y), windowed(x * y)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a = 2.0 * mx * my + C1
    b = 2.0 * cxy + C2
    c = mx * mx + my * my + C1
    d = vx + vy + C2
    s = (a * b) / (c * d)
    # S as a function of (mu_x, var_x, cov_xy); then var_x = E[x^2] - mu_x^2,
    # cov_xy = E[xy] - mu_x mu_y
    ds_dmx = (2.0 * my * b) / (c * d) - s * (2.0 * mx) / c
    ds_dvx = -s / d
    ds_dcxy = 2.0 * a / (c * d)
    return {"s": s, "d_mu": ds_dmx + ds_dvx * (-2.0 * mx) + ds_dcxy * (-my), "d_exx": ds_dvx,
            "d_exy": ds_dcxy, "mu_x": mx, "mu_y": my, "var_x": vx, "var_y": vy, "cov": cxy}


def _views(images: np.ndarray, cams):
    off = 0
    for c in cams:
        n = 3 * c.width * c.height
        yield images[off:off + n].reshape(3, c.height, c.width), slice(off, off + n)
        off += n


def recon_loss(images, target, cams, lam: float = LAMBDA_SSIM) -> dict:
    """L_recon and dL_recon / d images for views packed [v][3][H_v][W_v]."""
    x_all = np.asarray(images, dtype=np.float64).ravel()
    y_all = np.asarray(target, dtype=np.float64).ravel()
    m = x_all.size
    l1 = np.abs(x_all - y_all).sum() / m
    grad = (1.0 - lam) * np.sign(x_all - y_all) / m
    s_sum = 0.0
    for (x, sl), (y, _) in zip(_views(x_all, cams), _views(y_all, cams)):
        g = np.zeros_like(x)
        for ch in range(3):
            mp = ssim_maps(x[ch], y[ch])
            s_sum += mp["s"].sum()
            # d S_total / d x(p) = sum_q w(q - p) [d_mu(q) + 2 x(p) d_exx(q) + y(p) d_exy(q)]
            # (the window is symmetric, so the transpose is the same windowed sum)
            g[ch] = windowed(mp["d_mu"]) + 2.0 * x[ch] * windowed(mp["d_exx"]) + y[ch] * windowed(mp["d_exy"])
        grad[sl] += (-lam / m) * g.ravel()
    l_ssim = 1.0 - s_sum / m
    return {"loss": (1.0 - lam) * l1 + lam * l_ssim, "l1": l1, "l_ssim": l_ssim, "grad": grad}
