"""Oracle: image-quality metrics (PSNR, SSIM) in float64.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.

The paper reports PSNR and SSIM (its "Image Quality" section) without
fixing their conventions.  Readings used here: images are RGB clamped to
[0, 1]; PSNR with MAX = 1 over all pixels and channels; SSIM after Wang et
al. 2004 with an 11x11 Gaussian window (sigma 1.5, truncated at radius 5),
K1 = 0.01, K2 = 0.03, computed per channel over the valid (unpadded) window
positions and averaged; tPSNR the PSNR (MAX = 1) of the frame-to-frame change
of the reconstruction against that of the reference, frames clamped first.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate1d


def psnr(a, b):
    a = np.clip(np.asarray(a, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(b, np.float64), 0.0, 1.0)
    mse = np.mean((a - b) ** 2)
    if mse == 0.0:
        return float("inf")
    return float(-10.0 * np.log10(mse))


def _gauss_window(sigma=1.5, radius=5):
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-0.5 * (x / sigma) ** 2)
    return g / g.sum()


def _filter_valid(img, g):
    r = (len(g) - 1) // 2
    out = correlate1d(img, g, axis=0, mode="constant")
    out = correlate1d(out, g, axis=1, mode="constant")
    return out[r:img.shape[0] - r, r:img.shape[1] - r]


def ssim(a, b, k1=0.01, k2=0.03):
    """Mean SSIM of [3, H, W] (or [H, W]) images."""
    a = np.clip(np.asarray(a, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(b, np.float64), 0.0, 1.0)
    if a.ndim == 2:
        a, b = a[None], b[None]
    g = _gauss_window()
    c1, c2 = (k1 * 1.0) ** 2, (k2 * 1.0) ** 2
    vals = []
    for ch in range(a.shape[0]):
        x, y = a[ch], b[ch]
        mx, my = _filter_valid(x, g), _filter_valid(y, g)
        sxx = _filter_valid(x * x, g) - mx * mx
        syy = _filter_valid(y * y, g) - my * my
        sxy = _filter_valid(x * y, g) - mx * my
        s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(s.mean())
    return float(np.mean(vals))


def tpsnr(o_prev, o, y_prev, y):
    c = lambda t: np.clip(np.asarray(t, np.float64), 0.0, 1.0)   # noqa: E731
    d = (c(o) - c(o_prev)) - (c(y) - c(y_prev))
    mse = np.mean(d ** 2)
    if mse == 0.0:
        return float("inf")
    return float(-10.0 * np.log10(mse))
