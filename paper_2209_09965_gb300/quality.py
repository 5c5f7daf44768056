"""Image-quality measurements of rendered frames (PSNR, SSIM, temporal PSNR)
on the device, for the benchmark's quality figures -- measurement, not part
of the render path.  Conventions (the paper reports PSNR, SSIM and tPSNR
without fixing them): RGB clamped to [0, 1]; PSNR with MAX = 1 over all
pixels and channels; SSIM after Wang et al. 2004, 11 x 11 Gaussian window
(sigma 1.5, radius 5), K1 = 0.01, K2 = 0.03, over the window positions
inside the image, averaged over the channels; tPSNR the PSNR (MAX = 1) of
the frame-to-frame change of the reconstruction against that of the
reference, (O_t - O_t-1) vs (Y_t - Y_t-1), the clamped frames differenced."""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F


def psnr(a: torch.Tensor, b: torch.Tensor) -> float:
    mse = torch.mean((a.clamp(0, 1) - b.clamp(0, 1)) ** 2).item()
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)


def _window(device, sigma=1.5, radius=5):
    x = torch.arange(-radius, radius + 1, dtype=torch.float64, device=device)
    g = torch.exp(-0.5 * (x / sigma) ** 2)
    return g / g.sum()


def ssim(a: torch.Tensor, b: torch.Tensor, k1=0.01, k2=0.03) -> float:
    """Mean SSIM of two [C, H, W] (or [H, W]) images, computed in float64."""
    x = a.clamp(0, 1).to(torch.float64)
    y = b.clamp(0, 1).to(torch.float64)
    if x.dim() == 2:
        x, y = x[None], y[None]
    c = x.shape[0]
    g = _window(x.device)
    gx = g.view(1, 1, 1, -1).expand(c, 1, 1, g.numel())
    gy = g.view(1, 1, -1, 1).expand(c, 1, g.numel(), 1)

    def filt(t):   # separable Gaussian, valid positions only
        return F.conv2d(F.conv2d(t[None], gx, groups=c), gy, groups=c)[0]

    mx, my = filt(x), filt(y)
    sxx = filt(x * x) - mx * mx
    syy = filt(y * y) - my * my
    sxy = filt(x * y) - mx * my
    c1, c2 = k1 * k1, k2 * k2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean(dim=(1, 2)).mean().item())


def tpsnr(o_prev: torch.Tensor, o: torch.Tensor, y_prev: torch.Tensor, y: torch.Tensor) -> float:
    """Temporal PSNR of one frame pair: the reconstruction's change against the reference's."""
    d = (o.clamp(0, 1) - o_prev.clamp(0, 1)) - (y.clamp(0, 1) - y_prev.clamp(0, 1))
    mse = torch.mean(d.to(torch.float64) ** 2).item()
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)
