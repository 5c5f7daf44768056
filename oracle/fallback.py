"""Oracle: error estimate and denser-mask fallback of a foveated frame.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.

Not in the paper (its frames have no quality guard); the reading used here:
probe pixels are those whose second hash -- the mask's hash with the seed
xor 0x9E3779B9 -- has its top 24 bits below 2^16 (1/256 of the frame) and
that the mask left out.  They are ray-marched like sampled pixels; the PSNR
of the reconstruction at the probes (RGB clamped to [0, 1]) estimates the
frame's PSNR.  While it is below the threshold and fewer than max_levels
re-renders were made, the frame is rendered again with P_b doubled (capped
at 1).
"""
from __future__ import annotations

import math

import numpy as np

from . import march as om
from . import mask as omask
from . import net as onet

SALT = 0x9E3779B9
PROBE_THRESHOLD = 1 << 16


def probe_ids(width, height, seed, frame, mask):
    ys, xs = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    h = omask.pixel_hash((seed ^ SALT) & 0xFFFFFFFF, frame, xs.astype(np.uint32), ys.astype(np.uint32))
    p = ((h >> np.uint32(8)).astype(np.int64) < PROBE_THRESHOLD) & (mask == 0)
    return np.flatnonzero(p.reshape(-1)).astype(np.int32)


def probe_psnr(rgb, probe_rgbam, ids):
    """PSNR of rgb [3,H,W] against the probe samples at ids."""
    if ids.size == 0:
        return 99.0
    r = np.clip(rgb.reshape(3, -1)[:, ids], 0, 1)
    p = np.clip(probe_rgbam.reshape(5, -1)[:3, ids], 0, 1)
    mse = np.mean((r - p) ** 2)
    return 99.0 if mse == 0 else -10.0 * math.log10(mse)


def render_adaptive(vol, tf, cam, fov, mp, params, min_psnr_db, max_levels):
    """(level, PSNR estimate, rgb) of the fallback rule in float64."""
    p_base = float(np.float32(fov.p_base))
    level = 0
    while True:
        m, ids, _ = omask.make_mask(cam.width, cam.height, fov.focal_px, fov.fovea_radius, fov.falloff_sigma,
                                    p_base, fov.seed, fov.frame)
        sp, _, _ = om.march(vol, tf, cam, mp, ids=ids)
        rgb = onet.forward(params, sp)
        pids = probe_ids(cam.width, cam.height, fov.seed, fov.frame, m)
        probe, _, _ = om.march(vol, tf, cam, mp, ids=pids)
        est = probe_psnr(rgb, probe, pids)
        if est >= min_psnr_db or level >= max_levels or p_base >= 1.0:
            return level, est, rgb
        p_base = min(1.0, float(np.float32(2.0 * p_base)))
        level += 1
