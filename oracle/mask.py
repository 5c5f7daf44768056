"""Oracle: foveated sample mask and its compaction (integer, bit-exact).

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.

Follows the paper's "Sample Maps" subsection:

* Eq. 1 / Eq. 2: the sampling threshold tau(u, v) = (1 - P_b) P_f(u, v) + P_b,
  with P_f an exponential falloff around the focal point.  Reading used here
  (the printed Eq. 1 is garbled: it has no (u, v) dependence): with d the
  distance of the pixel centre from the focal point divided by the half
  diagonal R = sqrt(W^2 + H^2) / 2, P_f(d) = 1 for d <= r0 (the fovea) and
  exp(-0.5 ((d - r0) / s)^2) beyond it.
* M(u, v) = 1 iff N(u, v) < tau(u, v) (strict), N a per-pixel noise value.
  The paper draws N from a looping series of pre-computed noise tiles
  ("Noise Patterns": tiles of 16^2 to 256^2 pixels, 64 of them, repeated over
  the frame and looped over time).  Two sources of N:
  - by default the top 24 bits of a stateless 32-bit integer hash of
    (seed, frame, x, y): the PCG-derived hash evaluated by Jarzynski and
    Olano, "Hash Functions for GPU Rendering" (JCGT 2020), nested over the
    four inputs;
  - given a series of K tiles of T x T 24-bit values (an input, like the
    paper's pre-computed tiles), N(x, y) = tile[frame mod K][y mod T][x mod T].
* tau is quantised so that CPU and GPU take the decision in integers: the
  squared half-pixel distance q = (2x + 1 - F_x)^2 + (2y + 1 - F_y)^2 (F the
  focal point in half pixels, rounded) selects bin q >> shift of a 16384-entry
  table; entry b holds floor(tau(d_b) 2^24) with d_b the distance of the bin's
  centre, or 2^24 where tau = 1.
* Eq. 3: C_max = mean of tau over the frame (the expected sampled fraction).
* Stream compaction ("Stream Compaction" subsection): the list of pixel ids
  y * W + x with M = 1.  The oracle returns it in row-major order.
"""
from __future__ import annotations

import math

import numpy as np

NBINS = 16384
ONE24 = 1 << 24

_U32 = np.uint32


def pcg_hash(v: np.ndarray) -> np.ndarray:
    """PCG-style 32-bit integer hash (Jarzynski and Olano 2020, after O'Neill's
    PCG RXS-M-XS output function).  Wrapping uint32 arithmetic."""
    v = np.asarray(v, dtype=_U32)
    state = v * _U32(747796405) + _U32(2891336453)
    word = ((state >> ((state >> _U32(28)) + _U32(4))) ^ state) * _U32(277803737)
    return (word >> _U32(22)) ^ word


def pixel_hash(seed: int, frame: int, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """h = H(x + H(y + H(frame + H(seed)))) with wrapping uint32 adds."""
    with np.errstate(over="ignore"):
        k = pcg_hash(np.array([seed & 0xFFFFFFFF], dtype=_U32))
        k = pcg_hash(np.array([frame & 0xFFFFFFFF], dtype=_U32) + k)
        hy = pcg_hash(np.asarray(ys, dtype=_U32) + k)
        return pcg_hash(np.asarray(xs, dtype=_U32) + hy)


def bin_shift(width: int, height: int) -> int:
    qmax = (2 * width) ** 2 + (2 * height) ** 2
    s = 0
    while (qmax >> s) >= NBINS:
        s += 1
    return s


def tau_of_distance(d: float, r0: float, s: float, p_base: float) -> float:
    """Eq. 2 with the Eq. 1 reading above; d in units of the half diagonal."""
    if d <= r0:
        pf = 1.0
    elif s <= 0.0:
        pf = 0.0
    else:
        z = (d - r0) / s
        pf = math.exp(-0.5 * z * z)
    return (1.0 - p_base) * pf + p_base


def tau_table(width: int, height: int, fovea_radius: float, falloff_sigma: float, p_base: float):
    """(tau_b as float64 [NBINS], T_b as uint32 [NBINS], shift).

    The profile parameters are single-precision values (as they are passed
    to the renderer); they are rounded to float32 first and the table is
    then evaluated in float64."""
    fovea_radius = float(np.float32(fovea_radius))
    falloff_sigma = float(np.float32(falloff_sigma))
    p_base = float(np.float32(p_base))
    shift = bin_shift(width, height)
    big_r = 0.5 * math.sqrt(float(width) * width + float(height) * height)
    taus = np.empty(NBINS, dtype=np.float64)
    thr = np.empty(NBINS, dtype=np.uint32)
    for b in range(NBINS):
        qc = (b + 0.5) * float(1 << shift)
        d = math.sqrt(qc) * 0.5 / big_r
        t = tau_of_distance(d, fovea_radius, falloff_sigma, p_base)
        taus[b] = t
        if t >= 1.0:
            thr[b] = ONE24
        elif t <= 0.0:
            thr[b] = 0
        else:
            thr[b] = int(math.floor(t * ONE24))
    return taus, thr, shift


def focal_half_pixels(fx: float, fy: float, width: int, height: int):
    """Focal point in half-pixel units, rounded, clamped to the frame."""
    f2x = int(math.floor(2.0 * float(np.float32(fx)) + 0.5))
    f2y = int(math.floor(2.0 * float(np.float32(fy)) + 0.5))
    return min(max(f2x, 0), 2 * width), min(max(f2y, 0), 2 * height)


def make_mask(width: int, height: int, focal_px, fovea_radius=0.10, falloff_sigma=0.10,
              p_base=0.05, seed=0, frame=0, noise=None):
    """Return (mask uint8 [H, W], ids int32 row-major, c_max float).
    noise: optional uint32 [K, T, T] tile series (values < 2^24) replacing the hash."""
    taus, thr, shift = tau_table(width, height, fovea_radius, falloff_sigma, p_base)
    f2x, f2y = focal_half_pixels(focal_px[0], focal_px[1], width, height)
    ys, xs = np.meshgrid(np.arange(height, dtype=np.int64), np.arange(width, dtype=np.int64),
                         indexing="ij")
    q = (2 * xs + 1 - f2x) ** 2 + (2 * ys + 1 - f2y) ** 2
    b = (q >> shift).astype(np.int64)
    if noise is None:
        h = pixel_hash(seed, frame, xs.astype(np.uint32), ys.astype(np.uint32))
        n24 = (h >> _U32(8)).astype(np.int64)
    else:
        noise = np.asarray(noise, dtype=np.uint32)
        k, t = noise.shape[0], noise.shape[1]
        n24 = noise[int(frame) % k][ys % t, xs % t].astype(np.int64)
    m = (n24 < thr[b].astype(np.int64)).astype(np.uint8)
    ids = np.flatnonzero(m.reshape(-1)).astype(np.int32)
    c_max = float(taus[b].mean())
    return m, ids, c_max
