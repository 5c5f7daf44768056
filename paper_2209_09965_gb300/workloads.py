"""Seeded synthetic inputs for the foveated volume renderer.

This module produces the INPUT bytes that both the CUDA path and the CPU
oracle consume: scalar volumes, transfer-function tables, cameras, focal
points and network weights.  It holds none of the method's arithmetic (no
mask, no ray marching, no network layer), only random draws and the
procedural shapes that stand in for the paper's CT / simulation datasets
(Table "datasets" of the paper), which are not available.

Recipes (all seeded, all deterministic on CPU):

* ``blob_volume``: sum of isotropic Gaussian blobs, centres U[sigma, n-sigma]^3,
  sigma ~ U[4, 12] voxels, amplitude ~ U[0.2, 1], clamped to [0, 1].
* ``value_noise_volume``: fractal value noise, ``octaves`` octaves with lattice
  spacing 32, 16, 8, 4 voxels and amplitudes 1, 1/2, 1/4, 1/8, lattice values
  U[0, 1], smoothstep-weighted trilinear interpolation, normalised to [0, 1].
* ``turbulence_volume``: the same octaves but summing |2 n - 1|.
* ``transfer_function``: 256-entry piecewise-linear RGBA table from 4 seeded
  control points (position U[0,1] sorted, rgb U[0,1], alpha U[0, alpha_max])
  plus implicit end points (0, rgb_0, 0) and (1, rgb_3, alpha_3).
* ``orbit_camera``: perspective pinhole on a seeded orbit around the volume.
* ``focal_point``: uniform in the central 50 % of the screen.
* ``stereo_pair``: two cameras whose eyes sit baseline / 2 to either side of
  an orbit eye along the image x axis, looking at the same target.
* ``multiview_views`` / ``multiview_volumes``: 16 views (4 stereo pairs at
  2064x2208, 4 at 1280x720, 4 at 3840x2160) over a 512^3 float16 noise volume
  and a 1024^3 uint8 blob volume, alternating between the two (TF peak
  opacities 0.08 and 0.15).
* ``net_weights``: Kaiming-uniform weights, zero biases, in the flat order
  given by ``NET_LAYERS``.

Voxel layout everywhere is x fastest: ``vol[z, y, x]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

# ---------------------------------------------------------------------------
# volumes
# ---------------------------------------------------------------------------


def _interp_matrix(n: int, spacing: int, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """[n, L] matrix mapping lattice values to voxel-centre values along one
    axis with smoothstep weights (value-noise interpolation)."""
    nlat = n // spacing + 2
    x = (torch.arange(n, dtype=dtype, device=device) + 0.5) / spacing
    j0 = torch.floor(x)
    t = x - j0
    w = t * t * (3.0 - 2.0 * t)
    m = torch.zeros(n, nlat, dtype=dtype, device=device)
    idx = j0.long()
    m[torch.arange(n, device=device), idx] = 1.0 - w
    m[torch.arange(n, device=device), idx + 1] = w
    return m


def _noise_octave(n: int, spacing: int, gen: torch.Generator, device) -> torch.Tensor:
    nlat = n // spacing + 2
    lat = torch.rand(nlat, nlat, nlat, generator=gen, dtype=torch.float64).to(device)
    m = _interp_matrix(n, spacing, device=device)
    # separable smoothstep-trilinear: apply the 1-D matrix along x, y, z
    v = torch.einsum("xa,cba->cbx", m, lat)
    v = torch.einsum("yb,cbx->cyx", m, v)
    v = torch.einsum("zc,cyx->zyx", m, v)
    return v


def value_noise_volume(n: int = 256, seed: int = 2, octaves: int = 4, base_spacing: int = 32,
                       device="cpu", turbulence: bool = False) -> torch.Tensor:
    """Fractal value noise in [0, 1], float64 tensor [n, n, n] on ``device``."""
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    acc = torch.zeros(n, n, n, dtype=torch.float64, device=device)
    amp_sum = 0.0
    for o in range(octaves):
        spacing = max(1, base_spacing >> o)
        amp = 0.5 ** o
        nv = _noise_octave(n, spacing, gen, device)
        if turbulence:
            nv = (2.0 * nv - 1.0).abs()
        acc += amp * nv
        amp_sum += amp
    return (acc / amp_sum).clamp_(0.0, 1.0)


def turbulence_volume(n: int, seed: int, octaves: int = 4, device="cpu") -> torch.Tensor:
    return value_noise_volume(n, seed, octaves, base_spacing=max(4, n // 8), device=device,
                              turbulence=True)


def blob_volume(n: int = 64, seed: int = 1, nblobs: int = 8, sigma_range=(4.0, 12.0),
                amp_range=(0.2, 1.0), device="cpu") -> torch.Tensor:
    """Sum of seeded isotropic Gaussian blobs, float64 [n, n, n] in [0, 1]."""
    rng = np.random.default_rng(seed)
    x = torch.arange(n, dtype=torch.float64, device=device) + 0.5
    acc = torch.zeros(n, n, n, dtype=torch.float64, device=device)
    scale = n / 64.0
    for _ in range(nblobs):
        sigma = rng.uniform(*sigma_range) * scale
        c = rng.uniform(sigma, n - sigma, size=3)
        a = rng.uniform(*amp_range)
        gx = torch.exp(-0.5 * ((x - c[0]) / sigma) ** 2)
        gy = torch.exp(-0.5 * ((x - c[1]) / sigma) ** 2)
        gz = torch.exp(-0.5 * ((x - c[2]) / sigma) ** 2)
        acc += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return acc.clamp_(0.0, 1.0)


def training_volume(n: int, seed: int, device="cpu") -> torch.Tensor:
    """Blobs plus 4-octave turbulence, quantised to uint16 (stored as int32
    carrier in torch since torch has no uint16 arithmetic on every version);
    returns a torch.int16 tensor holding the uint16 bit pattern."""
    b = blob_volume(n, seed, nblobs=8, device=device)
    t = turbulence_volume(n, seed + 7919, device=device)
    v = (0.65 * b + 0.35 * t).clamp_(0.0, 1.0)
    q = torch.round(v * 65535.0).to(torch.int32)
    return (q - 65536 * (q >= 32768).to(torch.int32)).to(torch.int16)


# ---------------------------------------------------------------------------
# transfer function, camera, focal point
# ---------------------------------------------------------------------------


def transfer_function(seed: int, n: int = 256, alpha_max: float = 0.5, npoints: int = 4) -> np.ndarray:
    """[n, 4] float32 RGBA table, piecewise linear through seeded control points."""
    rng = np.random.default_rng(seed)
    xs = np.sort(rng.uniform(0.0, 1.0, npoints))
    rgb = rng.uniform(0.0, 1.0, (npoints, 3))
    al = rng.uniform(0.0, alpha_max, npoints)
    px = np.concatenate([[0.0], xs, [1.0]])
    prgb = np.concatenate([rgb[:1], rgb, rgb[-1:]], axis=0)
    pa = np.concatenate([[0.0], al, al[-1:]])
    g = np.arange(n, dtype=np.float64) / (n - 1)
    out = np.empty((n, 4), dtype=np.float64)
    for c in range(3):
        out[:, c] = np.interp(g, px, prgb[:, c])
    out[:, 3] = np.interp(g, px, pa)
    return out.astype(np.float32)


@dataclass
class Camera:
    eye: tuple
    target: tuple
    up: tuple
    fov_y_deg: float
    width: int
    height: int


def orbit_camera(seed: int, frame: int = 0, nframes: int = 64, width: int = 1920, height: int = 1080,
                 fov_y_deg: float = 45.0, radius_factor=1.8, extent=(1.0, 1.0, 1.0)) -> Camera:
    """Seeded orbit: start azimuth U[0, 2 pi), elevation amplitude U[0.2, 0.6] rad,
    one revolution per ``nframes`` frames, radius = radius_factor x box diagonal.
    A (near, far) radius_factor gives an oscillating zoom (two zoom cycles per
    revolution), like the paper's fly-through of rotation plus oscillating zoom."""
    rng = np.random.default_rng(seed)
    az0 = rng.uniform(0.0, 2.0 * math.pi)
    el_amp = rng.uniform(0.2, 0.6)
    diag = math.sqrt(sum(e * e for e in extent))
    if isinstance(radius_factor, (tuple, list)):
        near, far = radius_factor
        z = 0.5 - 0.5 * math.cos(4.0 * math.pi * frame / nframes)
        r = (near + (far - near) * z) * diag
    else:
        r = radius_factor * diag
    az = az0 + 2.0 * math.pi * frame / nframes
    el = el_amp * math.sin(2.0 * math.pi * frame / nframes + 0.7)
    eye = (r * math.cos(el) * math.cos(az), r * math.sin(el), r * math.cos(el) * math.sin(az))
    return Camera(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=fov_y_deg,
                  width=width, height=height)


def random_camera(rng: np.random.Generator, width: int, height: int, rmin=0.9, rmax=1.8,
                  fov_y_deg: float = 45.0) -> Camera:
    """Random view direction on the sphere, random radius factor, small target jitter."""
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    r = rng.uniform(rmin, rmax) * math.sqrt(3.0)
    tgt = rng.uniform(-0.15, 0.15, 3)
    eye = tgt + r * v
    up = (0.0, 1.0, 0.0) if abs(v[1]) < 0.95 else (1.0, 0.0, 0.0)
    return Camera(eye=tuple(float(e) for e in eye), target=tuple(float(t) for t in tgt), up=up,
                  fov_y_deg=fov_y_deg, width=width, height=height)


def focal_point(seed: int, frame: int, width: int, height: int) -> tuple:
    """Focal point in pixel units, uniform in the central 50 % of the screen."""
    rng = np.random.default_rng([int(seed), int(frame)])
    return (float(width * rng.uniform(0.25, 0.75)), float(height * rng.uniform(0.25, 0.75)))


@dataclass
class Foveation:
    """Focal point in pixels; radius / falloff in fractions of the half diagonal."""
    focal_px: tuple
    fovea_radius: float = 0.10
    falloff_sigma: float = 0.10
    p_base: float = 0.05
    seed: int = 0
    frame: int = 0


# ---------------------------------------------------------------------------
# blue-noise sample-map tiles
# ---------------------------------------------------------------------------

def blue_noise_ranks(tile: int = 64, seed: int = 0, sigma: float = 1.5, initial: float = 0.1) -> np.ndarray:
    """Void-and-cluster ranking of a tile x tile torus (Ulichney, "The
    void-and-cluster method for dither array generation", 1993): a seeded
    initial pattern of ones relaxed by moving the tightest cluster into the
    largest void until stable, then ranked by removing tightest clusters
    (ranks below the initial count) and filling largest voids (ranks above).
    Cluster / void energies are a toroidal Gaussian filter of the pattern.
    Returns int64 [tile, tile], a permutation of 0 .. tile^2 - 1."""
    n = tile * tile
    d = np.minimum(np.arange(tile), tile - np.arange(tile)).astype(np.float64)
    kern = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * sigma * sigma))   # centred at (0, 0)

    def splat(energy, p, sign):
        y, x = divmod(int(p), tile)
        energy += sign * np.roll(np.roll(kern, y, axis=0), x, axis=1)

    rng = np.random.default_rng(seed)
    ones = np.zeros(n, bool)
    ones[rng.choice(n, max(1, int(initial * n)), replace=False)] = True
    energy = np.zeros((tile, tile))
    for p in np.flatnonzero(ones):
        splat(energy, p, 1.0)
    flat = energy.reshape(-1)
    for _ in range(4 * n):                       # relax: tightest cluster -> largest void
        c = int(np.argmax(np.where(ones, flat, -np.inf)))
        ones[c] = False
        splat(energy, c, -1.0)
        v = int(np.argmin(np.where(ones, np.inf, flat)))
        ones[v] = True
        splat(energy, v, 1.0)
        if v == c:
            break
    ranks = np.full(n, -1, np.int64)
    n1 = int(ones.sum())
    pat, e = ones.copy(), energy.copy()
    ef = e.reshape(-1)
    for r in range(n1 - 1, -1, -1):              # ranks below n1: remove tightest clusters
        c = int(np.argmax(np.where(pat, ef, -np.inf)))
        pat[c] = False
        splat(e, c, -1.0)
        ranks[c] = r
    pat, e = ones.copy(), energy.copy()
    ef = e.reshape(-1)
    for r in range(n1, n):                       # ranks from n1: fill largest voids
        v = int(np.argmin(np.where(pat, np.inf, ef)))
        pat[v] = True
        splat(e, v, 1.0)
        ranks[v] = r
    return ranks.reshape(tile, tile)


GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0


def blue_noise_tiles(tile: int = 64, frames: int = 64, seed: int = 0) -> np.ndarray:
    """A looping series of sample-map noise tiles (the paper draws its masks
    from a pre-computed series of 64 spatio-temporal blue-noise tiles, which
    are not available here): frame 0 is the void-and-cluster ranking scaled
    to 24 bits, frame k adds k times the golden-ratio conjugate modulo 1, so
    every frame is a rank shift of a blue-noise tile and every pixel's values
    over the frames form an additive low-discrepancy sequence.  uint32
    [frames, tile, tile], values < 2^24."""
    ranks = blue_noise_ranks(tile, seed)
    n = tile * tile
    base = ((2 * ranks + 1) << 23) // n                        # (rank + 1/2) / n in 24-bit fixed point
    out = np.empty((frames, tile, tile), np.uint32)
    for k in range(frames):
        off = int(math.floor(math.fmod(k * GOLDEN, 1.0) * (1 << 24)))
        out[k] = ((base + off) & ((1 << 24) - 1)).astype(np.uint32)
    return out


# Default light of the shadowed shading mode: from above (+y is the orbit's up), off to one side.
LIGHT_DIR = (0.35, 0.85, 0.40)


@dataclass
class MarchParams:
    """shading: 0 none, 1 Phong headlight, 2 Phong lit by a directional light
    along light_dir (world space, towards the light) with one shadow ray per
    sample at shadow_rate x the main step (the paper's renderer uses 4)."""
    step_vox: float = 0.5
    term_alpha: float = 0.99
    bg: tuple = (0.0, 0.0, 0.0)
    shading: int = 1
    light_dir: tuple = LIGHT_DIR
    shadow_rate: int = 4


# ---------------------------------------------------------------------------
# network weights
# ---------------------------------------------------------------------------

# (name, cin, cout, ksize) in the flat weight order; each layer stores
# W[cout][cin][k][k] followed by b[cout], float32.
NET_LAYERS = (
    ("enc0a", 5, 16, 3), ("enc0b", 16, 16, 3),
    ("enc1a", 16, 32, 3), ("enc1b", 32, 32, 3),
    ("bota", 32, 64, 3), ("botb", 64, 64, 3),
    ("dec1a", 96, 32, 3), ("dec1b", 32, 32, 3),
    ("dec0a", 48, 16, 3), ("dec0b", 16, 16, 3),
    ("head", 16, 29, 1),
)


# The recurrent network: enc0a also takes the previous output's RGB.
NET_LAYERS_RECURRENT = (("enc0a", 8, 16, 3),) + NET_LAYERS[1:]


def recurrent_weights(flat: np.ndarray, history_scale: float = 0.0, seed: int = 0) -> np.ndarray:
    """Recurrent weights from plain ones: enc0a's weights for the three
    history channels are appended (zeros by default, so the recurrent
    network starts as the plain one; seeded uniform in +-history_scale
    otherwise)."""
    parts = split_weights(np.asarray(flat, np.float32))
    w, b = parts["enc0a"]
    rng = np.random.default_rng(seed)
    extra = rng.uniform(-history_scale, history_scale, (w.shape[0], 3) + w.shape[2:]).astype(np.float32)
    parts["enc0a"] = (np.concatenate([w, extra], axis=1), b)
    return np.concatenate([np.concatenate([parts[n][0].ravel(), parts[n][1].ravel()])
                           for n, _, _, _ in NET_LAYERS_RECURRENT]).astype(np.float32)


# The two-stage network (direct prediction D, then kernel prediction K on D's
# output): block widths (encoder per scale, coarsest block, decoder per
# scale), and its layers in the flat weight order of fvn_wnet_weight_count.
WNET_PAPER = ((64, 64, 80), 96, (64, 64, 80))   # the paper's e64-e64-e80-d96-d80-d64-d64
WNET_SLIM = ((16, 32), 64, (16, 32))            # the single network's widths


def wnet_layers(cfg) -> tuple:
    enc, bot, dec = cfg
    n = len(enc)
    d_enc = []
    for s in range(n):
        d_enc += [(f"d_enc{s}a", 5 if s == 0 else enc[s - 1], enc[s], 3), (f"d_enc{s}b", enc[s], enc[s], 3)]
    d_dec = []
    for s in range(n - 1, -1, -1):
        below = bot if s == n - 1 else dec[s + 1]
        d_dec += [(f"d_dec{s}a", below + enc[s], dec[s], 3), (f"d_dec{s}b", dec[s], dec[s], 3)]
    k_enc = []
    for s in range(n):
        k_enc += [(f"k_enc{s}", dec[s] + (enc[s - 1] if s > 0 else 0), enc[s], 1), (f"k_enc{s}_taps", enc[s], 9, 1)]
    k_dec = []
    for s in range(n - 1, -1, -1):
        below = bot if s == n - 1 else dec[s + 1]
        k_dec += [(f"k_dec{s}", below + dec[s], dec[s], 1), (f"k_dec{s}_taps", dec[s], 9, 1),
                  (f"k_dec{s}_blend", dec[s], 1, 1)]
    return tuple(d_enc + [("d_bota", enc[-1], bot, 3), ("d_botb", bot, bot, 3)] + d_dec + [("d_out", dec[0], 3, 1)]
                 + k_enc + [("k_bot", enc[-1] + bot, bot, 1), ("k_bot_taps", bot, 9, 1)] + k_dec)


def wnet_weights(cfg, seed: int = 3) -> np.ndarray:
    """Seeded initial weights of the two-stage network: Kaiming-uniform for
    the convolutions, small weights on the tap and blend heads, tap biases
    that favour the centre tap (every kernel starts close to the identity,
    so the first output is close to D's), zero other biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ci, co, k in wnet_layers(cfg):
        bound = math.sqrt(6.0 / (ci * k * k))
        head = name.endswith("_taps") or name.endswith("_blend")
        parts.append(rng.uniform(-bound, bound, co * ci * k * k) * (0.1 if head else 1.0))
        b = np.zeros(co)
        if name.endswith("_taps"):
            b[4] = 3.0
        parts.append(b)
    return np.concatenate(parts).astype(np.float32)


def net_param_count(layers=NET_LAYERS) -> int:
    return sum(co * ci * k * k + co for _, ci, co, k in layers)


def net_weights(seed: int = 3, layers=NET_LAYERS) -> np.ndarray:
    """Seeded Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co, k in layers:
        bound = math.sqrt(6.0 / (ci * k * k))
        parts.append(rng.uniform(-bound, bound, co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def split_weights(flat: np.ndarray, layers=NET_LAYERS) -> dict:
    """Views of the flat weight vector as {name: (W[co,ci,k,k], b[co])}."""
    out, off = {}, 0
    for name, ci, co, k in layers:
        nw = co * ci * k * k
        w = flat[off:off + nw].reshape(co, ci, k, k)
        off += nw
        b = flat[off:off + co]
        off += co
        out[name] = (w, b)
    assert off == flat.size
    return out


def stereo_pair(cam: Camera, baseline: float = 0.03) -> tuple:
    """(left, right): the eye moved by -/+ baseline / 2 (world units, the
    volume's longest side is 1) along the image x axis, same target."""
    eye = np.array(cam.eye, np.float64)
    fwd = np.array(cam.target, np.float64) - eye
    right = np.cross(fwd, np.array(cam.up, np.float64))
    right /= np.linalg.norm(right)
    out = []
    for sgn in (-0.5, 0.5):
        e = eye + sgn * baseline * right
        out.append(Camera(eye=tuple(float(v) for v in e), target=cam.target, up=cam.up, fov_y_deg=cam.fov_y_deg,
                          width=cam.width, height=cam.height))
    return tuple(out)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------


def dense_small_workload(seed: int = 1, frame: int = 0):
    """64^3 float32 blobs, 128x128 camera, 4-point TF: the small dense case."""
    vol = blob_volume(64, seed).to(torch.float32).numpy()
    tf = transfer_function(seed, alpha_max=0.5)
    cam = orbit_camera(seed, frame, width=128, height=128)
    return vol, tf, cam, MarchParams(shading=0)


def foveated_1080p_workload(seed: int = 2, frame: int = 0, n: int = 256, width: int = 1920,
                            height: int = 1080, vol: np.ndarray | None = None):
    """256^3 float32 fractal value noise, 1920x1080, Phong, step 0.5 voxel."""
    if vol is None:
        vol = value_noise_volume(n, seed).to(torch.float32).numpy()
    tf = transfer_function(seed + 1000, alpha_max=0.08)
    cam = orbit_camera(seed, frame, width=width, height=height, radius_factor=(0.85, 1.75))
    fov = Foveation(focal_px=focal_point(seed, frame, width, height), seed=seed, frame=frame)
    return vol, tf, cam, fov, MarchParams(shading=1)


# 4 stereo pairs at 2064x2208 (8 views), 4 views at 1280x720, 4 at 3840x2160
MULTIVIEW_SIZES = ((2064, 2208),) * 8 + ((1280, 720),) * 4 + ((3840, 2160),) * 4


def multiview_volumes(device="cpu", n_noise: int = 512, n_blobs: int = 1024, seed: int = 50):
    """(float16 fractal value noise n_noise^3, uint8 Gaussian blobs n_blobs^3)."""
    noise = value_noise_volume(n_noise, seed + 1, device=device).to(torch.float16)
    blobs = blob_volume(n_blobs, seed + 2, device=device)
    blobs = torch.round(blobs.mul_(255.0)).to(torch.uint8)
    return noise, blobs


def multiview_transfer_functions(seed: int = 50):
    """Transfer functions of the noise and the blob volume (peak opacities
    inside the range the network is trained on)."""
    return transfer_function(seed + 1000, alpha_max=0.08), transfer_function(seed + 2000, alpha_max=0.15)


def multiview_views(seed: int = 50, frame: int = 0, sizes=MULTIVIEW_SIZES, nframes: int = 64):
    """The views of one batched frame: list of dicts with w, h, volume (0 =
    noise, 1 = blobs), cam and fov.  Views 0-7 are four stereo pairs (pair k
    renders volume k % 2); the other views alternate between the volumes."""
    views = []
    i = 0
    while i < len(sizes):
        w, h = sizes[i]
        k = len(views)
        paired = i + 1 < len(sizes) and sizes[i + 1] == sizes[i] and i < 8
        cam = orbit_camera(seed + k, frame, nframes=nframes, width=w, height=h, radius_factor=(0.85, 1.75))
        cams = stereo_pair(cam) if paired else (cam,)
        vol = (k // 2) % 2 if paired else k % 2
        for c in cams:
            fov = Foveation(focal_px=focal_point(seed + k, frame, w, h), seed=seed + k, frame=frame)
            views.append({"w": w, "h": h, "volume": vol, "cam": c, "fov": fov})
        i += len(cams)
    return views
