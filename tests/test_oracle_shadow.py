"""Pins for the oracle's shadowed shading mode (shading 2: one shadow ray per
sample towards a directional light at a quarter of the main sample rate) --
closed forms for homogeneous media, geometric invariants, an occluder, and a
numpy/scipy brute force on tiny grids.  No GPU."""
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from oracle import march as om
from paper_2209_09965_gb300.workloads import Camera, MarchParams

CUTOFF = 2.0 ** -14


def axis_camera(vox_origin, dims, direction=(1.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """1x1 camera whose single ray starts at a voxel-space point and runs along ``direction``."""
    nmax = max(dims)
    eye = tuple((vox_origin[a] - 0.5 * dims[a]) / nmax for a in range(3))
    tgt = tuple(eye[a] + direction[a] for a in range(3))
    return Camera(eye=eye, target=tgt, up=up, fov_y_deg=45.0, width=1, height=1)


def const_tf(rgb, alpha, n=256):
    tf = np.zeros((n, 4), np.float32)
    tf[:, :3] = rgb
    tf[:, 3] = alpha
    return tf


def exit_distance_bisection(p, L, dims):
    """Distance along L at which p leaves the box [0, n], by bisection on "inside"."""
    def inside(s):
        q = p + s * L
        return bool(np.all(q >= 0.0) and np.all(q <= dims))
    lo, hi = 0.0, 4.0 * float(np.max(dims))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if inside(mid) else (lo, mid)
    return lo


def homogeneous_T(alpha, s_exit, dt, rate):
    """Closed form of the shadow ray in a medium of constant TF opacity: the
    exponents sum to rate (x - 1) for x = s_exit / ds > 1 (full steps j = 1..J-1
    plus the partial last one), i.e. (1 - alpha)^((s_exit - ds) / dt), unless
    the cutoff stops it at the first full step that falls below 2^-14."""
    ds = rate * dt
    x = s_exit / ds
    if x <= 1.0:
        return 1.0
    nfull = math.ceil(x) - 2          # samples with a full exponent: j = 1 .. ceil(x) - 2
    for j in range(1, nfull + 1):
        t = (1.0 - alpha) ** (rate * j)
        if t < CUTOFF:
            return t
    return (1.0 - alpha) ** (rate * (x - 1.0))


@pytest.mark.parametrize("rate,dt", [(4, 0.5), (1, 0.5), (2, 0.25), (8, 0.5)])
def test_homogeneous_shadow_closed_form(rate, dt):
    rng = np.random.default_rng(rate * 10 + int(dt * 4))
    dims = np.array([20.0, 14.0, 9.0])
    vol = np.full((9, 14, 20), 0.5, np.float32)
    alpha = float(np.float32(0.03))
    tf = const_tf((1, 1, 1), alpha)
    pts = rng.uniform(0.0, 1.0, (64, 3)) * dims
    for _ in range(6):
        L = rng.normal(size=3)
        L /= np.linalg.norm(L)
        T = om.shadow(vol, tf, pts, L, dt, rate)
        ref = [homogeneous_T(alpha, exit_distance_bisection(p, L, dims), dt, rate) for p in pts]
        assert np.max(np.abs(T - np.array(ref))) < 1e-12


def test_shadow_cutoff_stops_at_first_full_step_below():
    dims = np.array([40.0, 8.0, 8.0])
    vol = np.full((8, 8, 40), 0.5, np.float32)
    alpha = float(np.float32(0.5))
    tf = const_tf((1, 1, 1), alpha)
    p = np.array([[1.3, 4.0, 4.0]])
    T = om.shadow(vol, tf, p, (1.0, 0.0, 0.0), 0.5, 4)[0]
    # (1 - a)^(4 j) < 2^-14 first at j = 4 (2^-16); the full march would go on to 2^-72
    assert T == 2.0 ** -16
    assert homogeneous_T(alpha, 40.0 - 1.3, 0.5, 4) == T


def test_shadow_direction_sign_and_axis_lights():
    # off-centre point: the light along +x and -x crosses different lengths of medium
    dims = np.array([32.0, 12.0, 12.0])
    vol = np.full((12, 12, 32), 0.5, np.float32)
    alpha = float(np.float32(0.02))
    tf = const_tf((1, 1, 1), alpha)
    p = np.array([[7.3, 6.1, 5.2]])
    tp = om.shadow(vol, tf, p, (1.0, 0.0, 0.0), 0.5, 4)[0]
    tm = om.shadow(vol, tf, p, (-1.0, 0.0, 0.0), 0.5, 4)[0]
    assert abs(tp - (1 - alpha) ** ((32.0 - 7.3 - 2.0) / 0.5)) < 1e-13
    assert abs(tm - (1 - alpha) ** ((7.3 - 2.0) / 0.5)) < 1e-13
    # the light direction is normalised
    assert om.shadow(vol, tf, p, (-5.0, 0.0, 0.0), 0.5, 4)[0] == tm
    # within one shadow step of the face: no shadow sample at all
    assert om.shadow(vol, tf, np.array([[31.0, 6.0, 6.0]]), (1.0, 0.0, 0.0), 0.5, 4)[0] == 1.0


def test_occluder_casts_shadow_only_towards_the_light():
    # empty volume (TF alpha(0) = 0 exactly) with an opaque slab at x in [20, 26)
    n = 32
    vol = np.zeros((n, n, n), np.float32)
    vol[:, :, 20:26] = 1.0
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 1.0
    tf[1:, 3] = 0.6
    p = np.array([[8.0, 16.0, 16.0]])
    assert om.shadow(vol, tf, p, (1.0, 0.0, 0.0), 0.5, 4)[0] < CUTOFF      # slab between p and the light
    assert om.shadow(vol, tf, p, (-1.0, 0.0, 0.0), 0.5, 4)[0] == 1.0       # nothing towards -x
    assert om.shadow(vol, tf, p, (0.0, 1.0, 0.0), 0.5, 4)[0] == 1.0        # parallel to the slab
    # a grazing light that passes above the slab's top (the slab spans all y, so use z extent)
    vol2 = np.zeros((n, n, n), np.float32)
    vol2[:8, :, 20:26] = 1.0                                                 # slab only for z < 8
    assert om.shadow(vol2, tf, np.array([[8.0, 16.0, 20.0]]), (1.0, 0.0, 0.0), 0.5, 4)[0] == 1.0
    assert om.shadow(vol2, tf, np.array([[8.0, 16.0, 4.0]]), (1.0, 0.0, 0.0), 0.5, 4)[0] < CUTOFF


def test_shadowed_pixel_constant_medium_closed_form():
    # ray along +x through a constant medium (zero gradient: c' = c (0.2 + 0.7 T))
    dims = (24, 16, 16)
    vol = np.full((16, 16, 24), 0.5, np.float32)
    c = np.array([0.8, 0.4, 0.6], np.float32).astype(np.float64)
    a = float(np.float32(0.05))
    tf = const_tf(c, a)
    o = (0.25, 5.3, 7.6)
    cam = axis_camera(o, dims)
    bg = np.array([0.1, 0.2, 0.3])
    # light along +y: every sample sees the same exit distance 16 - 5.3
    mp = MarchParams(0.5, 0.999, tuple(bg), 2, light_dir=(0.0, 1.0, 0.0), shadow_rate=4)
    out, amb, ns = om.march(vol, tf, cam, mp)
    nsamp = 48                                                   # x in [0.25, 24), dt = 0.5
    T = (1 - a) ** ((16 - 5.3 - 2.0) / 0.5)
    A = 1 - (1 - a) ** nsamp
    assert ns == nsamp and (amb[0, 0] & 3) == 0
    assert np.allclose(out[:3, 0, 0], c * (0.2 + 0.7 * T) * A + (1 - A) * bg, atol=1e-13)
    # light along the ray: sample k at x_k = 0.25 + 0.5 k exits after 24 - x_k
    mp = MarchParams(0.5, 0.999, tuple(bg), 2, light_dir=(1.0, 0.0, 0.0), shadow_rate=4)
    out, _, _ = om.march(vol, tf, cam, mp)
    acc = np.zeros(3)
    for k in range(nsamp):
        x = 0.25 + 0.5 * k
        Tk = homogeneous_T(a, 24.0 - x, 0.5, 4)
        acc += (1 - a) ** k * a * c * (0.2 + 0.7 * Tk)
    assert np.allclose(out[:3, 0, 0], acc + (1 - A) * bg, atol=1e-13)


def test_shadowed_phong_constant_gradient_closed_form():
    # field along x only; ray in the x-y plane at angle theta; light at angle phi in the x-z plane
    nx, ny, nz = 64, 16, 16
    xs = np.arange(nx) + 0.5
    vol = np.broadcast_to((0.1 + 0.012 * xs).astype(np.float32), (nz, ny, nx)).copy()
    theta, phi = 2.6, 0.3                     # the ray runs towards -x, the light sits towards +x
    d = np.array([math.cos(theta), math.sin(theta), 0.0])
    L = np.array([math.cos(phi), 0.0, math.sin(phi)])
    o = (60.0, 3.0, 6.0)
    cam = axis_camera(o, (nx, ny, nz), direction=tuple(d))
    c = np.array([0.9, 0.5, 0.2], np.float32).astype(np.float64)
    a = float(np.float32(0.02))
    mp = MarchParams(0.5, 0.99, (0, 0, 0), 2, light_dir=tuple(L), shadow_rate=4)
    out, amb, ns = om.march(vol, const_tf(c, a), cam, mp)
    # n = -x: |n.L| = cos(phi); H = (L - d) / |L - d|: |n.H| = |L_x - d_x| / |L - d|
    ndl = math.cos(phi)
    h = L - d
    ndh = abs(h[0]) / np.linalg.norm(h)
    assert ns == 51                           # leaves through y = 16 at t = 13 / sin(theta) = 25.2
    assert ndh > 0.9                          # a specular term that matters
    dims = np.array([nx, ny, nz], np.float64)
    p0 = np.array(o)
    acc, A = np.zeros(3), 0.0
    for k in range(ns):
        p = p0 + (0.5 * k) * d
        T = homogeneous_T(a, exit_distance_bisection(p, L, dims), 0.5, 4)
        col = np.clip(c * (0.2 + 0.7 * T * ndl) + 0.3 * T * ndh ** 32, 0, 1)
        acc += (1 - A) * a * col
        A += (1 - A) * a
    assert amb[0, 0] == 0
    # the bisection fixes the exit distances to ~1e-13 voxels
    assert np.allclose(out[:3, 0, 0], acc, atol=1e-10)
    assert abs(out[3, 0, 0] - A) < 1e-13
    # (L + d) instead of (L - d) in the half vector would give another specular term
    assert abs(abs(L[0] + d[0]) / np.linalg.norm(L + d) - ndh) > 0.1


def _brute_force_shadowed(vol, tf, cam, mp):
    """Independent per-pixel march with shadows: numpy camera, scipy trilinear,
    np.interp TF, bisection for the shadow ray's exit distance."""
    nz, ny, nx = vol.shape
    dims = np.array([nx, ny, nz], np.float64)
    nmax = dims.max()
    f = np.subtract(cam.target, cam.eye)
    f = f / np.linalg.norm(f)
    r = np.cross(f, cam.up)
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(cam.fov_y_deg) / 2)
    o = np.array(cam.eye) * nmax + dims / 2
    v64 = np.clip(vol.astype(np.float64), 0, 1)
    L = np.array(mp.light_dir, np.float64)
    L = L / np.linalg.norm(L)
    grid = np.arange(tf.shape[0]) / (tf.shape[0] - 1)
    tf64 = tf.astype(np.float64)

    def val(p):
        return map_coordinates(v64, [[p[2] - 0.5], [p[1] - 0.5], [p[0] - 0.5]], order=1, mode="nearest")[0]

    def opacity(v):
        return np.interp(v, grid, tf64[:, 3])

    def light(p):
        ds = mp.shadow_rate * mp.step_vox
        se = exit_distance_bisection(p, L, dims)
        T, s = 1.0, ds
        while s < se and T >= CUTOFF:
            frac = min(1.0, (se - s) / ds)
            T *= (1.0 - opacity(val(p + s * L))) ** (mp.shadow_rate * frac)
            s += ds
        return T

    out = np.zeros((4, cam.height, cam.width))
    for y in range(cam.height):
        for x in range(cam.width):
            sx = (2 * (x + 0.5) / cam.width - 1) * th * cam.width / cam.height
            sy = (1 - 2 * (y + 0.5) / cam.height) * th
            d = f + sx * r + sy * u
            d = d / np.linalg.norm(d)
            with np.errstate(divide="ignore"):
                t0 = (0 - o) / d
                t1 = (dims - o) / d
            tn = max(np.minimum(t0, t1).max(), 0.0)
            tfar = np.maximum(t0, t1).min()
            C, A, k = np.zeros(3), 0.0, 0
            while tn < tfar:
                t = tn + k * mp.step_vox
                if t >= tfar:
                    break
                k += 1
                p = o + t * d
                v = val(p)
                col = np.array([np.interp(v, grid, tf64[:, ch]) for ch in range(4)])
                if col[3] > 0:
                    T = light(p)
                    g = np.array([val(p + e) - val(p - e) for e in np.eye(3)]) * 0.5
                    gn = np.linalg.norm(g)
                    if gn >= 1e-6:
                        hv = (L - d) / np.linalg.norm(L - d)
                        ndl, ndh = abs(g @ L) / gn, abs(g @ hv) / gn
                        col[:3] = np.clip(col[:3] * (0.2 + 0.7 * T * ndl) + 0.3 * T * ndh ** 32, 0, 1)
                    else:
                        col[:3] = np.clip(col[:3] * (0.2 + 0.7 * T), 0, 1)
                C += (1 - A) * col[3] * col[:3]
                A += (1 - A) * col[3]
                if A >= mp.term_alpha:
                    break
            out[:3, y, x] = C + (1 - A) * np.array(mp.bg)
            out[3, y, x] = A
    return out


@pytest.mark.parametrize("n,rate,seed", [(3, 4, 0), (4, 4, 1), (4, 2, 2), (5, 1, 3)])
def test_brute_force_tiny_grids_shadowed(n, rate, seed):
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0, 1, (n, n + 1, n + 2)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rng.uniform(0, 1, 3)
    tf[:, 3] = np.linspace(0.0, 0.5, 256)
    tf[:, 1] = np.linspace(0.9, 0.2, 256)
    v = rng.normal(size=3)
    cam = Camera(eye=tuple(1.6 * v / np.linalg.norm(v)), target=(0.02, -0.03, 0.01), up=(0, 1, 0),
                 fov_y_deg=45.0, width=7, height=6)
    light = tuple(rng.normal(size=3))
    mp = MarchParams(0.5, 0.95, (0.1, 0.2, 0.3), 2, light_dir=light, shadow_rate=rate)
    out, amb, ns = om.march(vol, tf, cam, mp)
    ref = _brute_force_shadowed(vol, tf, cam, mp)
    ok = amb == 0
    assert ok.mean() > 0.8
    # the bisection fixes exit distances to ~1e-13; everything else is FP64 rounding
    assert np.max(np.abs(out[:4][:, ok] - ref[:, ok])) < 1e-9


def test_headlight_mode_unchanged_by_light_fields():
    rng = np.random.default_rng(9)
    vol = rng.uniform(0, 1, (6, 7, 8)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 0.6
    tf[:, 3] = np.linspace(0, 0.3, 256)
    cam = Camera(eye=(0.4, 0.9, 1.5), target=(0, 0, 0), up=(0, 1, 0), fov_y_deg=45.0, width=12, height=9)
    a, _, _ = om.march(vol, tf, cam, MarchParams(0.5, 0.99, (0, 0, 0), 1))
    b, _, _ = om.march(vol, tf, cam, MarchParams(0.5, 0.99, (0, 0, 0), 1, light_dir=(1.0, -2.0, 0.5),
                                                 shadow_rate=2))
    assert np.array_equal(a, b)


# Plausible mistakes planted in a compiled copy of the oracle's source (the
# oracle itself is not touched); each must break at least one pin above.
SHADOW_MUTANTS = [
    ("no partial last step", "if (e > 1.0) e = 1.0;", "e = 1.0;",
     [lambda: test_homogeneous_shadow_closed_form(4, 0.5)]),
    ("a shadow sample at the point itself", "for (int64_t j = 1; (double)j * ds < se; ++j) {",
     "for (int64_t j = 0; (double)j * ds < se; ++j) {", [lambda: test_homogeneous_shadow_closed_form(4, 0.5)]),
    ("exit face flipped", "double s = ((L[a] > 0.0 ? (double)v->n[a] : 0.0) - p[a]) / L[a];",
     "double s = ((L[a] > 0.0 ? 0.0 : (double)v->n[a]) - p[a]) / L[a];",
     [lambda: test_homogeneous_shadow_closed_form(4, 0.5), test_shadow_direction_sign_and_axis_lights]),
    ("L + dir as the half vector", "double h[3] = {L[0] - d[0], L[1] - d[1], L[2] - d[2]};",
     "double h[3] = {L[0] + d[0], L[1] + d[1], L[2] + d[2]};", [test_shadowed_phong_constant_gradient_closed_form]),
    ("unshadowed specular term", "col[ch] = clamp01(col[ch] * (0.2 + 0.7 * T * ndl) + 0.3 * T * spec);",
     "col[ch] = clamp01(col[ch] * (0.2 + 0.7 * T * ndl) + 0.3 * spec);",
     [test_shadowed_phong_constant_gradient_closed_form]),
    ("unshadowed flat-region term", "for (int ch = 0; ch < 3; ++ch) col[ch] = clamp01(col[ch] * (0.2 + 0.7 * T));",
     "for (int ch = 0; ch < 3; ++ch) col[ch] = clamp01(col[ch] * (0.2 + 0.7));",
     [test_shadowed_pixel_constant_medium_closed_form]),
]


@pytest.mark.parametrize("what,old,new,pins", SHADOW_MUTANTS, ids=[m[0] for m in SHADOW_MUTANTS])
def test_planted_mistakes_fail_the_pins(what, old, new, pins, tmp_path, monkeypatch):
    import subprocess
    src = open(om._SRC).read()
    assert src.count(old) == 1, what
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c), "-lm"])
    monkeypatch.setattr(om, "_lib", None)
    monkeypatch.setattr(om, "build", lambda force=False: str(so))
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught: {what}"
