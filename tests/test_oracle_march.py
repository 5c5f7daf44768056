"""Pins for the oracle ray marcher against closed forms, a library
interpolator and brute force -- no GPU."""
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from oracle import march as om
from paper_2209_09965_gb300.workloads import Camera, MarchParams


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


def test_trilinear_matches_library_interpolator():
    rng = np.random.default_rng(0)
    vol = rng.uniform(0, 1, (5, 6, 7)).astype(np.float32)       # [z, y, x]
    pts = rng.uniform(-2.0, 9.0, (500, 3))                       # (x, y, z) voxel units, incl. outside
    ours = om.trilinear(vol, pts)
    ref = map_coordinates(vol.astype(np.float64), [pts[:, 2] - 0.5, pts[:, 1] - 0.5, pts[:, 0] - 0.5],
                          order=1, mode="nearest")
    assert np.max(np.abs(ours - ref)) < 1e-12


def test_ray_geometry_closed_form():
    cam = Camera(eye=(0.3, -1.2, 2.5), target=(0.05, 0.1, -0.2), up=(0.0, 1.0, 0.0), fov_y_deg=45.0,
                 width=33, height=21)
    f = np.subtract(cam.target, cam.eye)
    f /= np.linalg.norm(f)
    o, d = om.ray(cam, (16, 16, 16), 16, 10)                     # centre pixel
    assert np.allclose(d, f, atol=1e-14)
    assert np.allclose(o, np.array(cam.eye) * 16 + 8, atol=1e-12)
    o, d = om.ray(cam, (16, 16, 16), 0, 0)                       # corner pixel
    t = math.tan(math.radians(22.5))
    expect = math.atan(t * math.hypot(33 / 21 * (1 - 1 / 33), 1 - 1 / 21))
    assert abs(math.acos(np.clip(d @ f, -1, 1)) - expect) < 1e-12


def test_constant_slab_closed_form():
    dims = (16, 16, 16)
    vol = np.full((16, 16, 16), 0.5, np.float32)
    cam = axis_camera((0.25, 8.3, 7.6), dims)
    c, a = np.array([0.2, 0.6, 0.9], np.float32).astype(np.float64), float(np.float32(0.1))
    bg = (0.3, 0.1, 0.7)
    for shading in (0, 1):                                       # zero gradient -> unshaded
        out, amb, ns = om.march(vol, const_tf(c, a), cam, MarchParams(0.5, 0.99, bg, shading))
        n = 32                                                   # t in [0, 15.75), dt = 0.5
        A = 1 - (1 - a) ** n
        assert ns == n and (amb[0, 0] & 3) == 0          # bit 2 flags the zero gradient
        assert np.allclose(out[:3, 0, 0], c * A + (1 - A) * np.array(bg), atol=1e-13)
        assert abs(out[3, 0, 0] - A) < 1e-13 and out[4, 0, 0] == 1.0


def test_early_termination_count():
    vol = np.full((16, 16, 16), 0.5, np.float32)
    cam = axis_camera((0.25, 8.3, 7.6), (16, 16, 16))
    out, _, ns = om.march(vol, const_tf((1, 1, 1), 0.3), cam, MarchParams(0.5, 0.99, (0, 0, 0), 0))
    a = float(np.float32(0.3))                                   # the TF table is float32
    k = math.ceil(math.log(0.01) / math.log(1 - a))              # first k with 1 - (1-a)^k >= 0.99
    assert ns == k == 13
    assert abs(out[3, 0, 0] - (1 - (1 - a) ** 13)) < 1e-13


def test_linear_ramp_gamma_closed_form():
    # v(x) = b0 + b1 x along the ray, alpha(v) = amax v, constant colour.
    n = 16
    b0, b1, amax = 0.1, 0.05, 0.2
    xs = np.arange(n) + 0.5
    vol = np.broadcast_to((b0 + b1 * xs).astype(np.float32), (n, n, n)).copy()
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = (0.4, 0.5, 0.6)
    tf[:, 3] = amax * np.arange(256) / 255.0
    cam = axis_camera((0.25, 8.3, 7.6), (n, n, n))
    out, amb, ns = om.march(vol, tf, cam, MarchParams(0.5, 0.999, (0, 0, 0), 0))
    # samples x_k = 0.25 + 0.5 k, k = 0..31; k = 0 and k = 31 fall in the clamped edge cells
    c0 = 1 - amax * (b0 + 0.25 * b1)
    c1 = 0.5 * amax * b1
    B = c0 / c1
    log_prod = 30 * math.log(c1) + math.lgamma(B) - math.lgamma(B - 30)   # prod_{k=1}^{30} (c0 - c1 k)
    T = math.exp(log_prod) * (1 - amax * (b0 + 0.5 * b1)) * (1 - amax * (b0 + 15.5 * b1))
    assert ns == 32
    # inputs are rounded to float32 (relative 6e-8), so the match is to ~1e-7
    assert abs(out[3, 0, 0] - (1 - T)) < 2e-7
    assert np.allclose(out[:3, 0, 0], np.array([0.4, 0.5, 0.6]) * (1 - T), atol=2e-7)


def test_phong_constant_gradient_closed_form():
    # field depends on x only, ray at angle theta in the x-y plane: |n.L| = cos(theta) everywhere
    nx, ny, nz = 64, 16, 4
    xs = np.arange(nx) + 0.5
    vol = np.broadcast_to((0.1 + 0.012 * xs).astype(np.float32), (nz, ny, nx)).copy()
    theta = 0.3
    cam = axis_camera((2.0, 8.0, 2.0), (nx, ny, nz), direction=(math.cos(theta), math.sin(theta), 0.0))
    c = np.array([0.9, 0.5, 0.2], np.float32).astype(np.float64)
    out, amb, ns = om.march(vol, const_tf(c, 0.3), cam, MarchParams(0.5, 0.99, (0, 0, 0), 1))
    ndl = math.cos(theta)
    shaded = np.clip(c * (0.2 + 0.7 * ndl) + 0.3 * ndl ** 32, 0, 1)
    a = float(np.float32(0.3))
    A = 1 - (1 - a) ** 13
    assert ns == 13
    assert np.allclose(out[:3, 0, 0], shaded * A, atol=1e-12)
    # gradient perpendicular to the ray: ambient only
    cam2 = axis_camera((2.0, 8.0, 2.0), (nx, ny, nz), direction=(0.0, 1.0, 0.0), up=(1.0, 0.0, 0.0))
    out2, _, ns2 = om.march(vol, const_tf(c, 0.3), cam2, MarchParams(0.5, 0.99, (0, 0, 0), 1))
    assert np.allclose(out2[:3, 0, 0], 0.2 * c * (1 - (1 - a) ** ns2), atol=1e-12)


def test_empty_volume_and_miss_give_background():
    bg = (0.25, 0.5, 0.75)
    vol = np.zeros((8, 8, 8), np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 1.0
    tf[1:, 3] = 0.5                                              # alpha(0) = 0 exactly
    cam = Camera(eye=(0.2, 0.3, 2.0), target=(0, 0, 0), up=(0, 1, 0), fov_y_deg=45.0, width=16, height=12)
    out, _, ns = om.march(vol, tf, cam, MarchParams(0.5, 0.99, bg, 1))
    assert ns > 0
    assert np.all(out[:3] == np.array(bg)[:, None, None]) and np.all(out[3] == 0) and np.all(out[4] == 1)
    # looking away from the box: no sample at all
    cam = Camera(eye=(0.2, 0.3, 2.0), target=(0.2, 0.3, 3.0), up=(0, 1, 0), fov_y_deg=45.0, width=16, height=12)
    out, _, ns = om.march(np.ones((8, 8, 8), np.float32), tf, cam, MarchParams(0.5, 0.99, bg, 1))
    assert ns == 0 and np.all(out[:3] == np.array(bg)[:, None, None]) and np.all(out[3] == 0)


def test_opaque_tf_gives_first_sample_colour():
    rng = np.random.default_rng(3)
    vol = rng.uniform(0, 1, (8, 8, 8)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    g = np.arange(256) / 255.0
    tf[:, 0], tf[:, 1], tf[:, 2], tf[:, 3] = g, 1 - g, 0.5, 1.0
    o = (0.6, 3.3, 4.1)
    cam = axis_camera(o, (8, 8, 8))
    out, _, ns = om.march(vol, tf, cam, MarchParams(0.5, 0.99, (0, 0, 0), 0))
    v = map_coordinates(vol.astype(np.float64), [[o[2] - 0.5], [o[1] - 0.5], [o[0] - 0.5]], order=1,
                        mode="nearest")[0]
    assert ns == 1
    assert np.allclose(out[:3, 0, 0], [v, 1 - v, 0.5], atol=1e-7)   # TF table is float32
    assert out[3, 0, 0] == 1.0


def _brute_force(vol, tf, cam, mp):
    """Independent per-pixel march: numpy camera, scipy trilinear, np.interp TF."""
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

    def val(p):
        return map_coordinates(v64, [[p[2] - 0.5], [p[1] - 0.5], [p[0] - 0.5]], order=1, mode="nearest")[0]

    grid = np.arange(tf.shape[0]) / (tf.shape[0] - 1)
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
            C, A = np.zeros(3), 0.0
            t = tn
            k = 0
            while tn < tfar:
                t = tn + k * mp.step_vox
                if t >= tfar:
                    break
                k += 1
                p = o + t * d
                v = val(p)
                col = np.array([np.interp(v, grid, tf[:, ch].astype(np.float64)) for ch in range(4)])
                if col[3] > 0 and mp.shading:
                    g = np.array([val(p + e) - val(p - e) for e in np.eye(3)]) * 0.5
                    gn = np.linalg.norm(g)
                    if gn >= 1e-6:
                        ndl = abs(g @ d) / gn
                        col[:3] = np.clip(col[:3] * (0.2 + 0.7 * ndl) + 0.3 * ndl ** 32, 0, 1)
                C += (1 - A) * col[3] * col[:3]
                A += (1 - A) * col[3]
                if A >= mp.term_alpha:
                    break
            out[:3, y, x] = C + (1 - A) * np.array(mp.bg)
            out[3, y, x] = A
    return out


@pytest.mark.parametrize("n,shading,seed", [(2, 0, 0), (3, 1, 1), (4, 1, 2), (4, 0, 3)])
def test_brute_force_tiny_grids(n, shading, seed):
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0, 1, (n, n + 1, n)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rng.uniform(0, 1, 3)
    tf[:, 3] = np.linspace(0.0, 0.6, 256)
    tf[:, 0] = np.linspace(0.1, 0.9, 256)
    v = rng.normal(size=3)
    cam = Camera(eye=tuple(1.6 * v / np.linalg.norm(v)), target=(0.02, -0.03, 0.01), up=(0, 1, 0),
                 fov_y_deg=45.0, width=9, height=7)
    mp = MarchParams(0.5, 0.95, (0.1, 0.2, 0.3), shading)
    out, amb, ns = om.march(vol, tf, cam, mp)
    ref = _brute_force(vol, tf, cam, mp)
    ok = amb == 0
    assert ok.mean() > 0.8
    assert np.max(np.abs(out[:4][:, ok] - ref[:, ok])) < 1e-9


def test_sparse_equals_dense_at_ids_and_zero_elsewhere():
    rng = np.random.default_rng(5)
    vol = rng.uniform(0, 1, (10, 12, 14)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = 0.7
    tf[:, 3] = np.linspace(0, 0.2, 256)
    cam = Camera(eye=(0.4, 0.9, 1.5), target=(0, 0, 0), up=(0, 1, 0), fov_y_deg=45.0, width=24, height=16)
    mp = MarchParams(0.5, 0.99, (0.2, 0.2, 0.2), 1)
    dense, _, nd = om.march(vol, tf, cam, mp)
    ids = np.sort(rng.choice(24 * 16, 50, replace=False)).astype(np.int32)
    sparse, _, ns = om.march(vol, tf, cam, mp, ids=ids)
    d = dense.reshape(5, -1)
    s = sparse.reshape(5, -1)
    assert np.array_equal(s[:, ids], d[:, ids])
    rest = np.setdiff1d(np.arange(24 * 16), ids)
    assert np.all(s[:, rest] == 0)
    assert 0 < ns < nd


def test_integer_dtypes_normalise():
    rng = np.random.default_rng(6)
    q8 = rng.integers(0, 256, (6, 6, 6)).astype(np.uint8)
    q16 = rng.integers(0, 65536, (6, 6, 6)).astype(np.uint16)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rng.uniform(0, 1, 3)
    tf[:, 3] = np.linspace(0, 0.3, 256)
    cam = Camera(eye=(0.3, 0.5, 1.4), target=(0, 0, 0), up=(0, 1, 0), fov_y_deg=45.0, width=10, height=10)
    mp = MarchParams(0.5, 0.99, (0, 0, 0), 1)
    a, amb, _ = om.march(q8, tf, cam, mp)
    b, _, _ = om.march((q8 / 255.0).astype(np.float32), tf, cam, mp)
    ok = amb == 0
    assert np.max(np.abs(a - b)[:, ok]) < 1e-6
    a, amb, _ = om.march(q16, tf, cam, mp)
    b, _, _ = om.march((q16 / 65535.0).astype(np.float32), tf, cam, mp)
    ok = amb == 0
    assert np.max(np.abs(a - b)[:, ok]) < 1e-6
    h = rng.uniform(0, 1, (6, 6, 6)).astype(np.float16)
    a, amb, _ = om.march(h, tf, cam, mp)
    b, _, _ = om.march(h.astype(np.float32), tf, cam, mp)
    assert np.array_equal(a, b)


# Plausible mistakes planted in a copy of the oracle's source (the oracle
# itself is not touched): each mutant is built with the oracle's own compiler
# flags and must break at least one of the pins above.
MUTANTS = [
    ("compositing without the accumulated transmittance",
     "double w = (1.0 - A) * alpha;", "double w = alpha;",
     ["test_constant_slab_closed_form"]),
    ("background added unattenuated",
     "rgba[0] = C[0] + (1.0 - A) * bg[0];", "rgba[0] = C[0] + bg[0];",
     ["test_constant_slab_closed_form", "test_empty_volume_and_miss_give_background"]),
    ("specular exponent 16 instead of 32",
     "for (int s = 0; s < 5; ++s) spec = spec * spec; /* ndl^32 */",
     "for (int s = 0; s < 4; ++s) spec = spec * spec; /* ndl^32 */",
     ["test_phong_constant_gradient_closed_form"]),
    ("transfer-function index scaled by n instead of n - 1",
     "double x = val * (double)(ntf - 1);", "double x = val * (double)ntf;",
     ["test_linear_ramp_gamma_closed_form"]),
    ("trilinear fractions of x and y swapped",
     "double tx = ux - fx, ty = uy - fy, tz = uz - fz;", "double tx = uy - fy, ty = ux - fx, tz = uz - fz;",
     ["test_trilinear_matches_library_interpolator"]),
    ("early termination past the threshold",
     "if (A >= term) { ++k; break; }", "if (A >= term + 0.005) { ++k; break; }",
     ["test_early_termination_count"]),
]


@pytest.mark.parametrize("what,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
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
    caught = []
    for name in pins:
        try:
            globals()[name]()
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {what}"
