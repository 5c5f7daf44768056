"""Pins for the oracle's sample mask (Eq. 1-3) -- no GPU."""
import math

import numpy as np
import pytest

from oracle import mask as om


def test_hash_is_uniform_24bit():
    # 2^20 pixels of one frame: the top 24 bits of the hash should be uniform
    ys, xs = np.meshgrid(np.arange(1024), np.arange(1024), indexing="ij")
    h = om.pixel_hash(7, 3, xs.ravel().astype(np.uint32), ys.ravel().astype(np.uint32))
    n = (h >> np.uint32(8)).astype(np.float64) / 2.0**24
    assert abs(n.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n.size)
    counts = np.bincount((n * 64).astype(int), minlength=64)
    exp = n.size / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 6 * math.sqrt(2 * 63)          # ~6 sigma of chi^2(63)
    # horizontally adjacent pixels are uncorrelated
    img = n.reshape(1024, 1024)
    c = np.corrcoef(img[:, 1:].ravel(), img[:, :-1].ravel())[0, 1]
    assert abs(c) < 5 / 1024
    # different frames and seeds give different masks
    h2 = om.pixel_hash(7, 4, xs.ravel().astype(np.uint32), ys.ravel().astype(np.uint32))
    h3 = om.pixel_hash(8, 3, xs.ravel().astype(np.uint32), ys.ravel().astype(np.uint32))
    assert (h2 == h).mean() < 1e-3 and (h3 == h).mean() < 1e-3


def test_pb_one_samples_everything():
    m, ids, cmax = om.make_mask(97, 61, (40.0, 20.0), p_base=1.0, seed=1, frame=2)
    assert m.all() and ids.size == 97 * 61 and cmax == 1.0


def test_flat_density_without_fovea():
    # r0 = 0 and a degenerate falloff leave tau = P_b everywhere: C_max = P_b exactly (Eq. 3)
    w, h, pb = 640, 480, 0.2
    m, ids, cmax = om.make_mask(w, h, (100.0, 100.0), fovea_radius=0.0, falloff_sigma=0.0, p_base=pb)
    assert abs(cmax - float(np.float32(pb))) < 1e-12          # parameters are single precision
    frac = m.mean()
    sigma = math.sqrt(pb * (1 - pb) / m.size)
    assert abs(frac - pb) < 4 * sigma


def test_fovea_is_fully_sampled_and_centred():
    w, h = 1920, 1080
    f = (700.0, 400.0)
    r0 = 0.10
    m, _, _ = om.make_mask(w, h, f, fovea_radius=r0, falloff_sigma=0.1, p_base=0.0, seed=5)
    big_r = 0.5 * math.hypot(w, h)
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    d = np.hypot(xs + 0.5 - f[0], ys + 0.5 - f[1]) / big_r
    # every pixel well inside the fovea is sampled (bins are < 4 px wide here)
    assert m[d < r0 - 4.0 / big_r].all()
    # far outside the falloff nothing is sampled when P_b = 0
    assert not m[d > r0 + 8 * 0.1].any()
    # the sampled set is centred on the focal point
    cy, cx = np.argwhere(m).mean(axis=0)
    assert abs(cx + 0.5 - f[0]) < 3 and abs(cy + 0.5 - f[1]) < 3


def test_tau_table_matches_eq2_closed_form():
    w, h = 1920, 1080
    r0, s, pb = 0.1, 0.1, 0.05
    taus, thr, shift = om.tau_table(w, h, r0, s, pb)
    assert thr.max() == 2**24 and np.all(np.diff(thr.astype(np.int64)) <= 0)      # non-increasing
    big_r = 0.5 * math.hypot(w, h)
    centres = np.sqrt((np.arange(om.NBINS) + 0.5) * 2.0**shift) * 0.5 / big_r
    # at d = r0 + s the falloff is exp(-1/2): interpolate the table there
    t = np.interp(r0 + s, centres, taus)
    assert abs(t - (pb + (1 - pb) * math.exp(-0.5))) < 2e-3
    # far away tau -> P_b
    assert abs(taus[-1] - pb) < 1e-6
    # quantisation: T = floor(tau 2^24)
    inner = taus < 1.0
    assert np.all(thr[inner] <= taus[inner] * 2**24) and np.all(thr[inner] > taus[inner] * 2**24 - 1)


def test_realised_density_follows_cmax():
    # the sampled fraction is binomial around C_max (Eq. 3), both overall and per ring
    w, h = 1920, 1080
    fp = (1000.0, 500.0)
    m, ids, cmax = om.make_mask(w, h, fp, seed=11, frame=9)
    taus, thr, shift = om.tau_table(w, h, 0.1, 0.1, 0.05)
    f2x, f2y = om.focal_half_pixels(*fp, w, h)
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    b = (((2 * xs + 1 - f2x) ** 2 + (2 * ys + 1 - f2y) ** 2) >> shift)
    p = thr[b] / 2.0**24
    sd = math.sqrt((p * (1 - p)).sum())
    assert abs(m.sum() - p.sum()) < 4 * sd
    assert abs(cmax - p.mean()) < 1e-6
    assert np.array_equal(ids, np.flatnonzero(m.ravel()))
    # expected density of this configuration is ~14.6 % of the frame
    assert 0.12 < cmax < 0.17


def test_mask_changes_with_frame():
    a, _, _ = om.make_mask(256, 256, (128.0, 128.0), seed=1, frame=0)
    b, _, _ = om.make_mask(256, 256, (128.0, 128.0), seed=1, frame=1)
    assert (a != b).mean() > 0.05


# ---- the tiled noise source (a looping series of pre-computed tiles) -------

def _flat_profile(p):
    """Profile with tau = p everywhere: no fovea, no falloff (table bins are
    evaluated at their centres, so even the bin of distance 0 has d > r0 = 0)."""
    return dict(fovea_radius=0.0, falloff_sigma=0.0, p_base=p)


def test_constant_tiles_reduce_to_threshold_only():
    w, h, fp = 96, 64, (40.3, 27.8)
    zero = np.zeros((1, 16, 16), np.uint32)
    m, ids, _ = om.make_mask(w, h, fp, noise=zero)
    assert m.all() and ids.size == w * h                        # 0 < T everywhere (P_b > 0)
    top = np.full((1, 16, 16), (1 << 24) - 1, np.uint32)
    m_top, _, _ = om.make_mask(w, h, fp, noise=top)
    fovea, _, _ = om.make_mask(w, h, fp, p_base=0.0, falloff_sigma=0.0, seed=5)   # hash, fovea only
    assert np.array_equal(m_top, fovea) and 0 < m_top.sum() < w * h


def test_tiles_repeat_over_the_frame_and_loop_over_frames():
    rng = np.random.default_rng(3)
    tiles = rng.integers(0, 1 << 24, (5, 32, 32), dtype=np.uint32)
    w, h, p = 100, 70, 0.3
    thr = int(np.floor(float(np.float32(p)) * (1 << 24)))
    for frame in (0, 3, 7):
        m, _, _ = om.make_mask(w, h, (10.25, 60.75), frame=frame, noise=tiles, **_flat_profile(p))
        ys, xs = np.mgrid[0:h, 0:w]
        expect = tiles[frame % 5][ys % 32, xs % 32] < thr
        assert np.array_equal(m.astype(bool), expect)
    a, _, _ = om.make_mask(w, h, (50.0, 35.0), frame=2, noise=tiles)
    b, _, _ = om.make_mask(w, h, (50.0, 35.0), frame=12, noise=tiles)
    assert np.array_equal(a, b)                                  # frame mod K


def test_blue_noise_tiles_give_the_expected_density():
    from paper_2209_09965_gb300 import workloads as wl
    tiles = wl.blue_noise_tiles(32, 6, seed=1)
    for p in (0.05, 0.1, 0.37):
        for frame in range(6):
            m, _, _ = om.make_mask(256, 128, (100.0, 60.0), frame=frame, noise=tiles, **_flat_profile(p))
            # a rank shift of a permutation: the count of values below the
            # threshold in each tile is p n to within one
            assert abs(m.mean() - p) <= 2.0 / (32 * 32)


def test_threshold_comparison_is_strict():
    """M = 1 iff N < T (strict, Eq. 2 as read): noise equal to the threshold
    samples nothing, one below it samples everything."""
    w, h, p = 40, 24, 0.3
    thr = int(np.floor(float(np.float32(p)) * (1 << 24)))
    at = np.full((1, 8, 8), thr, np.uint32)
    below = np.full((1, 8, 8), thr - 1, np.uint32)
    m_at, ids_at, _ = om.make_mask(w, h, (20.0, 12.0), noise=at, **_flat_profile(p))
    m_below, _, _ = om.make_mask(w, h, (20.0, 12.0), noise=below, **_flat_profile(p))
    assert not m_at.any() and ids_at.size == 0
    assert m_below.all()


@pytest.mark.parametrize("w,h", [(1920, 1080), (333, 200)])
def test_fovea_is_symmetric_about_a_centred_focal_point(w, h):
    """Distances are measured from pixel centres: with the focal point at the
    frame's centre, a fovea-only mask (tau 0 or 1, so no noise enters) is
    mirror-symmetric in x and in y."""
    m, _, _ = om.make_mask(w, h, (w / 2.0, h / 2.0), fovea_radius=0.1, falloff_sigma=0.0, p_base=0.0, seed=3)
    assert 0 < m.sum() < w * h
    assert np.array_equal(m, m[:, ::-1]) and np.array_equal(m, m[::-1, :])


# Plausible mistakes planted in a copy of the oracle's source (the oracle
# itself is not touched); each must break at least one of the pins above.
MASK_MUTANTS = [
    ("non-strict comparison", "m = (n24 < thr[b].astype(np.int64))", "m = (n24 <= thr[b].astype(np.int64))",
     ["test_threshold_comparison_is_strict"]),
    ("distances from pixel corners", "q = (2 * xs + 1 - f2x) ** 2 + (2 * ys + 1 - f2y) ** 2",
     "q = (2 * xs - f2x) ** 2 + (2 * ys - f2y) ** 2", ["test_fovea_is_symmetric_about_a_centred_focal_point"]),
    ("Gaussian without the factor 1/2", "pf = math.exp(-0.5 * z * z)", "pf = math.exp(-z * z)",
     ["test_tau_table_matches_eq2_closed_form"]),
    ("P_b added without scaling the falloff", "return (1.0 - p_base) * pf + p_base", "return pf + p_base",
     ["test_tau_table_matches_eq2_closed_form"]),
    ("threshold rounded up", "thr[b] = int(math.floor(t * ONE24))", "thr[b] = int(math.ceil(t * ONE24))",
     ["test_tau_table_matches_eq2_closed_form"]),
]


@pytest.mark.parametrize("what,old,new,pins", MASK_MUTANTS, ids=[m[0] for m in MASK_MUTANTS])
def test_planted_mistakes_fail_the_pins(what, old, new, pins, monkeypatch):
    import types
    src = open(om.__file__).read()
    assert src.count(old) == 1, what
    mutant = types.ModuleType("mask_mutant")
    exec(compile(src.replace(old, new), "mask_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "om", mutant)
    caught = []
    for name in pins:
        fn = globals()[name]
        try:
            if name == "test_fovea_is_symmetric_about_a_centred_focal_point":
                fn(1920, 1080)
            else:
                fn()
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {what}"
