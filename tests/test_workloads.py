"""The seeded input generators: shapes, ranges, determinism.  No GPU."""
import numpy as np
import torch

from paper_2209_09965_gb300 import workloads as wl


def test_volumes_deterministic_and_in_range():
    a = wl.value_noise_volume(32, seed=4).numpy()
    b = wl.value_noise_volume(32, seed=4).numpy()
    c = wl.value_noise_volume(32, seed=5).numpy()
    assert a.shape == (32, 32, 32) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0 and a.max() <= 1 and 0.3 < a.mean() < 0.7
    bl = wl.blob_volume(64, seed=1).numpy()
    assert bl.min() >= 0 and bl.max() <= 1 and bl.max() > 0.15
    tv = wl.training_volume(32, seed=3).numpy().view(np.uint16)
    assert tv.dtype == np.uint16 and tv.max() > 20000


def test_transfer_function_shape_and_endpoints():
    tf = wl.transfer_function(7, alpha_max=0.3)
    assert tf.shape == (256, 4) and tf.dtype == np.float32
    assert tf[0, 3] == 0.0 and tf[:, 3].max() <= 0.3
    assert np.all(tf >= 0) and np.all(tf <= 1)


def test_weights_layout():
    w = wl.net_weights(3)
    assert w.size == wl.net_param_count()
    parts = wl.split_weights(w)
    assert parts["enc0a"][0].shape == (16, 5, 3, 3) and parts["head"][0].shape == (29, 16, 1, 1)
    assert np.all(parts["bota"][1] == 0)


def test_cameras_and_focal_points():
    cam = wl.orbit_camera(2, 5)
    r = np.linalg.norm(cam.eye)
    assert abs(r - 1.8 * np.sqrt(3)) < 1e-9 and cam.width == 1920
    fx, fy = wl.focal_point(2, 5, 1920, 1080)
    assert 480 <= fx <= 1440 and 270 <= fy <= 810


def test_stereo_pair_geometry():
    cam = wl.orbit_camera(4, 3, width=320, height=200)
    left, right = wl.stereo_pair(cam, baseline=0.05)
    el, er, e = (np.array(c.eye) for c in (left, right, cam))
    assert abs(np.linalg.norm(er - el) - 0.05) < 1e-12
    assert np.allclose((el + er) / 2, e, atol=1e-12)            # centred on the orbit eye
    fwd = np.array(cam.target) - e
    assert abs(np.dot(er - el, fwd)) < 1e-12                     # baseline across the view direction
    assert abs(np.dot(er - el, np.array(cam.up))) < 1e-12
    assert left.target == cam.target and right.width == 320


def test_multiview_views_layout():
    views = wl.multiview_views(seed=50)
    sizes = [(v["w"], v["h"]) for v in views]
    assert sizes == list(wl.MULTIVIEW_SIZES) and len(views) == 16
    for k in range(4):                                           # four stereo pairs
        a, b = views[2 * k], views[2 * k + 1]
        assert a["volume"] == b["volume"] == k % 2
        assert a["fov"].focal_px == b["fov"].focal_px and a["fov"].seed == b["fov"].seed
        assert abs(np.linalg.norm(np.array(a["cam"].eye) - np.array(b["cam"].eye)) - 0.03) < 1e-12
    assert {v["volume"] for v in views[8:]} == {0, 1}
    assert views == wl.multiview_views(seed=50)                  # seeded


def test_multiview_volumes_small():
    noise, blobs = wl.multiview_volumes(n_noise=16, n_blobs=32, seed=50)
    assert noise.dtype == torch.float16 and noise.shape == (16, 16, 16)
    assert blobs.dtype == torch.uint8 and blobs.shape == (32, 32, 32) and int(blobs.max()) > 30


def test_blue_noise_tiles_are_blue_permutations():
    t = 32
    ranks = wl.blue_noise_ranks(t, seed=4)
    assert np.array_equal(np.sort(ranks.reshape(-1)), np.arange(t * t))
    tiles = wl.blue_noise_tiles(t, 8, seed=4)
    assert tiles.dtype == np.uint32 and tiles.shape == (8, t, t) and int(tiles.max()) < (1 << 24)
    # frame k is frame 0 shifted by k times the golden-ratio conjugate (mod 2^24)
    off = (tiles[3].astype(np.int64) - tiles[0].astype(np.int64)) % (1 << 24)
    assert np.all(off == off.flat[0])
    assert abs(off.flat[0] / (1 << 24) - (3 * wl.GOLDEN) % 1.0) < 1e-6

    def mean_nn(mask):
        ys, xs = np.nonzero(mask)
        p = np.stack([xs, ys], 1).astype(float)
        d = np.abs(p[:, None] - p[None])
        d = np.minimum(d, t - d)
        dd = np.sqrt((d ** 2).sum(-1))
        np.fill_diagonal(dd, np.inf)
        return dd.min(1).mean()

    # blue: at 10 % density the sampled pixels keep ~1.5x the nearest-neighbour
    # distance of white noise, whose expectation is 0.5 / sqrt(0.1) = 1.58 px
    for k in (0, 3, 7):
        m = tiles[k] < int(0.1 * (1 << 24))
        assert mean_nn(m) > 2.1
    white = np.random.default_rng(0).random((t, t)) < 0.1
    assert mean_nn(white) < 1.9
