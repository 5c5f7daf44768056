"""The seeded input generators: shapes, ranges, determinism.  No GPU."""
import numpy as np

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
