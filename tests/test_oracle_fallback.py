"""Pins for the oracle's error estimate / fallback rule -- no GPU."""
import math

import numpy as np

from oracle import fallback as ofb
from oracle import mask as omask


def test_probes_are_outside_the_mask_at_1_in_256():
    w, h = 1024, 768
    m, _, _ = omask.make_mask(w, h, (500.0, 400.0), seed=3, frame=4)
    ids = ofb.probe_ids(w, h, 3, 4, m)
    assert np.all(m.reshape(-1)[ids] == 0)
    n_out = int((m == 0).sum())
    p = 1 / 256
    assert abs(ids.size - n_out * p) < 5 * math.sqrt(n_out * p * (1 - p))
    # independent of the mask's own hash: the probe density is the same in and out of the fovea
    ids2 = ofb.probe_ids(w, h, 3, 4, np.zeros_like(m))
    assert abs(ids2.size - w * h * p) < 5 * math.sqrt(w * h * p)


def test_probe_psnr_closed_form():
    rgb = np.full((3, 8, 8), 0.5)
    probe = np.zeros((5, 8, 8))
    probe[:3] = 0.5 + 0.1
    ids = np.array([0, 5, 17, 63], np.int32)
    assert abs(ofb.probe_psnr(rgb, probe, ids) - 20.0) < 1e-9
    assert ofb.probe_psnr(rgb, probe, np.zeros(0, np.int32)) == 99.0
