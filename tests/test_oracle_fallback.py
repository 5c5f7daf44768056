"""Pins for the oracle's error estimate / fallback rule -- no GPU."""
import math

import numpy as np
import pytest

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


def _tiny_case(p_base):
    from oracle import net as onet
    from paper_2209_09965_gb300 import workloads as wl
    vol = wl.value_noise_volume(12, seed=4, octaves=2, base_spacing=4).numpy().astype(np.float32)
    tf = wl.transfer_function(9, alpha_max=0.3)
    cam = wl.orbit_camera(4, 3, width=20, height=12)
    fov = wl.Foveation(focal_px=(10.0, 6.0), seed=4, frame=3, p_base=p_base)
    params = onet.unpack(wl.net_weights(3))
    return vol, tf, cam, fov, wl.MarchParams(shading=1), params


def test_fallback_doubles_pb_up_to_the_cap():
    """The fallback rule: a threshold never met doubles P_b on every level
    (0.3 -> 0.6 -> 1.0, capped) and stops at the cap after two re-renders
    even with levels to spare; a threshold always met renders once."""
    vol, tf, cam, fov, mp, params = _tiny_case(0.3)
    level, est, rgb = ofb.render_adaptive(vol, tf, cam, fov, mp, params, min_psnr_db=1e9, max_levels=5)
    assert level == 2 and rgb.shape[-2:] == (12, 20)
    level, _, _ = ofb.render_adaptive(vol, tf, cam, fov, mp, params, min_psnr_db=-1e9, max_levels=5)
    assert level == 0
    level, _, _ = ofb.render_adaptive(vol, tf, cam, fov, mp, params, min_psnr_db=1e9, max_levels=1)
    assert level == 1


FALLBACK_MUTANTS = [
    ("probes inside the mask", "< PROBE_THRESHOLD) & (mask == 0)", "< PROBE_THRESHOLD)",
     ["test_probes_are_outside_the_mask_at_1_in_256"]),
    ("probes at 1 in 128", "PROBE_THRESHOLD = 1 << 16", "PROBE_THRESHOLD = 1 << 17",
     ["test_probes_are_outside_the_mask_at_1_in_256"]),
    ("probes from the mask's own hash", "omask.pixel_hash((seed ^ SALT) & 0xFFFFFFFF,", "omask.pixel_hash(seed,",
     ["test_probes_are_outside_the_mask_at_1_in_256"]),
    ("P_b grown by 1.5 instead of doubled", "p_base = min(1.0, float(np.float32(2.0 * p_base)))",
     "p_base = min(1.0, float(np.float32(1.5 * p_base)))", ["test_fallback_doubles_pb_up_to_the_cap"]),
    ("the level limit ignored", "if est >= min_psnr_db or level >= max_levels or p_base >= 1.0:",
     "if est >= min_psnr_db or p_base >= 1.0:", ["test_fallback_doubles_pb_up_to_the_cap"]),
]


@pytest.mark.parametrize("what,old,new,pins", FALLBACK_MUTANTS, ids=[m[0] for m in FALLBACK_MUTANTS])
def test_planted_mistakes_fail_the_pins(what, old, new, pins, monkeypatch):
    """Each mistake, planted in a copy of the fallback oracle's source (the
    oracle itself is not touched), breaks at least one pin above."""
    import types
    src = open(ofb.__file__).read()
    assert src.count(old) == 1, what
    mutant = types.ModuleType("oracle.fallback_mutant")
    mutant.__package__ = "oracle"
    exec(compile(src.replace(old, new), "fallback_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "ofb", mutant)
    caught = []
    for name in pins:
        try:
            globals()[name]()
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {what}"
