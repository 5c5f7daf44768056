"""FP8 (E4M3) tensor-core reconstruction: calibrated per-tensor activation
scales, per-output-channel weight scales, FP32 accumulation.  Parity is a
stated PSNR against the FP64 oracle (no max-abs bound at 3 mantissa bits)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import march as om
from oracle import mask as omask
from oracle import net as onet
from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FP8_MIN_PSNR_DB = 30.0     # FP8 output vs the FP64 oracle's output on the same input


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def _psnr(a, b):
    mse = np.mean((np.clip(a, 0, 1) - np.clip(b, 0, 1)) ** 2)
    return -10 * math.log10(max(mse, 1e-20))


def test_fp8_needs_calibration_then_tracks_the_oracle(fvn):
    wpath = os.path.join(ROOT, "paper_2209_09965_gb300", "weights", "fvn_16_32_64.npy")
    weights = np.load(wpath).astype(np.float32) if os.path.exists(wpath) else wl.net_weights(3)
    W, H = 320, 240
    vol, tf, _, _, mp = wl.foveated_1080p_workload(seed=4, frame=0, n=96)
    cam = wl.orbit_camera(4, 3, width=W, height=H, radius_factor=(0.85, 1.75))
    _, ids, _ = omask.make_mask(W, H, (150.0, 110.0), seed=4, frame=3)
    sp, _, _ = om.march(vol, tf, cam, mp, ids=ids)
    sp32 = sp.astype(np.float32)
    ref = onet.forward(onet.unpack(weights), sp32.astype(np.float64))
    ctx = fvn.Context()
    ctx.load_weights(weights)
    x = torch.from_numpy(sp32).cuda()
    y16 = torch.empty(3, H, W, device="cuda")
    y8 = torch.empty(3, H, W, device="cuda")
    with pytest.raises(fvn.FvnError, match="calibrate"):
        ctx.reconstruct(x, W, H, y8, precision=fvn.PREC_FP8)
    ctx.calibrate_fp8(x, W, H)
    ctx.reconstruct(x, W, H, y16, precision=fvn.PREC_FP16)
    ctx.reconstruct(x, W, H, y8, precision=fvn.PREC_FP8)
    ctx.device_status()
    o16, o8 = y16.cpu().numpy(), y8.cpu().numpy()
    ctx.close()
    assert np.abs(o16 - ref).max() < 2e-2
    assert np.isfinite(o8).all()
    p8 = _psnr(o8, ref)
    print(f"FP8 vs FP64 oracle: PSNR {p8:.2f} dB, max-abs {np.abs(o8 - ref).max():.4f}; "
          f"FP16 vs oracle PSNR {_psnr(o16, ref):.2f} dB")
    assert p8 >= FP8_MIN_PSNR_DB
