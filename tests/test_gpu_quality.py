"""Quality gate of the learned part: on held-out frames (a volume family and
seed the network never saw), the trained network (direct prediction +
kernel prediction, FP16 tensor-core inference) beats (i) push-pull hole
filling of the same sparse samples, (ii) the same architecture trained for
direct prediction only, and (iii) the untrained network; and reaches
>= 35 dB mean PSNR against the dense render."""
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WDIR = os.path.join(ROOT, "paper_2209_09965_gb300", "weights")


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def psnr(a, b):
    mse = torch.mean((a.clamp(0, 1) - b.clamp(0, 1)) ** 2).item()
    return -10 * math.log10(max(mse, 1e-20))


def push_pull(sp):
    """Classic push-pull fill of the sparse RGB (test-side baseline)."""
    rgb, m = sp[0:3][None], sp[4:5][None]
    levels = [(rgb * m, m)]
    while min(levels[-1][1].shape[-2:]) > 1:
        c, w = levels[-1]
        h2, w2 = c.shape[-2] // 2 * 2, c.shape[-1] // 2 * 2
        c2 = F.avg_pool2d(c[..., :h2, :w2], 2) * 4
        wt = F.avg_pool2d(w[..., :h2, :w2], 2) * 4
        levels.append((c2, wt))
    fill = levels[-1][0] / levels[-1][1].clamp_min(1e-8)
    for c, w in reversed(levels[:-1]):
        up = F.interpolate(fill, size=c.shape[-2:], mode="bilinear", align_corners=False)
        own = c / w.clamp_min(1e-8)
        a = w.clamp(0, 1)
        fill = a * own + (1 - a) * up
    return fill[0]


def recon(fvn, weights, sp):
    ctx = fvn.Context()
    ctx.load_weights(weights)
    out = torch.empty(3, sp.shape[1], sp.shape[2], device="cuda")
    ctx.reconstruct(sp, sp.shape[2], sp.shape[1], out)
    torch.cuda.synchronize()
    ctx.close()
    return out


def test_trained_network_beats_baselines(fvn):
    wpath = os.path.join(WDIR, "fvn_16_32_64.npy")
    dpath = os.path.join(WDIR, "fvn_direct_only.npy")
    if not (os.path.exists(wpath) and os.path.exists(dpath)):
        pytest.skip("trained weights not present")
    trained = np.load(wpath).astype(np.float32)
    direct = np.load(dpath).astype(np.float32).copy()
    # direct-only weights: force the blend to the direct prediction (a = 0)
    parts = wl.split_weights(direct)
    parts["head"][0][28] = 0.0
    parts["head"][1][28] = -1e4
    untrained = wl.net_weights(3)
    W, H = 1920, 1080
    vol_np, tf_np, _, _, mp = wl.foveated_1080p_workload(seed=7, frame=0)
    dev = torch.device("cuda")
    vol = torch.from_numpy(vol_np).to(dev)
    tf = torch.from_numpy(tf_np).to(dev)
    ctx = fvn.Context()
    scores = {"trained": [], "direct_only": [], "push_pull": [], "untrained": []}
    for f in (0, 16, 40):
        cam = wl.orbit_camera(7, f, width=W, height=H, radius_factor=(0.85, 1.75))
        fov = wl.Foveation(focal_px=wl.focal_point(7, f, W, H), seed=7, frame=f)
        dense = torch.empty(5, H, W, device=dev)
        sp = torch.empty(5, H, W, device=dev)
        mask = torch.empty(H, W, dtype=torch.uint8, device=dev)
        ids = torch.empty(W * H, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        ctx.march(vol, tf, cam, mp, dense)
        ctx.make_mask(fov, W, H, mask, ids, cnt)
        ctx.march(vol, tf, cam, mp, sp, ids=ids, count=cnt)
        torch.cuda.synchronize()
        ref = dense[0:3]
        scores["trained"].append(psnr(recon(fvn, trained, sp), ref))
        scores["direct_only"].append(psnr(recon(fvn, direct, sp), ref))
        scores["untrained"].append(psnr(recon(fvn, untrained, sp), ref))
        scores["push_pull"].append(psnr(push_pull(sp), ref))
    ctx.close()
    mean = {k: float(np.mean(v)) for k, v in scores.items()}
    print("PSNR dB", mean)
    assert mean["trained"] > mean["push_pull"]
    assert mean["trained"] > mean["direct_only"]
    assert mean["trained"] > mean["untrained"] + 10
    assert mean["trained"] >= 35.0


def test_two_stage_beats_kernels_on_the_sparse_samples(fvn):
    """The paper's reconstruction (kernels applied to D's coarse image, at
    several scales, with its own widths) against the single network whose one
    kernel filters the sparse samples, at an equal training budget on
    held-out frames: the paper's two-stage network wins by more than 1 dB and
    beats the two-stage network with the single network's widths.  (At those
    slim widths the two forms trade places between frame sets, so no order
    is asserted between them.)"""
    files = {k: os.path.join(WDIR, v) for k, v in (
        ("single", "fvn_16_32_64_4k.npy"), ("slim", "fvn_wnet_slim_4k.npy"), ("paper", "fvn_wnet_paper_4k.npy"))}
    if not all(os.path.exists(p) for p in files.values()):
        pytest.skip("ablation weights not present")
    W, H = 1920, 1080
    vol_np, tf_np, _, _, mp = wl.foveated_1080p_workload(seed=7, frame=0)
    dev = torch.device("cuda")
    vol = torch.from_numpy(vol_np).to(dev)
    tf = torch.from_numpy(tf_np).to(dev)
    ctx = {k: fvn.Context() for k in files}
    try:
        ctx["single"].load_weights(np.load(files["single"]).astype(np.float32))
        ctx["slim"].load_wnet_weights(wl.WNET_SLIM, np.load(files["slim"]).astype(np.float32))
        ctx["paper"].load_wnet_weights(wl.WNET_PAPER, np.load(files["paper"]).astype(np.float32))
        scores = {k: [] for k in files}
        dense = torch.empty(5, H, W, device=dev)
        sp = torch.empty(5, H, W, device=dev)
        out = torch.empty(3, H, W, device=dev)
        for f in (0, 16, 40):
            cam = wl.orbit_camera(7, f, width=W, height=H, radius_factor=(0.85, 1.75))
            fov = wl.Foveation(focal_px=wl.focal_point(7, f, W, H), seed=7, frame=f)
            ctx["single"].march(vol, tf, cam, mp, dense)
            ctx["single"].render(vol, tf, cam, fov, mp, out, rgbam_out=sp)
            for k, c in ctx.items():
                if k == "single":
                    c.reconstruct(sp, W, H, out)
                else:
                    c.reconstruct_wnet(sp, W, H, out)
                torch.cuda.synchronize()
                scores[k].append(psnr(out, dense[0:3]))
        mean = {k: float(np.mean(v)) for k, v in scores.items()}
        print("PSNR dB", mean)
        assert mean["paper"] > mean["single"] + 1.0
        assert mean["paper"] > mean["slim"]
    finally:
        for c in ctx.values():
            c.close()
