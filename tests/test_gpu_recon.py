"""GPU parity: the FP16 tensor-core reconstruction network (fvn_reconstruct)
and the whole frame (fvn_render) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import mask as omask
from oracle import march as om
from oracle import net as onet
from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP16_TOL = 2e-2        # max-abs, FP16 operands / FP32 accumulation vs FP64


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


@pytest.fixture(scope="module")
def ctx(fvn):
    c = fvn.Context()
    c.load_weights(wl.net_weights(3))
    yield c
    c.device_status()          # no bounded tensor-core wait gave up
    c.close()


def sparse_input(h, w, seed, density=0.15):
    rng = np.random.default_rng(seed)
    sp = np.zeros((5, h, w), np.float32)
    m = rng.uniform(size=(h, w)) < density
    yy, xx = np.mgrid[0:h, 0:w]
    base = 0.5 + 0.4 * np.sin(xx / 7.0)[None] * np.cos(yy / 5.0)[None] * np.array([1.0, 0.7, 0.4, 0.9])[:, None, None]
    sp[0:4] = (base + 0.05 * rng.normal(size=(4, h, w))) * m
    sp[4] = m
    return sp


def gpu_recon(ctx, sp, precision=0):
    dev = torch.device("cuda")
    _, h, w = sp.shape
    x = torch.from_numpy(sp).to(dev)
    y = torch.full((3, h, w), 77.0, dtype=torch.float32, device=dev)
    ctx.reconstruct(x, w, h, y, precision=precision)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("h,w,seed", [(64, 128, 0), (48, 200, 1), (45, 70, 2), (4, 4, 3), (1, 9, 4), (130, 67, 5)])
def test_recon_fp16_matches_oracle(ctx, h, w, seed):
    sp = sparse_input(h, w, seed)
    out = gpu_recon(ctx, sp)
    ref = onet.forward(onet.unpack(wl.net_weights(3)), sp)
    assert np.abs(out - ref).max() < FP16_TOL


def test_recon_other_weights(fvn):
    c = fvn.Context()
    w = wl.net_weights(11)
    rng = np.random.default_rng(12)
    w = (w + rng.normal(size=w.size).astype(np.float32) * 0.02).astype(np.float32)   # non-zero biases too
    c.load_weights(w)
    sp = sparse_input(96, 160, 6, density=0.3)
    out = gpu_recon(c, sp)
    ref = onet.forward(onet.unpack(w), sp)
    c.close()
    assert np.abs(out - ref).max() < FP16_TOL


def test_recon_1080p_sampled_windows(ctx):
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=0)
    _, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    sp, _, _ = om.march(vol, tf, cam, mp, ids=ids)
    sp = sp.astype(np.float32)
    out = gpu_recon(ctx, sp)
    params = onet.unpack(wl.net_weights(3))
    # the network's receptive field is < 32 px: a window cropped with a
    # 48-px margin on a multiple-of-4 grid reproduces the full-frame output
    rng = np.random.default_rng(3)
    for (y0, x0) in [(0, 0), (1080 - 64, 1920 - 64), (512, 960)] + [tuple(4 * rng.integers(0, [254, 464])) for _ in range(3)]:
        y0, x0 = int(y0), int(x0)
        ya, xa = max(0, y0 - 48), max(0, x0 - 48)
        yb, xb = min(1080, y0 + 64 + 48), min(1920, x0 + 64 + 48)
        crop = sp[:, ya:yb, xa:xb]
        ref = onet.forward(params, crop)
        got = out[:, y0:y0 + 64, x0:x0 + 64]
        want = ref[:, y0 - ya:y0 - ya + 64, x0 - xa:x0 - xa + 64]
        # windows on the right / bottom edge of the frame see the frame's own padding
        assert np.abs(got - want).max() < FP16_TOL, (y0, x0)


def test_recon_empty_and_full_masks(ctx):
    sp = np.zeros((5, 32, 48), np.float32)
    out = gpu_recon(ctx, sp)
    ref = onet.forward(onet.unpack(wl.net_weights(3)), sp)
    assert np.abs(out - ref).max() < FP16_TOL
    sp = sparse_input(32, 48, 9, density=1.0)
    out = gpu_recon(ctx, sp)
    ref = onet.forward(onet.unpack(wl.net_weights(3)), sp)
    assert np.abs(out - ref).max() < FP16_TOL


def test_render_matches_oracle_chain(ctx):
    w, h = 200, 120
    vol = wl.value_noise_volume(64, seed=4).to(torch.float32).numpy()
    tf = wl.transfer_function(5, alpha_max=0.1)
    cam = wl.orbit_camera(4, 7, width=w, height=h)
    fov = wl.Foveation(focal_px=(90.0, 70.0), seed=4, frame=7)
    mp = wl.MarchParams(shading=1)
    dev = torch.device("cuda")
    rgb = torch.zeros(3, h, w, device=dev)
    rgbam = torch.zeros(5, h, w, device=dev)
    ctx.render(torch.from_numpy(vol).to(dev), torch.from_numpy(tf).to(dev), cam, fov, mp, rgb, rgbam_out=rgbam)
    torch.cuda.synchronize()
    _, ids, _ = omask.make_mask(w, h, fov.focal_px, seed=fov.seed, frame=fov.frame)
    from tests.parity import march_parity
    march_parity(vol, tf, cam, mp, rgbam.cpu().numpy(), ids=ids)
    ref = onet.forward(onet.unpack(wl.net_weights(3)), rgbam.cpu().numpy().astype(np.float64))
    assert np.abs(rgb.cpu().numpy() - ref).max() < FP16_TOL


def test_reconstruct_needs_weights(fvn):
    c = fvn.Context()
    x = torch.zeros(5, 8, 8, device="cuda")
    y = torch.zeros(3, 8, 8, device="cuda")
    with pytest.raises(fvn.FvnError, match="no weights"):
        c.reconstruct(x, 8, 8, y)
    with pytest.raises(fvn.FvnError, match="expected"):
        c.load_weights(np.zeros(10, np.float32))
    c.close()


def test_render_adaptive_follows_oracle_rule(fvn):
    """Denser-mask fallback: probe ids, estimate and chosen level against the oracle rule."""
    from oracle import fallback as ofb
    w, h = 160, 120
    vol = wl.value_noise_volume(48, seed=6).to(torch.float32).numpy()
    tf = wl.transfer_function(6, alpha_max=0.1)
    cam = wl.orbit_camera(6, 2, width=w, height=h, radius_factor=(0.85, 1.75))
    fov = wl.Foveation(focal_px=(70.0, 60.0), seed=6, frame=2)
    mp = wl.MarchParams(shading=1)
    weights = wl.net_weights(3)
    params = onet.unpack(weights)
    c = fvn.Context()
    c.load_weights(weights)
    dev = torch.device("cuda")
    v = torch.from_numpy(vol).to(dev)
    t = torch.from_numpy(tf).to(dev)
    rgb = torch.zeros(3, h, w, device=dev)
    lvl0, est0 = c.render_adaptive(v, t, cam, fov, mp, rgb, min_psnr_db=0.0, max_levels=3)
    ref0, eref0, _ = ofb.render_adaptive(vol, tf, cam, fov, mp, params, 0.0, 3)
    assert lvl0 == ref0 == 0
    assert abs(est0 - eref0) < 0.5
    lvl, est = c.render_adaptive(v, t, cam, fov, mp, rgb, min_psnr_db=200.0, max_levels=3)
    ref, eref, rgb_ref = ofb.render_adaptive(vol, tf, cam, fov, mp, params, 200.0, 3)
    assert lvl == ref == 3
    assert abs(est - eref) < 0.5
    assert np.abs(rgb.cpu().numpy() - rgb_ref).max() < FP16_TOL
    c.device_status()
    c.close()



def test_render_cuda_graph_replay(ctx):
    """fvn_render captured in a CUDA graph replays to the result of the direct call."""
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=3, n=64, width=320, height=180)
    dev = torch.device("cuda")
    v = torch.from_numpy(vol).to(dev)
    t = torch.from_numpy(tf).to(dev)
    rgb = torch.empty(3, 180, 320, device=dev)
    sparse = torch.empty(5, 180, 320, device=dev)
    ctx.render(v, t, cam, fov, mp, rgb, rgbam_out=sparse)          # sizes the workspaces
    torch.cuda.synchronize()
    ref, ref_sparse = rgb.clone(), sparse.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        ctx.render(v, t, cam, fov, mp, rgb, rgbam_out=sparse)
    rgb.fill_(-1.0)
    sparse.fill_(-1.0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref) and torch.equal(sparse, ref_sparse)


@pytest.mark.parametrize("h,w", [(1080, 1920), (130, 67)])
def test_recon_tile_rows_are_bit_identical(fvn, h, w):
    """The tile-shape options (output rows per tile of the half-resolution,
    quarter-resolution and first decoder convolutions) change the launch
    shape, not the arithmetic: every combination gives the same frame, FP16
    and FP8."""
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        x = torch.from_numpy(sparse_input(h, w, 9)).cuda()
        c.calibrate_fp8(x, w, h)
        for prec in (fvn.PREC_FP16, fvn.PREC_FP8):
            ref = torch.empty(3, h, w, device="cuda")
            c.reconstruct(x, w, h, ref, precision=prec)
            for a, b, d in ((2, 1, 2), (2, 4, 1), (4, 4, 2), (2, 2, 1)):
                c.set_option(fvn.OPT_CONV_ROWS_HALF, a)
                c.set_option(fvn.OPT_CONV_ROWS_QUARTER, b)
                c.set_option(fvn.OPT_CONV_ROWS_DEC1, d)
                out = torch.full((3, h, w), 7.0, device="cuda")
                c.reconstruct(x, w, h, out, precision=prec)
                torch.cuda.synchronize()
                assert torch.equal(out, ref), (prec, a, b, d)
            c.set_option(fvn.OPT_CONV_ROWS_HALF, 4)
            c.set_option(fvn.OPT_CONV_ROWS_QUARTER, 2)
            c.set_option(fvn.OPT_CONV_ROWS_DEC1, 1)
        with pytest.raises(fvn.FvnError, match="tile rows"):
            c.set_option(fvn.OPT_CONV_ROWS_HALF, 3)
        c.device_status()
    finally:
        c.close()


@pytest.mark.parametrize("h,w,seed", [(64, 128, 0), (45, 70, 2), (4, 4, 3), (130, 67, 5), (1080, 1920, 6)])
def test_recon_fused_decoder_upsampling_matches_oracle(fvn, h, w, seed):
    """FVN_OPT_CONV_FUSE_UP_DEC1: the first decoder convolution up-samples the
    bottleneck output itself (half precision); the frame still meets the FP16
    bar against the oracle, for every tile-row setting of that layer."""
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        c.set_option(fvn.OPT_CONV_FUSE_UP_DEC1, 1)
        sp = sparse_input(h, w, seed)
        ref = onet.forward(onet.unpack(wl.net_weights(3)), sp) if h * w < 100000 else None
        outs = []
        for rows in (1, 2):
            c.set_option(fvn.OPT_CONV_ROWS_DEC1, rows)
            outs.append(gpu_recon(c, sp))
        assert np.array_equal(outs[0], outs[1])
        c.set_option(fvn.OPT_CONV_FUSE_UP_DEC1, 0)
        sep = gpu_recon(c, sp)
        assert np.abs(outs[0] - sep).max() < 1e-2
        if ref is not None:
            assert np.abs(outs[0] - ref).max() < FP16_TOL
        c.device_status()
    finally:
        c.close()
