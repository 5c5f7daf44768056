"""GPU: sample masks from a looping series of noise tiles (the paper's
pre-computed blue-noise tiles; fvn_set_noise_tiles) -- bit-exact against the
oracle for several frame and tile sizes, frames past the end of the series,
the render and the batch, going back to the hash, and the argument checks."""
import numpy as np
import pytest
import torch

from oracle import mask as omask
from paper_2209_09965_gb300 import workloads as wl
from tests.parity import march_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


@pytest.fixture(scope="module")
def ctx(fvn):
    c = fvn.Context()
    yield c
    c.device_status()
    c.close()


def gpu_mask(ctx, fov, w, h):
    dev = torch.device("cuda")
    mask = torch.full((h, w), 7, dtype=torch.uint8, device=dev)
    ids = torch.full((w * h,), -1, dtype=torch.int32, device=dev)
    count = torch.full((1,), -5, dtype=torch.int32, device=dev)
    ctx.make_mask(fov, w, h, mask, ids, count)
    torch.cuda.synchronize()
    n = int(count.item())
    return mask.cpu().numpy(), ids[:n].cpu().numpy(), n


@pytest.mark.parametrize("tile,frames", [(16, 1), (64, 5), (256, 64)])
@pytest.mark.parametrize("w,h,fp,frame", [
    (1920, 1080, (960.0, 540.0), 0),
    (1920, 1080, (500.5, 300.25), 70),        # past the end of the series
    (97, 61, (40.0, 20.0), 3),                # ragged
    (1, 1, (0.5, 0.5), 9),
    (333, 1, (100.0, 0.5), 4),
])
def test_tiled_mask_bit_exact(ctx, tile, frames, w, h, fp, frame):
    tiles = wl.blue_noise_tiles(tile, frames, seed=tile) if tile <= 64 else \
        np.random.default_rng(7).integers(0, 1 << 24, (frames, tile, tile), dtype=np.uint32)
    ctx.set_noise_tiles(tiles)
    try:
        fov = wl.Foveation(focal_px=fp, seed=11, frame=frame)
        m, ids, n = gpu_mask(ctx, fov, w, h)
        m_ref, ids_ref, _ = omask.make_mask(w, h, fp, seed=11, frame=frame, noise=tiles)
        assert np.array_equal(m, m_ref)
        assert n == ids_ref.size and np.array_equal(np.sort(ids), ids_ref)
    finally:
        ctx.set_noise_tiles(None)


def test_back_to_the_hash(ctx):
    fov = wl.Foveation(focal_px=(300.0, 200.0), seed=5, frame=2)
    ctx.set_noise_tiles(wl.blue_noise_tiles(32, 4, seed=0))
    a, _, _ = gpu_mask(ctx, fov, 640, 360)
    ctx.set_noise_tiles(None)
    b, _, _ = gpu_mask(ctx, fov, 640, 360)
    ref, _, _ = omask.make_mask(640, 360, fov.focal_px, seed=5, frame=2)
    assert np.array_equal(b, ref) and not np.array_equal(a, b)


def test_render_and_batch_with_tiles(fvn):
    dev = torch.device("cuda")
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        tiles = wl.blue_noise_tiles(64, 8, seed=2)
        c.set_noise_tiles(tiles)
        vol_np = wl.blob_volume(48, seed=11).numpy().astype(np.float32)
        vol = torch.from_numpy(vol_np).to(dev)
        tf_np = wl.transfer_function(31, alpha_max=0.3)
        tf = torch.from_numpy(tf_np).to(dev)
        mp = wl.MarchParams(shading=1)
        views = []
        for i, (w, h) in enumerate([(160, 120), (97, 61)]):
            cam = wl.orbit_camera(30 + i, i, width=w, height=h, radius_factor=(1.0, 1.4))
            fov = wl.Foveation(focal_px=wl.focal_point(30 + i, i, w, h), seed=30 + i, frame=5 + 7 * i)
            views.append({"vol": vol, "tf": tf, "cam": cam, "fov": fov,
                          "rgb": torch.full((3, h, w), 5.0, device=dev),
                          "rgbam": torch.full((5, h, w), 9.0, device=dev)})
        c.render_batch(views, mp)
        for v in views:
            w, h = v["cam"].width, v["cam"].height
            rgb = torch.empty(3, h, w, device=dev)
            rgbam = torch.empty(5, h, w, device=dev)
            c.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb, rgbam_out=rgbam)
            torch.cuda.synchronize()
            assert torch.equal(v["rgb"], rgb) and torch.equal(v["rgbam"], rgbam)
            f = v["fov"]
            m, ids, _ = omask.make_mask(w, h, f.focal_px, f.fovea_radius, f.falloff_sigma, f.p_base, f.seed,
                                        f.frame, noise=tiles)
            got = rgbam.cpu().numpy()
            assert np.array_equal(got[4] != 0, m != 0)
            march_parity(vol_np, tf_np, v["cam"], mp, got, ids=ids)
        c.device_status()
    finally:
        c.close()


def test_noise_argument_errors(ctx, fvn):
    good = wl.blue_noise_tiles(16, 2, seed=0)
    ctx.set_noise_tiles(good)
    try:
        for bad in (np.zeros((1, 48, 48), np.uint32), np.zeros((1, 8, 8), np.uint32),
                    np.zeros((1, 512, 512), np.uint32), np.zeros((257, 16, 16), np.uint32),
                    np.full((1, 16, 16), 1 << 24, np.uint32)):
            with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
                ctx.set_noise_tiles(bad)
        # the installed tiles survive a rejected call
        fov = wl.Foveation(focal_px=(60.0, 40.0), seed=1, frame=1)
        m, _, _ = gpu_mask(ctx, fov, 128, 96)
        ref, _, _ = omask.make_mask(128, 96, fov.focal_px, seed=1, frame=1, noise=good)
        assert np.array_equal(m, ref)
    finally:
        ctx.set_noise_tiles(None)
