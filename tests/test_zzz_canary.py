"""Out-of-bounds writes, without a sanitizer: every output buffer sits
between two guard regions filled with a sentinel, and after each call
through the C ABI the guards must be intact -- mask, ids and count, dense
and sparse marches, the FP16 reconstruction (both kernel families), the
whole frame, the two-stage network and its kernels, and the training
kernels -- on odd frame sizes (1 x 1, widths not a multiple of 4, ragged
tiles).  Also the 1x1 training convolutions' remaining shapes against the
oracle: planes whose length is not a multiple of 4 (scalar staging) and
more than 128 channels (channel groups spread over CTAs).  Collected last,
so a failure here comes after every other test has run."""
import math

import numpy as np
import pytest
import torch

from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
GUARD = 4096
SENTINEL = {torch.float32: 12345.0, torch.int32: -777, torch.uint8: 77}


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


class Guarded:
    """A device tensor of the given shape inside a larger sentinel-filled array."""

    def __init__(self, shape, dtype=torch.float32):
        self.n = math.prod(shape)
        self.buf = torch.full((self.n + 2 * GUARD,), SENTINEL[dtype], dtype=dtype, device=DEV)
        self.t = self.buf[GUARD:GUARD + self.n].view(shape)
        self.dtype = dtype

    def intact(self):
        torch.cuda.synchronize()
        s = SENTINEL[self.dtype]
        return bool((self.buf[:GUARD] == s).all()) and bool((self.buf[GUARD + self.n:] == s).all())


def scene(w, h, seed):
    vol = torch.from_numpy(wl.blob_volume(40, seed=seed).numpy().astype(np.float32)).to(DEV)
    tf = torch.from_numpy(wl.transfer_function(seed, alpha_max=0.3)).to(DEV)
    cam = wl.orbit_camera(seed, 1, width=w, height=h, radius_factor=(1.0, 1.4))
    fov = wl.Foveation(focal_px=(w * 0.4, h * 0.6), seed=seed, frame=2)
    return vol, tf, cam, fov


@pytest.mark.parametrize("w,h", [(1, 1), (97, 61), (130, 7), (3, 200)])
def test_frame_path_stays_in_bounds(fvn, w, h):
    ctx = fvn.Context()
    try:
        ctx.load_weights(wl.net_weights(3))
        vol, tf, cam, fov = scene(w, h, 5)
        mask, ids, count = Guarded((h, w), torch.uint8), Guarded((w * h,), torch.int32), Guarded((1,), torch.int32)
        ctx.make_mask(fov, w, h, mask.t, ids.t, count.t)
        assert mask.intact() and ids.intact() and count.intact()
        for shading in (0, 1, 2):
            mp = wl.MarchParams(shading=shading)
            dense, sparse = Guarded((5, h, w)), Guarded((5, h, w))
            ctx.march(vol, tf, cam, mp, dense.t)
            ctx.march(vol, tf, cam, mp, sparse.t, ids=ids.t, count=count.t)
            assert dense.intact() and sparse.intact(), f"march, shading {shading}"
        rgb = Guarded((3, h, w))
        ctx.reconstruct(sparse.t, w, h, rgb.t)
        assert rgb.intact()
        rgb2, rgbam = Guarded((3, h, w)), Guarded((5, h, w))
        ctx.render(vol, tf, cam, fov, wl.MarchParams(shading=1), rgb2.t, rgbam_out=rgbam.t)
        assert rgb2.intact() and rgbam.intact()
        ctx.device_status()
    finally:
        ctx.close()


@pytest.mark.parametrize("w,h", [(1, 1), (37, 21), (64, 48)])
def test_two_stage_stays_in_bounds(fvn, w, h):
    ctx = fvn.Context()
    try:
        cfg = ((3, 5), 6, (4, 5))
        ctx.load_wnet_weights(cfg, wl.wnet_weights(cfg, 2))
        sp = torch.rand(5, h, w, device=DEV)
        rgb = Guarded((3, h, w))
        ctx.reconstruct_wnet(sp, w, h, rgb.t)
        assert rgb.intact()
        ctx.device_status()
    finally:
        ctx.close()
    n, hh, ww = 2, 2 * ((h + 1) // 2), 2 * ((w + 1) // 2)
    img, lg = torch.rand(n, 3, hh, ww, device=DEV), torch.rand(n, 9, hh, ww, device=DEV)
    out, gi, gl = Guarded((n, 3, hh, ww)), Guarded((n, 3, hh, ww)), Guarded((n, 9, hh, ww))
    fvn.filter3_fwd(img, lg, out.t)
    fvn.filter3_bwd(img, lg, torch.rand(n, 3, hh, ww, device=DEV), gi.t, gl.t)
    assert out.intact() and gi.intact() and gl.intact()
    y, z = torch.rand(n, 3, hh // 2, ww // 2, device=DEV), torch.rand(n, 1, hh, ww, device=DEV)
    x, gj, gy, gz = Guarded((n, 3, hh, ww)), Guarded((n, 3, hh, ww)), Guarded((n, 3, hh // 2, ww // 2)), \
        Guarded((n, 1, hh, ww))
    fvn.wnet_join_fwd(img, y, z, x.t)
    fvn.wnet_join_bwd(img, y, z, torch.rand(n, 3, hh, ww, device=DEV), gj.t, gy.t, gz.t)
    assert x.intact() and gj.intact() and gy.intact() and gz.intact()


@pytest.mark.parametrize("k,ca,cb,cout,h,w", [(3, 5, 3, 16, 17, 70), (1, 7, 0, 9, 5, 3), (3, 16, 0, 29, 1, 1),
                                             (1, 40, 24, 140, 6, 10)])
def test_training_kernels_stay_in_bounds(fvn, k, ca, cb, cout, h, w):
    n = 2
    xa = torch.rand(n, ca, h, w, device=DEV)
    xb = torch.rand(n, cb, h, w, device=DEV) if cb else None
    wt = torch.rand(cout, ca + cb, k, k, device=DEV) - 0.5
    b = torch.rand(cout, device=DEV)
    y = Guarded((n, cout, h, w))
    fvn.conv_fwd(xa, xb, wt, b, True, y.t)
    assert y.intact()
    gxa, gw, gb = Guarded((n, ca, h, w)), Guarded(tuple(wt.shape)), Guarded((cout,))
    gxb = Guarded((n, cb, h, w)) if cb else None
    fvn.conv_bwd(xa, xb, wt, torch.rand(n, cout, h, w, device=DEV), y.t, gxa.t, None if gxb is None else gxb.t,
                 gw.t, gb.t)
    assert gxa.intact() and gw.intact() and gb.intact() and (gxb is None or gxb.intact())
    if h % 2 == 0 and w % 2 == 0:
        p = Guarded((n, ca, h // 2, w // 2))
        fvn.avgpool2_fwd(xa, p.t)
        u = Guarded((n, ca, 2 * h, 2 * w))
        fvn.upsample2_fwd(xa, u.t)
        assert p.intact() and u.intact()


@pytest.mark.parametrize("ca,cb,cout,h,w", [(5, 3, 9, 7, 13), (130, 0, 200, 3, 5), (96, 80, 176, 8, 8)])
def test_1x1_training_convolution_shapes(fvn, ca, cb, cout, h, w):
    from oracle import net as onet
    rng = np.random.default_rng(ca + cout)
    n = 2
    xa = rng.normal(size=(n, ca, h, w))
    xb = rng.normal(size=(n, cb, h, w)) if cb else None
    wt = rng.normal(size=(cout, ca + cb, 1, 1)) * 0.2
    b = rng.normal(size=cout) * 0.1
    x = xa if xb is None else np.concatenate([xa, xb], 1)
    z = onet.conv2d(x, wt, b)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV)   # noqa: E731
    y = torch.empty(n, cout, h, w, device=DEV)
    fvn.conv_fwd(T(xa), None if xb is None else T(xb), T(wt), T(b), True, y)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - np.maximum(z, 0)).max() < 1e-4
    gy = rng.normal(size=z.shape)
    gx_ref, gw_ref, gb_ref = onet.conv2d_backward(x, wt, gy * (z > 0))
    gxa = torch.empty(n, ca, h, w, device=DEV)
    gxb = torch.empty(n, cb, h, w, device=DEV) if cb else None
    gw, gb = torch.empty(cout, ca + cb, 1, 1, device=DEV), torch.empty(cout, device=DEV)
    fvn.conv_bwd(T(xa), None if xb is None else T(xb), T(wt), T(gy), y, gxa, gxb, gw, gb)
    torch.cuda.synchronize()
    gx = gxa.cpu().numpy() if gxb is None else np.concatenate([gxa.cpu().numpy(), gxb.cpu().numpy()], 1)
    assert np.abs(gx - gx_ref).max() < 1e-3 * max(1.0, np.abs(gx_ref).max())
    assert np.abs(gw.cpu().numpy() - gw_ref).max() < 1e-3 * max(1.0, np.abs(gw_ref).max())
    assert np.abs(gb.cpu().numpy() - gb_ref).max() < 1e-3 * max(1.0, np.abs(gb_ref).max())
