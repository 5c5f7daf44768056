"""GPU: batched multi-view render (fvn_render_batch).

Every view of a batch must equal fvn_render of that view alone, bit for bit
(same mask, same rays, same network tiles), over views of uneven sizes,
several volumes of different voxel types and several transfer functions; the
batch's sparse frames are also checked against the FP64 oracle march
directly, and a CUDA-graph replay of the batch must reproduce it."""
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
    c.load_weights(wl.net_weights(3))
    yield c
    c.device_status()
    c.close()


def _volumes():
    """Three small volumes of three voxel types (host numpy + device copies)."""
    dev = torch.device("cuda")
    u8 = np.round(wl.blob_volume(48, seed=11).numpy() * 255.0).astype(np.uint8)
    f16 = wl.value_noise_volume(40, seed=12, base_spacing=8).numpy().astype(np.float16)
    f32 = wl.blob_volume(32, seed=13).to(torch.float32).numpy()
    host = [u8, f16, f32]
    return host, [torch.from_numpy(v).to(dev) for v in host]


def _views(specs, vols_d, tfs_d, dev):
    views = []
    for (w, h, vi, ti, seed, frame, shift) in specs:
        cam = wl.orbit_camera(seed, frame, width=w, height=h, radius_factor=(1.0, 1.4))
        if shift:   # stereo partner: eye moved sideways along the image x axis
            cam = wl.stereo_pair(cam, 2.0 * shift)[1]
        fov = wl.Foveation(focal_px=wl.focal_point(seed, frame, w, h), seed=seed, frame=frame)
        views.append({"vol": vols_d[vi], "tf": tfs_d[ti], "cam": cam, "fov": fov,
                      "rgb": torch.full((3, h, w), 5.0, device=dev),
                      "rgbam": torch.full((5, h, w), 9.0, device=dev)})
    return views


SPECS = [  # w, h, volume, tf, seed, frame, stereo shift
    (160, 120, 0, 0, 21, 0, 0.0),
    (160, 120, 0, 0, 21, 0, 0.03),        # stereo partner of the first view
    (96, 64, 1, 1, 22, 3, 0.0),
    (200, 100, 2, 0, 23, 7, 0.0),
    (61, 45, 1, 1, 24, 9, 0.0),           # ragged: no multiple of any tile
    (128, 128, 2, 1, 25, 2, 0.0),
]


def _setup():
    dev = torch.device("cuda")
    host, vols_d = _volumes()
    tfs = [wl.transfer_function(31, alpha_max=0.3), wl.transfer_function(32, alpha_max=0.5)]
    tfs_d = [torch.from_numpy(t).to(dev) for t in tfs]
    return dev, host, vols_d, tfs, tfs_d


def test_batch_equals_single_views(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    views = _views(SPECS, vols_d, tfs_d, dev)
    ns = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx.render_batch(views, mp, nsamples=ns)
    torch.cuda.synchronize()
    ns_single = torch.zeros(1, dtype=torch.int64, device=dev)
    for v in views:
        w, h = v["cam"].width, v["cam"].height
        rgb = torch.empty(3, h, w, device=dev)
        rgbam = torch.empty(5, h, w, device=dev)
        ctx.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb, rgbam_out=rgbam)
        mask = torch.empty(h, w, dtype=torch.uint8, device=dev)
        ids = torch.empty(w * h, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        ctx.make_mask(v["fov"], w, h, mask, ids, cnt)
        scratch = torch.empty(5, h, w, device=dev)
        ctx.march(v["vol"], v["tf"], v["cam"], mp, scratch, ids=ids, count=cnt, nsamples=ns_single)
        torch.cuda.synchronize()
        assert torch.equal(v["rgbam"], rgbam), f"sparse frame of the {w}x{h} view differs from fvn_render"
        assert torch.equal(v["rgb"], rgb), f"output of the {w}x{h} view differs from fvn_render"
        assert torch.equal(scratch, rgbam)
    assert int(ns.item()) == int(ns_single.item()) > 0


def test_batch_sparse_frames_match_oracle(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    views = _views(SPECS, vols_d, tfs_d, dev)
    ctx.render_batch(views, mp)
    torch.cuda.synchronize()
    for (w, h, vi, ti, *_), v in zip(SPECS, views):
        f = v["fov"]
        m, ids, _ = omask.make_mask(w, h, f.focal_px, f.fovea_radius, f.falloff_sigma, f.p_base, f.seed, f.frame)
        got = v["rgbam"].cpu().numpy()
        assert np.array_equal(got[4].reshape(-1) != 0, m.reshape(-1) != 0), "batch mask differs from the oracle"
        unsampled = m.reshape(-1) == 0
        assert np.all(got.reshape(5, -1)[:, unsampled] == 0.0)
        march_parity(host[vi], tfs[ti], v["cam"], mp, got, ids=ids)


def test_batch_fp8_equals_single_views(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    views = _views(SPECS[:4], vols_d, tfs_d, dev)
    # calibrate the FP8 scales on the views' own sparse frames (FP16 pass first)
    ctx.render_batch(views, mp)
    for i, v in enumerate(views):
        ctx.calibrate_fp8(v["rgbam"], v["cam"].width, v["cam"].height, reset=(i == 0))
    ctx.render_batch(views, mp, precision=fvn.PREC_FP8)
    torch.cuda.synchronize()
    for v in views:
        w, h = v["cam"].width, v["cam"].height
        rgb = torch.empty(3, h, w, device=dev)
        ctx.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb, precision=fvn.PREC_FP8)
        torch.cuda.synchronize()
        assert torch.equal(v["rgb"], rgb)


def test_batch_cuda_graph_replay(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    views = _views(SPECS, vols_d, tfs_d, dev)
    ctx.render_batch(views, mp)          # sizes the workspace (the one synchronising call)
    torch.cuda.synchronize()
    ref = [v["rgb"].clone() for v in views]
    for v in views:
        v["rgb"].fill_(-1.0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        ctx.render_batch(views, mp)
    for v in views:
        v["rgb"].fill_(-1.0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for v, r in zip(views, ref):
        assert torch.equal(v["rgb"], r)


def test_batch_single_view_equals_render(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=0)
    views = _views([(77, 50, 0, 1, 41, 1, 0.0)], vols_d, tfs_d, dev)
    ctx.render_batch(views, mp)
    v = views[0]
    rgb = torch.empty(3, 50, 77, device=dev)
    ctx.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb)
    torch.cuda.synchronize()
    assert torch.equal(v["rgb"], rgb)


def test_batch_argument_errors(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
        ctx.render_batch([], mp)
    views = _views([(32, 32, 0, 0, 1, 0, 0.0)] * (fvn.MAX_VIEWS + 1), vols_d, tfs_d, dev)
    with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
        ctx.render_batch(views, mp)
    # five distinct volumes
    extra = [torch.zeros(8 + i, 8, 8, device=dev) for i in range(5)]
    views = _views([(16, 16, i, 0, 1, i, 0.0) for i in range(5)], extra, tfs_d, dev)
    with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
        ctx.render_batch(views, mp)
    views = _views([(16, 16, 0, 0, 1, 0, 0.0)], vols_d, tfs_d, dev)
    views[0]["rgb"] = None
    with pytest.raises((fvn.FvnError, ValueError)):
        ctx.render_batch(views, mp)


@pytest.mark.parametrize("mode", ["all", "some"])
def test_batch_adaptive_equals_single_view_fallback(ctx, fvn, mode):
    """fvn_render_batch_adaptive applies the denser-mask fallback to every
    view: each view ends with the output, level and estimate that
    fvn_render_adaptive gives for it alone -- with a threshold every view
    misses (all re-render up to max_levels), and with one between the views'
    first estimates (some re-render, the others keep their first frame)."""
    dev, host, vols_d, tfs, tfs_d = _setup()
    mp = wl.MarchParams(shading=1)
    single = []
    first = []
    for v in _views(SPECS, vols_d, tfs_d, dev):
        lvl, est = ctx.render_adaptive(v["vol"], v["tf"], v["cam"], v["fov"], mp, v["rgb"], min_psnr_db=-1.0,
                                       max_levels=0)
        first.append(est)
    thr = 99.5 if mode == "all" else float(np.median(first))
    for v in _views(SPECS, vols_d, tfs_d, dev):
        lvl, est = ctx.render_adaptive(v["vol"], v["tf"], v["cam"], v["fov"], mp, v["rgb"], min_psnr_db=thr,
                                       max_levels=2)
        torch.cuda.synchronize()
        single.append((lvl, est, v["rgb"].clone()))
    views = _views(SPECS, vols_d, tfs_d, dev)
    levels, ests = ctx.render_batch_adaptive(views, mp, min_psnr_db=thr, max_levels=2)
    torch.cuda.synchronize()
    for (lvl, est, rgb), v, bl, be in zip(single, views, levels, ests):
        assert bl == lvl and be == est
        assert torch.equal(v["rgb"], rgb)
    if mode == "all":
        assert all(x == 2 for x in levels)
    else:
        assert 0 < sum(1 for x in levels if x > 0) < len(levels)


def test_batch_adaptive_argument_errors(ctx, fvn):
    dev, host, vols_d, tfs, tfs_d = _setup()
    views = _views(SPECS[:2], vols_d, tfs_d, dev)
    with pytest.raises(fvn.FvnError, match="max_levels"):
        ctx.render_batch_adaptive(views, wl.MarchParams(shading=1), max_levels=9)
    assert float(views[0]["rgb"].min()) == 5.0           # nothing was enqueued
