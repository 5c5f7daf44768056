"""GPU parity of the shadowed shading mode (shading 2: a directional light,
one shadow ray per sample at 1 / shadow_rate of the main sample rate) against
the FP64 oracle, 1e-4 max-abs per channel, through the C ABI: every voxel
type (shadow rays read a cell volume of 2 x 2 voxel blocks in the voxel
type; the gradient-volume option does not apply to them), the cooperative
march modes, sparse 1080p, random lights including axis-aligned ones, the
batched march with several transfer functions (whose opacity-pair tables
share shared memory), and the argument checks."""
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


def run_march(ctx, vol, tf, cam, mp, ids=None):
    dev = torch.device("cuda")
    v = torch.from_numpy(np.ascontiguousarray(vol)).to(dev)
    t = torch.from_numpy(tf).to(dev)
    out = torch.full((5, cam.height, cam.width), 123.0, dtype=torch.float32, device=dev)
    ns = torch.zeros(1, dtype=torch.int64, device=dev)
    if ids is None:
        ctx.march(v, t, cam, mp, out, nsamples=ns)
    else:
        ids = np.asarray(ids, np.int32)
        i = torch.from_numpy(ids if ids.size else np.zeros(1, np.int32)).to(dev)
        c = torch.tensor([ids.size], dtype=torch.int32, device=dev)
        ctx.march(v, t, cam, mp, out, ids=i, count=c, nsamples=ns)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(ns.item())


def shadow_params(rate=4, light=wl.LIGHT_DIR, term=0.99, bg=(0.0, 0.0, 0.0)):
    return wl.MarchParams(0.5, term, bg, 2, light_dir=tuple(light), shadow_rate=rate)


@pytest.mark.parametrize("rate", [4, 1, 3])
def test_shadow_dense_small_blobs(ctx, rate):
    vol, tf, cam, _ = wl.dense_small_workload(seed=1, frame=5)
    mp = shadow_params(rate)
    out, ns = run_march(ctx, vol, tf, cam, mp)
    march_parity(vol, tf, cam, mp, out)
    assert ns > 0 and np.all(out[4] == 1.0)


@pytest.mark.parametrize("grad_volume", [0, 1])
@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
def test_shadow_dtypes(ctx, fvn, grad_volume, dtype):
    base = wl.value_noise_volume(36, seed=9, base_spacing=8).numpy()
    vol = {"u8": np.round(base * 255).astype(np.uint8), "u16": np.round(base * 65535).astype(np.uint16),
           "f16": base.astype(np.float16), "f32": base.astype(np.float32)}[dtype]
    vol_t = vol.view(np.int16) if dtype == "u16" else vol
    tf = wl.transfer_function(6, alpha_max=0.2)
    cam = wl.orbit_camera(5, 3, width=80, height=56, radius_factor=(0.9, 1.3))
    mp = shadow_params(4, light=(-0.5, 0.7, 0.2))
    try:
        ctx.set_option(fvn.OPT_MARCH_GRADIENT_VOLUME, grad_volume)    # does not apply to shadowed marches
        out, _ = run_march(ctx, vol_t, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)
        ids = np.arange(1, 80 * 56, 3, dtype=np.int32)
        outs, _ = run_march(ctx, vol_t, tf, cam, mp, ids=ids)
        march_parity(vol, tf, cam, mp, outs, ids=ids)
    finally:
        ctx.set_option(fvn.OPT_MARCH_GRADIENT_VOLUME, 1)


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2), (5, 3)])
def test_shadow_tiny_grids_random_cameras_and_lights(ctx, n, seed):
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0, 1, (n, n + 1, n + 2)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rng.uniform(0, 1, 3)
    tf[:, 0] = np.linspace(0.1, 0.9, 256)
    tf[:, 3] = np.linspace(0.0, 0.6, 256)
    lights = [tuple(rng.normal(size=3)), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.3, -0.8)]
    for k in range(4):
        v = rng.normal(size=3)
        r = [1.6, 0.3, 0.05, 2.5][k]           # outside, inside, near centre, far
        eye = tuple(r * v / np.linalg.norm(v))
        cam = wl.Camera(eye=eye, target=(0.02, -0.03, 0.01), up=(0, 1, 0), fov_y_deg=60.0, width=13, height=9)
        mp = shadow_params([4, 1, 2, 4][k], light=lights[k], term=0.95, bg=(0.1, 0.2, 0.3))
        out, _ = run_march(ctx, vol, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)


@pytest.mark.parametrize("coop", [4, 32])
def test_shadow_cooperative_modes(ctx, fvn, coop):
    vol, tf, cam, _ = wl.dense_small_workload(seed=1, frame=21)
    mp = shadow_params(4)
    try:
        ctx.set_option(fvn.OPT_MARCH_COOP_DENSE, coop)
        ctx.set_option(fvn.OPT_MARCH_COOP, coop)
        out, _ = run_march(ctx, vol, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)
        ids = np.arange(0, 128 * 128, 5, dtype=np.int32)
        outs, _ = run_march(ctx, vol, tf, cam, mp, ids=ids)
        march_parity(vol, tf, cam, mp, outs, ids=ids)
    finally:
        ctx.set_option(fvn.OPT_MARCH_COOP_DENSE, 0)
        ctx.set_option(fvn.OPT_MARCH_COOP, 0)


def test_shadow_sparse_1080p_sampled(ctx):
    vol, tf, cam, fov, _ = wl.foveated_1080p_workload(seed=2, frame=4)
    mp = shadow_params(4)
    _, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    out, ns = run_march(ctx, vol, tf, cam, mp, ids=ids)
    sample = np.sort(np.random.default_rng(4).choice(ids, 4000, replace=False)).astype(np.int32)
    march_parity(vol, tf, cam, mp, out, ids=sample)
    flat = out.reshape(5, -1)
    rest = np.setdiff1d(np.arange(1920 * 1080), ids)
    assert np.all(flat[:, rest] == 0.0) and np.all(flat[4, ids] == 1.0)
    assert ns > 0


def test_shadow_light_changes_image(ctx):
    vol, tf, cam, _ = wl.dense_small_workload(seed=1, frame=5)
    a, _ = run_march(ctx, vol, tf, cam, shadow_params(4, light=(1.0, 0.0, 0.0)))
    b, _ = run_march(ctx, vol, tf, cam, shadow_params(4, light=(-1.0, 0.0, 0.0)))
    c, _ = run_march(ctx, vol, tf, cam, wl.MarchParams(shading=1))
    assert np.abs(a[:3] - b[:3]).max() > 0.05
    assert np.abs(a[:3] - c[:3]).max() > 0.05
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[3], c[3])      # opacity does not depend on light


def test_shadow_batch_equals_single_views(fvn):
    dev = torch.device("cuda")
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        u8 = np.round(wl.blob_volume(40, seed=11).numpy() * 255.0).astype(np.uint8)
        f32 = wl.value_noise_volume(32, seed=12, base_spacing=8).numpy().astype(np.float32)
        vols = [torch.from_numpy(u8).to(dev), torch.from_numpy(f32).to(dev)]
        tfs = [torch.from_numpy(wl.transfer_function(31, alpha_max=0.3)).to(dev),
               torch.from_numpy(wl.transfer_function(32, alpha_max=0.5, n=77)).to(dev)]
        mp = shadow_params(4, light=(0.2, 0.9, -0.3))
        views = []
        for i, (w, h) in enumerate([(96, 64), (61, 45), (128, 72)]):
            cam = wl.orbit_camera(20 + i, i, width=w, height=h, radius_factor=(1.0, 1.4))
            fov = wl.Foveation(focal_px=wl.focal_point(20 + i, i, w, h), seed=20 + i, frame=i)
            views.append({"vol": vols[i % 2], "tf": tfs[(i // 2) % 2], "cam": cam, "fov": fov,
                          "rgb": torch.full((3, h, w), 5.0, device=dev),
                          "rgbam": torch.full((5, h, w), 9.0, device=dev)})
        c.render_batch(views, mp)
        for v in views:
            w, h = v["cam"].width, v["cam"].height
            rgb = torch.empty(3, h, w, device=dev)
            rgbam = torch.empty(5, h, w, device=dev)
            c.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb, rgbam_out=rgbam)
            torch.cuda.synchronize()
            assert torch.equal(v["rgbam"], rgbam) and torch.equal(v["rgb"], rgb)
        # the batch's sparse frames against the oracle
        host = [u8, f32]
        for i, v in enumerate(views):
            f = v["fov"]
            w, h = v["cam"].width, v["cam"].height
            _, ids, _ = omask.make_mask(w, h, f.focal_px, f.fovea_radius, f.falloff_sigma, f.p_base, f.seed, f.frame)
            march_parity(host[i % 2], v["tf"].cpu().numpy(), v["cam"], mp, v["rgbam"].cpu().numpy(), ids=ids)
        c.device_status()
    finally:
        c.close()


def test_shadow_argument_errors(ctx, fvn):
    vol, tf, cam, _ = wl.dense_small_workload(seed=1)
    dev = torch.device("cuda")
    v = torch.from_numpy(vol).to(dev)
    t = torch.from_numpy(tf).to(dev)
    out = torch.zeros(5, cam.height, cam.width, device=dev)
    for bad, msg in ((wl.MarchParams(shading=3), "shading"),
                     (shadow_params(light=(0.0, 0.0, 0.0)), "light_dir"),
                     (shadow_params(light=(float("nan"), 1.0, 0.0)), "light_dir"),
                     (shadow_params(rate=0), "shadow_rate"),
                     (shadow_params(rate=65), "shadow_rate")):
        out.fill_(7.0)
        with pytest.raises(fvn.FvnError, match=msg):
            ctx.march(v, t, cam, bad, out)
        torch.cuda.synchronize()
        assert torch.all(out == 7.0)                       # untouched on error
    # the light fields are ignored by the other shading modes
    a, _ = run_march(ctx, vol, tf, cam, wl.MarchParams(shading=1, light_dir=(0.0, 0.0, 0.0), shadow_rate=0))
    b, _ = run_march(ctx, vol, tf, cam, wl.MarchParams(shading=1))
    assert np.array_equal(a, b)


def test_shadow_sample_counting_option(ctx, fvn):
    vol, tf, cam, _ = wl.dense_small_workload(seed=1, frame=5)
    mp = shadow_params(4)
    _, n0 = run_march(ctx, vol, tf, cam, mp)
    try:
        ctx.set_option(fvn.OPT_MARCH_COUNT_SHADOW, 1)
        _, n1 = run_march(ctx, vol, tf, cam, mp)
        _, h1 = run_march(ctx, vol, tf, cam, wl.MarchParams(shading=1))
    finally:
        ctx.set_option(fvn.OPT_MARCH_COUNT_SHADOW, 0)
    _, h0 = run_march(ctx, vol, tf, cam, wl.MarchParams(shading=1))
    assert n1 > n0 > 0                      # shadow-ray samples added on top of the primary ones
    assert h1 == h0                         # no shadow rays without shading 2


def test_shadow_without_termination_and_empty_volume(ctx, fvn):
    # a thin TF and term_alpha = 1: every ray and every shadow ray runs to the box's far side
    vol, _, cam, _ = wl.dense_small_workload(seed=1)
    tf = wl.transfer_function(5, alpha_max=0.02)
    mp = shadow_params(4, term=1.0, bg=(0.1, 0.2, 0.3))
    out, _ = run_march(ctx, vol, tf, cam, mp)
    march_parity(vol, tf, cam, mp, out)
    # an empty volume (TF opacity 0 at 0): the background everywhere, no shadow work
    empty = np.zeros((16, 16, 16), np.float32)
    tf0 = np.zeros((256, 4), np.float32)
    tf0[:, :3] = 1.0
    tf0[1:, 3] = 0.5
    cam2 = wl.Camera(eye=(0.2, 0.3, 2.0), target=(0, 0, 0), up=(0, 1, 0), fov_y_deg=45.0, width=24, height=16)
    ctx.set_option(fvn.OPT_MARCH_COUNT_SHADOW, 1)
    try:
        out, ns = run_march(ctx, empty, tf0, cam2, mp)
    finally:
        ctx.set_option(fvn.OPT_MARCH_COUNT_SHADOW, 0)
    _, ns_primary = run_march(ctx, empty, tf0, cam2, mp)
    assert np.all(out[0] == np.float32(0.1)) and np.all(out[2] == np.float32(0.3)) and np.all(out[3] == 0.0)
    assert ns == ns_primary > 0          # samples, but no shadow-ray samples
