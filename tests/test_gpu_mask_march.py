"""GPU parity: fused mask + compaction (bit-exact) and the ray march
(1e-4 max-abs) against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import mask as omask
from oracle import march as om
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
    c.close()


def gpu_mask(ctx, fov, w, h):
    dev = torch.device("cuda")
    mask = torch.full((h, w), 7, dtype=torch.uint8, device=dev)
    ids = torch.full((w * h,), -1, dtype=torch.int32, device=dev)
    count = torch.full((1,), -5, dtype=torch.int32, device=dev)
    ctx.make_mask(fov, w, h, mask, ids, count)
    torch.cuda.synchronize()
    n = int(count.item())
    return mask.cpu().numpy(), ids[:n].cpu().numpy(), n, ids.cpu().numpy()


@pytest.mark.parametrize("w,h,seed,frame,fp", [
    (1920, 1080, 2, 0, (960.0, 540.0)),
    (1920, 1080, 2, 17, (500.5, 300.25)),
    (1920, 1080, 99, 63, (1600.0, 900.0)),
    (1280, 720, 4, 5, (-20.0, 800.0)),          # focal point outside: clamped
    (3840, 2160, 7, 1, (1000.0, 1000.0)),
    (97, 61, 1, 2, (40.0, 20.0)),               # ragged: not a multiple of the 32 x 8 tile
    (1, 1, 3, 3, (0.5, 0.5)),
    (1, 300, 3, 4, (0.5, 150.0)),
    (333, 1, 3, 4, (100.0, 0.5)),
])
def test_mask_bit_exact(ctx, fvn, w, h, seed, frame, fp):
    fov = wl.Foveation(focal_px=fp, seed=seed, frame=frame)
    m, ids, n, ids_full = gpu_mask(ctx, fov, w, h)
    m_ref, ids_ref, cmax = omask.make_mask(w, h, fp, seed=seed, frame=frame)
    assert np.array_equal(m, m_ref)
    assert n == ids_ref.size
    assert np.array_equal(np.sort(ids), ids_ref)          # order is unspecified: compare as sets
    assert np.all(ids_full[n:] == -1)                     # nothing written past count


@pytest.mark.parametrize("pb,r0,s", [(1.0, 0.1, 0.1), (0.0, 0.0, 0.0), (0.3, 0.25, 0.05)])
def test_mask_profiles(ctx, pb, r0, s):
    fov = wl.Foveation(focal_px=(321.0, 123.0), fovea_radius=r0, falloff_sigma=s, p_base=pb, seed=8, frame=9)
    m, ids, n, _ = gpu_mask(ctx, fov, 640, 360)
    m_ref, ids_ref, _ = omask.make_mask(640, 360, fov.focal_px, r0, s, pb, seed=8, frame=9)
    assert np.array_equal(m, m_ref) and np.array_equal(np.sort(ids), ids_ref)
    if pb == 1.0:
        assert n == 640 * 360


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


def test_march_dense_small_blobs(ctx):
    vol, tf, cam, mp = wl.dense_small_workload(seed=1)
    out, ns = run_march(ctx, vol, tf, cam, mp)
    err, namb = march_parity(vol, tf, cam, mp, out)
    _, amb, ns_ref = om.march(vol, tf, cam, mp)
    assert abs(ns - ns_ref) <= 2 * max(1, namb)
    assert np.all(out[4] == 1.0)


@pytest.mark.parametrize("shading", [0, 1])
@pytest.mark.parametrize("frame", [0, 21])
def test_march_dense_small_blobs_frames(ctx, shading, frame):
    vol, tf, cam, mp = wl.dense_small_workload(seed=1, frame=frame)
    mp = wl.MarchParams(shading=shading)
    out, _ = run_march(ctx, vol, tf, cam, mp)
    march_parity(vol, tf, cam, mp, out)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
def test_march_volume_dtypes(ctx, dtype):
    base = wl.value_noise_volume(40, seed=3, base_spacing=8).numpy()
    vol = {"u8": np.round(base * 255).astype(np.uint8), "u16": np.round(base * 65535).astype(np.uint16),
           "f16": base.astype(np.float16), "f32": base.astype(np.float32)}[dtype]
    vol_t = vol.view(np.int16) if dtype == "u16" else vol
    tf = wl.transfer_function(4, alpha_max=0.15)
    cam = wl.orbit_camera(3, 2, width=72, height=40)
    mp = wl.MarchParams(shading=1)
    out, _ = run_march(ctx, vol_t, tf, cam, mp)
    march_parity(vol, tf, cam, mp, out)


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2), (4, 3)])
def test_march_tiny_grids_random_cameras(ctx, n, seed):
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0, 1, (n, n + 1, n)).astype(np.float32)
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rng.uniform(0, 1, 3)
    tf[:, 0] = np.linspace(0.1, 0.9, 256)
    tf[:, 3] = np.linspace(0.0, 0.6, 256)
    for k in range(4):
        v = rng.normal(size=3)
        r = [1.6, 0.3, 0.05, 2.5][k]           # outside, inside, near centre, far
        eye = tuple(r * v / np.linalg.norm(v))
        cam = wl.Camera(eye=eye, target=(0.02, -0.03, 0.01), up=(0, 1, 0), fov_y_deg=60.0, width=13, height=9)
        mp = wl.MarchParams(0.5, 0.95, (0.1, 0.2, 0.3), k % 2)
        out, _ = run_march(ctx, vol, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)


def test_march_sparse_1080p_full_frame(ctx):
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=0)
    _, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    perm = np.random.default_rng(0).permutation(ids)      # any order
    out, ns = run_march(ctx, vol, tf, cam, mp, ids=perm)
    err, namb = march_parity(vol, tf, cam, mp, out, ids=ids)
    flat = out.reshape(5, -1)
    rest = np.setdiff1d(np.arange(1920 * 1080), ids)
    assert np.all(flat[:, rest] == 0.0)
    assert np.all(flat[4, ids] == 1.0)


def test_march_dense_1080p_sampled(ctx):
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=3, frame=5)
    out, ns = run_march(ctx, vol, tf, cam, mp)
    sample = np.sort(np.random.default_rng(1).choice(1920 * 1080, 60000, replace=False)).astype(np.int32)
    march_parity(vol, tf, cam, mp, out, ids=sample)
    assert ns > 0


def test_march_empty_id_list(ctx):
    vol, tf, cam, mp = wl.dense_small_workload(seed=1)
    out, ns = run_march(ctx, vol, tf, cam, mp, ids=np.zeros(0, np.int32))
    assert ns == 0 and np.all(out == 0.0)


def test_march_argument_errors(ctx, fvn):
    vol, tf, cam, mp = wl.dense_small_workload(seed=1)
    dev = torch.device("cuda")
    v = torch.from_numpy(vol).to(dev)
    t = torch.from_numpy(tf).to(dev)
    out = torch.zeros(5, cam.height, cam.width, device=dev)
    bad = wl.MarchParams(step_vox=0.0)
    with pytest.raises(fvn.FvnError, match="step_vox"):
        ctx.march(v, t, cam, bad, out)
    cam2 = wl.Camera(eye=(1, 1, 1), target=(1, 1, 1), up=(0, 1, 0), fov_y_deg=45, width=8, height=8)
    with pytest.raises(fvn.FvnError, match="eye equals target"):
        ctx.march(v, t, cam2, mp, out)


def test_march_masked_equals_sparse_march(ctx):
    """Naive rejection computes exactly the rays compaction computes."""
    vol, tf, cam, mp = wl.dense_small_workload(seed=1)
    cam = wl.Camera(**{**cam.__dict__, "width": 96, "height": 72})
    fov = wl.Foveation(focal_px=(40.0, 30.0), seed=3, frame=1)
    dev = torch.device("cuda")
    v = torch.from_numpy(vol).to(dev)
    t = torch.from_numpy(tf).to(dev)
    mask = torch.empty(72, 96, dtype=torch.uint8, device=dev)
    ids = torch.empty(96 * 72, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    ctx.make_mask(fov, 96, 72, mask, ids, count)
    a = torch.full((5, 72, 96), 9.0, device=dev)
    b = torch.full((5, 72, 96), 7.0, device=dev)
    na = torch.zeros(1, dtype=torch.int64, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx.march(v, t, cam, mp, a, ids=ids, count=count, nsamples=na)
    ctx.march_masked(v, t, cam, mp, mask, b, nsamples=nb)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and int(na.item()) == int(nb.item())


def run_march_masked(ctx, vol, tf, cam, mp, mask_np):
    dev = torch.device("cuda")
    v = torch.from_numpy(np.ascontiguousarray(vol)).to(dev)
    t = torch.from_numpy(tf).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(mask_np, dtype=np.uint8)).to(dev)
    out = torch.full((5, cam.height, cam.width), 123.0, dtype=torch.float32, device=dev)
    ns = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx.march_masked(v, t, cam, mp, m, out, nsamples=ns)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(ns.item())


@pytest.mark.parametrize("shading", [0, 1])
def test_march_masked_matches_oracle_small(ctx, shading):
    """Naive rejection (the paper's "Stream Compaction" comparison: a kernel
    over the whole frame whose unsampled pixels are discarded in place)
    against the oracle at the sampled pixels; the others are written 0."""
    vol, tf, cam, mp = wl.dense_small_workload(seed=1, frame=7)
    mp = wl.MarchParams(shading=shading)
    cam = wl.Camera(**{**cam.__dict__, "width": 99, "height": 70})
    m, ids, _ = omask.make_mask(99, 70, (40.0, 30.0), 0.15, 0.1, 0.2, seed=3, frame=1)
    out, ns = run_march_masked(ctx, vol, tf, cam, mp, m)
    _, namb = march_parity(vol, tf, cam, mp, out, ids=ids)
    flat = out.reshape(5, -1)
    rest = np.setdiff1d(np.arange(99 * 70), ids)
    assert np.all(flat[:, rest] == 0.0) and np.all(flat[4, ids] == 1.0)
    _, _, ns_ref = om.march(vol, tf, cam, mp, ids=ids)
    assert abs(ns - ns_ref) <= 2 * max(1, namb)


def test_march_masked_matches_oracle_1080p(ctx):
    """Naive rejection on the foveated 1080p frame: a sample of the sampled
    pixels against the oracle, every unsampled pixel 0."""
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=11)
    m, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    out, ns = run_march_masked(ctx, vol, tf, cam, mp, m)
    sample = np.sort(np.random.default_rng(5).choice(ids, 40000, replace=False)).astype(np.int32)
    march_parity(vol, tf, cam, mp, out, ids=sample)
    flat = out.reshape(5, -1)
    rest = np.setdiff1d(np.arange(1920 * 1080), ids)
    assert np.all(flat[:, rest] == 0.0) and np.all(flat[4, ids] == 1.0)


def test_march_ambiguity_margins_1080p(ctx):
    """How often FP32 takes the other side of a discontinuity, and how close
    to it.  Every sampled pixel of a foveated 1080p frame against the oracle:
    the pixels whose FP32 result differs from the oracle's beyond the bar
    must be pixels the oracle flags, within its windows (the sample count
    (t_far - t_near) / dt within 1e-3 of an integer, A within 1e-6 of the
    termination threshold at some step), and the flagged rays at most 2 % of
    the frame's.  Prints the measured figures: how
    many rays each window flags, how many actually took the other side, and
    the largest margin among those (how much of the window FP32 needed)."""
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=3)
    _, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    out, _ = run_march(ctx, vol, tf, cam, mp, ids=ids)
    ref, amb, _, mg = om.march(vol, tf, cam, mp, ids=ids, margins=True)
    g = out.reshape(5, -1)[:, ids].astype(np.float64)
    r = ref.reshape(5, -1)[:, ids]
    err = np.abs(g - r).max(axis=0)
    a = amb.reshape(-1)[ids]
    span_m = mg[0].reshape(-1)[ids]
    term_m = mg[1].reshape(-1)[ids]
    flipped = err >= 1e-4
    disc = (a & 3) != 0
    by_count = flipped & (span_m < 1e-3) & ~(term_m < 1e-6)
    by_term = flipped & (term_m < 1e-6) & ~(span_m < 1e-3)
    both = flipped & (term_m < 1e-6) & (span_m < 1e-3)
    unflagged = ~disc & ((a & 4) == 0)
    print(f"\n[ambiguity] rays {ids.size}: flagged by count {float((a & 1).astype(bool).mean()):.5f}, "
          f"by termination {float(((a & 2) != 0).mean()):.5f}, total {float(disc.mean()):.5f}; "
          f"other side taken: {int(flipped.sum())} ({float(flipped.mean()):.6f}): by count {int(by_count.sum())} "
          f"(largest count margin {float(span_m[by_count].max()) if by_count.any() else 0.0:.3e} of 1e-3), "
          f"by termination {int(by_term.sum())} (largest termination margin "
          f"{float(term_m[by_term].max()) if by_term.any() else 0.0:.3e} of 1e-6), both {int(both.sum())}; "
          f"unflagged max err {float(err[unflagged].max()):.3e}, 99.9th percentile "
          f"{float(np.percentile(err[unflagged], 99.9)):.3e}")
    # every pixel that took the other side lies inside a window of the oracle's flags
    assert np.all(disc[flipped]), "an unflagged pixel differs beyond 1e-4"
    assert float(err[unflagged].max()) < 1e-4
    assert float(disc.mean()) <= 0.02


@pytest.mark.parametrize("coop", [1, 4, 32])
def test_march_cooperative_finish_small(ctx, fvn, coop):
    """Warp-cooperative finishing of the last rays (32 samples per step,
    product-scan compositing) matches the oracle like the sequential march;
    coop = 32 marches every ray cooperatively."""
    try:
        ctx.set_option(fvn.OPT_MARCH_COOP_DENSE, coop)
        ctx.set_option(fvn.OPT_MARCH_COOP, coop)
        for shading, frame in ((0, 0), (1, 21)):
            vol, tf, cam, mp = wl.dense_small_workload(seed=1, frame=frame)
            mp = wl.MarchParams(shading=shading)
            out, ns = run_march(ctx, vol, tf, cam, mp)
            _, namb = march_parity(vol, tf, cam, mp, out)
            _, _, ns_ref = om.march(vol, tf, cam, mp)
            assert abs(ns - ns_ref) <= 2 * max(1, namb)
        # no termination (thin TF, opacity stays far below 1): every ray marches to the far side
        vol, _, cam, _ = wl.dense_small_workload(seed=1)
        tf = wl.transfer_function(5, alpha_max=0.02)
        mp = wl.MarchParams(0.5, 1.0, (0.1, 0.2, 0.3), 1)
        out, _ = run_march(ctx, vol, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)
    finally:
        ctx.set_option(fvn.OPT_MARCH_COOP_DENSE, 0)
        ctx.set_option(fvn.OPT_MARCH_COOP, 0)


@pytest.mark.parametrize("coop", [4, 32])
def test_march_cooperative_finish_sparse_1080p(ctx, fvn, coop):
    vol, tf, cam, fov, mp = wl.foveated_1080p_workload(seed=2, frame=9)
    _, ids, _ = omask.make_mask(1920, 1080, fov.focal_px, seed=fov.seed, frame=fov.frame)
    try:
        ctx.set_option(fvn.OPT_MARCH_COOP, coop)
        out, ns = run_march(ctx, vol, tf, cam, mp, ids=ids)
    finally:
        ctx.set_option(fvn.OPT_MARCH_COOP, 0)
    sample = np.sort(np.random.default_rng(2).choice(ids, 40000, replace=False)).astype(np.int32)
    march_parity(vol, tf, cam, mp, out, ids=sample)
    seq, ns_seq = run_march(ctx, vol, tf, cam, mp, ids=ids)
    assert abs(ns - ns_seq) <= 0.001 * ns_seq


@pytest.mark.parametrize("grad_volume", [0, 1])
@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
def test_march_stencil_and_gradient_volume(ctx, fvn, grad_volume, dtype):
    """Shaded marches read either the 32-voxel stencil of the padded copy or
    the gradient volume (value + central differences per voxel); both meet
    the oracle's bars, on every voxel type, dense and sparse."""
    base = wl.value_noise_volume(36, seed=9, base_spacing=8).numpy()
    vol = {"u8": np.round(base * 255).astype(np.uint8), "f16": base.astype(np.float16),
           "f32": base.astype(np.float32)}[dtype]
    tf = wl.transfer_function(6, alpha_max=0.2)
    cam = wl.orbit_camera(5, 3, width=80, height=56, radius_factor=(0.9, 1.3))
    mp = wl.MarchParams(shading=1)
    try:
        ctx.set_option(fvn.OPT_MARCH_GRADIENT_VOLUME, grad_volume)
        out, ns = run_march(ctx, vol, tf, cam, mp)
        march_parity(vol, tf, cam, mp, out)
        ids = np.arange(0, 80 * 56, 3, dtype=np.int32)
        outs, _ = run_march(ctx, vol, tf, cam, mp, ids=ids)
        march_parity(vol, tf, cam, mp, outs, ids=ids)
    finally:
        ctx.set_option(fvn.OPT_MARCH_GRADIENT_VOLUME, 1)
    _, _, ns_ref = om.march(vol, tf, cam, mp)
    assert abs(ns - ns_ref) <= max(2, ns_ref // 10000)


@pytest.mark.parametrize("shading", [0, 1, 2])
def test_volume_generation_reuses_the_prepared_copy(fvn, shading):
    """fvn_volume.generation != 0 lets the context reuse its prepared copy of
    the volume: the same frame as a fresh preparation, a copy that stays
    while the generation does (even if the caller broke the contract and
    changed the voxels), and a new preparation once the generation changes."""
    c = fvn.Context()
    try:
        vol, tf, cam, mp = wl.dense_small_workload(seed=1, frame=5)
        mp = wl.MarchParams(shading=shading)
        dev = torch.device("cuda")
        v = torch.from_numpy(np.ascontiguousarray(vol)).to(dev)
        t = torch.from_numpy(tf).to(dev)

        def march(gen):
            out = torch.zeros(5, cam.height, cam.width, device=dev)
            c.march(v, t, cam, mp, out, generation=gen)
            torch.cuda.synchronize()
            return out.clone()

        fresh = march(0)
        assert torch.equal(march(7), fresh) and torch.equal(march(7), fresh)
        v.mul_(0.5)                                   # voxels changed, generation not: the old copy is used
        assert torch.equal(march(7), fresh)
        changed = march(0)
        assert not torch.equal(changed, fresh)
        assert torch.equal(march(8), changed)         # a new generation prepares again
        march_parity(v.cpu().numpy(), tf, cam, mp, changed.cpu().numpy())
    finally:
        c.close()


def test_stage_times(fvn):
    """FVN_OPT_STAGE_TIMING: fvn_render records its stage boundaries; the
    five stage times are non-negative and add up to the frame's time."""
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        vol, tf, cam, mp = wl.dense_small_workload(seed=1, frame=2)
        mp = wl.MarchParams(shading=1)
        dev = torch.device("cuda")
        v, t = torch.from_numpy(vol).to(dev), torch.from_numpy(tf).to(dev)
        fov = wl.Foveation(focal_px=(60.0, 60.0), seed=1, frame=2)
        rgb = torch.empty(3, cam.height, cam.width, device=dev)
        with pytest.raises(fvn.FvnError, match="stage timing"):
            c.stage_times()
        c.set_option(fvn.OPT_STAGE_TIMING, 1)
        for gen in (0, 3, 3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.render(v, t, cam, fov, mp, rgb, generation=gen)
            e1.record()
            st = c.stage_times()
            torch.cuda.synchronize()
            assert set(st) == set(fvn.STAGES) and all(x >= 0.0 for x in st.values())
            assert sum(st.values()) <= e0.elapsed_time(e1) + 1e-3
        out = torch.empty(5, cam.height, cam.width, device=dev)
        c.march(v, t, cam, mp, out)                  # not a render: the last frame's times stay
        assert c.stage_times() == st
        c.set_option(fvn.OPT_STAGE_TIMING, 0)
        with pytest.raises(fvn.FvnError, match="stage timing"):
            c.stage_times()
    finally:
        c.close()
