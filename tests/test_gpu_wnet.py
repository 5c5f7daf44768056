"""GPU parity of the two-stage network (direct prediction D, kernel
prediction K applied to D's output at several scales) against the FP64
oracle: the per-pixel filter and the decoder join with their gradients, the
whole network through fvn_reconstruct_wnet (the paper's widths and small
ones, ragged frames), its training step, a full-size property, and the
argument checks."""
import numpy as np
import pytest
import torch

from oracle import net as onet
from oracle import wnet as W
from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")
TINY = ((3, 5), 6, (4, 5))


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV)


def N(t):
    return t.detach().cpu().numpy().astype(np.float64)


def sparse_input(n, h, w, seed, density=0.25):
    rng = np.random.default_rng(seed)
    sp = np.zeros((n, 5, h, w), np.float32)
    m = rng.uniform(size=(n, h, w)) < density
    sp[:, 0:4] = rng.uniform(0.05, 0.95, (n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    return sp


@pytest.mark.parametrize("n,h,w", [(2, 7, 13), (1, 1, 1), (1, 64, 96), (3, 33, 2)])
def test_filter_matches_oracle(fvn, n, h, w):
    rng = np.random.default_rng(h * w)
    img = rng.normal(size=(n, 3, h, w)).astype(np.float32)
    lg = (rng.normal(size=(n, 9, h, w)) * 3).astype(np.float32)
    go = rng.normal(size=(n, 3, h, w)).astype(np.float32)
    out = torch.full((n, 3, h, w), 7.0, device=DEV)
    fvn.filter3_fwd(T(img), T(lg), out)
    ref, cache = W.filter3(img.astype(np.float64), lg.astype(np.float64))
    assert np.abs(N(out) - ref).max() < 2e-5
    gi, gl = torch.full_like(out, 7.0), torch.full((n, 9, h, w), 7.0, device=DEV)
    fvn.filter3_bwd(T(img), T(lg), T(go), gi, gl)
    rgi, rgl = W.filter3_backward(go.astype(np.float64), cache)
    assert np.abs(N(gi) - rgi).max() < 2e-5
    assert np.abs(N(gl) - rgl).max() < 2e-5


@pytest.mark.parametrize("n,h,w", [(2, 6, 10), (1, 2, 2), (1, 64, 96), (2, 130, 4)])
def test_join_matches_oracle(fvn, n, h, w):
    rng = np.random.default_rng(h + w)
    j = rng.normal(size=(n, 3, h, w)).astype(np.float32)
    y = rng.normal(size=(n, 3, h // 2, w // 2)).astype(np.float32)
    z = (rng.normal(size=(n, 1, h, w)) * 2).astype(np.float32)
    gx = rng.normal(size=(n, 3, h, w)).astype(np.float32)
    x = torch.full((n, 3, h, w), 7.0, device=DEV)
    fvn.wnet_join_fwd(T(j), T(y), T(z), x)
    ref, cache = W.join(j.astype(np.float64), y.astype(np.float64), z[:, 0].astype(np.float64))
    assert np.abs(N(x) - ref).max() < 2e-5
    gj, gy, gz = torch.full_like(x, 7.0), torch.full((n, 3, h // 2, w // 2), 7.0, device=DEV), \
        torch.full((n, 1, h, w), 7.0, device=DEV)
    fvn.wnet_join_bwd(T(j), T(y), T(z), T(gx), gj, gy, gz)
    rj, ry, rz = W.join_backward(gx.astype(np.float64), cache)
    assert np.abs(N(gj) - rj).max() < 2e-5
    assert np.abs(N(gy) - ry).max() < 2e-5
    assert np.abs(N(gz)[:, 0] - rz).max() < 2e-5


@pytest.mark.parametrize("cfg,h,w,seed", [
    (TINY, 12, 16, 0),
    (TINY, 13, 7, 1),            # ragged: padded to 16 x 8 and cropped
    (TINY, 1, 1, 2),
    (((8,), 4, (6,)), 9, 11, 3),
    (wl.WNET_SLIM, 45, 70, 4),
    (wl.WNET_PAPER, 21, 37, 5),
    (((4, 5, 6, 7), 9, (3, 4, 5, 6)), 40, 48, 6),
])
def test_reconstruct_matches_oracle(fvn, cfg, h, w, seed):
    flat = wl.wnet_weights(cfg, seed)
    # perturb the heads so the kernels and blends are far from the initial ones
    flat = flat + np.random.default_rng(seed).normal(size=flat.size).astype(np.float32) * 0.05
    sp = sparse_input(1, h, w, seed)[0]
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        rgb = torch.full((3, h, w), 7.0, device=DEV)
        c.reconstruct_wnet(T(sp), w, h, rgb)
        torch.cuda.synchronize()
        ref = W.forward(W.unpack(flat, cfg), cfg, sp.astype(np.float64))
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(N(rgb) - ref).max() < 1e-4 * scale
        again = torch.empty_like(rgb)
        c.reconstruct_wnet(T(sp), w, h, again)
        torch.cuda.synchronize()
        assert torch.equal(rgb, again)
        c.device_status()
    finally:
        c.close()


def test_training_composition_equals_the_library_pass(fvn):
    """train.wnet_forward launches the same kernels in the same order as
    fvn_reconstruct_wnet: identical output on a frame that needs no padding."""
    from paper_2209_09965_gb300 import train
    cfg = wl.WNET_SLIM
    flat = wl.wnet_weights(cfg, 11)
    sp = sparse_input(1, 64, 96, 12)
    P = train.Params(flat, DEV, wl.wnet_layers(cfg))
    with torch.no_grad():
        out = train.wnet_forward(P, T(sp), cfg)
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        rgb = torch.empty(3, 64, 96, device=DEV)
        c.reconstruct_wnet(T(sp[0]), 96, 64, rgb)
        torch.cuda.synchronize()
        assert torch.equal(out[0], rgb)
    finally:
        c.close()


def test_training_step_matches_oracle(fvn):
    from paper_2209_09965_gb300 import train
    cfg = TINY
    rng = np.random.default_rng(21)
    flat = wl.wnet_weights(cfg, 21) + rng.normal(size=W.param_count(cfg)).astype(np.float32) * 0.05
    flat = flat.astype(np.float32)
    sp = sparse_input(2, 16, 24, 22)
    y = rng.uniform(size=(2, 3, 16, 24)).astype(np.float32)
    P = train.Params(flat, DEV, wl.wnet_layers(cfg))
    out = train.wnet_forward(P, T(sp), cfg)
    loss = train._Loss.apply(out, T(y), 1.0)
    P.g.zero_()
    loss.backward()
    torch.cuda.synchronize()
    params = W.unpack(flat, cfg)
    ref, cache = W.forward(params, cfg, sp.astype(np.float64), return_cache=True)
    lv, g = onet.loss_l1_grad(ref, y)
    assert np.abs(N(out) - ref).max() < 1e-4
    assert abs(float(loss.item()) - lv) < 1e-5
    grads = W.pack(W.backward(params, cache, g), cfg)
    got = N(P.g)
    assert np.abs(got - grads).max() < 2e-3 * np.abs(grads).max()


def test_full_size_constant_image(fvn):
    """The paper's widths at 1920 x 1080 in the benchmark's launch
    configuration: with D's output layer set to a constant, K's filters and
    joins must return that constant at every pixel (the filters are
    normalised, the joins add up(pooled difference) = 0)."""
    cfg = wl.WNET_PAPER
    flat = wl.wnet_weights(cfg, 5) + np.random.default_rng(5).normal(size=W.param_count(cfg)).astype(np.float32) * 0.05
    flat = flat.astype(np.float32)
    layers = wl.wnet_layers(cfg)
    off = 0
    for name, ci, co, k in layers:
        if name == "d_out":
            flat[off:off + co * ci * k * k] = 0.0
            flat[off + co * ci * k * k:off + co * ci * k * k + co] = (0.25, 0.5, 0.75)
        off += co * ci * k * k + co
    w, h = 1920, 1080
    sp = torch.from_numpy(sparse_input(1, h, w, 9)[0]).to(DEV)
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        rgb = torch.full((3, h, w), 7.0, device=DEV)
        c.reconstruct_wnet(sp, w, h, rgb)
        torch.cuda.synchronize()
        ref = torch.tensor([0.25, 0.5, 0.75], device=DEV)[:, None, None]
        assert float((rgb - ref).abs().max()) < 1e-5
        c.device_status()
    finally:
        c.close()


def test_argument_errors(fvn):
    c = fvn.Context()
    try:
        rgb = torch.empty(3, 8, 8, device=DEV)
        sp = torch.zeros(5, 8, 8, device=DEV)
        with pytest.raises(fvn.FvnError, match="FVN_ERR_STATE"):
            c.reconstruct_wnet(sp, 8, 8, rgb)
        with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
            c.load_wnet_weights(TINY, np.zeros(10, np.float32))
        bad = wl.wnet_weights(TINY, 0)
        bad[3] = np.nan
        with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
            c.load_wnet_weights(TINY, bad)
        with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
            c.load_wnet_weights(((4,) * 5, 4, (4,) * 5), np.zeros(10, np.float32))
        c.load_wnet_weights(TINY, wl.wnet_weights(TINY, 0))
        with pytest.raises(fvn.FvnError, match="FVN_ERR_ARG"):
            c.reconstruct_wnet(sp, 0, 8, rgb)
        c.reconstruct_wnet(sp, 8, 8, rgb)
        torch.cuda.synchronize()
        c.device_status()
    finally:
        c.close()


def test_training_runs(fvn):
    from paper_2209_09965_gb300 import train
    w, log = train.train(steps=10, nvol=2, vol_n=64, log_every=5, batch=2, wnet=wl.WNET_SLIM)
    assert w.size == W.param_count(wl.WNET_SLIM)
    assert all(np.isfinite(v) for _, v in log)


# The tensor-core path (FVN_OPT_WNET_TENSOR_CORES): FP16 operands and
# activations, FP32 accumulation.  Bar: 2e-2 of the output's scale against
# the FP64 oracle -- FP16 keeps 11 significant bits, and the error of some
# 30 layers in sequence stays near 1e-2 of the scale.
TC_TOL = 2e-2


@pytest.mark.parametrize("cfg,h,w,seed", [
    (wl.WNET_PAPER, 40, 48, 3),        # the paper's widths: 3x3 up to 176 input channels, 1x1 up to 176
    (wl.WNET_PAPER, 37, 131, 4),       # ragged: padded to multiples of 8, tiles across 126-pixel rows
    (wl.WNET_SLIM, 64, 96, 5),
    (((8, 16), 24, (8, 16)), 9, 300, 6),
])
def test_reconstruct_tensor_cores_matches_oracle(fvn, cfg, h, w, seed):
    flat = wl.wnet_weights(cfg, seed)
    flat = flat + np.random.default_rng(seed).normal(size=flat.size).astype(np.float32) * 0.05
    sp = sparse_input(1, h, w, seed)[0]
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        c.set_option(fvn.OPT_WNET_TENSOR_CORES, 1)
        rgb = torch.full((3, h, w), 7.0, device=DEV)
        c.reconstruct_wnet(T(sp), w, h, rgb)
        torch.cuda.synchronize()
        c.device_status()
        ref = W.forward(W.unpack(flat, cfg), cfg, sp.astype(np.float64))
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(N(rgb) - ref).max() < TC_TOL * scale
        again = torch.empty_like(rgb)
        c.reconstruct_wnet(T(sp), w, h, again)
        torch.cuda.synchronize()
        assert torch.equal(rgb, again)       # no atomics: the same result every time
    finally:
        c.close()


def test_tensor_cores_full_frame_agrees_with_fp32_path(fvn):
    """At 1080p (every tile position, 1 CTA per SM over many tiles) the
    tensor-core pass stays within the FP16 bar of the FP32 pass."""
    cfg = wl.WNET_PAPER
    flat = wl.wnet_weights(cfg, 3)
    h, w = 1080, 1920
    sp = T(sparse_input(1, h, w, 9, density=0.1)[0])
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        ref = torch.empty(3, h, w, device=DEV)
        c.reconstruct_wnet(sp, w, h, ref)
        c.set_option(fvn.OPT_WNET_TENSOR_CORES, 1)
        out = torch.empty(3, h, w, device=DEV)
        c.reconstruct_wnet(sp, w, h, out)
        torch.cuda.synchronize()
        c.device_status()
        scale = max(1.0, float(ref.abs().max()))
        assert float((out - ref).abs().max()) < TC_TOL * scale
    finally:
        c.close()


def test_tensor_cores_reject_unsupported_widths(fvn):
    c = fvn.Context()
    try:
        c.load_wnet_weights(TINY, wl.wnet_weights(TINY, 1))
        c.set_option(fvn.OPT_WNET_TENSOR_CORES, 1)
        rgb = torch.empty(3, 8, 8, device=DEV)
        with pytest.raises(fvn.FvnError, match="multiple of 8"):
            c.reconstruct_wnet(torch.zeros(5, 8, 8, device=DEV), 8, 8, rgb)
    finally:
        c.close()


def test_tensor_core_option_is_checked(fvn):
    c = fvn.Context()
    try:
        with pytest.raises(fvn.FvnError, match="two-stage tensor-core option"):
            c.set_option(fvn.OPT_WNET_TENSOR_CORES, 2)
    finally:
        c.close()


@pytest.mark.parametrize("cfg,h,w,seed", [
    (wl.WNET_PAPER, 40, 48, 3),
    (wl.WNET_PAPER, 37, 131, 4),       # ragged: padded frame, tiles across 126- and 128-pixel rows
    (wl.WNET_SLIM, 64, 96, 5),
    (((8, 16), 24, (8, 16)), 9, 300, 6),   # a 24-channel coarse input (3 chunks) keeps the separate pass
    (wl.WNET_PAPER, 1080, 1920, 7),
])
def test_fused_upsampling_equals_the_separate_pass(fvn, cfg, h, w, seed):
    """The decoder convolutions that up-sample their coarse input themselves
    (FVN_OPT_WNET_FUSED_UPSAMPLING = 1, the default) give the same bits as
    the separate up-sampling pass: the same interpolation, operation for
    operation, only computed in shared memory."""
    flat = wl.wnet_weights(cfg, seed)
    flat = flat + np.random.default_rng(seed).normal(size=flat.size).astype(np.float32) * 0.05
    sp = T(sparse_input(1, h, w, seed, density=0.1)[0])
    c = fvn.Context()
    try:
        c.load_wnet_weights(cfg, flat)
        c.set_option(fvn.OPT_WNET_TENSOR_CORES, 1)
        fused = torch.full((3, h, w), 7.0, device=DEV)
        c.reconstruct_wnet(sp, w, h, fused)
        c.set_option(fvn.OPT_WNET_FUSED_UPSAMPLING, 0)
        sep = torch.full((3, h, w), -7.0, device=DEV)
        c.reconstruct_wnet(sp, w, h, sep)
        torch.cuda.synchronize()
        c.device_status()
        assert torch.equal(fused, sep)
        assert bool(torch.isfinite(fused).all())
    finally:
        c.close()


def test_fused_upsampling_option_is_checked(fvn):
    c = fvn.Context()
    try:
        with pytest.raises(fvn.FvnError, match="fused up-sampling option"):
            c.set_option(fvn.OPT_WNET_FUSED_UPSAMPLING, 2)
    finally:
        c.close()
