"""GPU: the training step's 3x3 layers on the tensor cores (forward and data
gradient as tcgen05 implicit GEMMs, BF16 operands, FP32 accumulation)
against the FP64 oracle, layer by layer and through the whole network's
forward and backward, through the C ABI.  The bars are those of 16-bit
operands: BF16 keeps 8 significant bits, so a layer's output differs from the
FP64 one by up to ~1 % of its scale."""
import numpy as np
import pytest
import torch

from oracle import net as onet

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
LAYER_TOL = 1.5e-2      # max-abs error / max |reference|, one layer
NET_TOL = 5e-2          # the same for the whole network's parameter gradients


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


# every 3x3 layer shape of the 16/32/64 network (input a + input b -> output),
# on ragged frames that span several tiles
@pytest.mark.parametrize("ca,cb,cout,h,w", [(5, 0, 16, 19, 150), (8, 0, 16, 9, 40), (16, 0, 16, 12, 131),
                                           (16, 0, 32, 10, 64), (32, 0, 32, 7, 129), (32, 0, 64, 6, 33),
                                           (64, 0, 64, 5, 20), (64, 32, 32, 9, 70), (32, 16, 16, 13, 260),
                                           (16, 0, 16, 1, 1)])
def test_tc_conv_forward_and_data_gradient(fvn, ca, cb, cout, h, w):
    rng = np.random.default_rng(ca * 7 + cb * 3 + cout)
    n = 2
    xa = rng.normal(size=(n, ca, h, w))
    xb = rng.normal(size=(n, cb, h, w)) if cb else None
    wt = rng.normal(size=(cout, ca + cb, 3, 3)) * 0.2
    b = rng.normal(size=cout) * 0.1
    x = xa if xb is None else np.concatenate([xa, xb], 1)
    z = onet.conv2d(x, wt, b)
    y_ref = np.maximum(z, 0)
    y = torch.full((n, cout, h, w), 9.0, device=DEV)
    fvn.conv3x3_fwd_bf16(T(xa), None if xb is None else T(xb), T(wt), T(b), True, y)
    fvn.train_device_status()
    assert np.abs(N(y) - y_ref).max() < LAYER_TOL * np.abs(y_ref).max()
    # data gradient through the ReLU of the FP64 forward (the saved output's mask)
    gy = rng.normal(size=y_ref.shape)
    gx_ref, _, _ = onet.conv2d_backward(x, wt, gy * (z > 0))
    gxa = torch.full((n, ca, h, w), 7.0, device=DEV)
    gxb = torch.full((n, cb, h, w), 7.0, device=DEV) if cb else None
    fvn.conv3x3_dgrad_bf16(T(gy), T(y_ref), T(wt), ca, cb, gxa, gxb)
    fvn.train_device_status()
    gx = N(gxa) if gxb is None else np.concatenate([N(gxa), N(gxb)], 1)
    assert np.abs(gx - gx_ref).max() < LAYER_TOL * np.abs(gx_ref).max()


def test_tc_conv_unsupported_shape_is_rejected(fvn):
    x = torch.zeros(1, 176, 4, 4, device=DEV)
    wt = torch.zeros(80, 176, 3, 3, device=DEV)
    y = torch.zeros(1, 80, 4, 4, device=DEV)
    with pytest.raises(fvn.FvnError, match="no tensor-core training convolution"):
        fvn.conv3x3_fwd_bf16(x, None, wt, torch.zeros(80, device=DEV), True, y)


def test_tc_whole_network_gradients_match_oracle(fvn):
    """train.forward (tc=True) + backward through the autograd shims against
    the FP64 oracle network: prediction, loss and every parameter gradient."""
    from paper_2209_09965_gb300 import train, workloads as wl
    rng = np.random.default_rng(7)
    flat = wl.net_weights(5)
    flat = (flat + rng.normal(size=flat.size).astype(np.float32) * 0.01).astype(np.float32)
    n, h, w = 2, 32, 136
    sp = np.zeros((n, 5, h, w), np.float32)
    m = rng.uniform(size=(n, h, w)) < 0.3
    sp[:, 0:4] = rng.uniform(size=(n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    tgt = rng.uniform(size=(n, 3, h, w)).astype(np.float32)
    P = train.Params(flat, DEV)
    pred = train.forward(P, T(sp), tc=True)
    loss = train._Loss.apply(pred, T(tgt), 1.0)
    P.g.zero_()
    loss.backward()
    fvn.train_device_status()
    params = onet.unpack(flat)
    ref, cache = onet.forward(params, sp.astype(np.float64), return_cache=True)
    lref, gref = onet.loss_l1_grad(ref, tgt)
    assert np.abs(N(pred) - ref).max() < 2e-2
    assert abs(float(loss.item()) - lref) < 1e-2 * abs(lref)
    ref_g = onet.pack(onet.backward(params, cache, gref))
    g = P.g.cpu().numpy().astype(np.float64)
    assert np.abs(g - ref_g).max() < NET_TOL * np.abs(ref_g).max()
    # and the FP32 path of the same step agrees with it to the same bar
    P2 = train.Params(flat, DEV)
    P2.g.zero_()
    train._Loss.apply(train.forward(P2, T(sp), tc=False), T(tgt), 1.0).backward()
    g32 = P2.g.cpu().numpy().astype(np.float64)
    assert np.abs(g - g32).max() < NET_TOL * np.abs(g32).max()


def test_tc_training_reduces_loss(fvn):
    from paper_2209_09965_gb300 import train
    _, log = train.train(steps=60, nvol=2, vol_n=64, log_every=20, batch=4)
    assert log[-1][1] < log[0][1]
    fvn.train_device_status()


# weight and bias gradients (a GEMM over the pixels): every layer shape, ragged
# widths across several 128-pixel segments, and the ReLU mask from the forward
@pytest.mark.parametrize("ca,cb,cout,h,w", [(5, 0, 16, 19, 150), (16, 0, 32, 10, 64), (32, 0, 64, 6, 33),
                                           (64, 0, 64, 5, 20), (64, 32, 32, 9, 70), (32, 16, 16, 13, 260),
                                           (48, 0, 48, 7, 129), (32, 0, 96, 4, 300), (16, 0, 16, 1, 1)])
def test_tc_conv_weight_gradient(fvn, ca, cb, cout, h, w):
    rng = np.random.default_rng(ca * 5 + cb + cout * 11)
    n = 2
    xa = rng.normal(size=(n, ca, h, w))
    xb = rng.normal(size=(n, cb, h, w)) if cb else None
    x = xa if xb is None else np.concatenate([xa, xb], 1)
    z = rng.normal(size=(n, cout, h, w))
    gy = rng.normal(size=z.shape)
    y = np.maximum(z, 0)
    _, gw_ref, gb_ref = onet.conv2d_backward(x, np.zeros((cout, ca + cb, 3, 3)), gy * (z > 0))
    gw = torch.full((cout, ca + cb, 3, 3), 5.0, device=DEV)
    gb = torch.full((cout,), 5.0, device=DEV)
    fvn.conv3x3_wgrad_bf16(T(xa), None if xb is None else T(xb), T(gy), T(y), gw, gb)
    fvn.train_device_status()
    assert np.abs(N(gw) - gw_ref).max() < LAYER_TOL * np.abs(gw_ref).max()
    assert np.abs(N(gb) - gb_ref).max() < LAYER_TOL * max(np.abs(gb_ref).max(), 1e-6)
    # without a ReLU mask
    _, gw2, gb2 = onet.conv2d_backward(x, np.zeros((cout, ca + cb, 3, 3)), gy)
    fvn.conv3x3_wgrad_bf16(T(xa), None if xb is None else T(xb), T(gy), None, gw, gb)
    fvn.train_device_status()
    assert np.abs(N(gw) - gw2).max() < LAYER_TOL * np.abs(gw2).max()
    assert np.abs(N(gb) - gb2).max() < LAYER_TOL * max(np.abs(gb2).max(), 1e-6)


# the 1x1 head fused with the kernel-prediction blend, forward and backward
# (FP32 throughout): sparse masks thin enough that some 5x5 neighbourhoods
# are empty (the direct-prediction branch), ragged frames across several
# 256-pixel tiles
@pytest.mark.parametrize("n,h,w,density", [(2, 37, 300, 0.05), (1, 8, 8, 0.5), (3, 1, 1, 1.0), (1, 64, 96, 0.0)])
def test_fused_head_and_blend(fvn, n, h, w, density):
    rng = np.random.default_rng(h * 31 + w)
    x = rng.normal(size=(n, 16, h, w))
    wt = rng.normal(size=(29, 16, 1, 1)) * 0.3
    b = rng.normal(size=29) * 0.1
    sparse = rng.uniform(size=(n, 5, h, w))
    sparse[:, 4] = (rng.uniform(size=(n, h, w)) < density).astype(np.float64)
    sparse[:, 0:4] *= sparse[:, 4:5]
    head_ref = onet.conv2d(x, wt, b)
    out_ref, cache = onet.kp_blend(head_ref, sparse)
    gout = rng.normal(size=out_ref.shape)
    gh = onet.kp_blend_backward(gout, cache)
    gx_ref, gw_ref, gb_ref = onet.conv2d_backward(x, wt, gh)
    head = torch.full((n, 29, h, w), 3.0, device=DEV)
    out = torch.full((n, 3, h, w), 3.0, device=DEV)
    fvn.head_kp_fwd(T(x), T(wt), T(b), T(sparse), head, out)
    gx = torch.full((n, 16, h, w), 3.0, device=DEV)
    gw = torch.full((29, 16, 1, 1), 3.0, device=DEV)
    gb = torch.full((29,), 3.0, device=DEV)
    fvn.head_kp_bwd(T(x), head, T(sparse), T(wt), T(gout), gx, gw, gb)
    torch.cuda.synchronize()
    tol = 1e-4
    for got, ref in ((head, head_ref), (out, out_ref), (gx, gx_ref), (gw, gw_ref), (gb, gb_ref)):
        assert np.abs(N(got) - ref).max() <= tol * max(np.abs(ref).max(), 1.0)


def test_graphed_step_matches_eager_steps(fvn):
    """A training step captured as a CUDA graph and replayed gives the eager
    steps' parameters (up to the order of the weight gradients' atomics) and
    its loss falls over the replays; Adam's step count advances on the
    device."""
    from paper_2209_09965_gb300 import train, workloads as wl
    rng = np.random.default_rng(3)
    flat = wl.net_weights(5)
    xs = torch.from_numpy(rng.uniform(size=(2, 5, 32, 48)).astype(np.float32)).to(DEV)
    xs[:, 4] = (xs[:, 4] < 0.3).float()
    ys = torch.from_numpy(rng.uniform(size=(2, 3, 32, 48)).astype(np.float32)).to(DEV)
    fwd = lambda P, x: train.forward(P, x, tc=True)  # noqa: E731
    Pe = train.Params(flat, DEV)
    losses_e = []
    for _ in range(4):
        Pe.g.zero_()
        loss = train._Loss.apply(fwd(Pe, xs), ys, 1.0)
        loss.backward()
        Pe.adam(1e-3)
        losses_e.append(float(loss.detach()))
    Pg = train.Params(flat, DEV)
    step = train.GraphedStep(Pg, xs, ys, fwd, lr=1e-3)
    assert torch.equal(Pg.p.detach(), train.Params(flat, DEV).p.detach())   # building left the weights alone
    losses_g = [float(step(xs, ys)) for _ in range(4)]
    fvn.train_device_status()
    assert Pg.step == 4 and int(step.step_t) == 4
    np.testing.assert_allclose(losses_g, losses_e, rtol=2e-3)
    assert np.abs(N(Pg.p) - N(Pe.p)).max() < 2e-3
    assert losses_g[-1] < losses_g[0]


def test_new_training_entry_points_reject_bad_arguments(fvn):
    """The tensor-core weight gradient and the fused head refuse what they
    cannot compute, before launching anything."""
    x = torch.zeros(1, 16, 4, 4, device=DEV)
    gy = torch.zeros(1, 100, 4, 4, device=DEV)
    gw = torch.zeros(100, 16, 3, 3, device=DEV)
    gb = torch.zeros(100, device=DEV)
    with pytest.raises(fvn.FvnError, match="no tensor-core weight gradient"):
        fvn.conv3x3_wgrad_bf16(x, None, gy, None, gw, gb)
    wt = torch.zeros(29, 16, 1, 1, device=DEV)
    b = torch.zeros(29, device=DEV)
    sp = torch.zeros(1, 5, 4, 4, device=DEV)
    head = torch.zeros(1, 29, 4, 4, device=DEV)
    out = torch.zeros(1, 3, 4, 4, device=DEV)
    empty = torch.zeros(0, 16, 4, 4, device=DEV)
    with pytest.raises(fvn.FvnError, match="null tensor|bad sizes"):   # an empty tensor has no storage
        fvn.head_kp_fwd(empty, wt, b, sp, head, out)
    step = torch.zeros(1, dtype=torch.int32, device=DEV)
    p = torch.zeros(8, device=DEV)
    with pytest.raises(TypeError):
        fvn.adam_step_dev(p, p, p, p, step.float())   # the step count is an int32 tensor
    fvn.train_device_status()


def test_tensor_core_training_matches_fp32_training_quality(fvn):
    """BF16 operands in training cost no reconstruction quality: the same
    network trained for the same steps from the same seed on the same
    self-rendered pairs, once with its 3x3 layers on the tensor cores and once
    on the FP32 kernels, reaches the same PSNR on held-out frames (a volume
    seed neither run saw) within 0.5 dB."""
    import math
    from paper_2209_09965_gb300 import train, workloads as wl
    ws = {}
    for name, tc in (("tc", True), ("fp32", False)):
        ws[name], _ = train.train(steps=1000, batch=8, lr=1e-3, seed=100, nvol=8, vol_n=256, log_every=1000,
                                  lr_final=1e-4, device=DEV, tc=tc)
    W, H = 960, 540
    vol_np, tf_np, _, _, mp = wl.foveated_1080p_workload(seed=7, frame=0)
    vol, tf = T(vol_np), T(tf_np)
    ctx = fvn.Context()
    scores = {k: [] for k in ws}
    try:
        for f in (0, 16, 40):
            cam = wl.orbit_camera(7, f, width=W, height=H, radius_factor=(0.85, 1.75))
            fov = wl.Foveation(focal_px=wl.focal_point(7, f, W, H), seed=7, frame=f)
            dense = torch.empty(5, H, W, device=DEV)
            sp = torch.empty(5, H, W, device=DEV)
            mask = torch.empty(H, W, dtype=torch.uint8, device=DEV)
            ids = torch.empty(W * H, dtype=torch.int32, device=DEV)
            cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
            ctx.march(vol, tf, cam, mp, dense)
            ctx.make_mask(fov, W, H, mask, ids, cnt)
            ctx.march(vol, tf, cam, mp, sp, ids=ids, count=cnt)
            for k, w in ws.items():
                c = fvn.Context()
                c.load_weights(w)
                out = torch.empty(3, H, W, device=DEV)
                c.reconstruct(sp, W, H, out)
                torch.cuda.synchronize()
                mse = torch.mean((out.clamp(0, 1) - dense[0:3].clamp(0, 1)) ** 2).item()
                scores[k].append(-10 * math.log10(max(mse, 1e-20)))
                c.close()
    finally:
        ctx.close()
    mean = {k: float(np.mean(v)) for k, v in scores.items()}
    print("held-out PSNR dB", mean)
    assert abs(mean["tc"] - mean["fp32"]) < 0.5
    assert min(mean.values()) > 25.0
