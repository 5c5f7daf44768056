"""GPU parity of the FP32 training kernels (forward and backward) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import net as onet

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


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


@pytest.mark.parametrize("k,ca,cb,cout,h,w", [(3, 5, 0, 16, 20, 37), (3, 16, 32, 16, 17, 16), (1, 16, 0, 29, 9, 40),
                                             (3, 64, 32, 32, 8, 8), (3, 3, 0, 5, 1, 1)])
def test_conv_forward_backward(fvn, k, ca, cb, cout, h, w):
    rng = np.random.default_rng(k * 100 + ca + cout)
    n = 2
    xa = rng.normal(size=(n, ca, h, w))
    xb = rng.normal(size=(n, cb, h, w)) if cb else None
    wt = rng.normal(size=(cout, ca + cb, k, k)) * 0.2
    b = rng.normal(size=cout) * 0.1
    x = xa if xb is None else np.concatenate([xa, xb], 1)
    z = onet.conv2d(x, wt, b)
    y_ref = np.maximum(z, 0)
    y = torch.empty(n, cout, h, w, device=DEV)
    fvn.conv_fwd(T(xa), None if xb is None else T(xb), T(wt), T(b), True, y)
    torch.cuda.synchronize()
    assert np.abs(N(y) - y_ref).max() < 1e-4
    gy = rng.normal(size=y_ref.shape)
    gz = gy * (z > 0)
    gx_ref, gw_ref, gb_ref = onet.conv2d_backward(x, wt, gz)
    gxa = torch.empty(n, ca, h, w, device=DEV)
    gxb = torch.empty(n, cb, h, w, device=DEV) if cb else None
    gw = torch.empty_like(T(wt))
    gb = torch.empty(cout, device=DEV)
    fvn.conv_bwd(T(xa), None if xb is None else T(xb), T(wt), T(gy), y, gxa, gxb, gw, gb)
    torch.cuda.synchronize()
    gx = N(gxa) if gxb is None else np.concatenate([N(gxa), N(gxb)], 1)
    # y > 0 on the GPU and z > 0 in FP64 agree except within rounding of 0
    assert np.abs(gx - gx_ref).max() < 1e-3 * max(1.0, np.abs(gx_ref).max())
    assert np.abs(N(gw) - gw_ref).max() < 1e-3 * max(1.0, np.abs(gw_ref).max())
    assert np.abs(N(gb) - gb_ref).max() < 1e-3 * max(1.0, np.abs(gb_ref).max())


def test_pool_upsample_and_adjoints(fvn):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 10, 14))
    y = torch.empty(2, 3, 5, 7, device=DEV)
    fvn.avgpool2_fwd(T(x), y)
    g = rng.normal(size=(2, 3, 5, 7))
    gx = torch.empty(2, 3, 10, 14, device=DEV)
    fvn.avgpool2_bwd(T(g), gx)
    u = torch.empty(2, 3, 20, 28, device=DEV)
    fvn.upsample2_fwd(T(x), u)
    gu = rng.normal(size=(2, 3, 20, 28))
    gux = torch.empty(2, 3, 10, 14, device=DEV)
    fvn.upsample2_bwd(T(gu), gux)
    torch.cuda.synchronize()
    assert np.abs(N(y) - onet.avgpool2(x)).max() < 1e-5
    assert np.abs(N(gx) - onet.avgpool2_backward(g)).max() < 1e-5
    assert np.abs(N(u) - onet.upsample2(x)).max() < 1e-5
    assert np.abs(N(gux) - onet.upsample2_backward(gu, 10, 14)).max() < 1e-4


def test_kp_blend_forward_backward(fvn):
    rng = np.random.default_rng(2)
    n, h, w = 2, 11, 13
    head = rng.normal(size=(n, 29, h, w))
    sp = np.zeros((n, 5, h, w))
    m = rng.uniform(size=(n, h, w)) < 0.3
    sp[:, 0:4] = rng.uniform(size=(n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    ref, cache = onet.kp_blend(head, sp)
    out = torch.empty(n, 3, h, w, device=DEV)
    fvn.kp_blend_fwd(T(head), T(sp), out)
    g = rng.normal(size=(n, 3, h, w))
    gh_ref = onet.kp_blend_backward(g, cache)
    gh = torch.empty(n, 29, h, w, device=DEV)
    fvn.kp_blend_bwd(T(head), T(sp), T(g), gh)
    torch.cuda.synchronize()
    assert np.abs(N(out) - ref).max() < 1e-5
    assert np.abs(N(gh) - gh_ref).max() < 1e-5


def test_loss_and_adam(fvn):
    rng = np.random.default_rng(3)
    p = rng.uniform(size=(2, 3, 9, 12))
    t = rng.uniform(size=(2, 3, 9, 12))
    lref, gref = onet.loss_l1_grad(p, t)
    loss = torch.zeros(1, device=DEV)
    g = torch.empty(2, 3, 9, 12, device=DEV)
    fvn.loss_l1grad(T(p), T(t), 1.0, loss, g)
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - lref) < 1e-5
    assert np.abs(N(g) - gref).max() < 1e-7
    prm = rng.normal(size=1000)
    grad = rng.normal(size=1000)
    m = np.zeros(1000)
    v = np.zeros(1000)
    tp, tg, tm, tv = T(prm), T(grad), T(m), T(v)
    for s in range(1, 4):
        prm, m, v = onet.adam_step(prm, grad, m, v, s)
        fvn.adam_step(tp, tg, tm, tv, s)
    torch.cuda.synchronize()
    assert np.abs(N(tp) - prm).max() < 1e-6


def test_whole_network_forward_and_gradients_match_oracle(fvn):
    """train.forward + backward through the autograd shims (every step in the
    library's FP32 kernels: tc=False) against the FP64 oracle network."""
    from paper_2209_09965_gb300 import train, workloads as wl
    rng = np.random.default_rng(7)
    flat = wl.net_weights(5)
    flat = (flat + rng.normal(size=flat.size).astype(np.float32) * 0.01).astype(np.float32)
    n, h, w = 2, 16, 24
    sp = np.zeros((n, 5, h, w), np.float32)
    m = rng.uniform(size=(n, h, w)) < 0.3
    sp[:, 0:4] = rng.uniform(size=(n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    tgt = rng.uniform(size=(n, 3, h, w)).astype(np.float32)
    P = train.Params(flat, DEV)
    pred = train.forward(P, T(sp), tc=False)
    loss = train._Loss.apply(pred, T(tgt), 1.0)
    P.g.zero_()
    loss.backward()
    torch.cuda.synchronize()
    params = onet.unpack(flat)
    ref, cache = onet.forward(params, sp.astype(np.float64), return_cache=True)
    lref, gref = onet.loss_l1_grad(ref, tgt)
    assert np.abs(N(pred) - ref).max() < 1e-4
    assert abs(float(loss.item()) - lref) < 1e-5
    grads = onet.backward(params, cache, gref)
    g = P.g.cpu().numpy().astype(np.float64)
    ref_g = onet.pack(grads)
    scale = np.abs(ref_g).max()
    assert np.abs(g - ref_g).max() < 2e-3 * scale


def test_training_reduces_loss(fvn):
    from paper_2209_09965_gb300 import train
    _, log = train.train(steps=60, nvol=2, vol_n=64, log_every=20, batch=4)
    first, last = log[0][1], log[-1][1]
    assert last < first
