"""Pins for the oracle network, kernel prediction, loss and optimiser --
against library routines (torch float64 on CPU), brute force, closed forms
and finite differences.  No GPU."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import metrics
from oracle import net as on
from paper_2209_09965_gb300 import workloads as wl




def T(a):
    return torch.from_numpy(np.asarray(a, np.float64))


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 2, 4, 5))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    out = on.conv2d(x, w, b)
    ref = np.zeros((1, 3, 4, 5))
    for o in range(3):
        for yy in range(4):
            for xx in range(5):
                s = b[o]
                for c in range(2):
                    for i in range(3):
                        for j in range(3):
                            sy, sx = yy + i - 1, xx + j - 1
                            if 0 <= sy < 4 and 0 <= sx < 5:
                                s += w[o, c, i, j] * x[0, c, sy, sx]
                ref[0, o, yy, xx] = s
    assert np.max(np.abs(out - ref)) < 1e-12


@pytest.mark.parametrize("k", [1, 3])
def test_conv_and_grads_match_torch(k):
    rng = np.random.default_rng(k)
    x = rng.normal(size=(2, 5, 7, 6))
    w = rng.normal(size=(4, 5, k, k))
    b = rng.normal(size=4)
    g = rng.normal(size=(2, 4, 7, 6))
    xt, wt, bt = T(x).requires_grad_(), T(w).requires_grad_(), T(b).requires_grad_()
    yt = F.conv2d(xt, wt, bt, padding=k // 2)
    yt.backward(T(g))
    assert np.max(np.abs(on.conv2d(x, w, b) - yt.detach().numpy())) < 1e-12
    gx, gw, gb = on.conv2d_backward(x, w, g)
    assert np.max(np.abs(gx - xt.grad.numpy())) < 1e-11
    assert np.max(np.abs(gw - wt.grad.numpy())) < 1e-11
    assert np.max(np.abs(gb - bt.grad.numpy())) < 1e-11


def test_pool_and_upsample_match_torch():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 6, 10))
    assert np.max(np.abs(on.avgpool2(x) - F.avg_pool2d(T(x), 2).numpy())) < 1e-14
    ref = F.interpolate(T(x), scale_factor=2, mode="bilinear", align_corners=False).numpy()
    assert np.max(np.abs(on.upsample2(x) - ref)) < 1e-14
    # adjoints
    gu = rng.normal(size=(2, 3, 12, 20))
    assert abs((on.upsample2(x) * gu).sum() - (x * on.upsample2_backward(gu, 6, 10)).sum()) < 1e-10
    gp = rng.normal(size=(2, 3, 3, 5))
    assert abs((on.avgpool2(x) * gp).sum() - (x * on.avgpool2_backward(gp)).sum()) < 1e-10


def _head_and_sparse(rng, n=1, h=9, w=11, density=0.3):
    head = rng.normal(size=(n, 29, h, w))
    sp = np.zeros((n, 5, h, w))
    m = rng.uniform(size=(n, h, w)) < density
    sp[:, 0:4] = rng.uniform(size=(n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    return head, sp


def test_kp_one_hot_is_shifted_copy():
    rng = np.random.default_rng(2)
    head, sp = _head_and_sparse(rng, density=1.0)                 # every pixel valid
    dy, dx = 1, -2
    q = (dy + 2) * 5 + (dx + 2)
    head[:, 3:28] = -1e3
    head[:, 3 + q] = 1e3
    head[:, 28] = 1e3                                             # a = 1 -> pure KP
    out, _ = on.kp_blend(head, sp)
    h, w = sp.shape[2:]
    inner = out[0, :, 0:h - dy, -dx:]                             # where p + q is inside the frame
    assert np.max(np.abs(inner - sp[0, 0:3, dy:, 0:w + dx])) < 1e-12
    head[:, 28] = -1e3                                            # a = 0 -> direct prediction
    out, _ = on.kp_blend(head, sp)
    assert np.max(np.abs(out - head[:, 0:3])) < 1e-12


def test_kp_uniform_logits_is_masked_box_filter_and_empty_window_falls_back():
    rng = np.random.default_rng(3)
    head, sp = _head_and_sparse(rng, density=0.2)
    head[:, 3:28] = 0.7
    head[:, 28] = 50.0
    out, _ = on.kp_blend(head, sp)
    a = 1 / (1 + math.exp(-50.0))
    h, w = sp.shape[2:]
    for y in range(h):
        for x in range(w):
            ys = slice(max(0, y - 2), min(h, y + 3))
            xs = slice(max(0, x - 2), min(w, x + 3))
            m = sp[0, 4, ys, xs]
            if m.sum() == 0:
                exp = head[0, 0:3, y, x]
            else:
                kp = (sp[0, 0:3, ys, xs] * m).sum(axis=(1, 2)) / m.sum()
                exp = a * kp + (1 - a) * head[0, 0:3, y, x]
            assert np.max(np.abs(out[0, :, y, x] - exp)) < 1e-12


def test_kp_blend_backward_finite_differences():
    rng = np.random.default_rng(4)
    head, sp = _head_and_sparse(rng, h=6, w=7, density=0.35)
    g = rng.normal(size=(1, 3, 6, 7))
    out, cache = on.kp_blend(head, sp)
    gh = on.kp_blend_backward(g, cache)
    eps = 1e-6
    idx = [tuple(rng.integers(0, s) for s in head.shape) for _ in range(40)]
    for i in idx:
        hp, hm = head.copy(), head.copy()
        hp[i] += eps
        hm[i] -= eps
        fd = ((on.kp_blend(hp, sp)[0] - on.kp_blend(hm, sp)[0]) * g).sum() / (2 * eps)
        assert abs(fd - gh[i]) < 1e-7 * max(1.0, abs(fd))


def _torch_forward(params, sparse):
    """The same network written with torch library layers, float64."""
    x = T(sparse)
    p = {k: (T(w), T(b)) for k, (w, b) in params.items()}

    def cbr(name, t):
        return F.relu(F.conv2d(t, p[name][0], p[name][1], padding=1))

    up = lambda t: F.interpolate(t, scale_factor=2, mode="bilinear", align_corners=False)
    e0 = cbr("enc0b", cbr("enc0a", x))
    e1 = cbr("enc1b", cbr("enc1a", F.avg_pool2d(e0, 2)))
    bt = cbr("botb", cbr("bota", F.avg_pool2d(e1, 2)))
    d1 = cbr("dec1b", cbr("dec1a", torch.cat([up(bt), e1], 1)))
    d0 = cbr("dec0b", cbr("dec0a", torch.cat([up(d1), e0], 1)))
    head = F.conv2d(d0, p["head"][0], p["head"][1])
    rgb_d, logit, zl = head[:, 0:3], head[:, 3:28], head[:, 28:29]
    wq = torch.softmax(logit, 1)
    c = F.unfold(x[:, 0:3], 5, padding=2).view(x.shape[0], 3, 25, *x.shape[2:])
    m = F.unfold(x[:, 4:5], 5, padding=2).view(x.shape[0], 25, *x.shape[2:])
    den = (wq * m).sum(1, keepdim=True)
    num = (wq[:, None] * m[:, None] * c).sum(2)
    kp = torch.where(den >= 1e-12, num / den.clamp_min(1e-300), rgb_d)
    a = torch.sigmoid(zl)
    return a * kp + (1 - a) * rgb_d


def _random_params(chans, seed):
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co, k in on.layer_table(chans):
        params[name] = (rng.normal(size=(co, ci, k, k)) * math.sqrt(2.0 / (ci * k * k)),
                        rng.normal(size=co) * 0.1)
    return params


def test_forward_matches_torch_composition():
    params = on.unpack(wl.net_weights(seed=5))
    rng = np.random.default_rng(6)
    _, sp = _head_and_sparse(rng, n=2, h=16, w=24, density=0.25)
    out = on.forward(params, sp)
    ref = _torch_forward(params, sp).numpy()
    assert np.max(np.abs(out - ref)) < 1e-11


def test_forward_pads_to_multiple_of_four():
    params = _random_params((4, 8, 8), 7)
    rng = np.random.default_rng(8)
    _, sp = _head_and_sparse(rng, n=1, h=10, w=13, density=0.4)
    out = on.forward(params, sp)
    big = np.zeros((1, 5, 12, 16))
    big[:, :, :10, :13] = sp
    ref = _torch_forward(params, big).numpy()[:, :, :10, :13]
    assert out.shape == (1, 3, 10, 13) and np.max(np.abs(out - ref)) < 1e-11


def test_backward_matches_autograd_and_finite_differences():
    chans = (4, 8, 8)
    params = _random_params(chans, 9)
    rng = np.random.default_rng(10)
    _, sp = _head_and_sparse(rng, n=2, h=8, w=8, density=0.4)
    g = rng.normal(size=(2, 3, 8, 8))
    out, cache = on.forward(params, sp, return_cache=True)
    grads = on.backward(params, cache, g)
    # autograd of the torch composition
    tp = {k: (T(w).requires_grad_(), T(b).requires_grad_()) for k, (w, b) in params.items()}
    import types
    yt = _torch_forward({k: (v[0], v[1]) for k, v in params.items()}, sp)   # value check
    assert np.max(np.abs(yt.numpy() - out)) < 1e-11
    x = T(sp)

    def fwd(pt):
        def cbr(name, t):
            return F.relu(F.conv2d(t, pt[name][0], pt[name][1], padding=1))
        up = lambda t: F.interpolate(t, scale_factor=2, mode="bilinear", align_corners=False)
        e0 = cbr("enc0b", cbr("enc0a", x))
        e1 = cbr("enc1b", cbr("enc1a", F.avg_pool2d(e0, 2)))
        bt = cbr("botb", cbr("bota", F.avg_pool2d(e1, 2)))
        d1 = cbr("dec1b", cbr("dec1a", torch.cat([up(bt), e1], 1)))
        d0 = cbr("dec0b", cbr("dec0a", torch.cat([up(d1), e0], 1)))
        head = F.conv2d(d0, pt["head"][0], pt["head"][1])
        rgb_d, logit, zl = head[:, 0:3], head[:, 3:28], head[:, 28:29]
        wq = torch.softmax(logit, 1)
        c = F.unfold(x[:, 0:3], 5, padding=2).view(x.shape[0], 3, 25, *x.shape[2:])
        m = F.unfold(x[:, 4:5], 5, padding=2).view(x.shape[0], 25, *x.shape[2:])
        den = (wq * m).sum(1, keepdim=True)
        num = (wq[:, None] * m[:, None] * c).sum(2)
        kp = torch.where(den >= 1e-12, num / den.clamp_min(1e-300), rgb_d)
        a = torch.sigmoid(zl)
        return a * kp + (1 - a) * rgb_d

    (fwd(tp) * T(g)).sum().backward()
    for name in params:
        assert np.max(np.abs(grads[name][0] - tp[name][0].grad.numpy())) < 1e-10, name
        assert np.max(np.abs(grads[name][1] - tp[name][1].grad.numpy())) < 1e-10, name
    # finite differences on a few weights of every layer
    eps = 1e-6
    for name in params:
        w = params[name][0]
        for _ in range(3):
            i = tuple(rng.integers(0, s) for s in w.shape)
            old = w[i]
            w[i] = old + eps
            fp = (on.forward(params, sp) * g).sum()
            w[i] = old - eps
            fm = (on.forward(params, sp) * g).sum()
            w[i] = old
            fd = (fp - fm) / (2 * eps)
            assert abs(fd - grads[name][0][i]) < 1e-6 * max(1.0, abs(fd)), name


def test_loss_closed_form_and_finite_differences():
    rng = np.random.default_rng(11)
    t = rng.uniform(size=(2, 3, 6, 7))
    # constant offset: the gradient terms vanish, L1 = |c|
    loss, _ = on.loss_l1_grad(t + 0.25, t)
    assert abs(loss - 0.25) < 1e-12
    p = rng.uniform(size=t.shape)
    loss, g = on.loss_l1_grad(p, t)
    eps = 1e-7
    for _ in range(30):
        i = tuple(rng.integers(0, s) for s in p.shape)
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (on.loss_l1_grad(pp, t)[0] - on.loss_l1_grad(pm, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6


def test_adam_first_steps_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.01, 2.0])
    p1, m, v = on.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-3)
    # after one step m_hat = g and v_hat = g^2: the update is lr * g / (|g| + eps)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
    # a constant gradient keeps m_hat = g, v_hat = g^2 at every step
    q, m, v = p, np.zeros(3), np.zeros(3)
    for s in range(1, 6):
        q, m, v = on.adam_step(q, g, m, v, s, lr=1e-3)
    assert np.allclose(q, p - 5e-3 * g / (np.abs(g) + 1e-8), atol=1e-13)


def test_psnr_ssim_closed_forms():
    rng = np.random.default_rng(12)
    a = rng.uniform(0.2, 0.8, (3, 32, 32))
    assert abs(metrics.psnr(a, a + 0.01) - 40.0) < 1e-9
    assert abs(metrics.ssim(a, a) - 1.0) < 1e-12
    x = np.full((3, 20, 20), 0.3)
    y = np.full((3, 20, 20), 0.6)
    c1 = 0.01 ** 2
    assert abs(metrics.ssim(x, y) - (2 * 0.18 + c1) / (0.09 + 0.36 + c1)) < 1e-12


def test_device_quality_metrics_match_the_oracle():
    """The benchmark's torch PSNR / SSIM equal the oracle's float64 ones."""
    import torch
    from paper_2209_09965_gb300 import quality
    rng = np.random.default_rng(12)
    a = rng.uniform(-0.1, 1.1, (3, 40, 57))
    b = np.clip(a + rng.normal(0, 0.05, a.shape), -0.2, 1.2)
    assert abs(quality.psnr(torch.from_numpy(a), torch.from_numpy(b)) - metrics.psnr(a, b)) < 1e-9
    assert abs(quality.ssim(torch.from_numpy(a), torch.from_numpy(b)) - metrics.ssim(a, b)) < 1e-12
    assert abs(quality.ssim(torch.from_numpy(a[0]), torch.from_numpy(b[0])) - metrics.ssim(a[0], b[0])) < 1e-12



def test_tpsnr_closed_form_and_device_metric():
    import torch
    from paper_2209_09965_gb300 import quality
    rng = np.random.default_rng(13)
    y0, y1 = rng.integers(0, 57, (2, 3, 16, 20)) / 64.0          # dyadic: the differences are exact
    # a reconstruction off by a constant (inside [0, 1]) changes exactly like the reference
    assert metrics.tpsnr(y0 + 0.0625, y1 + 0.0625, y0, y1) == float("inf")
    # a static reconstruction of a changing reference: the error is the reference's change
    d = y1 - y0
    assert abs(metrics.tpsnr(y0, y0, y0, y1) - (-10 * np.log10(np.mean(d ** 2)))) < 1e-12
    o0 = np.clip(y0 + rng.normal(0, 0.03, y0.shape), -0.1, 1.1)
    o1 = np.clip(y1 + rng.normal(0, 0.03, y1.shape), -0.1, 1.1)
    t = [torch.from_numpy(v) for v in (o0, o1, y0, y1)]
    assert abs(quality.tpsnr(*t) - metrics.tpsnr(o0, o1, y0, y1)) < 1e-9


# ---- recurrent variant: the previous output as three more input channels ----

def _recurrent_from(flat5, rng=None, scale=0.0):
    """The 8-input network equal to a 5-input one plus prev-channel weights (zero or random)."""
    p = on.unpack(flat5)
    w, b = p["enc0a"]
    extra = np.zeros((w.shape[0], 3, 3, 3)) if rng is None else rng.normal(0, scale, (w.shape[0], 3, 3, 3))
    p["enc0a"] = (np.concatenate([w, extra], axis=1), b)
    return p


def test_recurrent_with_zero_history_weights_is_the_plain_network():
    rng = np.random.default_rng(21)
    flat = wl.net_weights(3)
    sparse = rng.uniform(0, 1, (2, 5, 12, 18))
    sparse[:, 4] = (rng.random((2, 12, 18)) < 0.4)
    prev = rng.uniform(-0.5, 1.5, (2, 3, 12, 18))
    plain = on.forward(on.unpack(flat), sparse)
    rec0 = _recurrent_from(flat)
    assert on.param_count(cin=8) == on.pack(rec0).size
    assert np.array_equal(on.unpack(on.pack(rec0))["enc0a"][0], rec0["enc0a"][0])
    assert np.allclose(on.forward(rec0, sparse, prev=prev), plain, atol=1e-13)
    rec = _recurrent_from(flat, rng, 0.3)
    # no history is zero history; history outside [0, 1] acts clamped
    assert np.array_equal(on.forward(rec, sparse), on.forward(rec, sparse, prev=np.zeros((2, 3, 12, 18))))
    assert np.array_equal(on.forward(rec, sparse, prev=prev), on.forward(rec, sparse, prev=np.clip(prev, 0, 1)))
    assert not np.allclose(on.forward(rec, sparse, prev=prev), plain, atol=1e-3)


def test_recurrent_history_enters_the_first_convolution_linearly():
    rng = np.random.default_rng(22)
    rec = _recurrent_from(wl.net_weights(4), rng, 0.3)
    sparse = rng.uniform(0, 1, (1, 5, 8, 12))
    prev = rng.uniform(0, 1, (1, 3, 8, 12))
    _, c1 = on.forward(rec, sparse, return_cache=True, prev=prev)
    _, c0 = on.forward(rec, sparse, return_cache=True)
    dz = c1["enc0a"][1] - c0["enc0a"][1]
    ref = F.conv2d(torch.from_numpy(prev), torch.from_numpy(rec["enc0a"][0][:, 5:]), padding=1).numpy()
    assert np.max(np.abs(dz - ref)) < 1e-12


def test_recurrent_backward_matches_finite_differences():
    rng = np.random.default_rng(23)
    rec = _recurrent_from(wl.net_weights(5), rng, 0.3)
    sparse = rng.uniform(0, 1, (1, 5, 8, 8))
    sparse[:, 4] = 1.0
    prev = rng.uniform(0, 1, (1, 3, 8, 8))
    gout = rng.normal(size=(1, 3, 8, 8))
    _, cache = on.forward(rec, sparse, return_cache=True, prev=prev)
    g = on.backward(rec, cache, gout)
    for (o, c, ky, kx) in [(0, 5, 1, 1), (3, 7, 0, 2), (9, 6, 2, 0)]:      # history-channel weights
        eps = 1e-6
        w = rec["enc0a"][0]
        old = w[o, c, ky, kx]
        w[o, c, ky, kx] = old + eps
        fp = np.sum(on.forward(rec, sparse, prev=prev) * gout)
        w[o, c, ky, kx] = old - eps
        fm = np.sum(on.forward(rec, sparse, prev=prev) * gout)
        w[o, c, ky, kx] = old
        assert abs((fp - fm) / (2 * eps) - g["enc0a"][0][o, c, ky, kx]) < 1e-6 * max(1.0, abs(fp - fm) / eps)


def test_temporal_loss_closed_form_and_gradient():
    rng = np.random.default_rng(24)
    y0, y1 = rng.uniform(0, 1, (2, 3, 6, 7))
    o0 = rng.uniform(0, 1, (3, 6, 7))
    # a reconstruction that follows the reference's change exactly: zero loss
    l, g = on.loss_temporal(o0 + (y1 - y0), o0, y1, y0)
    assert l < 1e-15
    o1 = rng.uniform(0, 1, (3, 6, 7))
    l, g = on.loss_temporal(o1, o0, y1, y0)
    assert abs(l - np.mean(np.abs((o1 - o0) - (y1 - y0)))) < 1e-15
    for idx in [(0, 0, 0), (2, 5, 6), (1, 3, 2)]:
        e = np.zeros_like(o1)
        e[idx] = 1e-7
        fd = (on.loss_temporal(o1 + e, o0, y1, y0)[0] - on.loss_temporal(o1 - e, o0, y1, y0)[0]) / 2e-7
        assert abs(fd - g[idx]) < 1e-6


def test_loss_gradient_terms_closed_form():
    """A prediction that differs from the target by a linear ramp a x + b y:
    the L1 term is the mean of |a x + b y|, and the forward differences are a
    along x and b along y at every pixel, so the two gradient terms add
    lam_g (|a| + |b|) (paper, "Loss": L1 plus the L1 of the image gradients)."""
    rng = np.random.default_rng(21)
    h, w, a, b = 6, 7, 0.03, -0.05
    yy, xx = np.mgrid[0:h, 0:w]
    d = a * xx + b * yy
    t = rng.uniform(size=(2, 3, h, w))
    for lam in (1.0, 0.5, 0.0):
        loss, _ = on.loss_l1_grad(t + d, t, lam)
        assert abs(loss - (np.abs(d).mean() + lam * (abs(a) + abs(b)))) < 1e-12


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Plausible mistakes planted in the oracle -- a transposed tap order, the
    sample mask missing from the kernel-prediction weights, the blend
    inverted, align-corners up-sampling, max instead of average pooling, a
    flipped convolution kernel, the gradient terms of the loss dropped, Adam
    without bias correction -- each break one of the pins above."""
    good_nb, good_upw, good_sig = on._neighbours, on._up_axis_weights, on.sigmoid
    good_conv, good_loss = on.conv2d, on.loss_l1_grad

    def nb_transposed(img, r=on.KP_R):   # taps ordered dx-major instead of dy-major
        n, c, h, w = img.shape
        p = np.zeros((n, c, h + 2 * r, w + 2 * r))
        p[:, :, r:r + h, r:r + w] = img
        return np.stack([p[:, :, r + dy:r + dy + h, r + dx:r + dx + w]
                         for dx in range(-r, r + 1) for dy in range(-r, r + 1)], axis=2)

    def nb_mask_ones(img, r=on.KP_R):    # every tap counted as sampled
        out = good_nb(img, r)
        return np.ones_like(out) if img.shape[1] == 1 else out

    def up_align_corners(n_in):
        m = np.zeros((2 * n_in, n_in))
        for o in range(2 * n_in):
            s = o * (n_in - 1) / (2 * n_in - 1)
            i0 = int(np.floor(s))
            i1 = min(i0 + 1, n_in - 1)
            m[o, i0] += 1.0 - (s - i0)
            m[o, i1] += s - i0
        return m

    def max_pool(x):
        n, c, h, w = x.shape
        return x.reshape(n, c, h // 2, 2, w // 2, 2).max(axis=(3, 5))

    def adam_no_bias_correction(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        return p - lr * m / (np.sqrt(v) + eps), m, v

    plants = [
        ("_neighbours", nb_transposed, test_kp_one_hot_is_shifted_copy),
        ("_neighbours", nb_mask_ones, test_kp_uniform_logits_is_masked_box_filter_and_empty_window_falls_back),
        ("sigmoid", lambda z: good_sig(-z), test_kp_one_hot_is_shifted_copy),
        ("_up_axis_weights", up_align_corners, test_pool_and_upsample_match_torch),
        ("avgpool2", max_pool, test_pool_and_upsample_match_torch),
        ("conv2d", lambda x, w, b: good_conv(x, w[:, :, ::-1, ::-1].copy(), b), test_conv_matches_direct_sum),
        ("loss_l1_grad", lambda p, t, lam_g=1.0: good_loss(p, t, 0.0), test_loss_gradient_terms_closed_form),
        ("adam_step", adam_no_bias_correction, test_adam_first_steps_closed_form),
    ]
    for name, bad, pin in plants:
        monkeypatch.setattr(on, name, bad)
        _fails(pin)
        monkeypatch.undo()
    # with the oracle restored every pin passes again
    for _, _, pin in plants:
        pin()
    assert on._neighbours is good_nb and on._up_axis_weights is good_upw


def test_ssim_brute_force_windows():
    """SSIM against an explicit loop over every valid 11 x 11 window with the
    normalised 2-D Gaussian weights (sigma 1.5) and centred (co)variances,
    per channel, then averaged (Wang et al. 2004)."""
    rng = np.random.default_rng(31)
    a = rng.uniform(size=(2, 14, 17))
    b = np.clip(a + rng.normal(0, 0.1, a.shape), 0, 1)
    x = np.arange(-5, 6)
    g1 = np.exp(-0.5 * (x / 1.5) ** 2)
    w2 = np.outer(g1, g1)
    w2 /= w2.sum()
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    vals = []
    for ch in range(a.shape[0]):
        s = []
        for i in range(a.shape[1] - 10):
            for j in range(a.shape[2] - 10):
                pa, pb = a[ch, i:i + 11, j:j + 11], b[ch, i:i + 11, j:j + 11]
                ma, mb = (w2 * pa).sum(), (w2 * pb).sum()
                va, vb = (w2 * (pa - ma) ** 2).sum(), (w2 * (pb - mb) ** 2).sum()
                cab = (w2 * (pa - ma) * (pb - mb)).sum()
                s.append((2 * ma * mb + c1) * (2 * cab + c2) / ((ma ** 2 + mb ** 2 + c1) * (va + vb + c2)))
        vals.append(np.mean(s))
    assert abs(metrics.ssim(a, b) - np.mean(vals)) < 1e-12


METRIC_MUTANTS = [
    ("SSIM over the padded border", "return out[r:img.shape[0] - r, r:img.shape[1] - r]", "return out",
     ["test_ssim_brute_force_windows"]),
    ("covariance without the means", "sxy = _filter_valid(x * y, g) - mx * my", "sxy = _filter_valid(x * y, g)",
     ["test_psnr_ssim_closed_forms", "test_ssim_brute_force_windows"]),
    ("window not normalised", "return g / g.sum()", "return g", ["test_ssim_brute_force_windows"]),
    ("PSNR with a peak of 255", "return float(-10.0 * np.log10(mse))\n\n\ndef _gauss_window",
     "return float(20.0 * np.log10(255.0) - 10.0 * np.log10(mse))\n\n\ndef _gauss_window",
     ["test_psnr_ssim_closed_forms"]),
    ("tPSNR without the reference's change", "d = (c(o) - c(o_prev)) - (c(y) - c(y_prev))",
     "d = c(o) - c(o_prev)", ["test_tpsnr_closed_form_and_device_metric"]),
]


@pytest.mark.parametrize("what,old,new,pins", METRIC_MUTANTS, ids=[m[0] for m in METRIC_MUTANTS])
def test_planted_metric_mistakes_fail_the_pins(what, old, new, pins, monkeypatch):
    """Each mistake, planted in a copy of the metrics oracle's source (the
    oracle itself is not touched), breaks at least one pin above."""
    import types
    src = open(metrics.__file__).read()
    assert src.count(old) == 1, what
    mutant = types.ModuleType("metrics_mutant")
    exec(compile(src.replace(old, new), "metrics_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "metrics", mutant)
    caught = []
    for name in pins:
        try:
            globals()[name]()
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {what}"


NET_SOURCE_MUTANTS = [
    ("history not clamped", "else np.clip(np.asarray(prev, np.float64), 0.0, 1.0)",
     "else np.asarray(prev, np.float64)", ["test_recurrent_with_zero_history_weights_is_the_plain_network"]),
    ("history before the sparse channels", "x = _pad4(np.concatenate([x_in, pv], axis=1))",
     "x = _pad4(np.concatenate([pv, x_in], axis=1))", ["test_recurrent_history_enters_the_first_convolution_linearly"]),
    ("temporal loss without the reference's change",
     "d = (np.asarray(o, np.float64) - o_prev) - (np.asarray(y, np.float64) - y_prev)",
     "d = np.asarray(o, np.float64) - o_prev", ["test_temporal_loss_closed_form_and_gradient"]),
]


@pytest.mark.parametrize("what,old,new,pins", NET_SOURCE_MUTANTS, ids=[m[0] for m in NET_SOURCE_MUTANTS])
def test_planted_recurrent_mistakes_fail_the_pins(what, old, new, pins, monkeypatch):
    """Each mistake, planted in a copy of the network oracle's source (the
    oracle itself is not touched), breaks at least one pin above."""
    import types
    src = open(on.__file__).read()
    assert src.count(old) == 1, what
    mutant = types.ModuleType("oracle.net_mutant")
    mutant.__package__ = "oracle"
    exec(compile(src.replace(old, new), "net_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "on", mutant)
    caught = []
    for name in pins:
        try:
            globals()[name]()
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin caught: {what}"
