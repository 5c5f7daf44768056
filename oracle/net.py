"""Oracle: FP64 reconstruction network, kernel-prediction blend, loss, Adam.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  Plain numpy in float64; the only
library primitive used as a step is the tensor contraction (``np.einsum``).

Network (the paper's "Reconstruction Network" section and Fig. "network
architecture": a U-Net with 3x3 convolutions of stride 1 and padding 1,
ReLU, average pooling down, bilinear up-sampling and skip connections; the
"Model Configuration" subsection gives two convolutions per block).  The
channel plan here is the slim 16/32/64 variant, three levels:

    enc0 : conv 5->c0, conv c0->c0                  (full resolution)
    pool 2x2 average
    enc1 : conv c0->c1, conv c1->c1                 (1/2)
    pool
    bot  : conv c1->c2, conv c2->c2                 (1/4)
    up x2 bilinear, concat [up, enc1]  -> dec1 : conv (c2+c1)->c1, conv c1->c1
    up x2 bilinear, concat [up, enc0]  -> dec0 : conv (c1+c0)->c0, conv c0->c0
    head : 1x1 conv c0 -> 29 = rgb_d (3) | kernel logits (25) | blend logit (1)

Every 3x3 convolution has a bias and is followed by ReLU; the head has no
activation.  Frames whose sides are not multiples of 4 are zero-padded at the
bottom / right and the output is cropped back.  Bilinear up-sampling uses
half-pixel centres (source coordinate (o + 0.5)/2 - 0.5, negative clamped to
0) and clamps the upper neighbour to the edge.

Kernel prediction and blend (the "Kernel Prediction" subsection predicts
per-pixel filter kernels and applies them; the reading used here applies one
5x5 kernel to the sparse samples and blends with the direct prediction):

    w_q  = softmax over the 25 logits (tap q = (dy + 2) * 5 + (dx + 2))
    den  = sum_q w_q M(p + q),  num = sum_q w_q M(p + q) c(p + q)
    kp   = num / den            (kp = rgb_d where den < 1e-12)
    a    = sigmoid(blend logit)
    out  = a kp + (1 - a) rgb_d

c is the sparse RGB, M the mask channel; neighbours outside the frame count
as M = 0.

Recurrent variant (the paper's "Recurrence" subsection: D's output is passed
back to its input layer in the next run, concatenated along the channels):
enc0 takes 8 channels, the 5 of the sparse frame and the previous frame's
output RGB clamped to [0, 1] (zeros for the first frame).  The paper's
recurrent connections between decoder blocks are not part of this variant.

Loss (replaces the paper's Eq. 4-7 perceptual / temporal terms, which need
VGG19 weights and optical flow): L1 + lambda_g * L1 of forward differences
along x and y, each term a mean over its own elements, lambda_g = 1.  For
the recurrent variant the temporal term of Eq. 6 without its optical-flow
part: L_t = mean |(O_t - O_t-1) - (Y_t - Y_t-1)|, combined as in Eq. 4 with
lambda_s = 0.8, lambda_t = 1.0.
Adam: beta = (0.9, 0.999), eps = 1e-8, bias-corrected, no weight decay.
"""
from __future__ import annotations

import numpy as np

KP_R = 2
KP_TAPS = 25
HEAD_C = 29


def layer_table(chans=(16, 32, 64), cin=5):
    c0, c1, c2 = chans
    return (
        ("enc0a", cin, c0, 3), ("enc0b", c0, c0, 3),
        ("enc1a", c0, c1, 3), ("enc1b", c1, c1, 3),
        ("bota", c1, c2, 3), ("botb", c2, c2, 3),
        ("dec1a", c2 + c1, c1, 3), ("dec1b", c1, c1, 3),
        ("dec0a", c1 + c0, c0, 3), ("dec0b", c0, c0, 3),
        ("head", c0, HEAD_C, 1),
    )


def param_count(chans=(16, 32, 64), cin=5):
    return sum(co * ci * k * k + co for _, ci, co, k in layer_table(chans, cin))


def unpack(flat, chans=(16, 32, 64), cin=None):
    """Flat float vector -> {name: (W[co,ci,k,k], b[co])} in float64.  The
    input width (5, or 8 for the recurrent variant) follows from the size
    unless given."""
    flat = np.asarray(flat, dtype=np.float64)
    if cin is None:
        cin = 8 if flat.size == param_count(chans, 8) else 5
    out, off = {}, 0
    for name, ci, co, k in layer_table(chans, cin):
        nw = co * ci * k * k
        out[name] = (flat[off:off + nw].reshape(co, ci, k, k), flat[off + nw:off + nw + co])
        off += nw + co
    if off != flat.size:
        raise ValueError(f"weight vector has {flat.size} entries, expected {off}")
    return out


def pack(params, chans=(16, 32, 64)):
    parts = []
    for name, _, _, _ in layer_table(chans, params["enc0a"][0].shape[1]):
        w, b = params[name]
        parts += [np.asarray(w, np.float64).ravel(), np.asarray(b, np.float64).ravel()]
    return np.concatenate(parts)


# ---------------------------------------------------------------------------
# layers (NCHW, float64)
# ---------------------------------------------------------------------------


def conv2d(x, w, b):
    """out[n,o,y,x] = b[o] + sum_{c,i,j} w[o,c,i,j] x[n,c,y+i-r,x+j-r], zero padding r."""
    k = w.shape[2]
    r = k // 2
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * r, wd + 2 * r))
    xp[:, :, r:r + h, r:r + wd] = x
    out = np.zeros((n, w.shape[0], h, wd))
    for i in range(k):
        for j in range(k):
            out += np.einsum("nchw,oc->nohw", xp[:, :, i:i + h, j:j + wd], w[:, :, i, j], optimize=True)
    return out + b[None, :, None, None]


def conv2d_backward(x, w, gout):
    """Gradients of conv2d w.r.t. x, w, b given dL/dout."""
    k = w.shape[2]
    r = k // 2
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2 * r, wd + 2 * r))
    xp[:, :, r:r + h, r:r + wd] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for i in range(k):
        for j in range(k):
            gw[:, :, i, j] = np.einsum("nohw,nchw->oc", gout, xp[:, :, i:i + h, j:j + wd], optimize=True)
            gxp[:, :, i:i + h, j:j + wd] += np.einsum("nohw,oc->nchw", gout, w[:, :, i, j], optimize=True)
    gb = gout.sum(axis=(0, 2, 3))
    return gxp[:, :, r:r + h, r:r + wd], gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    n, c, h, w = x.shape
    return x.reshape(n, c, h // 2, 2, w // 2, 2).mean(axis=(3, 5))


def avgpool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) * 0.25


def _up_axis_weights(n_in):
    """Interpolation matrix [2 n_in, n_in] of x2 bilinear, half-pixel centres."""
    m = np.zeros((2 * n_in, n_in))
    for o in range(2 * n_in):
        src = (o + 0.5) / 2.0 - 0.5
        if src < 0.0:
            src = 0.0
        i0 = int(np.floor(src))
        t = src - i0
        i1 = min(i0 + 1, n_in - 1)
        m[o, i0] += 1.0 - t
        m[o, i1] += t
    return m


def upsample2(x):
    my = _up_axis_weights(x.shape[2])
    mx = _up_axis_weights(x.shape[3])
    return np.einsum("yh,nchw,xw->ncyx", my, x, mx, optimize=True)


def upsample2_backward(g, in_h, in_w):
    my = _up_axis_weights(in_h)
    mx = _up_axis_weights(in_w)
    return np.einsum("yh,ncyx,xw->nchw", my, g, mx, optimize=True)


def sigmoid(z):
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def _neighbours(img, r=KP_R):
    """[N, C, H, W] -> [N, C, 25, H, W] of p + q with zero outside the frame."""
    n, c, h, w = img.shape
    p = np.zeros((n, c, h + 2 * r, w + 2 * r))
    p[:, :, r:r + h, r:r + w] = img
    taps = []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            taps.append(p[:, :, r + dy:r + dy + h, r + dx:r + dx + w])
    return np.stack(taps, axis=2)


def kp_blend(head, sparse):
    """head [N,29,H,W], sparse [N,5,H,W] (R,G,B,A,M) -> (out [N,3,H,W], cache)."""
    rgb_d = head[:, 0:3]
    logits = head[:, 3:3 + KP_TAPS]
    zl = head[:, 28]
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    wq = e / e.sum(axis=1, keepdims=True)                      # [N,25,H,W]
    nb_c = _neighbours(sparse[:, 0:3])                           # [N,3,25,H,W]
    nb_m = _neighbours(sparse[:, 4:5])[:, 0]                     # [N,25,H,W]
    wm = wq * nb_m
    den = wm.sum(axis=1)                                         # [N,H,W]
    num = np.einsum("nqhw,ncqhw->nchw", wm, nb_c)
    valid = den >= 1e-12
    safe = np.where(valid, den, 1.0)
    kp = np.where(valid[:, None], num / safe[:, None], rgb_d)
    a = sigmoid(zl)[:, None]
    out = a * kp + (1.0 - a) * rgb_d
    cache = dict(rgb_d=rgb_d, wq=wq, nb_c=nb_c, nb_m=nb_m, den=den, safe=safe, valid=valid, kp=kp, a=a)
    return out, cache


def kp_blend_backward(gout, cache):
    """dL/dhead [N,29,H,W] given dL/dout [N,3,H,W]."""
    a, kp, rgb_d, valid = cache["a"], cache["kp"], cache["rgb_d"], cache["valid"]
    wq, nb_c, nb_m, safe = cache["wq"], cache["nb_c"], cache["nb_m"], cache["safe"]
    g = np.zeros((gout.shape[0], HEAD_C) + gout.shape[2:])
    g_kp = gout * a
    g_rgbd = gout * (1.0 - a)
    g_a = (gout * (kp - rgb_d)).sum(axis=1)                      # [N,H,W]
    g[:, 28] = g_a * (a[:, 0] * (1.0 - a[:, 0]))
    # where den < 1e-12, kp = rgb_d
    g_rgbd = g_rgbd + np.where(valid[:, None], 0.0, g_kp)
    g[:, 0:3] = g_rgbd
    # kp_c = sum_q w_q m_q c_qc / sum_q w_q m_q  ->  dkp_c/dw_q = m_q (c_qc - kp_c) / den
    gkv = np.where(valid[:, None], g_kp, 0.0)
    d_w = np.einsum("nchw,nqhw,ncqhw->nqhw", gkv, nb_m, nb_c - kp[:, :, None]) / safe[:, None]
    # softmax backward: dl_q = w_q (d_w_q - sum_r w_r d_w_r)
    g[:, 3:28] = wq * (d_w - (wq * d_w).sum(axis=1, keepdims=True))
    return g


# ---------------------------------------------------------------------------
# whole network
# ---------------------------------------------------------------------------


def _pad4(x):
    n, c, h, w = x.shape
    h4, w4 = -(-h // 4) * 4, -(-w // 4) * 4
    if (h4, w4) == (h, w):
        return x
    xp = np.zeros((n, c, h4, w4))
    xp[:, :, :h, :w] = x
    return xp


def forward(params, sparse, return_cache=False, prev=None):
    """sparse [N,5,H,W] (or [5,H,W]) float -> rgb [N,3,H,W] (or [3,H,W]).
    With recurrent parameters (8 input channels) ``prev`` is the previous
    output [N,3,H,W] (None: zeros), clamped to [0, 1] as input."""
    single = sparse.ndim == 3
    x_in = np.asarray(sparse, np.float64)
    if single:
        x_in = x_in[None]
    n, _, h, w = x_in.shape
    if params["enc0a"][0].shape[1] == 8:
        pv = np.zeros((n, 3, h, w)) if prev is None else np.clip(np.asarray(prev, np.float64), 0.0, 1.0)
        if pv.ndim == 3:
            pv = pv[None]
        x = _pad4(np.concatenate([x_in, pv], axis=1))
    else:
        x = _pad4(x_in)
    cache = {"x": x}

    def cbr(name, inp):
        wgt, b = params[name]
        z = conv2d(inp, wgt, b)
        cache[name] = (inp, z)
        return relu(z)

    e0 = cbr("enc0b", cbr("enc0a", x))
    p0 = avgpool2(e0)
    e1 = cbr("enc1b", cbr("enc1a", p0))
    p1 = avgpool2(e1)
    bt = cbr("botb", cbr("bota", p1))
    u1 = upsample2(bt)
    d1 = cbr("dec1b", cbr("dec1a", np.concatenate([u1, e1], axis=1)))
    u0 = upsample2(d1)
    d0 = cbr("dec0b", cbr("dec0a", np.concatenate([u0, e0], axis=1)))
    wh, bh = params["head"]
    head = conv2d(d0, wh, bh)
    cache.update(e0=e0, e1=e1, bt=bt, d1=d1, d0=d0, head=head)
    sp = _pad4(x_in)
    out, kcache = kp_blend(head, sp)
    cache["kp"] = kcache
    out = out[:, :, :h, :w]
    if single:
        out = out[0]
    return (out, cache) if return_cache else out


def backward(params, cache, gout):
    """dL/dparams (same dict layout) given dL/dout [N,3,H,W] (unpadded)."""
    grads = {}
    x = cache["x"]
    n, _, hp, wp = x.shape
    g = np.zeros((n, 3, hp, wp))
    g[:, :, :gout.shape[2], :gout.shape[3]] = gout
    g_head = kp_blend_backward(g, cache["kp"])
    gd0, gw, gb = conv2d_backward(cache["d0"], params["head"][0], g_head)
    grads["head"] = (gw, gb)

    def cbr_back(name, gy):
        inp, z = cache[name]
        gz = gy * (z > 0)
        gi, gw_, gb_ = conv2d_backward(inp, params[name][0], gz)
        grads[name] = (gw_, gb_)
        return gi

    c0 = cache["e0"].shape[1]
    c1 = cache["e1"].shape[1]
    g = cbr_back("dec0a", cbr_back("dec0b", gd0))
    gu0, ge0 = g[:, :-c0], g[:, -c0:]
    gd1 = upsample2_backward(gu0, cache["d1"].shape[2], cache["d1"].shape[3])
    g = cbr_back("dec1a", cbr_back("dec1b", gd1))
    gu1, ge1 = g[:, :-c1], g[:, -c1:]
    gbt = upsample2_backward(gu1, cache["bt"].shape[2], cache["bt"].shape[3])
    gp1 = cbr_back("bota", cbr_back("botb", gbt))
    ge1 = ge1 + avgpool2_backward(gp1)
    gp0 = cbr_back("enc1a", cbr_back("enc1b", ge1))
    ge0 = ge0 + avgpool2_backward(gp0)
    cbr_back("enc0a", cbr_back("enc0b", ge0))
    return grads


# ---------------------------------------------------------------------------
# loss and optimiser
# ---------------------------------------------------------------------------


def loss_l1_grad(pred, target, lam_g=1.0):
    """(loss, dL/dpred) for L1 + lam_g (L1 of d/dx + L1 of d/dy), per-term means."""
    pred = np.asarray(pred, np.float64)
    target = np.asarray(target, np.float64)
    d = pred - target
    l1 = np.abs(d).mean()
    dx = d[..., :, 1:] - d[..., :, :-1]
    dy = d[..., 1:, :] - d[..., :-1, :]
    lx = np.abs(dx).mean()
    ly = np.abs(dy).mean()
    g = np.sign(d) / d.size
    sx = lam_g * np.sign(dx) / dx.size
    sy = lam_g * np.sign(dy) / dy.size
    g[..., :, 1:] += sx
    g[..., :, :-1] -= sx
    g[..., 1:, :] += sy
    g[..., :-1, :] -= sy
    return l1 + lam_g * (lx + ly), g


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015); returns new (p, m, v). step >= 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def loss_temporal(o, o_prev, y, y_prev):
    """(L_t, dL_t/do): mean |(o - o_prev) - (y - y_prev)| (the temporal L1 term
    without optical flow); o_prev is a constant of the step."""
    d = (np.asarray(o, np.float64) - o_prev) - (np.asarray(y, np.float64) - y_prev)
    return float(np.mean(np.abs(d))), np.sign(d) / d.size
