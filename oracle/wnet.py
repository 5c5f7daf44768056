"""Oracle: FP64 two-stage reconstruction network (direct prediction D, then
kernel prediction K applied to D's output in sequence at several scales).

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  Plain numpy in float64; the 3x3 / 1x1
convolutions, pooling and up-sampling are the ones of ``oracle.net``.

The paper's "Reconstruction Network" section builds FoVolNet from two U-Nets
run in sequence: D predicts a coarse image O_d directly and keeps the hidden
states H_d of its decoder blocks; K turns H_d into per-pixel filter kernels
at several scales, in its encoder and its decoder blocks, and passes O_d
through them one after the other ("Model Configuration": both follow the
block plan e64-e64-e80-d96-d80-d64-d64, D's blocks hold two 3x3 convolutions
each with ReLU, K's blocks one 1x1 convolution; encoder blocks end in a 2x2
average pool, decoder blocks up-sample bilinearly).  The paper does not give
the size of the predicted kernels, how the image moves between K's scales,
nor how its skip connections join; the readings used here:

Widths ``cfg = (enc, bot, dec)``: ``enc[s]`` and ``dec[s]`` are the widths of
the encoder and decoder blocks at scale s (resolution 2^-s), ``bot`` that of
the block at the coarsest scale L = len(enc).  The paper's plan reads as
enc = (64, 64, 80), bot = 96, dec = (64, 64, 80) -- its d96 is the block
between the two halves, so there are four blocks going down (three of them
pooled) and three coming up, which matches the text's count of encoder
and decoder blocks (4 and 3).  The frame is zero-padded at the bottom / right to a multiple of
2^L and the output cropped back.

D (3x3 convolutions with bias, each followed by ReLU):
    E_0 = CBR(CBR(x));  E_s = CBR(CBR(pool E_(s-1)))            s = 1..L-1
    B   = CBR(CBR(pool E_(L-1)))                                  scale L
    U_s = CBR(CBR([up U_(s+1), E_s]))   s = L-1..0, U_L = B
    O_d = 1x1 conv of U_0 to 3 channels (no activation)
    H_d = (U_0, ..., U_(L-1), B)

K (1x1 convolutions with bias; G = ReLU(conv(input)), then linear 1x1 heads
give the block's 9 tap logits and, in the decoder blocks, one blend logit
z):
    G_0 = [U_0];  G_s = [pool G_(s-1), U_s];  G_L = [pool G_(L-1), B]
    G'_s = [up G'_(s+1), U_s]                   s = L-1..0, G'_L = G_L
    (brackets: the inputs concatenated, resampled input first)

Image path through K (each block filters the image with its 3x3 kernels,
in order):
    I_0 = O_d;  J_s = F(I_s, k_enc s);  I_(s+1) = pool J_s
    Y_L = F(I_L, k_bot)
    X_s = J_s + sigmoid(z_s) up(Y_(s+1) - pool J_s);  Y_s = F(X_s, k_dec s)
    output = Y_0
The decoder's join X_s swaps the low frequencies of the encoder's image J_s
for those of the coarser filtered image, in the predicted proportion
sigmoid(z_s): near 0 it keeps J_s, near 1 it takes all of the coarse image's
low band (the usual join of multi-scale kernel prediction).  F is a per-pixel 3x3 filter whose weights are the softmax of
its 9 logits over the taps inside the frame (the frame at that scale):
    F(I, l)(p) = sum_q w_q(p) I(p + q),   w_q = exp(l_q) / sum_r exp(l_r),
    q, r over {-1, 0, 1}^2 with p + q in the frame.
So F keeps a constant image constant, and with it the whole of K: a constant
O_d comes out unchanged, whatever K's weights.
"""
from __future__ import annotations

import numpy as np

from . import net as on

TAPS = 9
PAPER = ((64, 64, 80), 96, (64, 64, 80))
SLIM = ((16, 32), 64, (16, 32))


def layer_table(cfg, cin=5):
    """(name, c_in, c_out, k) of every convolution, in the flat weight order."""
    enc, bot, dec = cfg
    L = len(enc)
    t = []
    ci = cin
    for s in range(L):
        t += [(f"d_enc{s}a", ci, enc[s], 3), (f"d_enc{s}b", enc[s], enc[s], 3)]
        ci = enc[s]
    t += [("d_bota", enc[-1], bot, 3), ("d_botb", bot, bot, 3)]
    prev = bot
    for s in reversed(range(L)):
        t += [(f"d_dec{s}a", prev + enc[s], dec[s], 3), (f"d_dec{s}b", dec[s], dec[s], 3)]
        prev = dec[s]
    t += [("d_out", dec[0], 3, 1)]
    for s in range(L):
        t += [(f"k_enc{s}", (enc[s - 1] if s else 0) + dec[s], enc[s], 1), (f"k_enc{s}_taps", enc[s], TAPS, 1)]
    t += [("k_bot", enc[-1] + bot, bot, 1), ("k_bot_taps", bot, TAPS, 1)]
    prev = bot
    for s in reversed(range(L)):
        t += [(f"k_dec{s}", prev + dec[s], dec[s], 1), (f"k_dec{s}_taps", dec[s], TAPS, 1),
              (f"k_dec{s}_blend", dec[s], 1, 1)]
        prev = dec[s]
    return tuple(t)


def param_count(cfg):
    return sum(co * ci * k * k + co for _, ci, co, k in layer_table(cfg))


def unpack(flat, cfg):
    flat = np.asarray(flat, np.float64)
    out, off = {}, 0
    for name, ci, co, k in layer_table(cfg):
        nw = co * ci * k * k
        out[name] = (flat[off:off + nw].reshape(co, ci, k, k), flat[off + nw:off + nw + co])
        off += nw + co
    if off != flat.size:
        raise ValueError(f"weight vector has {flat.size} entries, expected {off}")
    return out


def pack(params, cfg):
    parts = []
    for name, _, _, _ in layer_table(cfg):
        w, b = params[name]
        parts += [np.asarray(w, np.float64).ravel(), np.asarray(b, np.float64).ravel()]
    return np.concatenate(parts)


# ---------------------------------------------------------------------------
# the per-pixel 3x3 filter and the decoder join
# ---------------------------------------------------------------------------


def _shifted(img):
    """[N, C, H, W] -> ([N, C, 9, H, W] of img(p + q), [9, H, W] in-frame flags),
    q = (dy, dx) row-major over {-1, 0, 1}^2, zero outside the frame."""
    n, c, h, w = img.shape
    p = np.zeros((n, c, h + 2, w + 2))
    p[:, :, 1:h + 1, 1:w + 1] = img
    inside = np.zeros((h + 2, w + 2))
    inside[1:h + 1, 1:w + 1] = 1.0
    vals, flags = [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            vals.append(p[:, :, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w])
            flags.append(inside[1 + dy:1 + dy + h, 1 + dx:1 + dx + w])
    return np.stack(vals, axis=2), np.stack(flags, axis=0)


def filter3(img, logits):
    """F(img, logits): img [N, C, H, W], logits [N, 9, H, W] -> (out, cache)."""
    nb, inside = _shifted(img)
    l = np.where(inside[None] > 0, logits, -np.inf)
    m = l.max(axis=1, keepdims=True)
    e = np.exp(l - m)
    wq = e / e.sum(axis=1, keepdims=True)                      # zero outside the frame
    out = np.einsum("nqhw,ncqhw->nchw", wq, nb)
    return out, dict(wq=wq, nb=nb, out=out)


def filter3_backward(gout, cache):
    """(dL/dimg, dL/dlogits) given dL/dout."""
    wq, nb, out = cache["wq"], cache["nb"], cache["out"]
    n, c, h, w = gout.shape
    # dout_c/dl_q = w_q (img_c(p + q) - out_c)
    d = np.einsum("nchw,ncqhw->nqhw", gout, nb - out[:, :, None])
    glog = wq * d
    # dout_c(p)/dimg_c(p + q) = w_q(p): scatter back to p + q
    gp = np.zeros((n, c, h + 2, w + 2))
    k = 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            gp[:, :, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w] += wq[:, k][:, None] * gout
            k += 1
    return gp[:, :, 1:h + 1, 1:w + 1], glog


def join(j, y, z):
    """X = J + sigmoid(z) up(Y - pool J): J [N, 3, H, W], Y [N, 3, H/2, W/2], z [N, H, W]."""
    d = y - on.avgpool2(j)
    u = on.upsample2(d)
    a = on.sigmoid(z)[:, None]
    return j + a * u, dict(u=u, a=a, shape=d.shape)


def join_backward(gx, cache):
    """(dL/dJ, dL/dY, dL/dz) given dL/dX."""
    u, a, shape = cache["u"], cache["a"], cache["shape"]
    gz = (gx * u).sum(axis=1) * (a[:, 0] * (1.0 - a[:, 0]))
    gd = on.upsample2_backward(gx * a, shape[2], shape[3])
    gj = gx - on.avgpool2_backward(gd)
    return gj, gd, gz


# ---------------------------------------------------------------------------
# whole network
# ---------------------------------------------------------------------------


def _pad(x, m):
    n, c, h, w = x.shape
    hp, wp = -(-h // m) * m, -(-w // m) * m
    if (hp, wp) == (h, w):
        return x
    xp = np.zeros((n, c, hp, wp))
    xp[:, :, :h, :w] = x
    return xp


def forward(params, cfg, sparse, return_cache=False):
    """sparse [N, 5, H, W] (or [5, H, W]) -> rgb [N, 3, H, W] (or [3, H, W])."""
    enc, bot, dec = cfg
    L = len(enc)
    single = sparse.ndim == 3
    x_in = np.asarray(sparse, np.float64)
    if single:
        x_in = x_in[None]
    n, _, h, w = x_in.shape
    x = _pad(x_in, 1 << L)
    c = {"x": x}

    def conv(name, inp, act):
        wgt, b = params[name]
        z = on.conv2d(inp, wgt, b)
        c[name] = (inp, z)
        return on.relu(z) if act else z

    def cbr2(pre, inp):
        return conv(pre + "b", conv(pre + "a", inp, True), True)

    # D
    E, t = [], x
    for s in range(L):
        E.append(cbr2(f"d_enc{s}", t))
        t = on.avgpool2(E[s])
    B = cbr2("d_bot", t)
    U = [None] * L
    prev = B
    for s in reversed(range(L)):
        U[s] = cbr2(f"d_dec{s}", np.concatenate([on.upsample2(prev), E[s]], axis=1))
        prev = U[s]
    o_d = conv("d_out", U[0], False)
    # K: features and logits
    G, le = [], []
    for s in range(L):
        inp = U[0] if s == 0 else np.concatenate([on.avgpool2(G[s - 1]), U[s]], axis=1)
        G.append(conv(f"k_enc{s}", inp, True))
        le.append(conv(f"k_enc{s}_taps", G[s], False))
    gb = conv("k_bot", np.concatenate([on.avgpool2(G[L - 1]), B], axis=1), True)
    lb = conv("k_bot_taps", gb, False)
    ld, zd = [None] * L, [None] * L
    prev = gb
    for s in reversed(range(L)):
        g = conv(f"k_dec{s}", np.concatenate([on.upsample2(prev), U[s]], axis=1), True)
        ld[s] = conv(f"k_dec{s}_taps", g, False)
        zd[s] = conv(f"k_dec{s}_blend", g, False)[:, 0]
        prev = g
    # image path
    J, fc_e, img = [], [], o_d
    for s in range(L):
        j, fc = filter3(img, le[s])
        J.append(j)
        fc_e.append(fc)
        img = on.avgpool2(j)
    y, fc_b = filter3(img, lb)
    fc_d, jc = [None] * L, [None] * L
    for s in reversed(range(L)):
        xs, jc[s] = join(J[s], y, zd[s])
        y, fc_d[s] = filter3(xs, ld[s])
    out = y[:, :, :h, :w]
    c.update(E=E, B=B, U=U, o_d=o_d, G=G, gb=gb, fc_e=fc_e, fc_b=fc_b, fc_d=fc_d, jc=jc, cfg=cfg)
    if single:
        out = out[0]
    return (out, c) if return_cache else out


def direct(params, cfg, sparse):
    """O_d alone (D's direct prediction), cropped like the output."""
    _, c = forward(params, cfg, sparse if sparse.ndim == 4 else sparse[None], return_cache=True)
    h, w = sparse.shape[-2:]
    o = c["o_d"][:, :, :h, :w]
    return o if sparse.ndim == 4 else o[0]


def backward(params, cache, gout):
    """dL/dparams {name: (gW, gb)} given dL/dout [N, 3, H, W] (unpadded)."""
    enc, bot, dec = cache["cfg"]
    L = len(enc)
    grads = {}
    x = cache["x"]
    n, _, hp, wp = x.shape
    gy = np.zeros((n, 3, hp, wp))
    gy[:, :, :gout.shape[2], :gout.shape[3]] = gout

    def conv_back(name, gz, act):
        inp, z = cache[name]
        if act:
            gz = gz * (z > 0)
        gi, gw, gb_ = on.conv2d_backward(inp, params[name][0], gz)
        grads[name] = (gw, gb_)
        return gi

    U, E, G = cache["U"], cache["E"], cache["G"]
    # image path, backwards
    g_ld, g_zd, g_J = [None] * L, [None] * L, [None] * L
    for s in range(L):
        gx, g_ld[s] = filter3_backward(gy, cache["fc_d"][s])
        g_J[s], gy, g_zd[s] = join_backward(gx, cache["jc"][s])
    gimg, g_lb = filter3_backward(gy, cache["fc_b"])
    g_le = [None] * L
    for s in reversed(range(L)):
        gj = g_J[s] + on.avgpool2_backward(gimg)
        gimg, g_le[s] = filter3_backward(gj, cache["fc_e"][s])
    g_od = gimg
    # K features, backwards
    g_U = [np.zeros_like(u) for u in U]
    g_B = np.zeros_like(cache["B"])
    g_prev = None                                   # dL/d G'_(s+1) flowing down
    for s in range(L):
        gg = conv_back(f"k_dec{s}_taps", g_ld[s], False) + conv_back(f"k_dec{s}_blend", g_zd[s][:, None], False)
        if g_prev is not None:
            gg = gg + g_prev
        gi = conv_back(f"k_dec{s}", gg, True)
        cu = gi.shape[1] - dec[s]
        g_U[s] += gi[:, cu:]
        hh, ww = U[s + 1].shape[2:] if s < L - 1 else cache["gb"].shape[2:]
        g_prev = on.upsample2_backward(gi[:, :cu], hh, ww)
    ggb = conv_back("k_bot_taps", g_lb, False) + g_prev
    gi = conv_back("k_bot", ggb, True)
    g_B += gi[:, enc[-1]:]
    g_G = on.avgpool2_backward(gi[:, :enc[-1]])
    for s in reversed(range(L)):
        gg = g_G + conv_back(f"k_enc{s}_taps", g_le[s], False)
        gi = conv_back(f"k_enc{s}", gg, True)
        if s == 0:
            g_U[0] += gi
        else:
            g_U[s] += gi[:, enc[s - 1]:]
            g_G = on.avgpool2_backward(gi[:, :enc[s - 1]])
    # D, backwards
    g_U[0] += conv_back("d_out", g_od, False)
    g_E = [None] * L
    for s in range(L):
        gi = conv_back(f"d_dec{s}a", conv_back(f"d_dec{s}b", g_U[s], True), True)
        cu = gi.shape[1] - enc[s]
        g_E[s] = gi[:, cu:]
        if s < L - 1:
            g_U[s + 1] += on.upsample2_backward(gi[:, :cu], U[s + 1].shape[2], U[s + 1].shape[3])
        else:
            g_B += on.upsample2_backward(gi[:, :cu], cache["B"].shape[2], cache["B"].shape[3])
    gt = conv_back("d_bota", conv_back("d_botb", g_B, True), True)
    for s in reversed(range(L)):
        ge = g_E[s] + on.avgpool2_backward(gt)
        gt = conv_back(f"d_enc{s}a", conv_back(f"d_enc{s}b", ge, True), True)
    return grads
