"""Training of the reconstruction network on self-rendered pairs.

The network keeps FP32 master weights, gradients and Adam state (paper:
"Model Precision & Optimization": train in full precision, run with the
weights truncated to 16 bit); its 3x3 layers' forward, data and weight
gradients run on the tensor cores with BF16 operands and FP32 accumulation
(``--fp32``: every layer on the FP32 kernels, as the shipped weights were
trained).  It is trained on pairs
(sparse input, dense target) rendered by this library's own ray marcher
from seeded procedural volumes (the paper trains on renders of its CT and
simulation datasets, "Dataset" / "Training" sections).  Loss: L1 plus L1 of
the image gradients (the paper's perceptual and temporal terms, Eq. 4-7,
need VGG19 weights and optical flow that are not available).  Optimiser:
Adam, lr 1e-3 with cosine decay to ``lr_final``.

The recurrent network (``--recurrent``; paper: "Recurrence", the output of
D passed back to its input in the next run) is trained on two-frame
sequences -- the second frame's camera turned about the target by a small
random angle, its focal point moved and its mask drawn for the next frame
index -- with the first frame's output (no gradient) as the second's
history input, and the loss of Eq. 4 with lambda_s = 0.8 on the spatial
term above and lambda_t = 1.0 on the temporal term of Eq. 6 without its
optical-flow part, L1 of (O_1 - O_0) - (Y_1 - Y_0).  It starts from plain
weights (``--init``) with zero weights on the history channels, so its
first step is the plain network.

The two-stage network (``--wnet slim|paper``; paper: "Reconstruction
Network", D's direct prediction refined by K's kernels at several scales)
trains with the same loss on the same pairs; its initial kernels are close
to the identity, so it starts from D's output.

Every forward and backward step runs in the library's CUDA kernels, called
through ``torch.autograd.Function`` shims; parameter gradients are written by
the backward kernels straight into one flat gradient buffer on which the
Adam kernel steps.  Assembling a batch (choosing crop windows, slicing the
rendered frame) uses plain tensor indexing.

The shipped weights were made with

    python -m paper_2209_09965_gb300.train --fp32 --steps 30000 --lr-final 1e-5 --log-every 1000 \
        --out paper_2209_09965_gb300/weights/fvn_16_32_64.npy
    python -m paper_2209_09965_gb300.train --fp32 --steps 8000 --direct-only \
        --out paper_2209_09965_gb300/weights/fvn_direct_only.npy
    python -m paper_2209_09965_gb300.train --fp32 --recurrent --steps 6000 --lr 3e-4 --lr-final 1e-5 \
        --init paper_2209_09965_gb300/weights/fvn_16_32_64.npy --log-every 500 \
        --out paper_2209_09965_gb300/weights/fvn_16_32_64_recurrent.npy

and the equal-budget ablation of the reconstruction with

    python -m paper_2209_09965_gb300.train --fp32 --steps 4000 --direct-only \
        --out paper_2209_09965_gb300/weights/fvn_direct_only_4k.npy
    python -m paper_2209_09965_gb300.train --fp32 --steps 4000 --out paper_2209_09965_gb300/weights/fvn_16_32_64_4k.npy
    python -m paper_2209_09965_gb300.train --steps 4000 --wnet slim \
        --out paper_2209_09965_gb300/weights/fvn_wnet_slim_4k.npy
    python -m paper_2209_09965_gb300.train --steps 4000 --wnet paper \
        --out paper_2209_09965_gb300/weights/fvn_wnet_paper_4k.npy
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np
import torch

from . import fvn
from . import workloads as wl

LAYERS = wl.NET_LAYERS


class Params:
    """Flat FP32 master weights with per-layer views, flat gradient and Adam moments."""

    def __init__(self, flat: np.ndarray, device, layers=LAYERS):
        self.p = torch.from_numpy(np.ascontiguousarray(flat, np.float32)).to(device).requires_grad_(True)
        self.g = torch.zeros_like(self.p, requires_grad=False)
        self.m = torch.zeros_like(self.g)
        self.v = torch.zeros_like(self.g)
        self.step = 0
        self.recurrent = layers[0][1] == 8
        self.views = {}
        off = 0
        for name, ci, co, k in layers:
            nw = co * ci * k * k
            self.views[name] = (off, nw, (co, ci, k, k))
            off += nw + co

    def w(self, name):
        off, nw, shape = self.views[name]
        return self.p[off:off + nw].view(shape)

    def b(self, name):
        off, nw, shape = self.views[name]
        return self.p[off + nw:off + nw + shape[0]]

    def gw(self, name):
        off, nw, shape = self.views[name]
        return self.g[off:off + nw].view(shape)

    def gb(self, name):
        off, nw, shape = self.views[name]
        return self.g[off + nw:off + nw + shape[0]]

    def adam(self, lr=1e-3):
        self.step += 1
        join_wgrad(self.g.device)
        fvn.adam_step(self.p.data, self.g, self.m, self.v, self.step, lr=lr)

    def numpy(self):
        return self.p.detach().cpu().numpy().astype(np.float32)


class GraphedStep:
    """One optimiser step -- zero the gradients, forward, loss, backward,
    Adam -- captured once as a CUDA graph and replayed: its ~46 launches cost
    the host one graph launch, and no Python runs between the kernels.

    fwd(P, xs) is the network's forward (e.g. forward with tc=True).  Each
    call copies the batch into the graph's static inputs (when given), bumps
    the device step counter Adam reads, replays, and returns the loss as a
    device scalar (no host sync).  Building the graph runs the step once
    eagerly on a side stream (lazy initialisation of the kernels) with the
    parameters, moments and step restored afterwards."""

    def __init__(self, P: Params, xs: torch.Tensor, ys: torch.Tensor, fwd, lr=1e-3, lam=1.0):
        self.P, self.fwd, self.lr, self.lam = P, fwd, lr, lam
        self.xs, self.ys = xs.detach().clone(), ys.detach().clone()
        self.step_t = torch.full((1,), P.step, dtype=torch.int32, device=xs.device)
        saved = [t.detach().clone() for t in (P.p, P.m, P.v, self.step_t)]
        side = torch.cuda.Stream(device=xs.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._body()
        torch.cuda.current_stream().wait_stream(side)
        with torch.no_grad():
            for t, v in zip((P.p, P.m, P.v, self.step_t), saved):
                t.copy_(v)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self.loss = self._body()

    def _body(self):
        P = self.P
        P.g.zero_()
        pred = self.fwd(P, self.xs)
        # the loss and its gradient in one kernel; the backward pass starts
        # from that gradient (no loss node, no multiply by dL/dL = 1)
        loss = torch.zeros(1, device=pred.device)
        g = torch.empty_like(pred)
        fvn.loss_l1grad(pred.detach(), self.ys, self.lam, loss, g)
        pred.backward(g)
        join_wgrad(P.g.device)
        self.step_t.add_(1)
        fvn.adam_step_dev(P.p.data, P.g, P.m, P.v, self.step_t, lr=self.lr)
        return loss[0]

    def __call__(self, xs: torch.Tensor = None, ys: torch.Tensor = None):
        if xs is not None:
            self.xs.copy_(xs)
        if ys is not None:
            self.ys.copy_(ys)
        self.graph.replay()
        self.P.step += 1
        return self.loss


class _Conv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xa, xb, w, b, relu, gw, gb):
        n, _, h, wd = xa.shape
        y = torch.empty(n, w.shape[0], h, wd, device=xa.device)
        fvn.conv_fwd(xa, xb, w.detach(), b.detach(), relu, y)
        ctx.save_for_backward(xa, xb, w, y if relu else None)
        ctx.gwb = (gw, gb)
        ctx.relu = relu
        return y

    @staticmethod
    def backward(ctx, gy):
        xa, xb, w, y = ctx.saved_tensors
        gy = gy.contiguous()
        gxa = torch.empty_like(xa) if ctx.needs_input_grad[0] else None
        gxb = torch.empty_like(xb) if (xb is not None and ctx.needs_input_grad[1]) else None
        gw, gb = ctx.gwb
        fvn.conv_bwd(xa, xb, w.detach(), gy, y, gxa, gxb, gw, gb)
        # parameter gradients went straight to the flat buffer
        return gxa, gxb, None, None, None, None, None


_WGRAD_STREAMS = {}


def _wgrad_stream(device) -> torch.cuda.Stream:
    """The side stream the tensor-core weight gradients run on (per device)."""
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    if key not in _WGRAD_STREAMS:
        _WGRAD_STREAMS[key] = torch.cuda.Stream(device=key)
    return _WGRAD_STREAMS[key]


def join_wgrad(device):
    """Make the current stream wait for the weight gradients issued so far."""
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    if key in _WGRAD_STREAMS:
        torch.cuda.current_stream(key).wait_stream(_WGRAD_STREAMS[key])


class _ConvTC(torch.autograd.Function):
    """A 3x3 layer on the tensor cores: forward and data gradient as tcgen05
    implicit GEMMs with BF16 operands and FP32 accumulation, the weight
    gradient as a tcgen05 GEMM over the pixels (written straight into the
    flat buffer)."""

    @staticmethod
    def forward(ctx, xa, xb, w, b, relu, gw, gb):
        n, _, h, wd = xa.shape
        y = torch.empty(n, w.shape[0], h, wd, device=xa.device)
        fvn.conv3x3_fwd_bf16(xa, xb, w.detach(), b.detach(), relu, y)
        ctx.save_for_backward(xa, xb, w, y if relu else None)
        ctx.gwb = (gw, gb)
        return y

    @staticmethod
    def backward(ctx, gy):
        xa, xb, w, y = ctx.saved_tensors
        gy = gy.contiguous()
        ca, cb = xa.shape[1], 0 if xb is None else xb.shape[1]
        gxa = torch.empty_like(xa) if ctx.needs_input_grad[0] else None
        gxb = torch.empty_like(xb) if (xb is not None and ctx.needs_input_grad[1]) else None
        if gxa is not None or gxb is not None:
            fvn.conv3x3_dgrad_bf16(gy, y, w.detach(), ca, cb, gxa, gxb)
        gw, gb = ctx.gwb
        if not torch.cuda.is_current_stream_capturing():
            # eager: the host issues every launch, and the side stream's
            # bookkeeping would cost more host time than its overlap saves
            fvn.conv3x3_wgrad_bf16(xa, xb, gy, y, gw, gb)
            return gxa, gxb, None, None, None, None, None
        # captured in a CUDA graph: the weight gradient on a side stream (joined
        # before the optimiser reads the gradients), beside the data gradients
        # of this and the earlier layers
        side = _wgrad_stream(gy.device)
        side.wait_stream(torch.cuda.current_stream(gy.device))
        with torch.cuda.stream(side):
            fvn.conv3x3_wgrad_bf16(xa, xb, gy, y, gw, gb)
        for t in (xa, xb, gy, y):
            if t is not None:
                t.record_stream(side)
        # the backward pass ends with the caller's stream waiting for them
        dev = gy.device
        torch.autograd.Variable._execution_engine.queue_callback(lambda: join_wgrad(dev))
        return gxa, gxb, None, None, None, None, None


class _Pool(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        n, c, h, w = x.shape
        y = torch.empty(n, c, h // 2, w // 2, device=x.device)
        fvn.avgpool2_fwd(x, y)
        ctx.shape = x.shape
        return y

    @staticmethod
    def backward(ctx, gy):
        gx = torch.empty(ctx.shape, device=gy.device)
        fvn.avgpool2_bwd(gy.contiguous(), gx)
        return gx


class _Up(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        n, c, h, w = x.shape
        y = torch.empty(n, c, 2 * h, 2 * w, device=x.device)
        fvn.upsample2_fwd(x, y)
        ctx.shape = x.shape
        return y

    @staticmethod
    def backward(ctx, gy):
        gx = torch.empty(ctx.shape, device=gy.device)
        fvn.upsample2_bwd(gy.contiguous(), gx)
        return gx


class _KP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, head, sparse):
        n, _, h, w = head.shape
        out = torch.empty(n, 3, h, w, device=head.device)
        fvn.kp_blend_fwd(head, sparse, out)
        ctx.save_for_backward(head, sparse)
        return out

    @staticmethod
    def backward(ctx, gout):
        head, sparse = ctx.saved_tensors
        gh = torch.empty_like(head)
        fvn.kp_blend_bwd(head, sparse, gout.contiguous(), gh)
        return gh, None


class _HeadKP(torch.autograd.Function):
    """The 1x1 head and the kernel-prediction blend fused: one kernel forward
    (the head's output kept for the backward pass), one backward (dL/dx and
    the head's weight gradients, written straight into the flat buffer)."""

    @staticmethod
    def forward(ctx, x, sparse, w, b, gw, gb):
        n, _, h, wd = x.shape
        head = torch.empty(n, 29, h, wd, device=x.device)
        out = torch.empty(n, 3, h, wd, device=x.device)
        fvn.head_kp_fwd(x, w.detach(), b.detach(), sparse, head, out)
        ctx.save_for_backward(x, head, sparse, w)
        ctx.gwb = (gw, gb)
        return out

    @staticmethod
    def backward(ctx, gout):
        x, head, sparse, w = ctx.saved_tensors
        gx = torch.empty_like(x)
        gw, gb = ctx.gwb
        fvn.head_kp_bwd(x, head, sparse, w.detach(), gout.contiguous(), gx, gw, gb)
        return gx, None, None, None, None, None


class _Filter3(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, logits):
        out = torch.empty_like(img)
        fvn.filter3_fwd(img, logits, out)
        ctx.save_for_backward(img, logits)
        return out

    @staticmethod
    def backward(ctx, gout):
        img, logits = ctx.saved_tensors
        gimg, glog = torch.empty_like(img), torch.empty_like(logits)
        fvn.filter3_bwd(img, logits, gout.contiguous(), gimg, glog)
        return gimg, glog


class _Join(torch.autograd.Function):
    @staticmethod
    def forward(ctx, j, y, z):
        x = torch.empty_like(j)
        fvn.wnet_join_fwd(j, y, z, x)
        ctx.save_for_backward(j, y, z)
        return x

    @staticmethod
    def backward(ctx, gx):
        j, y, z = ctx.saved_tensors
        gj, gy, gz = torch.empty_like(j), torch.empty_like(y), torch.empty_like(z)
        fvn.wnet_join_bwd(j, y, z, gx.contiguous(), gj, gy, gz)
        return gj, gy, gz


class _Loss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, target, lam):
        loss = torch.zeros(1, device=pred.device)
        g = torch.empty_like(pred)
        fvn.loss_l1grad(pred, target, lam, loss, g)
        ctx.save_for_backward(g)
        return loss[0]

    @staticmethod
    def backward(ctx, gl):
        (g,) = ctx.saved_tensors
        return g * gl, None, None   # on the device: no host sync inside the backward pass


def forward(P: Params, sparse: torch.Tensor, direct_only: bool = False, prev: torch.Tensor = None,
            tc: bool = True):
    """Network forward on [N, 5, H, W] (H, W multiples of 4); returns [N, 3, H, W].
    The recurrent network also takes prev, the previous output [N, 3, H, W]
    (None: zeros), clamped to [0, 1].  tc: the 3x3 layers on the tensor cores
    (BF16 operands, FP32 accumulation) and the head fused with the blend;
    False: every layer on the FP32 kernels."""
    conv = _ConvTC if tc else _Conv

    def cbr(name, xa, xb=None):
        return conv.apply(xa, xb, P.w(name), P.b(name), True, P.gw(name), P.gb(name))

    if P.recurrent:
        n, _, h, w = sparse.shape
        hist = torch.zeros(n, 3, h, w, device=sparse.device) if prev is None else prev.detach().clamp(0, 1)
        e0 = cbr("enc0b", cbr("enc0a", sparse, hist.contiguous()))
    else:
        e0 = cbr("enc0b", cbr("enc0a", sparse))
    e1 = cbr("enc1b", cbr("enc1a", _Pool.apply(e0)))
    bt = cbr("botb", cbr("bota", _Pool.apply(e1)))
    d1 = cbr("dec1b", cbr("dec1a", _Up.apply(bt), e1))
    d0 = cbr("dec0b", cbr("dec0a", _Up.apply(d1), e0))
    if tc and not direct_only:
        return _HeadKP.apply(d0, sparse, P.w("head"), P.b("head"), P.gw("head"), P.gb("head"))
    head = _Conv.apply(d0, None, P.w("head"), P.b("head"), False, P.gw("head"), P.gb("head"))
    if direct_only:
        return head[:, 0:3].contiguous()
    return _KP.apply(head, sparse)


def wnet_forward(P: Params, sparse: torch.Tensor, cfg):
    """The two-stage network (fvn_reconstruct_wnet's layer sequence) on
    [N, 5, H, W], H and W multiples of 2^levels: D's direct prediction O_d and
    decoder states, K's per-block kernels and blend logits, then O_d through
    K's kernels in order.  Returns [N, 3, H, W]."""
    enc, _, _ = cfg
    n_lv = len(enc)

    def conv(name, xa, xb=None, relu=True):
        return _Conv.apply(xa, xb, P.w(name), P.b(name), relu, P.gw(name), P.gb(name))

    e, t = [], sparse
    for s in range(n_lv):
        e.append(conv(f"d_enc{s}b", conv(f"d_enc{s}a", t)))
        t = _Pool.apply(e[s])
    bt = conv("d_botb", conv("d_bota", t))
    u, below = [None] * n_lv, bt
    for s in reversed(range(n_lv)):
        u[s] = conv(f"d_dec{s}b", conv(f"d_dec{s}a", _Up.apply(below), e[s]))
        below = u[s]
    o_d = conv("d_out", u[0], relu=False)
    g, taps_e = [], []
    for s in range(n_lv):
        g.append(conv("k_enc0", u[0]) if s == 0 else conv(f"k_enc{s}", _Pool.apply(g[s - 1]), u[s]))
        taps_e.append(conv(f"k_enc{s}_taps", g[s], relu=False))
    gb = conv("k_bot", _Pool.apply(g[-1]), bt)
    taps_b = conv("k_bot_taps", gb, relu=False)
    taps_d, blend_d, below = [None] * n_lv, [None] * n_lv, gb
    for s in reversed(range(n_lv)):
        gd = conv(f"k_dec{s}", _Up.apply(below), u[s])
        taps_d[s] = conv(f"k_dec{s}_taps", gd, relu=False)
        blend_d[s] = conv(f"k_dec{s}_blend", gd, relu=False)
        below = gd
    j, img = [], o_d
    for s in range(n_lv):
        j.append(_Filter3.apply(img, taps_e[s]))
        img = _Pool.apply(j[s])
    y = _Filter3.apply(img, taps_b)
    for s in reversed(range(n_lv)):
        y = _Filter3.apply(_Join.apply(j[s], y, blend_d[s]), taps_d[s])
    return y


# ---------------------------------------------------------------------------
# self-rendered training pairs
# ---------------------------------------------------------------------------
class PairSource:
    """Crops of 1920x1080 frames of procedural volumes: the dense march of
    the crop's pixels is the target; the sparse input is the same samples
    kept where the foveated mask is set (the sparse march of a pixel equals
    its dense march)."""

    def __init__(self, ctx: fvn.Context, device, nvol=64, vol_n=512, seed=100, frame_w=1920, frame_h=1080,
                 crop=256, value_noise_share=0.5):
        self.ctx, self.dev = ctx, device
        self.W, self.H, self.crop = frame_w, frame_h, crop
        self.rng = np.random.default_rng(seed)
        self.vols = []
        for i in range(nvol):
            s = seed + i
            if i < int(nvol * (1 - value_noise_share)):
                v = wl.training_volume(vol_n, s, device=device)               # uint16 blobs + turbulence
            else:
                base = [16, 32, 64][i % 3] * vol_n // 256
                v = wl.value_noise_volume(vol_n, s, base_spacing=max(4, base), device=device)
                v = torch.round(v * 65535.0).to(torch.int32)
                v = (v - 65536 * (v >= 32768).to(torch.int32)).to(torch.int16)
            self.vols.append(v.contiguous())
        self.rgbam = torch.empty(5, frame_h, frame_w, device=device)
        self.mask = torch.empty(frame_h, frame_w, dtype=torch.uint8, device=device)
        self.ids_all = torch.empty(frame_w * frame_h, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        yy, xx = torch.meshgrid(torch.arange(crop, device=device), torch.arange(crop, device=device), indexing="ij")
        self.local = (yy * frame_w + xx).reshape(-1).to(torch.int32)

    def _render_crop(self, vol, tf, cam, mp, fov, x0, y0, xs, ys):
        """Dense march of the crop's pixels (target) and the masked copy (input)."""
        c, W, H = self.crop, self.W, self.H
        ids = self.local + (y0 * W + x0)
        cnt = torch.tensor([ids.numel()], dtype=torch.int32, device=self.dev)
        self.ctx.march(vol, tf, cam, mp, self.rgbam, ids=ids, count=cnt)
        self.ctx.make_mask(fov, W, H, self.mask, self.ids_all, self.count)
        win = self.rgbam[:, y0:y0 + c, x0:x0 + c]
        m = self.mask[y0:y0 + c, x0:x0 + c].to(torch.float32)
        ys.copy_(win[0:3])
        xs[0:4] = win[0:4] * m
        xs[4] = m

    def _draw(self):
        r, W, H, c = self.rng, self.W, self.H, self.crop
        vol = self.vols[r.integers(len(self.vols))]
        tf = torch.from_numpy(wl.transfer_function(int(r.integers(1 << 30)), alpha_max=r.uniform(0.03, 0.2)))
        cam = wl.random_camera(r, W, H, rmin=0.8, rmax=1.8)
        mp = wl.MarchParams(shading=int(r.uniform() < 0.85))
        fov = wl.Foveation(focal_px=(r.uniform(0.0, W), r.uniform(0.0, H)), fovea_radius=r.uniform(0.05, 0.15),
                           falloff_sigma=r.uniform(0.05, 0.15), p_base=r.uniform(0.03, 0.1),
                           seed=int(r.integers(1 << 30)), frame=int(r.integers(1 << 20)))
        # crop window: mostly around the screen centre where the volume is
        x0 = int(np.clip(r.normal(W / 2, W / 5) - c / 2, 0, W - c))
        y0 = int(np.clip(r.normal(H / 2, H / 5) - c / 2, 0, H - c))
        return vol, tf.to(self.dev), cam, mp, fov, x0, y0

    def sample(self, batch):
        c = self.crop
        xs = torch.empty(batch, 5, c, c, device=self.dev)
        ys = torch.empty(batch, 3, c, c, device=self.dev)
        for b in range(batch):
            vol, tf, cam, mp, fov, x0, y0 = self._draw()
            self._render_crop(vol, tf, cam, mp, fov, x0, y0, xs[b], ys[b])
        return xs, ys

    def sample_sequence(self, batch, max_angle_deg=6.0):
        """Two consecutive frames per crop: the second camera turned about the
        target around the up axis by U[0, max_angle] degrees, the focal point
        moved by up to 2 % of the width, the mask drawn for the next frame."""
        c, r = self.crop, self.rng
        xs = torch.empty(2, batch, 5, c, c, device=self.dev)
        ys = torch.empty(2, batch, 3, c, c, device=self.dev)
        for b in range(batch):
            vol, tf, cam, mp, fov, x0, y0 = self._draw()
            self._render_crop(vol, tf, cam, mp, fov, x0, y0, xs[0, b], ys[0, b])
            a = math.radians(r.uniform(0.0, max_angle_deg)) * (1 if r.uniform() < 0.5 else -1)
            up = np.asarray(cam.up, np.float64) / np.linalg.norm(cam.up)
            rel = np.asarray(cam.eye, np.float64) - np.asarray(cam.target, np.float64)
            rel = (rel * math.cos(a) + np.cross(up, rel) * math.sin(a) + up * (up @ rel) * (1 - math.cos(a)))
            cam1 = wl.Camera(eye=tuple(np.asarray(cam.target) + rel), target=cam.target, up=cam.up,
                             fov_y_deg=cam.fov_y_deg, width=cam.width, height=cam.height)
            d = 0.02 * self.W
            fov1 = wl.Foveation(focal_px=(fov.focal_px[0] + r.uniform(-d, d), fov.focal_px[1] + r.uniform(-d, d)),
                                fovea_radius=fov.fovea_radius, falloff_sigma=fov.falloff_sigma, p_base=fov.p_base,
                                seed=fov.seed, frame=fov.frame + 1)
            self._render_crop(vol, tf, cam1, mp, fov1, x0, y0, xs[1, b], ys[1, b])
        return xs, ys


LAMBDA_S, LAMBDA_T = 0.8, 1.0   # Eq. 4 weights of the spatial and temporal terms


def train(steps=3000, batch=8, lr=1e-3, seed=100, nvol=64, vol_n=512, out=None, direct_only=False,
          init_seed=3, log_every=100, device=None, lr_final=1e-4, recurrent=False, init=None, max_angle_deg=6.0,
          wnet=None, tc=True):
    """wnet: widths (enc, bot, dec) to train the two-stage network instead;
    tc: the single network's 3x3 layers on the tensor cores (False: FP32)."""
    device = device or torch.device("cuda")
    ctx = fvn.Context()
    src = PairSource(ctx, device, nvol=nvol, vol_n=vol_n, seed=seed)
    if wnet is not None:
        flat = np.load(init).astype(np.float32) if init else wl.wnet_weights(wnet, init_seed)
    else:
        flat = np.load(init).astype(np.float32) if init else wl.net_weights(init_seed)
    if wnet is not None:
        P = Params(flat, device, wl.wnet_layers(wnet))
    elif recurrent:
        if flat.size == wl.net_param_count():
            flat = wl.recurrent_weights(flat)
        P = Params(flat, device, wl.NET_LAYERS_RECURRENT)
    else:
        P = Params(flat, device)
    log = []
    t0 = time.time()
    for it in range(1, steps + 1):
        P.g.zero_()
        if recurrent:
            x, y = src.sample_sequence(batch, max_angle_deg)
            with torch.no_grad():
                o0 = forward(P, x[0], tc=tc)
            o1 = forward(P, x[1], prev=o0, tc=tc)
            loss = LAMBDA_S * _Loss.apply(o1, y[1], 1.0) + \
                LAMBDA_T * _Loss.apply(o1 - o0, (y[1] - y[0]).contiguous(), 0.0)
        else:
            x, y = src.sample(batch)
            pred = wnet_forward(P, x, wnet) if wnet is not None else forward(P, x, direct_only, tc=tc)
            loss = _Loss.apply(pred, y, 1.0)
        loss.backward()
        # cosine decay from lr to lr_final over the run
        cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * (it - 1) / max(1, steps - 1)))
        P.adam(cur)
        if it % log_every == 0 or it == 1:
            lv = float(loss.item())
            log.append((it, lv))
            print(f"step {it} loss {lv:.5f} lr {cur:.2e} {time.time() - t0:.1f}s", flush=True)
    w = P.numpy()
    if out:
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        np.save(out, w)
    ctx.close()
    return w, log


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--nvol", type=int, default=64)
    ap.add_argument("--vol-n", type=int, default=512)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--direct-only", action="store_true")
    ap.add_argument("--recurrent", action="store_true")
    ap.add_argument("--init", default=None, help="start from these weights (.npy)")
    ap.add_argument("--max-angle", type=float, default=6.0, help="recurrent: camera turn between frames, degrees")
    ap.add_argument("--wnet", choices=("slim", "paper"), default=None,
                    help="train the two-stage network with the single network's widths or the paper's")
    ap.add_argument("--out", default=None)
    ap.add_argument("--fp32", action="store_true",
                    help="every layer on the FP32 kernels (the shipped weights were trained so)")
    a = ap.parse_args()
    cfg = {"slim": wl.WNET_SLIM, "paper": wl.WNET_PAPER}.get(a.wnet)
    train(a.steps, a.batch, a.lr, a.seed, a.nvol, a.vol_n, a.out, a.direct_only, log_every=a.log_every,
          lr_final=a.lr_final, recurrent=a.recurrent, init=a.init, max_angle_deg=a.max_angle, wnet=cfg,
          tc=not a.fp32)


if __name__ == "__main__":
    main()
