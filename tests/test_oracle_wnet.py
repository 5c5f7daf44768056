"""Pins for the oracle's two-stage network (direct prediction D, then kernels
predicted by K applied to D's output at several scales): the per-pixel
filter against brute force and a library box filter, invariants of the
whole network that fix its image path (constant images, identity kernels,
pure shifts), the decoder join against torch's pooling and bilinear
resampling, and every layer's gradient against finite differences.  No GPU."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F
from scipy.signal import convolve2d

from oracle import wnet as W

TINY = ((3, 5), 6, (4, 5))


def rand_params(cfg, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return W.unpack(rng.normal(size=W.param_count(cfg)) * scale, cfg)


def set_layer(P, name, w=0.0, b=None):
    wt, bt = P[name]
    P[name] = (np.full_like(wt, w), bt.copy() if b is None else np.asarray(b, np.float64) * np.ones_like(bt))


def test_filter_brute_force():
    rng = np.random.default_rng(0)
    img = rng.normal(size=(1, 3, 4, 5))
    lg = rng.normal(size=(1, 9, 4, 5)) * 2
    out, _ = W.filter3(img, lg)
    for y in range(4):
        for x in range(5):
            taps = [(q, y + q // 3 - 1, x + q % 3 - 1) for q in range(9)]
            taps = [(q, yy, xx) for q, yy, xx in taps if 0 <= yy < 4 and 0 <= xx < 5]
            e = [np.exp(lg[0, q, y, x]) for q, _, _ in taps]
            for c in range(3):
                ref = sum(ei * img[0, c, yy, xx] for ei, (_, yy, xx) in zip(e, taps)) / sum(e)
                assert abs(out[0, c, y, x] - ref) < 1e-12


def test_filter_uniform_logits_is_a_normalised_box():
    rng = np.random.default_rng(1)
    img = rng.normal(size=(2, 3, 9, 11))
    out, _ = W.filter3(img, np.full((2, 9, 9, 11), 0.7))
    ones = np.ones((3, 3))
    cnt = convolve2d(np.ones((9, 11)), ones, mode="same")
    for n in range(2):
        for c in range(3):
            ref = convolve2d(img[n, c], ones, mode="same") / cnt
            assert np.abs(out[n, c] - ref).max() < 1e-12


@pytest.mark.parametrize("q", range(9))
def test_filter_one_hot_logits_shift(q):
    rng = np.random.default_rng(q)
    img = rng.normal(size=(1, 3, 8, 10))
    lg = np.zeros((1, 9, 8, 10))
    lg[:, q] = 80.0
    out, _ = W.filter3(img, lg)
    dy, dx = q // 3 - 1, q % 3 - 1
    ref = np.roll(img, (-dy, -dx), axis=(2, 3))
    assert np.abs(out[..., 1:-1, 1:-1] - ref[..., 1:-1, 1:-1]).max() < 1e-12


def test_join_matches_torch_resampling():
    rng = np.random.default_rng(2)
    j = rng.normal(size=(2, 3, 6, 10))
    y = rng.normal(size=(2, 3, 3, 5))
    z = rng.normal(size=(2, 6, 10)) * 3
    x, _ = W.join(j, y, z)
    jt = torch.from_numpy(j)
    d = torch.from_numpy(y) - F.avg_pool2d(jt, 2)
    ref = jt + torch.sigmoid(torch.from_numpy(z))[:, None] * F.interpolate(d, scale_factor=2, mode="bilinear",
                                                                           align_corners=False)
    assert np.abs(x - ref.numpy()).max() < 1e-12


def test_plan_of_the_paper():
    """e64-e64-e80 pooled, d96 at 1/8, then d80-d64-d64 coming up: the
    decoder inputs concatenate the up-sampled block and the skip."""
    t = {name: (ci, co, k) for name, ci, co, k in W.layer_table(W.PAPER)}
    assert t["d_enc0a"] == (5, 64, 3) and t["d_enc2b"] == (80, 80, 3)
    assert t["d_bota"] == (80, 96, 3) and t["d_botb"] == (96, 96, 3)
    assert t["d_dec2a"] == (96 + 80, 80, 3) and t["d_dec1a"] == (80 + 64, 64, 3) and t["d_dec0a"] == (64 + 64, 64, 3)
    assert all(k == 1 for name, (_, _, k) in t.items() if name.startswith("k_"))
    assert t["k_bot"] == (80 + 96, 96, 1) and t["k_dec0"] == (64 + 64, 64, 1)
    assert W.param_count(W.PAPER) == sum(co * ci * k * k + co for ci, co, k in t.values())


@pytest.mark.parametrize("hw", [(8, 12), (7, 13), (1, 1)])
def test_constant_image_passes_through_k(hw):
    """F keeps a constant image, so does the join; a constant O_d (D's output
    layer with zero weights) leaves K unchanged, whatever K's weights."""
    P = rand_params(TINY, 3)
    set_layer(P, "d_out", 0.0, [0.3, 0.55, 0.8])
    sp = np.random.default_rng(4).uniform(size=(2, 5) + hw)
    out = W.forward(P, TINY, sp)
    ref = np.array([0.3, 0.55, 0.8])[None, :, None, None] * np.ones((2, 3) + hw)
    assert np.abs(out - ref).max() < 1e-12


def test_identity_kernels_return_the_direct_prediction():
    """Centre-tap kernels everywhere: J_s = I_s, Y_L = pool J_(L-1), so each
    join adds up(pool J_s - pool J_s) = 0 and the output is O_d, for any
    blend weights."""
    P = rand_params(TINY, 5)
    for name, _, co, _ in W.layer_table(TINY):
        if name.endswith("_taps"):
            set_layer(P, name, 0.0, [80.0 if q == 4 else 0.0 for q in range(9)])
    sp = np.random.default_rng(6).uniform(size=(1, 5, 12, 16))
    out = W.forward(P, TINY, sp)
    assert np.abs(out - W.direct(P, TINY, sp)).max() < 1e-12


def test_closed_join_gives_two_full_resolution_shifts():
    """Blend weights ~0 keep the encoder's image at every join, so the output
    is the full-resolution decoder filter applied to the full-resolution
    encoder filter: with one-hot kernels, two shifts of O_d."""
    P = rand_params(TINY, 7)
    for name, _, co, _ in W.layer_table(TINY):
        if name.endswith("_blend"):
            set_layer(P, name, 0.0, [-80.0])
    set_layer(P, "k_enc0_taps", 0.0, [80.0 if q == 5 else 0.0 for q in range(9)])    # (0, +1)
    set_layer(P, "k_dec0_taps", 0.0, [80.0 if q == 7 else 0.0 for q in range(9)])    # (+1, 0)
    sp = np.random.default_rng(8).uniform(size=(1, 5, 12, 16))
    od = W.direct(P, TINY, sp)
    out = W.forward(P, TINY, sp)
    ref = np.roll(od, (-1, -1), axis=(2, 3))
    assert np.abs(out[..., :-2, :-2] - ref[..., :-2, :-2]).max() < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(9)
    flat = rng.normal(size=W.param_count(TINY)) * 0.4
    sp = rng.uniform(size=(2, 5, 7, 9))
    P = W.unpack(flat, TINY)
    out, cache = W.forward(P, TINY, sp, return_cache=True)
    g = rng.normal(size=out.shape)
    ga = W.pack(W.backward(P, cache, g), TINY)

    def loss(f):
        return float((W.forward(W.unpack(f, TINY), TINY, sp) * g).sum())

    off = 0
    for name, ci, co, k in W.layer_table(TINY):
        n = co * ci * k * k + co
        for i in list(rng.choice(n - co, 2, replace=False)) + [n - co + int(rng.integers(co))]:
            e = np.zeros_like(flat)
            e[off + i] = 1e-6
            fd = (loss(flat + e) - loss(flat - e)) / 2e-6
            assert abs(fd - ga[off + i]) < 1e-6 * max(1.0, abs(fd)), name
        off += n


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """A join without the pooled subtraction, or a filter normalised over all
    nine taps at the border, breaks one of the pins above."""
    P = rand_params(TINY, 3)
    set_layer(P, "d_out", 0.0, [0.3, 0.55, 0.8])
    sp = np.random.default_rng(4).uniform(size=(1, 5, 8, 12))
    good = W.join

    def bad_join(j, y, z):
        x, c = good(j, y, z)
        return x - c["a"] * W.on.upsample2(-W.on.avgpool2(j)), c
    monkeypatch.setattr(W, "join", bad_join)
    assert np.abs(W.forward(P, TINY, sp) - np.array([0.3, 0.55, 0.8])[None, :, None, None]).max() > 1e-3
    monkeypatch.setattr(W, "join", good)

    def bad_filter(img, logits):
        nb, _ = W._shifted(img)
        e = np.exp(logits - logits.max(axis=1, keepdims=True))
        wq = e / e.sum(axis=1, keepdims=True)
        out = np.einsum("nqhw,ncqhw->nchw", wq, nb)
        return out, dict(wq=wq, nb=nb, out=out)
    monkeypatch.setattr(W, "filter3", bad_filter)
    assert np.abs(W.forward(P, TINY, sp) - np.array([0.3, 0.55, 0.8])[None, :, None, None]).max() > 1e-3


@pytest.mark.parametrize("cfg", [((5,), 4, (6,)), ((3, 4, 5), 6, (4, 3, 5))])
def test_constant_image_at_other_depths(cfg):
    """The image-path invariant with one and three levels (ragged frame)."""
    P = rand_params(cfg, 13)
    set_layer(P, "d_out", 0.0, [0.1, 0.2, 0.9])
    sp = np.random.default_rng(14).uniform(size=(1, 5, 11, 19))
    out = W.forward(P, cfg, sp)
    assert np.abs(out - np.array([0.1, 0.2, 0.9])[None, :, None, None]).max() < 1e-12


def test_flops_of_the_benchmark_roofline():
    """The two-stage roofline numerator: every convolution's 2 cin cout k^2 at
    its scale (4^-s of the pixels), plus 2 x 27 flops per filtered pixel at
    each of the image path's filters."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2209_09965_gb300 import workloads as wl
    enc, bot, dec = W.PAPER
    conv = 0.0
    scale = {"d_out": 0}
    for s in range(3):
        for pre in ("d_enc", "d_dec", "k_enc", "k_dec"):
            scale[f"{pre}{s}"] = s
    for name, ci, co, k in W.layer_table(W.PAPER):
        key = name if name == "d_out" else name[:6]
        s = 3 if "bot" in name else scale[key]
        conv += 2 * ci * co * k * k / 4 ** s
    filters = (1 + 1 / 4 + 1 / 16) * 2 + 1 / 64        # encoder and decoder filters per scale, the coarsest
    assert bench.wnet_flops_per_px(wl, W.PAPER) == pytest.approx(conv + filters * 54, rel=1e-12)
    assert 470e3 < conv < 480e3


WNET_MUTANTS = [
    ("filter taps in transposed order",
     "    for dy in (-1, 0, 1):\n        for dx in (-1, 0, 1):\n            vals.append(",
     "    for dx in (-1, 0, 1):\n        for dy in (-1, 0, 1):\n            vals.append(",
     [lambda: test_filter_one_hot_logits_shift(1)]),
    ("join blend inverted", "a = on.sigmoid(z)[:, None]", "a = on.sigmoid(-z)[:, None]",
     [test_join_matches_torch_resampling]),
    ("filter weights not normalised", "wq = e / e.sum(axis=1, keepdims=True)", "wq = e",
     [test_filter_uniform_logits_is_a_normalised_box]),
]


@pytest.mark.parametrize("what,old,new,pins", WNET_MUTANTS, ids=[m[0] for m in WNET_MUTANTS])
def test_planted_source_mistakes_fail_the_pins(what, old, new, pins, monkeypatch):
    """Each mistake, planted in a copy of the two-stage oracle's source (the
    oracle itself is not touched), breaks at least one pin above."""
    import types
    src = open(W.__file__).read()
    assert src.count(old) == 1, what
    mutant = types.ModuleType("oracle.wnet_mutant")
    mutant.__package__ = "oracle"
    exec(compile(src.replace(old, new), "wnet_mutant", "exec"), mutant.__dict__)
    monkeypatch.setitem(globals(), "W", mutant)
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught: {what}"
