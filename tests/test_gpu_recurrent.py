"""GPU parity of the recurrent network (the previous output as three more
input channels of the first layer; fvn_reconstruct_recurrent,
fvn_render_recurrent, batch views with a history) against the FP64 oracle,
and its training step (forward, gradients, temporal loss) against the
oracle's."""
import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP16_TOL = 2e-2
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def rec_weights(seed=3, scale=0.3):
    return wl.recurrent_weights(wl.net_weights(seed), history_scale=scale, seed=seed + 100)


@pytest.fixture(scope="module")
def ctx(fvn):
    c = fvn.Context()
    c.load_weights(rec_weights())
    yield c
    c.device_status()
    c.close()


def sparse_input(h, w, seed, density=0.2):
    rng = np.random.default_rng(seed)
    sp = np.zeros((5, h, w), np.float32)
    m = rng.uniform(size=(h, w)) < density
    sp[0:4] = rng.uniform(0.1, 0.9, (4, h, w)) * m
    sp[4] = m
    return sp


def history(h, w, seed):
    return np.random.default_rng(seed).uniform(-0.2, 1.2, (3, h, w)).astype(np.float32)   # clamped on input


def run(ctx, sp, prev=None, precision=0):
    _, h, w = sp.shape
    y = torch.full((3, h, w), 77.0, device=DEV)
    p = None if prev is None else torch.from_numpy(prev).to(DEV)
    ctx.reconstruct(torch.from_numpy(sp).to(DEV), w, h, y, precision=precision, prev=p)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("h,w,seed", [(64, 128, 0), (45, 70, 1), (1, 9, 2), (130, 67, 3)])
def test_recurrent_recon_matches_oracle(ctx, h, w, seed):
    sp, prev = sparse_input(h, w, seed), history(h, w, seed + 50)
    params = onet.unpack(rec_weights())
    out = run(ctx, sp, prev)
    ref = onet.forward(params, sp, prev=prev)
    assert np.abs(out - ref).max() < FP16_TOL
    # no history reads zeros; the history changes the output
    out0 = run(ctx, sp)
    assert np.array_equal(out0, run(ctx, sp, np.zeros((3, h, w), np.float32)))
    assert np.abs(out0 - onet.forward(params, sp)).max() < FP16_TOL
    assert np.abs(out - out0).max() > 1e-2


def test_zero_history_weights_give_the_plain_network(fvn):
    plain = wl.net_weights(3)
    a, b = fvn.Context(), fvn.Context()
    try:
        a.load_weights(plain)
        b.load_weights(wl.recurrent_weights(plain))
        sp = sparse_input(72, 96, 7)
        pa = run(a, sp)
        pb = run(b, sp, history(72, 96, 8))
        assert np.abs(pa - pb).max() < 1e-6
    finally:
        a.close()
        b.close()


def test_history_needs_recurrent_weights(fvn):
    c = fvn.Context()
    try:
        c.load_weights(wl.net_weights(3))
        with pytest.raises(fvn.FvnError, match="FVN_ERR_STATE"):
            run(c, sparse_input(16, 16, 0), history(16, 16, 1))
        assert fvn.weight_count_recurrent() == fvn.weight_count() + 16 * 3 * 9
    finally:
        c.close()


def test_render_and_batch_with_history(fvn):
    c = fvn.Context()
    try:
        c.load_weights(rec_weights(5))
        vol = torch.from_numpy(wl.blob_volume(48, seed=11).numpy().astype(np.float32)).to(DEV)
        tf = torch.from_numpy(wl.transfer_function(31, alpha_max=0.3)).to(DEV)
        mp = wl.MarchParams(shading=1)
        views = []
        for i, (w, h) in enumerate([(160, 120), (97, 61)]):
            cam = wl.orbit_camera(40 + i, i, width=w, height=h, radius_factor=(1.0, 1.4))
            fov = wl.Foveation(focal_px=wl.focal_point(40 + i, i, w, h), seed=40 + i, frame=i)
            views.append({"vol": vol, "tf": tf, "cam": cam, "fov": fov,
                          "rgb": torch.full((3, h, w), 5.0, device=DEV),
                          "rgbam": torch.full((5, h, w), 9.0, device=DEV),
                          "prev": torch.from_numpy(history(h, w, 60 + i)).to(DEV)})
        c.render_batch(views, mp)
        for v in views:
            w, h = v["cam"].width, v["cam"].height
            rgb = torch.empty(3, h, w, device=DEV)
            rgbam = torch.empty(5, h, w, device=DEV)
            c.render(v["vol"], v["tf"], v["cam"], v["fov"], mp, rgb, rgbam_out=rgbam, prev=v["prev"])
            again = torch.empty(3, h, w, device=DEV)
            c.reconstruct(rgbam, w, h, again, prev=v["prev"])
            torch.cuda.synchronize()
            assert torch.equal(v["rgb"], rgb) and torch.equal(rgb, again)
        c.device_status()
    finally:
        c.close()


def test_recurrent_fp8(fvn):
    c = fvn.Context()
    try:
        c.load_weights(rec_weights(6, 0.2))
        sp, prev = sparse_input(96, 128, 9, density=0.3), history(96, 128, 10)
        c.calibrate_fp8(torch.from_numpy(sp).to(DEV), 128, 96)
        out = run(c, sp, prev, precision=fvn.PREC_FP8)
        ref = onet.forward(onet.unpack(rec_weights(6, 0.2)), sp, prev=prev)
        mse = np.mean((out - ref) ** 2)
        assert -10 * np.log10(mse) > 30.0
    finally:
        c.close()


def test_recurrent_training_step_matches_oracle(fvn):
    """train.forward with a history input, the spatial + temporal loss and
    their gradients through the library's FP32 kernels against the oracle."""
    from paper_2209_09965_gb300 import train
    rng = np.random.default_rng(17)
    flat = rec_weights(7, 0.2)
    flat = (flat + rng.normal(size=flat.size).astype(np.float32) * 0.01).astype(np.float32)
    n, h, w = 2, 16, 20
    sp = np.zeros((n, 5, h, w), np.float32)
    m = rng.uniform(size=(n, h, w)) < 0.3
    sp[:, 0:4] = rng.uniform(size=(n, 4, h, w)) * m[:, None]
    sp[:, 4] = m
    o_prev = rng.uniform(-0.1, 1.1, (n, 3, h, w)).astype(np.float32)
    y0, y1 = rng.uniform(size=(2, n, 3, h, w)).astype(np.float32)
    P = train.Params(flat, DEV, wl.NET_LAYERS_RECURRENT)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)   # noqa: E731
    o1 = train.forward(P, T(sp), prev=T(o_prev), tc=False)
    loss = train.LAMBDA_S * train._Loss.apply(o1, T(y1), 1.0) + \
        train.LAMBDA_T * train._Loss.apply(o1 - T(o_prev), T(y1 - y0), 0.0)
    P.g.zero_()
    loss.backward()
    torch.cuda.synchronize()
    params = onet.unpack(flat)
    ref, cache = onet.forward(params, sp.astype(np.float64), return_cache=True, prev=o_prev)
    ls, gs = onet.loss_l1_grad(ref, y1)
    lt, gt = onet.loss_temporal(ref, o_prev, y1, y0)
    assert np.abs(o1.detach().cpu().numpy() - ref).max() < 1e-4
    assert abs(float(loss.item()) - (train.LAMBDA_S * ls + train.LAMBDA_T * lt)) < 1e-5
    grads = onet.pack(onet.backward(params, cache, train.LAMBDA_S * gs + train.LAMBDA_T * gt))
    g = P.g.cpu().numpy().astype(np.float64)
    assert np.abs(g - grads).max() < 2e-3 * np.abs(grads).max()


def test_recurrent_training_runs(fvn):
    from paper_2209_09965_gb300 import train
    w, log = train.train(steps=20, nvol=2, vol_n=64, log_every=10, batch=2, recurrent=True)
    assert w.size == wl.net_param_count(wl.NET_LAYERS_RECURRENT)
    assert all(np.isfinite(v) for _, v in log)
