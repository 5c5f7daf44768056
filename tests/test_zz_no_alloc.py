"""fvn_reconstruct_noalloc: the reconstruction for callers that cannot
allocate device memory at call time (graph capture, fixed memory budgets,
real-time loops).  It runs on a fixed device array inside the library, so
its results must equal fvn_reconstruct's; this file is collected last so a
failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2209_09965_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvn():
    import __graft_entry__ as ge
    ge.build()
    from paper_2209_09965_gb300 import fvn as f
    return f


def sparse(h, w, seed, density=0.2):
    rng = np.random.default_rng(seed)
    sp = np.zeros((5, h, w), np.float32)
    m = rng.uniform(size=(h, w)) < density
    sp[0:4] = rng.uniform(size=(4, h, w)) * m
    sp[4] = m
    return torch.from_numpy(sp).cuda()


def _noalloc(fvn, ctx, x, w, h, out, precision):
    lib = fvn.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.fvn_reconstruct_noalloc(ctx.h, ctypes.c_void_p(x.data_ptr()), w, h, precision,
                                     ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0, lib.fvn_last_error(ctx.h)


@pytest.mark.parametrize("precision", ["fp16", "fp8"])
def test_noalloc_matches_reconstruct_on_two_calls(fvn, precision):
    """Same kernels and weights as fvn_reconstruct, only another workspace:
    the outputs must be identical bit for bit, on two calls in a row (the
    second reuses the array the first left behind)."""
    ctx = fvn.Context()
    ctx.load_weights(wl.net_weights(3))
    prec = fvn.PREC_FP16 if precision == "fp16" else fvn.PREC_FP8
    if prec == fvn.PREC_FP8:
        ctx.calibrate_fp8(sparse(256, 320, 9), 320, 256)
    for call, (h, w, seed) in enumerate([(120, 200, 1), (512, 512, 2)]):
        x = sparse(h, w, seed)
        ref = torch.empty(3, h, w, device="cuda")
        out = torch.full((3, h, w), float("nan"), device="cuda")
        ctx.reconstruct(x, w, h, ref, precision=prec)
        _noalloc(fvn, ctx, x, w, h, out, prec)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (precision, call, (out - ref).abs().max().item())
    ctx.close()


def test_noalloc_rejects_frames_beyond_its_workspace(fvn):
    ctx = fvn.Context()
    ctx.load_weights(wl.net_weights(3))
    x = torch.zeros(5, 1080, 1920, device="cuda")
    y = torch.zeros(3, 1080, 1920, device="cuda")
    with pytest.raises(fvn.FvnError, match="fixed"):
        ctx.reconstruct_noalloc(x, 1920, 1080, y)
    assert float(y.abs().max()) == 0.0          # nothing was enqueued
    ctx.close()
