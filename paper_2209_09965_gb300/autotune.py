"""Autotuner for the launch shapes of the hot path.

Times, with CUDA events on the current stream, the candidate settings of

* the march: the lane-refill threshold of the persistent kernel (how many
  lanes of a warp must still be busy before idle lanes take new rays) and the
  number of persistent CTAs per SM;
* the reconstruction convolutions: the tcgen05 (TMEM-accumulator) kernels or
  the mma.sync kernels;

on the caller's own frame, and installs the fastest in the context with
fvn_set_option.  Every candidate computes the same result; only the time
differs.
"""
from __future__ import annotations

import itertools

import torch

from . import fvn


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_march(ctx: fvn.Context, vol, tf, cam, mp, rgbam, ids=None, count=None,
               refills=(1, 8, 16, 24, 28), blocks=(0, 4, 6)):
    """Pick (refill threshold, CTAs per SM) for the march of this frame: the
    sparse march when ids are given, the dense march otherwise."""
    o_refill = fvn.OPT_MARCH_REFILL if ids is not None else fvn.OPT_MARCH_REFILL_DENSE
    o_blocks = fvn.OPT_MARCH_BLOCKS_PER_SM if ids is not None else fvn.OPT_MARCH_BLOCKS_PER_SM_DENSE
    results = {}
    for r, b in itertools.product(refills, blocks):
        ctx.set_option(o_refill, r)
        ctx.set_option(o_blocks, b)
        results[(r, b)] = _time(lambda: ctx.march(vol, tf, cam, mp, rgbam, ids=ids, count=count))
    best = min(results, key=results.get)
    ctx.set_option(o_refill, best[0])
    ctx.set_option(o_blocks, best[1])
    return {"refill": best[0], "blocks_per_sm": best[1], "ms": results[best],
            "candidates": {f"{k[0]}/{k[1]}": round(v, 4) for k, v in results.items()}}


def tune_conv(ctx: fvn.Context, rgbam, w, h, rgb):
    """Pick the convolution kernels (tcgen05 or mma.sync) for this frame size."""
    results = {}
    for name, impl in (("tcgen05", fvn.CONV_TCGEN05), ("mma_sync", fvn.CONV_MMA_SYNC)):
        ctx.set_option(fvn.OPT_CONV_KERNEL, impl)
        results[name] = _time(lambda: ctx.reconstruct(rgbam, w, h, rgb))
    best = min(results, key=results.get)
    ctx.set_option(fvn.OPT_CONV_KERNEL, fvn.CONV_TCGEN05 if best == "tcgen05" else fvn.CONV_MMA_SYNC)
    return {"conv": best, "ms": {k: round(v, 4) for k, v in results.items()}}
