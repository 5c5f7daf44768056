"""Autotuner for the launch shapes of the hot path.

Times, with CUDA events on the current stream, the candidate settings of

* the march: the lane-refill threshold of the persistent kernel (how many
  lanes of a warp must still be busy before idle lanes take new rays), the
  cooperative-finish threshold (how few rays a warp must have left before it
  marches them with all 32 lanes) and the number of persistent CTAs per SM;
* the network: the output rows per tile of its half-resolution,
  quarter-resolution and first decoder convolutions;

on the caller's own frame, and installs the fastest in the context with
fvn_set_option.  Every candidate computes the same result (the cooperative
finish up to FP32 rounding order); only the time differs.
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
               refills=(1, 8, 16, 24), blocks=(0, 4), coops=(0, 2, 4, 8, 16, 32)):
    """Pick (refill threshold, cooperative-finish threshold, CTAs per SM) for
    the march of this frame: the sparse march when ids are given, the dense
    march otherwise."""
    sparse = ids is not None
    o_refill = fvn.OPT_MARCH_REFILL if sparse else fvn.OPT_MARCH_REFILL_DENSE
    o_blocks = fvn.OPT_MARCH_BLOCKS_PER_SM if sparse else fvn.OPT_MARCH_BLOCKS_PER_SM_DENSE
    o_coop = fvn.OPT_MARCH_COOP if sparse else fvn.OPT_MARCH_COOP_DENSE
    results = {}
    for r, c, b in itertools.product(refills, coops, blocks):
        ctx.set_option(o_refill, r)
        ctx.set_option(o_coop, c)
        ctx.set_option(o_blocks, b)
        results[(r, c, b)] = _time(lambda: ctx.march(vol, tf, cam, mp, rgbam, ids=ids, count=count))
    best = min(results, key=results.get)
    ctx.set_option(o_refill, best[0])
    ctx.set_option(o_coop, best[1])
    ctx.set_option(o_blocks, best[2])
    return {"refill": best[0], "coop": best[1], "blocks_per_sm": best[2], "ms": results[best],
            "candidates": {f"{k[0]}/{k[1]}/{k[2]}": round(v, 4) for k, v in results.items()}}


def tune_conv_tiles(ctx: fvn.Context, rgbam, w, h, rgb, precision=fvn.PREC_FP16, halves=(2, 4), quarters=(1, 2, 4),
                    dec1=(1, 2), fuse_up=(0, 1)):
    """Pick the network's tile shapes for this frame size: output rows per tile
    of the half-resolution 32-channel convolutions, of the quarter-resolution
    bottleneck and of the first decoder convolution (every choice gives the
    same output bit for bit; fewer rows per tile mean more, smaller tiles for
    the persistent CTAs, more rows less halo re-reading), and whether the first
    decoder convolution up-samples its input itself (the same result up to
    FP16 rounding of the interpolation)."""
    results = {}
    for a, b, c, f in itertools.product(halves, quarters, dec1, fuse_up):
        ctx.set_option(fvn.OPT_CONV_ROWS_HALF, a)
        ctx.set_option(fvn.OPT_CONV_ROWS_QUARTER, b)
        ctx.set_option(fvn.OPT_CONV_ROWS_DEC1, c)
        ctx.set_option(fvn.OPT_CONV_FUSE_UP_DEC1, f)
        results[(a, b, c, f)] = _time(lambda: ctx.reconstruct(rgbam, w, h, rgb, precision=precision), reps=5)
    best = min(results, key=results.get)
    ctx.set_option(fvn.OPT_CONV_ROWS_HALF, best[0])
    ctx.set_option(fvn.OPT_CONV_ROWS_QUARTER, best[1])
    ctx.set_option(fvn.OPT_CONV_ROWS_DEC1, best[2])
    ctx.set_option(fvn.OPT_CONV_FUSE_UP_DEC1, best[3])
    return {"rows_half": best[0], "rows_quarter": best[1], "rows_dec1": best[2], "fuse_up_dec1": best[3],
            "ms": results[best], "candidates": {"/".join(map(str, k)): round(v, 4) for k, v in results.items()}}
