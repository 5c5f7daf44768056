// K-streamed tensor-core convolution of FP16 chunk-planar tensors (included
// by conv_tc.cu), for layers too wide to keep their weights and every input
// chunk of a tile in shared memory -- the two-stage network's 64-176-channel
// 3x3 layers and its 1x1 layers (paper: "Reconstruction Network", "Model
// Configuration").  Same arithmetic as the other convolutions: bias, optional
// ReLU, FP16 operands, FP32 accumulation in TMEM.
//
// A tile is TR output rows x TO pixels (3x3: TO = 126 of a 128-pixel halo
// row; 1x1: TO = 128, no halo).  Its K dimension -- input chunks x taps -- is
// streamed in groups of two chunks (16 channels, one MMA K step per tap):
// each ring stage holds one group's halo planes (TMA, zero-filled outside
// the frame and past the last chunk) and that group's weights (one bulk copy
// of a layout packed at load time: [group][tap][2 chunks][COUTP][16 B]).
//   warp 0     producer: TMA + bulk copies into a ring of NS stages;
//   warp 1     MMA issuer: per stage TAPS x TR MMAs (M = 128, N = COUTP,
//              K = 16) into one of two TMEM accumulators;
//   warps 2-5  epilogue: one pixel per thread, bias, ReLU, FP16 chunk stores
//              and / or FP32 planar stores (the small heads);
//   warps 6-13 (UP only) up-sampling, below.
// UP (decoder layers): the first ch0 chunks of the input are the bilinear x2
// up-sampling of source 0, a coarse tensor of half the height and width,
// computed in the kernel: for those groups the producer loads the coarse
// block under the tile (TR / 2 + 2 rows x 66 pixels per chunk) instead of the
// fine halo, and the up-sampling warps interpolate it into the stage's two
// halo planes (zero outside the frame) before the MMA warp, which waits on a
// per-stage "ready" barrier, reads them.  The interpolation is that of the
// separate up-sampling pass, operation for operation, so the results are
// the same bits.
// Every mbarrier wait has an iteration limit; a wait that gives up sets the
// error flag and the roles leave their loops.
#pragma once

#include "resample.cuh"

namespace fvn {
namespace ks {

constexpr int kThreads = 192;
constexpr int kHXW = 128;   // halo pixels per row (one TMA box row per chunk)

template <int COUTP, int TR, int NS, bool K1, bool UP = false>
struct Layout {
    static constexpr int HY = K1 ? TR : TR + 2;
    static constexpr int TO = K1 ? kHXW : kHXW - 2;              // output pixels per tile row
    static constexpr int TAPS = K1 ? 1 : 9;
    // one chunk plane of a stage; the MMA rows of the two unstored lanes of a
    // 3x3 tile read 32 bytes past the last halo row, kept zero
    static constexpr uint32_t plane = (HY * kHXW * 16 + 32 + 127) / 128 * 128;
    static constexpr uint32_t halo = 2 * plane;
    static constexpr uint32_t wgrp = TAPS * 2 * COUTP * 16;      // one group's weights
    // UP: coarse rows / columns under the HY x 128 fine pixels of a tile
    // (fine halo rows / columns start even - 1 for 3x3 and even for 1x1)
    static constexpr int CR = TR / 2 + 2, CC = kHXW / 2 + 2;
    static constexpr uint32_t cplane = (CR * CC * 16 + 127) / 128 * 128;
    static constexpr uint32_t coarse = UP ? 2 * cplane : 0;
    static constexpr uint32_t stage = halo + wgrp + coarse;
    static constexpr size_t bias_off = (size_t)NS * stage;
    static constexpr size_t bar_off = bias_off + COUTP * 4;
    static constexpr int nbar = 2 * NS + 5 + (UP ? NS : 0);      // full, empty, tfull, tempty, drain, ready
    static constexpr size_t bytes = bar_off + nbar * 8 + 16;
    static constexpr int up_warps = 8;
    static constexpr int threads = kThreads + (UP ? 32 * up_warps : 0);
    static_assert(!UP || TR % 2 == 0, "up-sampled tiles start on an even fine row");
    static constexpr uint32_t acc = TR * COUTP;                   // TMEM columns of one accumulator
    static constexpr uint32_t tmem_cols = 2 * acc <= 32 ? 32 : 2 * acc <= 64 ? 64 : 2 * acc <= 128 ? 128
                                        : 2 * acc <= 256 ? 256 : 512;
    static_assert(2 * acc <= 512, "two accumulators must fit in TMEM");
    static_assert(COUTP % 16 == 0 && COUTP <= 256, "unsupported output channels");
    static_assert(bytes <= 227 * 1024, "shared memory");
};

struct Args {
    CUtensorMap map0, map1;           // sources: chunk-planar FP16 [chunks][H][W][16 B]
    int ch0;                          // chunks of source 0 (the rest, if any, from source 1)
    int has1;
    int groups;                       // K groups of two chunks
    const uint4* w;                   // [groups][TAPS][2][COUTP][16 B] FP16
    const float* bias;                // [COUTP], zero padded
    uint4* out;                       // chunk-planar FP16 output, out_chunks chunks (NULL: none)
    int out_chunks;
    float* out32;                     // FP32 planar output [cout][H][W] (NULL: none)
    int cout, relu;
    int H, W, tiles_x, ntiles;
    int Hc, Wc;                       // UP: size of the coarse source 0
    int* error;
};

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

template <int COUTP, int TR, int NS, bool K1, bool UP>
__global__ void __launch_bounds__(Layout<COUTP, TR, NS, K1, UP>::threads)
    conv_ks_kernel(const __grid_constant__ Args a) {
    using L = Layout<COUTP, TR, NS, K1, UP>;
    constexpr int HY = L::HY, TO = L::TO;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sBias = reinterpret_cast<float*>(smem + L::bias_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + L::nbar);
    const uint32_t full0 = tc::smem_addr(bars), empty0 = full0 + 8 * NS;
    const uint32_t tfull0 = full0 + 16 * NS, tempty0 = tfull0 + 16;
    const uint32_t ready0 = tempty0 + 16 + 8;   // UP: after the drain barrier
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {   // the ring zeroed once (the over-read slack of the halo planes stays zero), bias
        uint4* z = reinterpret_cast<uint4*>(smem);
        for (int i = tid; i < (int)(L::bias_off / 16); i += L::threads) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < COUTP; i += L::threads) sBias[i] = __ldg(a.bias + i);
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(bars + s, 1);
            tc::mbar_init(bars + NS + s, 1);
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(bars + 2 * NS + k, 1);
            tc::mbar_init(bars + 2 * NS + 2 + k, 4);
        }
        tc::mbar_init(bars + 2 * NS + 4, 1);
        if (UP)
            for (int s = 0; s < NS; ++s) tc::mbar_init(bars + 2 * NS + 5 + s, L::up_warps);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, L::tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool failed = false;

    if (warp == 0) {
        // ---- producer: per tile, per group, the halo planes and the weights
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < a.ntiles && !failed; tile += gridDim.x) {
                const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
                const int x0 = tx * TO - (K1 ? 0 : 1), y0 = ty * TR - (K1 ? 0 : 1);
                const int cx0 = ((x0 + 1) >> 1) - 1, cy0 = ((y0 + 1) >> 1) - 1;   // UP: coarse block origin
                for (int g = 0; g < a.groups; ++g, ++i) {
                    const int s = i % NS, k = i / NS;
                    if (k > 0 && !ws::wait(empty0 + 8 * s, (k - 1) & 1)) {
                        failed = true;
                        break;
                    }
                    const uint32_t full = full0 + 8 * s;
                    const uint32_t dst = tc::smem_addr(smem + (size_t)s * L::stage);
                    if (UP && 2 * g < a.ch0) {   // the coarse block of an up-sampled group
                        ws::mbar_expect_tx(full, 2u * L::CR * L::CC * 16 + L::wgrp);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            ws::tma_load_3d(dst + L::halo + L::wgrp + kk * L::cplane, &a.map0, 2 * cx0, cy0,
                                            2 * g + kk, full);
                    } else {
                        ws::mbar_expect_tx(full, 2u * HY * kHXW * 16 + L::wgrp);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const int c = 2 * g + kk;   // past the last chunk: out of the map's range, zero-filled
                            const bool first = !UP && (c < a.ch0 || !a.has1);
                            ws::tma_load_3d(dst + kk * L::plane, first ? &a.map0 : &a.map1, 2 * x0, y0,
                                            first ? c : c - a.ch0, full);
                        }
                    }
                    bulk_load(dst + L::halo, a.w + (size_t)g * (L::wgrp / 16), L::wgrp, full);
                }
            }
            if (failed)   // let the copies already issued land before the CTA exits
                for (int j = (i > NS ? i - NS : 0); j < i; ++j) ws::wait(full0 + 8 * (j % NS), (j / NS) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_f16(128, COUTP);
            int i = 0, t = 0;
            for (int tile = blockIdx.x; tile < a.ntiles && !failed; tile += gridDim.x, ++t) {
                const int acc = t & 1;
                if (t >= 2 && !ws::wait(tempty0 + 8 * acc, ((t >> 1) - 1) & 1)) {
                    failed = true;
                    break;
                }
                for (int g = 0; g < a.groups; ++g, ++i) {
                    const int s = i % NS;
                    if (!ws::wait(full0 + 8 * s, (i / NS) & 1) || (UP && !ws::wait(ready0 + 8 * s, (i / NS) & 1))) {
                        failed = true;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t st = tc::smem_addr(smem + (size_t)s * L::stage);
                    const uint64_t a0 = tc::smem_desc(st, L::plane, 128);
                    const uint64_t b0 = tc::smem_desc(st + L::halo, COUTP * 16, 128);
#pragma unroll 1
                    for (int tap = 0; tap < L::TAPS; ++tap) {
                        const int dy = K1 ? 0 : tap / 3, dx = K1 ? 0 : tap - (tap / 3) * 3;
                        const uint64_t bd = b0 + (uint64_t)(tap * 2 * COUTP);
#pragma unroll
                        for (int r = 0; r < TR; ++r) {
                            const uint32_t d = tmem + (uint32_t)(acc * L::acc + r * COUTP);
                            const uint64_t ad = a0 + (uint64_t)((r + dy) * kHXW + dx);
                            tc::mma_f16(d, ad, bd, idesc, (g | tap) != 0);
                        }
                    }
                    tc::mma_commit(bars + NS + s);   // the stage is free once these MMAs are done
                }
                if (failed) break;
                tc::mma_commit(bars + 2 * NS + acc);   // the accumulator is ready for the epilogue
            }
            // every MMA issued must finish before the TMEM is freed: on success the last
            // accumulator's commit covers them, after a give-up one more commit (bounded wait)
            if (t > 0 && !failed) ws::wait(tfull0 + 8 * ((t - 1) & 1), ((t - 1) >> 1) & 1);
            if (failed && i > 0) {
                tc::mma_commit(bars + 2 * NS + 4);
                ws::wait(tc::smem_addr(bars + 2 * NS + 4), 0);
            }
        }
    } else if (warp < 6) {
        // ---- epilogue: warps 2-5, one pixel (TMEM lane) per thread
        const int q = warp & 3;
        const int px = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const long long plane = (long long)a.H * a.W;
        int t = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++t) {
            const int acc = t & 1;
            if (!ws::wait(tfull0 + 8 * acc, (t >> 1) & 1)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
            const int x = tx * TO + px;
            const bool xin = px < TO && x < a.W;
#pragma unroll 1
            for (int r = 0; r < TR; ++r) {
                const int y = ty * TR + r;
                const bool in = xin && y < a.H;
                const long long pix = (long long)y * a.W + x;
#pragma unroll 1
                for (int cb = 0; cb < COUTP; cb += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + lane_base + (uint32_t)(acc * L::acc + r * COUTP + cb), v);   // whole warp
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] += sBias[cb + j];
                        if (a.relu) v[j] = fmaxf(v[j], 0.f);
                    }
                    if (in) {
                        if (a.out) {
                            if (cb / 8 < a.out_chunks) a.out[(cb / 8) * plane + pix] = pack8h(v);
                            if (cb / 8 + 1 < a.out_chunks) a.out[(cb / 8 + 1) * plane + pix] = pack8h(v + 8);
                        }
                        if (a.out32) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (cb + j < a.cout) a.out32[(cb + j) * plane + pix] = v[j];
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) ws::mbar_arrive(tempty0 + 8 * acc);
        }
    } else if constexpr (UP) {
        // ---- up-sampling: warps 6-13 take every stage in the order of the
        // ring; for an up-sampled group, thread u writes (chunk, halo column)
        // items u, u + 256, .. down the HY halo rows, holding the x
        // interpolations of the two coarse rows it last used (consecutive fine
        // rows share one); then every stage is released to the MMA warp.
        const int ut = tid - kThreads;
        constexpr int NUT = 32 * L::up_warps;
        int i = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !failed; tile += gridDim.x) {
            const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
            const int x0 = tx * TO - (K1 ? 0 : 1), y0 = ty * TR - (K1 ? 0 : 1);
            const int cx0 = ((x0 + 1) >> 1) - 1, cy0 = ((y0 + 1) >> 1) - 1;
            for (int g = 0; g < a.groups; ++g, ++i) {
                const int s = i % NS;
                if (!ws::wait(full0 + 8 * s, (i / NS) & 1)) {
                    failed = true;
                    break;
                }
                if (2 * g < a.ch0) {
                    unsigned char* st = smem + (size_t)s * L::stage;
                    const unsigned char* cb = st + L::halo + L::wgrp;
                    for (int it = ut; it < 2 * kHXW; it += NUT) {
                        const int kk = it / kHXW, p = it - kk * kHXW;
                        uint4* dst = reinterpret_cast<uint4*>(st + kk * L::plane) + p;
                        const int gx = x0 + p;
                        if (gx < 0 || gx >= a.W) {
#pragma unroll
                            for (int j = 0; j < HY; ++j) dst[j * kHXW] = make_uint4(0, 0, 0, 0);
                            continue;
                        }
                        int ix0, ix1;
                        float fx;
                        up_src(gx, a.Wc, ix0, ix1, fx);
                        const uint4* crow = reinterpret_cast<const uint4*>(cb + kk * L::cplane);
                        const int lx0 = ix0 - cx0, lx1 = ix1 - cx0;
                        float ra[8], rb[8];   // x interpolations of local coarse rows ya, yb
                        int ya = -1, yb = -1;
#pragma unroll
                        for (int j = 0; j < HY; ++j) {
                            const int gy = y0 + j;
                            if (gy < 0 || gy >= a.H) {
                                dst[j * kHXW] = make_uint4(0, 0, 0, 0);
                                continue;
                            }
                            int iy0, iy1;
                            float fy;
                            up_src(gy, a.Hc, iy0, iy1, fy);
                            const int ly0 = iy0 - cy0, ly1 = iy1 - cy0;
                            if (ly0 != ya) {
                                if (ly0 == yb) {
#pragma unroll
                                    for (int k = 0; k < 8; ++k) ra[k] = rb[k];
                                } else {
                                    up_xlerp8(crow[ly0 * L::CC + lx0], crow[ly0 * L::CC + lx1], fx, ra);
                                }
                                ya = ly0;
                            }
                            if (ly1 != yb) {
                                if (ly1 == ya) {
#pragma unroll
                                    for (int k = 0; k < 8; ++k) rb[k] = ra[k];
                                } else {
                                    up_xlerp8(crow[ly1 * L::CC + lx0], crow[ly1 * L::CC + lx1], fx, rb);
                                }
                                yb = ly1;
                            }
                            dst[j * kHXW] = up_ylerp8(ra, rb, fy);
                        }
                    }
                    tc::fence_async_smem();   // generic-proxy writes, read next by the tensor core
                }
                __syncwarp();
                if (lane == 0) ws::mbar_arrive(ready0 + 8 * s);
            }
        }
    }
    if (failed) atomicExch(a.error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, L::tmem_cols);
    }
}

}  // namespace ks
}  // namespace fvn
