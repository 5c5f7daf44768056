// Warp-specialised tensor-core convolution with TMA staging (included by
// conv_tc.cu).  Same arithmetic as conv3x3_tc_kernel's plain layers (paper:
// "Reconstruction Network"): 3x3 conv, bias, ReLU, optional fused 2x2 average
// pooling, FP16 or FP8 operands, FP32 accumulation in TMEM; the input is one
// tensor or the channel concatenation of two (the up-sampled coarse
// level and the skip tensor of a decoder layer).
//
// One persistent CTA of 6 warps per SM (or two, when they fit) runs three
// roles concurrently over its tiles (TR rows x 126 pixels):
//   warp 0     producer: TMA loads of the tile's halo (one box of 128
//              pixels x 16 bytes x TR+2 rows per channel chunk, zero-filled
//              outside the frame) into a ring of NS shared-memory stages;
//   warp 1     MMA issuer: tcgen05.mma per output row into one of two TMEM
//              accumulators; commits free the stage and hand the accumulator
//              to the epilogue;
//   warps 2-5  epilogue: tcgen05.ld of one pixel per thread, scale, bias,
//              ReLU, FP16 / FP8 stores, pooling.
// Activations are chunk-planar ([C / chunk][H][W][16 B]), so each TMA box
// row is 128 contiguous 16-byte vectors.
// so loads, MMAs and stores of consecutive tiles overlap.  Every mbarrier wait
// has an iteration limit; a wait that gives up sets the error flag, and every
// role then leaves its loop, waits (bounded) for its own operations in
// flight, and the TMEM is freed.
#pragma once

#include <cuda.h>

namespace fvn {
namespace ws {

constexpr int kThreads = 192;
// A tile row is 126 output pixels computed as one MMA of M = 128 (the last
// two TMEM lanes are not stored), so that its halo row is 128 pixels = 2048
// contiguous bytes per channel chunk: one TMA box row (256 8-byte elements).
// Loading rows of 16-byte elements instead runs the copy engine far below
// its bandwidth.
constexpr int kTW = 128;              // MMA M = pixels per TMEM accumulator row
constexpr int kTO = 126;              // output pixels per tile row
constexpr int kHXW = 128;             // halo pixels per row
constexpr uint32_t kLimit = 1u << 26;

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < kLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// FUSE (row-fused MMAs): each halo row is multiplied once by the three
// vertical taps' weights stacked along N (N = 3 COUT), accumulating into the
// three output rows it feeds; the accumulators of a tile are laid out so
// that those three are adjacent (output row r at column COUT (TR + 1 - r)),
// which halves the operand reads of the tensor core at TR = 4.  The weights
// are then kept as [dx][chunk][dy][COUT][16 B].
//
// UPC > 0 (decoder layers): the first UPC chunks of the input are the
// bilinear x2 up-sampling of a coarse tensor, computed in the kernel: the
// producer loads the coarse rows / columns under the tile (CR x CC pixels
// per chunk) next to each stage, and up-sampling warps interpolate them into
// the stage's first UPC chunk planes before the MMAs read it.  CB1: one
// coarse buffer for all stages (where per-stage ones would leave room for
// fewer stages): the producer loads a tile's coarse block once the
// up-sampling warps have released the previous one.
template <int CIN, int COUT, int TR, int NS, bool F8, bool FUSE = false, int UPC = 0, bool CB1 = false>
struct Layout {
    static constexpr int EB = F8 ? 1 : 2;
    static constexpr int CPC = 16 / EB;                      // channels per 16-byte chunk
    static constexpr int CH = CIN / CPC;                     // chunks per pixel = K per tap / chunk
    static constexpr int HY = TR + 2;
    // one chunk plane of a stage; the MMA rows of the two unstored lanes read
    // 32 bytes past the last halo row, kept zero
    static constexpr uint32_t plane = (HY * kHXW * 16 + 32 + 127) / 128 * 128;
    static constexpr uint32_t stage = CH * plane;
    // coarse rows and columns under the HY x 128 fine halo of a tile
    static constexpr int CR = (TR + 1) / 2 + 2, CC = kHXW / 2 + 1;
    static constexpr uint32_t cchunk = (CR * CC * 16 + 127) / 128 * 128;     // one coarse chunk (TMA target)
    static constexpr uint32_t coarse = UPC * cchunk;                          // per stage
    static constexpr size_t w_bytes = 9ull * CIN * COUT * EB;
    static constexpr size_t stage_off = (w_bytes + 1023) / 1024 * 1024;
    static constexpr size_t zero_off = stage_off + (size_t)NS * stage;   // zero A operand (FUSE)
    static constexpr size_t zero_bytes = FUSE ? 2 * kTW * 16 : 0;
    static constexpr size_t coarse_off = zero_off + zero_bytes;
    static constexpr size_t bias_off = coarse_off + (size_t)(CB1 ? 1 : NS) * coarse;
    static constexpr size_t bar_off = bias_off + 2 * COUT * 4;
    static constexpr int nbar = 2 * NS + 4 + (UPC ? NS : 0) + (CB1 ? 1 : 0);   // full, empty, tfull, tempty, ready, coarse free
    static constexpr size_t bytes = bar_off + nbar * 8 + 16;
    static constexpr int up_warps = 8;                                 // up-sampling warps (UPC > 0)
    static constexpr int threads = 64 + 32 * 4 + (UPC ? 32 * up_warps : 0);
    static_assert(UPC == 0 || 2 * CC <= 256, "coarse box wider than a TMA box");
    static_assert(!CB1 || UPC > 0, "a shared coarse buffer needs up-sampled chunks");
    static constexpr uint32_t acc = (FUSE ? TR + 4 : TR) * COUT;   // TMEM columns of one accumulator
    static constexpr uint32_t tmem_cols = 2 * acc <= 32 ? 32 : 2 * acc <= 64 ? 64 : 2 * acc <= 128 ? 128
                                        : 2 * acc <= 256 ? 256 : 512;
    static_assert(2 * acc <= 512, "two accumulators must fit in TMEM");
    static_assert(!FUSE || acc <= 256, "the zeroing MMA covers at most 256 columns");
    static_assert(!FUSE || 9ull * CIN * COUT * EB >= (size_t)acc * 32, "zeroing MMA reads B from the weights");
    static_assert(CIN % (2 * CPC) == 0, "K per tap must be a multiple of the MMA K");
    static_assert(COUT % 16 == 0 && COUT <= 64, "unsupported output channels");
};

// One image of a launch: its input tensor maps (source 0 = the first CH0
// chunks, source 1 = the rest), outputs and size.
struct Img {
    CUtensorMap map0, map1;
    void* out;                        // [Hl][Wl][COUT]
    void* pooled;                     // [Hl/2][Wl/2][COUT]
    int Hl, Wl;
    int tiles_x, tile0;
};

struct Args {
    const void* w;                    // [9][CIN/CPC][COUT][16 B]
    const float* bias;
    const float* wscale;              // FP8: per output channel weight scale
    float out_q, pool_q;              // FP8: 1 / s of the output / pooled tensor
    int ntiles, nimg;
    int* error;
    Img img[kMaxViews];
};

__device__ __forceinline__ int find_img(const Args& a, int tile) {
    int i = 0;
    while (i + 1 < a.nimg && tile >= a.img[i + 1].tile0) ++i;
    return i;
}

// Store COUT channels of one pixel into a chunk-planar tensor ([C / chunk]
// planes of H x W 16-byte vectors; plane = H W).
template <int COUT, bool F8>
__device__ __forceinline__ void store_px(void* base, long long plane, long long pix, const float* v, float q) {
    uint4* o = static_cast<uint4*>(base) + pix;
    if (F8) {
#pragma unroll
        for (int c = 0; c < COUT; c += 16) {
            float s[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) s[j] = v[c + j] * q;
            o[(c / 16) * plane] = pack16q(s);
        }
    } else {
#pragma unroll
        for (int c = 0; c < COUT; c += 8) o[(c / 8) * plane] = pack8h(v + c);
    }
}

// The up-sampling of the decoder input works on half2 pairs (the operands
// the tensor core reads are FP16 / FP8 anyway): a 16-byte chunk is NP = 4
// (FP16) or 8 (FP8, widened from E4M3) pairs.
template <bool F8>
__device__ __forceinline__ void chunk_to_h2(uint4 u, __half2* h) {
    if (F8) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const __half2_raw r =
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((w[i] >> (16 * j)) & 0xFFFFu), __NV_E4M3);
                h[2 * i + j] = *reinterpret_cast<const __half2*>(&r);
            }
    } else {
        const __half2* p = reinterpret_cast<const __half2*>(&u);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = p[i];
    }
}
template <bool F8>
__device__ __forceinline__ uint4 h2_to_chunk(const __half2* h) {
    if (F8) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t lo = __nv_cvt_halfraw2_to_fp8x2(*reinterpret_cast<const __half2_raw*>(&h[2 * i]),
                                                           __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi = __nv_cvt_halfraw2_to_fp8x2(*reinterpret_cast<const __half2_raw*>(&h[2 * i + 1]),
                                                           __NV_SATFINITE, __NV_E4M3);
            w[i] = lo | (hi << 16);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    uint4 u;
    __half2* p = reinterpret_cast<__half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = h[i];
    return u;
}

// One coarse row of a chunk interpolated along x at a fine column: the
// coarse pixels lx0, lx1 of `row` (16-byte chunks) with weight fx on lx1.
template <bool F8>
__device__ __forceinline__ void coarse_hlerp(const uint4* row, int lx0, int lx1, __half2 fx, __half2* h) {
    constexpr int NP = F8 ? 8 : 4;
    __half2 p0[NP], p1[NP];
    chunk_to_h2<F8>(row[lx0], p0);
    chunk_to_h2<F8>(row[lx1], p1);
#pragma unroll
    for (int j = 0; j < NP; ++j) h[j] = __hfma2(fx, __hsub2(p1[j], p0[j]), p0[j]);
}

// CIN: K per tap (padded); CHG: chunks read from memory (the others stay
// zero); CH0: chunks from source 0 (UPC > 0: CH0 == UPC chunks up-sampled
// from the coarse tensor of source 0).
template <int CIN, int CHG, int CH0, int COUT, int TR, int NS, bool POOL, bool F8, bool FUSE, int UPC = 0,
          bool CB1 = false>
__global__ void __launch_bounds__(Layout<CIN, COUT, TR, NS, F8, FUSE, UPC, CB1>::threads)
    conv3x3_ws_kernel(const __grid_constant__ Args a) {
    using L = Layout<CIN, COUT, TR, NS, F8, FUSE, UPC, CB1>;
    constexpr int CH = L::CH, HY = L::HY, kThreads = L::threads;
    static_assert(UPC == 0 || UPC == CH0, "up-sampled chunks are source 0");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem;
    unsigned char* sStage = smem + L::stage_off;
    float* sBias = reinterpret_cast<float*>(smem + L::bias_off);
    float* sScale = sBias + COUT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + L::nbar);
    const uint32_t full0 = tc::smem_addr(bars), empty0 = full0 + 8 * NS;
    const uint32_t tfull0 = full0 + 16 * NS, tempty0 = tfull0 + 16;
    const uint32_t ready0 = tempty0 + 16;   // UPC: stage's up-sampled planes written
    const uint32_t cfree0 = ready0 + 8 * NS;   // CB1: the coarse buffer read by the up-sampling warps

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {   // resident weights, bias, scales; chunks never loaded stay zero
        const uint4* src = static_cast<const uint4*>(a.w);
        uint4* dst = reinterpret_cast<uint4*>(sW);
        for (int i = tid; i < (int)(L::w_bytes / 16); i += kThreads) {
            int d = i;
            if (FUSE) {   // [tap][chunk][o] -> [dx][chunk][dy][o]
                const int o = i % COUT, t2 = i / COUT, ch = t2 % CH, tap = t2 / CH;
                d = (((tap % 3) * CH + ch) * 3 + tap / 3) * COUT + o;
            }
            dst[d] = __ldg(src + i);
        }
        if (FUSE)
            for (int i = tid; i < (int)(L::zero_bytes / 16); i += kThreads)
                reinterpret_cast<uint4*>(smem + L::zero_off)[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < COUT; i += kThreads) {
            sBias[i] = __ldg(a.bias + i);
            sScale[i] = F8 ? __ldg(a.wscale + i) : 1.0f;
        }
        for (int s = 0; s < NS; ++s) {
            if (CHG < CH)
                for (int i = tid; i < (int)((CH - CHG) * L::plane / 16); i += kThreads)
                    reinterpret_cast<uint4*>(sStage + (size_t)s * L::stage + CHG * L::plane)[i] = make_uint4(0, 0, 0, 0);
            constexpr int slack = (int)(L::plane - HY * kHXW * 16) / 16;
            for (int i = tid; i < CHG * slack; i += kThreads)
                reinterpret_cast<uint4*>(sStage + (size_t)s * L::stage + (i / slack) * L::plane +
                                         HY * kHXW * 16)[i % slack] = make_uint4(0, 0, 0, 0);
        }
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
        if (UPC)
            for (int k = 0; k < NS; ++k) tc::mbar_init(bars + 2 * NS + 4 + k, L::up_warps);
        if (CB1) tc::mbar_init(bars + 3 * NS + 4, L::up_warps);
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
    // the prologue above only read weights; the activations come from the previous kernel
    tc::grid_dep_wait();
    tc::grid_dep_launch();
    bool failed = false;

    if (warp == 0) {
        // ---- producer -------------------------------------------------------
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS, k = i / NS;
                // CB1: the previous tile's coarse block read before this tile's
                // is loaded over it (nothing of this tile is issued before)
                if ((k > 0 && !wait(empty0 + 8 * s, (k - 1) & 1)) || (CB1 && i > 0 && !wait(cfree0, (i - 1) & 1))) {
                    failed = true;
                    break;
                }
                const Img& im = a.img[find_img(a, tile)];
                const int lt = tile - im.tile0;
                const int ty = lt / im.tiles_x, tx = lt - ty * im.tiles_x;
                const uint32_t full = full0 + 8 * s;
                const uint32_t dst = tc::smem_addr(sStage + (size_t)s * L::stage);
                if constexpr (UPC > 0) {
                    // the coarse rows / columns under the tile (source 0), then
                    // the fine chunks of source 1 straight into the stage
                    mbar_expect_tx(full, (uint32_t)(CHG - UPC) * HY * kHXW * 16 + (uint32_t)UPC * L::CR * L::CC * 16);
                    const uint32_t cdst = tc::smem_addr(smem + L::coarse_off + (CB1 ? 0 : (size_t)s * L::coarse));
#pragma unroll
                    for (int c = 0; c < UPC; ++c)
                        tma_load_3d(cdst + c * L::cchunk, &im.map0, 2 * (((tx * kTO) >> 1) - 1), ((ty * TR) >> 1) - 1,
                                    c, full);
#pragma unroll
                    for (int c = UPC; c < CHG; ++c)
                        tma_load_3d(dst + c * L::plane, &im.map1, 2 * (tx * kTO - 1), ty * TR - 1, c - UPC, full);
                } else {
                    mbar_expect_tx(full, (uint32_t)CHG * HY * kHXW * 16);
#pragma unroll
                    for (int c = 0; c < CHG; ++c) {
                        const bool first = c < CH0;
                        tma_load_3d(dst + c * L::plane, first ? &im.map0 : &im.map1, 2 * (tx * kTO - 1),
                                    ty * TR - 1, first ? c : c - CH0, full);
                    }
                }
            }
            // on failure, let the loads already issued land before the CTA exits
            if (failed)
                for (int j = (i > NS ? i - NS : 0); j < i; ++j) wait(full0 + 8 * (j % NS), (j / NS) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer -----------------------------------------------------
        if (lane == 0) {
            constexpr int NB = FUSE ? 3 * COUT : COUT;      // N of one MMA
            constexpr uint32_t idesc = F8 ? tc::idesc_e4m3(128, NB) : tc::idesc_f16(128, NB);
            constexpr uint32_t idesc_z = F8 ? tc::idesc_e4m3(128, L::acc) : tc::idesc_f16(128, L::acc);
            const uint64_t b0 = tc::smem_desc(tc::smem_addr(sW), NB * 16, 128);
            const uint64_t z0 = tc::smem_desc(tc::smem_addr(smem + L::zero_off), kTW * 16, 128);
            int i = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS, acc = i & 1;
                // UPC: the stage is complete once the up-sampling warps have written their planes
                const uint32_t in_bar = UPC ? ready0 + 8 * s : full0 + 8 * s;
                if (!wait(in_bar, (i / NS) & 1) || (i >= 2 && !wait(tempty0 + 8 * acc, ((i >> 1) - 1) & 1))) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t a0 = tc::smem_desc(tc::smem_addr(sStage + (size_t)s * L::stage), L::plane, 128);
                if (FUSE) {
                    // zero the tile's accumulators (a zero A operand times finite weights) ...
                    if (F8) tc::mma_e4m3(tmem + (uint32_t)(acc * L::acc), z0, b0, idesc_z, 0);
                    else tc::mma_f16(tmem + (uint32_t)(acc * L::acc), z0, b0, idesc_z, 0);
                    // ... then halo row j feeds output rows j, j - 1, j - 2 in one MMA per (dx, K chunk)
#pragma unroll 1
                    for (int j = 0; j < HY; ++j) {
                        const uint32_t d = tmem + (uint32_t)(acc * L::acc + COUT * (TR + 1 - j));
#pragma unroll 1
                        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                            for (int kc = 0; kc < CH / 2; ++kc) {
                                const uint64_t ad = a0 + (uint64_t)((2 * kc) * (L::plane >> 4) + j * kHXW + dx);
                                const uint64_t bd = b0 + (uint64_t)((dx * CH + 2 * kc) * NB);
                                if (F8) tc::mma_e4m3(d, ad, bd, idesc, 1);
                                else tc::mma_f16(d, ad, bd, idesc, 1);
                            }
                        }
                    }
                } else {
                    // rows innermost: consecutive MMAs accumulate into
                    // different rows' accumulators, so they do not wait on
                    // one another
#pragma unroll 1
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                        for (int kc = 0; kc < CH / 2; ++kc) {
                            const uint64_t bd = b0 + (uint64_t)((tap * CH + 2 * kc) * COUT);
#pragma unroll
                            for (int r = 0; r < TR; ++r) {
                                const uint32_t d = tmem + (uint32_t)(acc * L::acc + r * COUT);
                                const uint64_t ad = a0 + (uint64_t)((2 * kc) * (L::plane >> 4) + (r + dy) * kHXW + dx);
                                if (F8) tc::mma_e4m3(d, ad, bd, idesc, (tap | kc) != 0);
                                else tc::mma_f16(d, ad, bd, idesc, (tap | kc) != 0);
                            }
                        }
                    }
                }
                tc::mma_commit(bars + NS + s);          // stage free once these MMAs are done
                tc::mma_commit(bars + 2 * NS + acc);    // accumulator ready for the epilogue
            }
            // every MMA issued must finish before the TMEM is freed
            if (i > 0) wait(tfull0 + 8 * ((i - 1) & 1), ((i - 1) >> 1) & 1);
        }
    } else if (warp < 6) {
        // ---- epilogue: warps 2-5, one pixel (TMEM lane) per thread ---------
        const int q = warp & 3;                 // TMEM lane quadrant of this warp
        const int px = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int i = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
            const int acc = i & 1;
            if (!wait(tfull0 + 8 * acc, (i >> 1) & 1)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const Img& im = a.img[find_img(a, tile)];
            const int lt = tile - im.tile0;
            const int ty = lt / im.tiles_x, tx = lt - ty * im.tiles_x;
            const int x = tx * kTO + px;
            const bool xin = px < kTO && x < im.Wl;
            float prev[COUT];
#pragma unroll 1
            for (int r = 0; r < TR; ++r) {
                const int y = ty * TR + r;
                float v[COUT];
#pragma unroll
                const int col = acc * L::acc + (FUSE ? COUT * (TR + 1 - r) : r * COUT);
#pragma unroll
                for (int c = 0; c < COUT; c += 16) tc::tmem_ld16(tmem + lane_base + col + c, v + c);
#pragma unroll
                for (int c = 0; c < COUT; ++c) v[c] = fmaxf(fmaf(v[c], sScale[c], sBias[c]), 0.f);
                if (y < im.Hl && xin)
                    store_px<COUT, F8>(im.out, (long long)im.Hl * im.Wl, (long long)y * im.Wl + x, v, a.out_q);
                if (POOL) {
                    if (r & 1) {
                        float sum[COUT];
#pragma unroll
                        for (int c = 0; c < COUT; ++c) {
                            sum[c] = prev[c] + v[c];
                            sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], 1);
                            sum[c] *= 0.25f;
                        }
                        if ((lane & 1) == 0 && y < im.Hl && xin)
                            store_px<COUT, F8>(im.pooled, (long long)(im.Hl >> 1) * (im.Wl >> 1),
                                               (long long)(y >> 1) * (im.Wl >> 1) + (x >> 1), sum, a.pool_q);
                    } else {
#pragma unroll
                        for (int c = 0; c < COUT; ++c) prev[c] = v[c];
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
        }
    } else if constexpr (UPC > 0) {
        // ---- up-sampling: warps 6.. write the stage's first UPC chunk planes
        // as the bilinear x2 up-sampling (half-pixel centres, edge clamp) of
        // the coarse rows the producer loaded, zero outside the fine frame
        // (half2 arithmetic: the interpolated values are FP16 / FP8 operands).
        // Thread t takes (chunk, fine halo column) items t, t + 32 up_warps, ..;
        // along a column it interpolates each coarse row along x once and
        // slides a pair of rows down the HY fine rows. ----
        constexpr int CPC = L::CPC;
        const int t = tid - 192;
        int i = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
            const int s = i % NS;
            if (!wait(full0 + 8 * s, (i / NS) & 1)) {
                failed = true;
                break;
            }
            const Img& im = a.img[find_img(a, tile)];
            const int lt = tile - im.tile0;
            const int ty = lt / im.tiles_x, tx = lt - ty * im.tiles_x;
            const int x0 = tx * kTO, y0 = ty * TR;
            const int Hc = im.Hl >> 1, Wc = im.Wl >> 1;
            const int cy0 = (y0 >> 1) - 1, cx0 = (x0 >> 1) - 1;   // coarse origin of the loaded block
            unsigned char* stg = sStage + (size_t)s * L::stage;
            const unsigned char* cbuf = smem + L::coarse_off + (CB1 ? 0 : (size_t)s * L::coarse);
            for (int item = t; item < UPC * kHXW; item += 32 * L::up_warps) {
                const int c = item / kHXW, p = item - c * kHXW;
                uint4* dst = reinterpret_cast<uint4*>(stg + (size_t)c * L::plane) + p;
                const int gx = x0 - 1 + p;
                if (gx < 0 || gx >= im.Wl) {
#pragma unroll
                    for (int j = 0; j < HY; ++j) dst[j * kHXW] = make_uint4(0, 0, 0, 0);
                    continue;
                }
                const int mx = gx >> 1;
                const int ix0 = (gx & 1) ? mx : max(mx - 1, 0), ix1 = min(ix0 + 1, Wc - 1);
                const __half2 fx = __float2half2_rn((gx & 1) ? 0.25f : (mx > 0 ? 0.75f : 0.0f));
                const int lx0 = ix0 - cx0, lx1 = ix1 - cx0;
                const uint4* crows = reinterpret_cast<const uint4*>(cbuf + (size_t)c * L::cchunk);
                constexpr int NP = CPC / 2;
                __half2 ha[NP], hb[NP];
                int ra = -1, rb = -1;                   // coarse rows held in ha / hb
#pragma unroll
                for (int j = 0; j < HY; ++j) {
                    const int gy = y0 - 1 + j;
                    if (gy < 0 || gy >= im.Hl) {
                        dst[j * kHXW] = make_uint4(0, 0, 0, 0);
                        continue;
                    }
                    const int my = gy >> 1;
                    const int iy0 = (gy & 1) ? my : max(my - 1, 0), iy1 = min(iy0 + 1, Hc - 1);
                    const __half2 fy = __float2half2_rn((gy & 1) ? 0.25f : (my > 0 ? 0.75f : 0.0f));
                    const int ly0 = iy0 - cy0, ly1 = iy1 - cy0;
                    if (ly0 != ra) {
                        if (ly0 == rb) {
#pragma unroll
                            for (int k = 0; k < NP; ++k) ha[k] = hb[k];
                        } else {
                            coarse_hlerp<F8>(crows + ly0 * L::CC, lx0, lx1, fx, ha);
                        }
                        ra = ly0;
                    }
                    if (ly1 != rb) {
                        if (ly1 == ra) {
#pragma unroll
                            for (int k = 0; k < NP; ++k) hb[k] = ha[k];
                        } else {
                            coarse_hlerp<F8>(crows + ly1 * L::CC, lx0, lx1, fx, hb);
                        }
                        rb = ly1;
                    }
                    __half2 v[NP];
#pragma unroll
                    for (int k = 0; k < NP; ++k) v[k] = __hfma2(fy, __hsub2(hb[k], ha[k]), ha[k]);
                    dst[j * kHXW] = h2_to_chunk<F8>(v);
                }
            }
            tc::fence_async_smem();   // generic-proxy writes, read next by the tensor core
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(ready0 + 8 * s);
                if (CB1) mbar_arrive(cfree0);
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

// ---------------------------------------------------------------------------
// Last decoder layer with the head, kernel prediction and blend (paper:
// "Kernel Prediction"): the 16 -> 16 conv (row-fused MMAs), then per tile a
// second MMA applies the 1x1 head (16 -> 29, padded to 32) to the layer's
// activations written back to shared memory as its A operand, and each
// epilogue thread finishes its pixel: softmax over the 25 kernel logits,
// weights times the sparse samples' mask, normalised by their sum (the
// direct RGB where no sample is in the window), blend by sigmoid(logit).
// The sparse R, G, B, M planes around the tile (TR + 4 rows x 136 columns,
// zero outside the frame) arrive by TMA with the halo.  16 epilogue warps in
// two groups that take alternate tiles (ping-pong: while one group waits for
// its head MMA the other runs its kernel prediction); within a group two
// warps per TMEM lane quadrant, each on half of the tile's rows.  Each group
// has its own conv accumulator, head accumulator and head A buffer.
constexpr int kHkEpi = 16;
constexpr int kHkThreads = 64 + 32 * kHkEpi;
constexpr int kSpW = kTW + 8;         // sparse window columns from (x0 - 2) rounded down to 4 floats

template <int CIN, int TR, int NS, bool F8>
struct HkLayout {
    using C = Layout<CIN, 16, TR, NS, F8, true>;
    static constexpr int SR = TR + 4;                               // sparse window rows
    static constexpr uint32_t sp_plane = SR * kSpW * 4;             // one float plane of the window
    static constexpr uint32_t stage = C::stage + 4 * sp_plane;      // conv halo + R, G, B, M
    static constexpr size_t w_bytes = C::w_bytes;
    static constexpr size_t hb_off = (w_bytes + 127) / 128 * 128;   // head B: [2][32][16 B]
    static constexpr size_t stage_off = (hb_off + 2 * 32 * 16 + 1023) / 1024 * 1024;
    static constexpr size_t zero_off = stage_off + (size_t)NS * stage;
    static constexpr size_t ha_bytes = (size_t)TR * 2 * kTW * 16;   // head A of one group: [TR][2][128][16 B]
    static constexpr size_t ha_off = zero_off + 2 * kTW * 16;
    static constexpr size_t bias_off = ha_off + 2 * ha_bytes;
    static constexpr size_t bar_off = bias_off + (16 + 16 + 32) * 4;
    static constexpr size_t bytes = bar_off + (2 * NS + 8) * 8 + 16;
    static constexpr uint32_t acc = C::acc;                         // conv accumulator columns
    static constexpr uint32_t head_col = 2 * acc;                   // head outputs: 2 x TR x 32 columns
    static constexpr uint32_t tmem_cols = head_col + 2 * TR * 32 <= 256 ? 256 : 512;
    static_assert(head_col + 2 * TR * 32 <= 512, "TMEM");
    static_assert(TR % (kHkEpi / 8) == 0, "rows split evenly over the warps of a group");
};

struct HkArgs {
    Args conv;                        // weights, bias, scales, tiles, images (map0 = d0a)
    const __half* head_w;             // [2][32][8] halves
    const float* head_b;              // [32]
    CUtensorMap sp[kMaxViews];        // sparse frame [5][H0][W0] float32 per view
    float* rgb[kMaxViews];
    int H0[kMaxViews], W0[kMaxViews];
};

template <int CIN, int CHG, int TR, int NS, bool F8>
__global__ void __launch_bounds__(kHkThreads, 1) conv3x3_ws_headkp_kernel(const __grid_constant__ HkArgs h) {
    using L = HkLayout<CIN, TR, NS, F8>;
    using LC = typename L::C;
    constexpr int CH = LC::CH, HY = LC::HY, COUT = 16;
    const Args& a = h.conv;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem;
    unsigned char* sStage = smem + L::stage_off;
    float* sBias = reinterpret_cast<float*>(smem + L::bias_off);
    float* sScale = sBias + 16;
    float* sHb = sBias + 32;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 8);
    const uint32_t full0 = tc::smem_addr(bars), empty0 = full0 + 8 * NS;
    const uint32_t tfull0 = full0 + 16 * NS, tempty0 = tfull0 + 16;
    const uint32_t hready0 = tempty0 + 16, hdone0 = hready0 + 16;   // per group

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const uint4* src = static_cast<const uint4*>(a.w);
        uint4* dst = reinterpret_cast<uint4*>(sW);
        for (int i = tid; i < (int)(L::w_bytes / 16); i += kHkThreads) {   // [tap][chunk][o] -> [dx][chunk][dy][o]
            const int o = i % COUT, t2 = i / COUT, ch = t2 % CH, tap = t2 / CH;
            dst[(((tap % 3) * CH + ch) * 3 + tap / 3) * COUT + o] = __ldg(src + i);
        }
        for (int i = tid; i < 2 * 32; i += kHkThreads)
            reinterpret_cast<uint4*>(smem + L::hb_off)[i] = __ldg(reinterpret_cast<const uint4*>(h.head_w) + i);
        for (int i = tid; i < 2 * kTW; i += kHkThreads)
            reinterpret_cast<uint4*>(smem + L::zero_off)[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < 16; i += kHkThreads) {
            sBias[i] = __ldg(a.bias + i);
            sScale[i] = F8 ? __ldg(a.wscale + i) : 1.0f;
        }
        for (int i = tid; i < 32; i += kHkThreads) sHb[i] = __ldg(h.head_b + i);
        for (int s = 0; s < NS; ++s) {
            if (CHG < CH)
                for (int i = tid; i < (int)((CH - CHG) * LC::plane / 16); i += kHkThreads)
                    reinterpret_cast<uint4*>(sStage + (size_t)s * L::stage + CHG * LC::plane)[i] = make_uint4(0, 0, 0, 0);
            constexpr int slack = (int)(LC::plane - HY * kHXW * 16) / 16;
            for (int i = tid; i < CHG * slack; i += kHkThreads)
                reinterpret_cast<uint4*>(sStage + (size_t)s * L::stage + (i / slack) * LC::plane +
                                         HY * kHXW * 16)[i % slack] = make_uint4(0, 0, 0, 0);
        }
    }
    if (tid == 0) {
        constexpr int GW = kHkEpi / 2;                 // warps of one epilogue group
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(bars + s, 1);
            tc::mbar_init(bars + NS + s, 1 + GW);      // conv MMAs done + the tile's group done with its samples
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(bars + 2 * NS + k, 1);
            tc::mbar_init(bars + 2 * NS + 2 + k, GW);
            tc::mbar_init(bars + 2 * NS + 4 + k, GW);  // head A of group k written
            tc::mbar_init(bars + 2 * NS + 6 + k, 1);   // head MMA of group k done
        }
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
    // the prologue above only read weights; the activations come from the previous kernel
    tc::grid_dep_wait();
    tc::grid_dep_launch();
    bool failed = false;

    if (warp == 0) {
        // ---- producer: conv halo + sparse window ---------------------------
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS, k = i / NS;
                if (k > 0 && !wait(empty0 + 8 * s, (k - 1) & 1)) {
                    failed = true;
                    break;
                }
                const int im_i = find_img(a, tile);
                const Img& im = a.img[im_i];
                const int lt = tile - im.tile0;
                const int ty = lt / im.tiles_x, tx = lt - ty * im.tiles_x;
                const uint32_t full = full0 + 8 * s;
                mbar_expect_tx(full, (uint32_t)CHG * HY * kHXW * 16 + 4u * L::SR * kSpW * 4);
                const uint32_t dst = tc::smem_addr(sStage + (size_t)s * L::stage);
#pragma unroll
                for (int c = 0; c < CHG; ++c)
                    tma_load_3d(dst + c * LC::plane, &im.map0, 2 * (tx * kTO - 1), ty * TR - 1, c, full);
                const uint32_t sp = dst + LC::stage;
                const int xs = (tx * kTO - 2) & ~3;   // 16-byte aligned start of the window
#pragma unroll
                for (int p = 0; p < 4; ++p)   // planes R, G, B, M (= 4) of the sparse frame
                    tma_load_3d(sp + p * L::sp_plane, &h.sp[im_i], xs, ty * TR - 2, p < 3 ? p : 4, full);
            }
            if (failed)
                for (int j = (i > NS ? i - NS : 0); j < i; ++j) wait(full0 + 8 * (j % NS), (j / NS) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer: row-fused conv, then the head of the previous tile ----
        if (lane == 0) {
            constexpr int NB = 3 * COUT;
            constexpr uint32_t idesc = F8 ? tc::idesc_e4m3(128, NB) : tc::idesc_f16(128, NB);
            constexpr uint32_t idesc_z = F8 ? tc::idesc_e4m3(128, LC::acc) : tc::idesc_f16(128, LC::acc);
            constexpr uint32_t idesc_h = tc::idesc_f16(128, 32);
            const uint64_t b0 = tc::smem_desc(tc::smem_addr(sW), NB * 16, 128);
            const uint64_t z0 = tc::smem_desc(tc::smem_addr(smem + L::zero_off), kTW * 16, 128);
            const uint64_t hb = tc::smem_desc(tc::smem_addr(smem + L::hb_off), 32 * 16, 128);
            auto head = [&](int t) -> bool {   // head MMA of the tile with index t (group t & 1)
                const int g = t & 1;
                if (!wait(hready0 + 8 * g, (t >> 1) & 1)) return false;
                tc::fence_after_sync();
#pragma unroll 1
                for (int r = 0; r < TR; ++r) {
                    const uint64_t ad = tc::smem_desc(
                        tc::smem_addr(smem + L::ha_off + g * L::ha_bytes + (size_t)r * 2 * kTW * 16), kTW * 16, 128);
                    tc::mma_f16(tmem + L::head_col + g * TR * 32 + 32 * r, ad, hb, idesc_h, 0);
                }
                tc::mma_commit(bars + 2 * NS + 6 + g);
                return true;
            };
            int i = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS, acc = i & 1;
                // the previous tile's head first, before this tile waits for its
                // accumulator: that wait ends only when the other group has
                // finished its kernel prediction of tile i - 2, and the head
                // issued behind it would serialise the two groups' kernel
                // predictions (the slow part of the epilogue) instead of
                // overlapping them with each other and with this tile's conv
                if (i >= 1 && !head(i - 1)) {
                    failed = true;
                    break;
                }
                if (!wait(full0 + 8 * s, (i / NS) & 1) || (i >= 2 && !wait(tempty0 + 8 * acc, ((i >> 1) - 1) & 1))) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t a0 = tc::smem_desc(tc::smem_addr(sStage + (size_t)s * L::stage), LC::plane, 128);
                if (F8) tc::mma_e4m3(tmem + (uint32_t)(acc * LC::acc), z0, b0, idesc_z, 0);
                else tc::mma_f16(tmem + (uint32_t)(acc * LC::acc), z0, b0, idesc_z, 0);
#pragma unroll 1
                for (int j = 0; j < HY; ++j) {
                    const uint32_t d = tmem + (uint32_t)(acc * LC::acc + COUT * (TR + 1 - j));
#pragma unroll 1
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int kc = 0; kc < CH / 2; ++kc) {
                            const uint64_t ad = a0 + (uint64_t)((2 * kc) * (LC::plane >> 4) + j * kHXW + dx);
                            const uint64_t bd = b0 + (uint64_t)((dx * CH + 2 * kc) * NB);
                            if (F8) tc::mma_e4m3(d, ad, bd, idesc, 1);
                            else tc::mma_f16(d, ad, bd, idesc, 1);
                        }
                    }
                }
                tc::mma_commit(bars + NS + s);
                tc::mma_commit(bars + 2 * NS + acc);
            }
            if (!failed && i >= 1 && !head(i - 1)) failed = true;
            // every MMA finished before the TMEM is freed
            if (i > 0) {
                wait(tfull0 + 8 * ((i - 1) & 1), ((i - 1) >> 1) & 1);
                if (!failed) wait(hdone0 + 8 * ((i - 1) & 1), ((i - 1) >> 1) & 1);
            }
        }
    } else {
        // ---- epilogue: group G (8 warps) takes the tiles i with i % 2 == G; in a
        // group, sub-group u (4 warps, one per lane quadrant) takes rows [u RG, (u + 1) RG) ----
        constexpr int RG = TR / (kHkEpi / 8);
        const int e = warp - 2, G = e >> 3, u = (e >> 2) & 1;
        const int q = warp & 3;
        const int px = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int r_lo = u * RG, r_hi = r_lo + RG;
        const uint32_t hready = hready0 + 8 * G, hdone = hdone0 + 8 * G;
        unsigned char* ha_base = smem + L::ha_off + G * L::ha_bytes;
        const uint32_t head_col = L::head_col + G * TR * 32;
        int i = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++i) {
            if ((i & 1) != G) continue;
            const int s = i % NS, acc = i & 1;
            if (!wait(tfull0 + 8 * acc, (i >> 1) & 1)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            // activations -> shared memory as the head's A operand
#pragma unroll 1
            for (int r = r_lo; r < r_hi; ++r) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + acc * LC::acc + COUT * (TR + 1 - r), v);
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = fmaxf(fmaf(v[c], sScale[c], sBias[c]), 0.f);
                unsigned char* ha = ha_base + (size_t)r * 2 * kTW * 16;
                *reinterpret_cast<uint4*>(ha + px * 16) = pack8h(v);
                *reinterpret_cast<uint4*>(ha + (kTW + px) * 16) = pack8h(v + 8);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(hready);
            if (!wait(hdone, (i >> 1) & 1)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const int im_i = find_img(a, tile);
            const Img& im = a.img[im_i];
            const int lt = tile - im.tile0;
            const int ty = lt / im.tiles_x, tx = lt - ty * im.tiles_x;
            const int x = tx * kTO + px;
            const int off = (tx * kTO - 2) - ((tx * kTO - 2) & ~3);   // window column of x0 - 2
            const int H0 = h.H0[im_i], W0 = h.W0[im_i];
            const long long plane = (long long)H0 * W0;
            const float* spR = reinterpret_cast<const float*>(sStage + (size_t)s * L::stage + LC::stage);
#pragma unroll 1
            for (int r = r_lo; r < r_hi; ++r) {
                const int y = ty * TR + r;
                float hd[32];
                tc::tmem_ld16(tmem + lane_base + head_col + 32 * r, hd);
                tc::tmem_ld16(tmem + lane_base + head_col + 32 * r + 16, hd + 16);
#pragma unroll
                for (int j = 0; j < 29; ++j) hd[j] += sHb[j];
                float mx = hd[3];
#pragma unroll
                for (int k = 1; k < 25; ++k) mx = fmaxf(mx, hd[3 + k]);
                // unnormalised softmax weights e_k: the normalisation cancels in
                // num / den, and den / sum(e) is the normalised sampled weight
                float es = 0.f, den = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
                for (int k = 0; k < 25; ++k) {
                    const float e = __expf(hd[3 + k] - mx);
                    const int o = (r + k / 5) * kSpW + off + px + k % 5;
                    const float wm = e * spR[3 * (L::sp_plane / 4) + o];
                    es += e;
                    den += wm;
                    n0 = fmaf(wm, spR[o], n0);
                    n1 = fmaf(wm, spR[(L::sp_plane / 4) + o], n1);
                    n2 = fmaf(wm, spR[2 * (L::sp_plane / 4) + o], n2);
                }
                float k0 = hd[0], k1 = hd[1], k2 = hd[2];
                if (den >= 1e-12f * es) {
                    k0 = n0 / den;
                    k1 = n1 / den;
                    k2 = n2 / den;
                }
                const float al = 1.0f / (1.0f + __expf(-hd[28]));
                if (y < H0 && px < kTO && x < W0) {
                    float* o = h.rgb[im_i] + (long long)y * W0 + x;
                    o[0] = fmaf(al, k0 - hd[0], hd[0]);
                    o[plane] = fmaf(al, k1 - hd[1], hd[1]);
                    o[2 * plane] = fmaf(al, k2 - hd[2], hd[2]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(tempty0 + 8 * acc);
                mbar_arrive(empty0 + 8 * s);
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

// Bilinear x2 up-sampling of fine rows 2 my and 2 my + 1 of one chunk plane
// of a chunk-planar tensor (half-pixel centres, edge clamp; Hl even), the
// block's threads striding over the columns: the two rows share a coarse
// row (the middle one from my = 1 on), interpolated along x once; each
// output is the same arithmetic as the up-sampling layers of
// conv3x3_tc_kernel apply while staging.
template <bool F8>
__device__ __forceinline__ void upsample2_rowpair(const void* __restrict__ coarse, void* __restrict__ fine, int Hl,
                                                  int Wl, int c, int my) {
    const int Hc = Hl >> 1, Wc = Wl >> 1;
    // fine row 2 my: coarse rows a, b with weight fe on b; fine row 2 my + 1: rows my, d with weight 1/4 on d
    const int ra = max(my - 1, 0), rb = min(ra + 1, Hc - 1), rd = min(my + 1, Hc - 1);
    const float fe = my > 0 ? 0.75f : 0.0f, fo = 0.25f;
    const uint4* base = static_cast<const uint4*>(coarse) + (long long)c * Hc * Wc;
    const uint4 *r0 = base + (long long)ra * Wc, *r1 = base + (long long)rb * Wc, *r2 = base + (long long)my * Wc,
                *r3 = base + (long long)rd * Wc;
    const bool c_is_b = my == rb, c_is_a = my == ra, d_is_b = rd == rb;
    uint4* out0 = static_cast<uint4*>(fine) + ((long long)c * Hl + 2 * my) * Wl;
    uint4* out1 = out0 + Wl;
    constexpr int CPC = F8 ? 16 : 8;
    auto xlerp = [&](const uint4* row, int ix0, int ix1, float fx, float* o) {
        float p0[16], p1[16];
        const uint4 u0 = __ldg(row + ix0), u1 = __ldg(row + ix1);
        if (F8) {
            unpack16q(u0, p0);
            unpack16q(u1, p1);
        } else {
            unpack8h(u0, p0);
            unpack8h(u1, p1);
        }
#pragma unroll
        for (int j = 0; j < CPC; ++j) o[j] = fmaf(fx, p1[j] - p0[j], p0[j]);
    };
    for (int gx = threadIdx.x; gx < Wl; gx += blockDim.x) {
        const int mx = gx >> 1;
        const int ix0 = (gx & 1) ? mx : max(mx - 1, 0), ix1 = min(ix0 + 1, Wc - 1);
        const float fx = (gx & 1) ? 0.25f : (mx > 0 ? 0.75f : 0.0f);
        float ta[16], tb[16], tc_[16], td[16], v[16];
        xlerp(r0, ix0, ix1, fx, ta);
        xlerp(r1, ix0, ix1, fx, tb);
        if (c_is_b) {
#pragma unroll
            for (int j = 0; j < CPC; ++j) tc_[j] = tb[j];
        } else if (c_is_a) {
#pragma unroll
            for (int j = 0; j < CPC; ++j) tc_[j] = ta[j];
        } else {
            xlerp(r2, ix0, ix1, fx, tc_);
        }
        if (d_is_b) {
#pragma unroll
            for (int j = 0; j < CPC; ++j) td[j] = tb[j];
        } else {
            xlerp(r3, ix0, ix1, fx, td);
        }
#pragma unroll
        for (int j = 0; j < CPC; ++j) v[j] = fmaf(fe, tb[j] - ta[j], ta[j]);
        out0[gx] = F8 ? pack16q(v) : pack8h(v);
#pragma unroll
        for (int j = 0; j < CPC; ++j) v[j] = fmaf(fo, td[j] - tc_[j], tc_[j]);
        out1[gx] = F8 ? pack16q(v) : pack8h(v);
    }
}

}  // namespace ws
}  // namespace fvn
