// Reconstruction convolutions on the 5th-generation tensor cores (tcgen05):
// implicit GEMM with the accumulators in tensor memory (paper: "Reconstruction
// Network"; the arithmetic is that of recon.cu's layers), with FP16 operands
// or FP8 E4M3 operands (paper: "Model Precision & Optimization" runs the
// network at reduced precision after training).
//
// Tile = TR output rows x 128 pixels.  For each row the GEMM is
// M = 128 pixels, N = COUT, K = 9 taps x CIN, issued as tcgen05.mma
// (kind::f16 with K = 16, or kind::f8f6f4 with K = 32) by one thread into a
// TMEM accumulator of COUT columns.  The input halo (TR+2 rows x 130 pixels)
// is staged in shared memory as planes of 16 bytes per pixel (8 FP16 or 16
// FP8 channels): that is the K-major, non-swizzled core-matrix layout the
// tensor core reads (8 pixels x 16 bytes contiguous), so the tap shift
// (dy, dx) is only a start-address offset of the operand descriptor
// (LBO = one channel plane, SBO = 128 B).  Weights stay resident in shared
// memory in the same layout ([tap][cin chunk][cout][16 B]).  Epilogue: each
// thread owns one pixel (one TMEM lane): scale, bias, ReLU, FP16 / FP8,
// 16-byte stores into chunk-planar tensors ([C / chunk][H][W][16 B], one
// plane per 16-byte channel chunk); fused 2x2 average pooling; for the last decoder conv a
// second MMA applies the 1x1 head (16 -> 29, padded to 32) from the
// activations written back to shared memory, and the thread finishes its
// pixel with the softmax 5x5 kernel prediction over the sparse samples
// (staged in shared memory) and the blend.
//
// FP8: an activation tensor t is stored as q = x / s_t (s_t = amax_t / 448
// from calibration); a layer's weights are stored as e4m3(w s_in / s_w[co])
// with the input scales folded in per input channel and one scale per output
// channel, so the accumulator times s_w[co] is the FP32 pre-activation.
#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace fvn {

namespace {

enum { TIN_ACT = 0, TIN_RGBAM = 1, TIN_UPCAT = 2 };
enum { TEPI_STORE = 0, TEPI_POOL = 1, TEPI_HEADKP = 2 };

constexpr int TW = 128;            // pixels per tile row = MMA M
constexpr int HXW = TW + 2;        // halo width
// 8 warps: warps w and w + 4 read the same TMEM lane quadrant (w % 4) and
// split the tile's rows in the epilogue.
constexpr int kThreads = 256;
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

__device__ __forceinline__ uint4 pack8h(const float* v) {
    uint4 r;
    __half2 h0 = __floats2half2_rn(v[0], v[1]), h1 = __floats2half2_rn(v[2], v[3]);
    __half2 h2 = __floats2half2_rn(v[4], v[5]), h3 = __floats2half2_rn(v[6], v[7]);
    r.x = *reinterpret_cast<uint32_t*>(&h0);
    r.y = *reinterpret_cast<uint32_t*>(&h1);
    r.z = *reinterpret_cast<uint32_t*>(&h2);
    r.w = *reinterpret_cast<uint32_t*>(&h3);
    return r;
}
__device__ __forceinline__ void unpack8h(uint4 u, float* v) {
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __half22float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ uint32_t pack4q(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}
__device__ __forceinline__ uint4 pack16q(const float* v) {
    return make_uint4(pack4q(v[0], v[1], v[2], v[3]), pack4q(v[4], v[5], v[6], v[7]),
                      pack4q(v[8], v[9], v[10], v[11]), pack4q(v[12], v[13], v[14], v[15]));
}
__device__ __forceinline__ void unpack16q(uint4 u, float* v) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const __half2_raw hr =
                __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((w[i] >> (16 * j)) & 0xFFFFu), __NV_E4M3);
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
            v[4 * i + 2 * j] = f.x;
            v[4 * i + 2 * j + 1] = f.y;
        }
    }
}

// CIN: padded input channels (the GEMM's K per tap); CG: channels of the
// tensor(s) read from memory (the rest of CIN is zero).
template <int CIN, int CG, int COUT, int TR, int MODE, int EPI, int CUP, bool F8>
struct TcLayout {
    static constexpr int EB = F8 ? 1 : 2;              // bytes per element
    static constexpr int CPC = 16 / EB;                // channels per 16-byte chunk
    static constexpr int CH = CIN / CPC;               // chunks per pixel (K per tap / chunk)
    static constexpr int CHG = CG / CPC;               // chunks read from memory
    static constexpr int HY = TR + 2;
    static constexpr int CR = TR / 2 + 3, CC = TW / 2 + 3;        // coarse halo (up-sampling)
    static constexpr size_t w_off = 0;
    static constexpr size_t w_bytes = 9ull * CIN * COUT * EB;
    static constexpr size_t halo_bytes = (size_t)CH * HY * HXW * 16;         // one halo buffer
    static constexpr size_t sp1_bytes = EPI == TEPI_HEADKP ? (size_t)(TR + 4) * (TW + 4) * 16 : 0;
    // two halo (and sparse-sample) buffers when they fit: the next tile is
    // staged while the tensor core works on the current one
    static constexpr size_t single_bytes = w_bytes + halo_bytes + sp1_bytes +
        (MODE == TIN_UPCAT ? (size_t)(CUP / CPC) * (TR / 2 + 3) * (TW / 2 + 3) * 16 : 0) +
        (EPI == TEPI_HEADKP ? (size_t)TR * 2 * TW * 16 + 2 * 32 * 16 : 0) + (2 * COUT + 32) * 4 + 16;
    // (only while two CTAs still fit on an SM: overlap across CTAs is worth more)
    static constexpr int NBUF = single_bytes + halo_bytes + sp1_bytes <= 112 * 1024 ? 2 : 1;
    static constexpr size_t halo_off = w_off + w_bytes;
    static constexpr size_t coarse_off = halo_off + NBUF * halo_bytes;
    static constexpr size_t coarse_bytes = MODE == TIN_UPCAT ? (size_t)(CUP / CPC) * CR * CC * 16 : 0;
    static constexpr size_t ha_off = coarse_off + coarse_bytes;     // head operand A: [TR][2][128][8] halves
    static constexpr size_t ha_bytes = EPI == TEPI_HEADKP ? (size_t)TR * 2 * TW * 16 : 0;
    static constexpr size_t hb_off = ha_off + ha_bytes;             // head weights: [2][32][8] halves
    static constexpr size_t hb_bytes = EPI == TEPI_HEADKP ? 2 * 32 * 16 : 0;
    static constexpr size_t sp_off = hb_off + hb_bytes;             // sparse R, G, B, M: [TR+4][TW+4] float4
    static constexpr size_t sp_bytes = NBUF * sp1_bytes;
    static constexpr size_t bias_off = sp_off + sp_bytes;           // bias [COUT], head bias [32], FP8 scales [COUT]
    static constexpr size_t bias_bytes = (2 * COUT + 32) * 4;
    static constexpr size_t bar_off = bias_off + bias_bytes;
    static constexpr size_t bytes = bar_off + 16;
    static constexpr uint32_t acc_cols = TR * COUT;
    static constexpr uint32_t need_cols = EPI == TEPI_HEADKP ? (acc_cols > TR * 32 ? acc_cols : TR * 32) : acc_cols;
    static constexpr uint32_t tmem_cols = need_cols <= 32 ? 32 : need_cols <= 64 ? 64 : need_cols <= 128 ? 128
                                        : need_cols <= 256 ? 256 : 512;
};

// One image of a batched launch: its tensors and sizes, and the first tile
// of the launch's tile range that belongs to it.
struct TcImg {
    const void* in;          // chunk-planar input, or the coarse level for up-sampling
    const void* skip;        // skip tensor (up-sampling layers)
    const float* rgbam;      // sparse frame [5][H0][W0] (first layer, KP)
    const float* prev;       // first layer, recurrent model: previous output [3][H0][W0] (NULL: zeros)
    void* out;               // [Hl][Wl][COUT]
    void* pooled;            // [Hl/2][Wl/2][COUT]
    float* rgb;              // [3][H0][W0] (KP layer)
    int H0, W0;
    int Hl, Wl;
    int tiles_x, tile0;
};

struct TcArgs {
    const void* w;           // [9][CIN/CPC][COUT][16 B]
    const float* bias;
    const float* wscale;     // FP8: per output channel weight scale
    float in_q;              // FP8 first layer: 1 / s of the sparse frame
    float out_q, pool_q;     // FP8: 1 / s of the output / pooled tensor
    const __half* head_w;    // [2][32][8] halves (KP layer)
    const float* head_b;     // [32]
    int ntiles;              // tiles of all images
    int nimg;
    int* error;              // set when a tensor-core wait gives up
    TcImg img[kMaxViews];
};

// Image of tile `tile` (the images' tile ranges are consecutive).
__device__ __forceinline__ int find_img(const TcArgs& a, int tile) {
    int i = 0;
    while (i + 1 < a.nimg && tile >= a.img[i + 1].tile0) ++i;
    return i;
}

// Store COUT channel values of one pixel (FP16, or FP8 after scaling by q)
// into a chunk-planar tensor: plane j holds channels [j CPC, (j + 1) CPC) of
// every pixel as 16-byte vectors ([C / CPC][H][W][16 B]; plane = H W).
template <int COUT, bool F8>
__device__ __forceinline__ void store_pixel(void* base, long long plane, long long pix, const float* v, float q) {
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

template <int CIN, int CG, int COUT, int TR, int MODE, int EPI, int CUP, bool F8>
__global__ void __launch_bounds__(kThreads) conv3x3_tc_kernel(const __grid_constant__ TcArgs a) {
    using L = TcLayout<CIN, CG, COUT, TR, MODE, EPI, CUP, F8>;
    constexpr int CH = L::CH, CHG = L::CHG, CPC = L::CPC, EB = L::EB, HY = L::HY;
    constexpr int CUPC = CUP / CPC;                   // up-sampled chunks
    static_assert(COUT % 16 == 0 && COUT <= 64, "unsupported conv shape");
    static_assert(CIN % (2 * CPC) == 0, "K per tap must be a multiple of the MMA K");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW = smem + L::w_off;
    unsigned char* sH0 = smem + L::halo_off;        // halo buffer 0 (buffer 1 follows)
    unsigned char* sC = smem + L::coarse_off;
    unsigned char* sHA = smem + L::ha_off;
    unsigned char* sHB = smem + L::hb_off;
    float* sBias = reinterpret_cast<float*>(smem + L::bias_off);
    float* sScale = sBias + COUT + 32;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tbase_s = reinterpret_cast<uint32_t*>(smem + L::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.w);
        uint4* dst = reinterpret_cast<uint4*>(sW);
        for (int i = tid; i < (int)(L::w_bytes / 16); i += kThreads) dst[i] = __ldg(src + i);
        for (int i = tid; i < COUT; i += kThreads) {
            sBias[i] = __ldg(a.bias + i);
            sScale[i] = F8 ? __ldg(a.wscale + i) : 1.0f;
        }
        if (EPI == TEPI_HEADKP) {
            const uint4* hs = reinterpret_cast<const uint4*>(a.head_w);
            for (int i = tid; i < 2 * 32; i += kThreads) reinterpret_cast<uint4*>(sHB)[i] = __ldg(hs + i);
            for (int i = tid; i < 32; i += kThreads) sBias[COUT + i] = __ldg(a.head_b + i);
        }
    }
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) {
        tc::tmem_alloc(tbase_s, L::tmem_cols);
        // give up the right to allocate again at once: while a CTA holds it,
        // no other CTA is scheduled on the SM
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tbase_s;
    // the prologue above only read weights; the activations come from the previous kernel
    tc::grid_dep_wait();
    tc::grid_dep_launch();
    const uint32_t sW_u = tc::smem_addr(sW), sH_u = tc::smem_addr(sH0);
    constexpr uint32_t idesc = F8 ? tc::idesc_e4m3(128, COUT) : tc::idesc_f16(128, COUT);
    uint32_t phase = 0;
    bool failed = false;

    // Stage the input halo (and the sparse samples of the KP layer) of a tile
    // into buffer `buf`.  Plain copies are left in flight (cp.async); the
    // up-sampling layers wait for theirs and interpolate here.
    auto stage = [&](int gtile, int buf) {
        const TcImg& im = a.img[find_img(a, gtile)];
        const unsigned char* gin = static_cast<const unsigned char*>(im.in);
        const unsigned char* gskip = static_cast<const unsigned char*>(im.skip);
        const int tile = gtile - im.tile0;
        const int ty = tile / im.tiles_x, tx = tile - ty * im.tiles_x;
        const int y0 = ty * TR, x0 = tx * TW;
        unsigned char* sH = smem + L::halo_off + (size_t)buf * L::halo_bytes;
        float4* sSP = reinterpret_cast<float4*>(smem + L::sp_off + (size_t)buf * L::sp1_bytes);
        if (MODE == TIN_RGBAM) {
            const long long plane = (long long)im.H0 * im.W0;
            for (int i = tid; i < HY * HXW; i += kThreads) {
                const int hy = i / HXW, hx = i - hy * HXW;
                const int gy = y0 + hy - 1, gx = x0 + hx - 1;
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = 0.f;
                if (gy >= 0 && gx >= 0 && gy < im.H0 && gx < im.W0) {
                    const float* p = im.rgbam + (long long)gy * im.W0 + gx;
#pragma unroll
                    for (int c = 0; c < 5; ++c) v[c] = __ldg(p + c * plane) * (F8 ? a.in_q : 1.0f);
                    if (im.prev) {   // the previous output, clamped to [0, 1], as channels 5..7
                        const float* q = im.prev + (long long)gy * im.W0 + gx;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            v[5 + c] = __saturatef(__ldg(q + c * plane)) * (F8 ? a.in_q : 1.0f);
                    }
                }
                *reinterpret_cast<uint4*>(sH + ((0 * HY + hy) * HXW + hx) * 16) = F8 ? pack16q(v) : pack8h(v);
#pragma unroll
                for (int c = 1; c < CH; ++c)
                    *reinterpret_cast<uint4*>(sH + ((c * HY + hy) * HXW + hx) * 16) = make_uint4(0, 0, 0, 0);
            }
        } else {
            constexpr int CS0 = MODE == TIN_UPCAT ? CUPC : 0;   // first chunk read from global
            for (int i = tid; i < (CH - CS0) * HY * HXW; i += kThreads) {
                const int c = CS0 + i / (HY * HXW);
                const int rem = i % (HY * HXW);
                const int hy = rem / HXW, hx = rem - hy * HXW;
                const int gy = y0 + hy - 1, gx = x0 + hx - 1;
                unsigned char* dst = sH + ((c * HY + hy) * HXW + hx) * 16;
                if (c < CHG && gy >= 0 && gx >= 0 && gy < im.Hl && gx < im.Wl) {
                    const long long pix = (long long)gy * im.Wl + gx;
                    const long long plane = (long long)im.Hl * im.Wl;
                    if (MODE == TIN_ACT) cp16(tc::smem_addr(dst), gin + (c * plane + pix) * 16);
                    else cp16(tc::smem_addr(dst), gskip + ((c - CS0) * plane + pix) * 16);
                } else {
                    *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
                }
            }
            if (MODE == TIN_UPCAT) {   // coarse rows / columns around the tile, clamped to the coarse frame
                const int Hc = im.Hl >> 1, Wc = im.Wl >> 1;
                const int cy0 = (y0 >> 1) - 1, cx0 = (x0 >> 1) - 1;
                for (int i = tid; i < CUPC * L::CR * L::CC; i += kThreads) {
                    const int c = i / (L::CR * L::CC);
                    const int rem = i % (L::CR * L::CC);
                    const int r = rem / L::CC, q = rem - r * L::CC;
                    const int cy = min(max(cy0 + r, 0), Hc - 1), cx = min(max(cx0 + q, 0), Wc - 1);
                    cp16(tc::smem_addr(sC + ((c * L::CR + r) * L::CC + q) * 16),
                         gin + (((long long)c * Hc + cy) * Wc + cx) * 16);
                }
            }
            if (MODE == TIN_UPCAT) {
                cp_wait_all();
                __syncthreads();
                const int Hc = im.Hl >> 1, Wc = im.Wl >> 1;
                const int cy0 = (y0 >> 1) - 1, cx0 = (x0 >> 1) - 1;
                for (int i = tid; i < HY * HXW; i += kThreads) {
                    const int hy = i / HXW, hx = i - hy * HXW;
                    const int gy = y0 + hy - 1, gx = x0 + hx - 1;
                    const bool inside = gy >= 0 && gx >= 0 && gy < im.Hl && gx < im.Wl;
                    // bilinear x2 with half-pixel centres: fine 2m -> coarse m-1 / m with weights
                    // 1/4, 3/4 (source clamped to 0 at m = 0), fine 2m+1 -> m / m+1 with 3/4, 1/4;
                    // the upper neighbour is clamped to the frame
                    const int my = gy >> 1, mx = gx >> 1;
                    const int iy0 = (gy & 1) ? my : max(my - 1, 0), ix0 = (gx & 1) ? mx : max(mx - 1, 0);
                    const float fy = (gy & 1) ? 0.25f : (my > 0 ? 0.75f : 0.0f);
                    const float fx = (gx & 1) ? 0.25f : (mx > 0 ? 0.75f : 0.0f);
                    const int iy1 = min(iy0 + 1, Hc - 1), ix1 = min(ix0 + 1, Wc - 1);
                    const int o00 = ((iy0 - cy0) * L::CC + (ix0 - cx0)) * 16, o01 = ((iy0 - cy0) * L::CC + (ix1 - cx0)) * 16;
                    const int o10 = ((iy1 - cy0) * L::CC + (ix0 - cx0)) * 16, o11 = ((iy1 - cy0) * L::CC + (ix1 - cx0)) * 16;
#pragma unroll
                    for (int c = 0; c < CUPC; ++c) {
                        unsigned char* dst = sH + ((c * HY + hy) * HXW + hx) * 16;
                        if (!inside) {
                            *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
                            continue;
                        }
                        const unsigned char* base = sC + (size_t)c * L::CR * L::CC * 16;
                        const uint4 u00 = *reinterpret_cast<const uint4*>(base + o00);
                        const uint4 u01 = *reinterpret_cast<const uint4*>(base + o01);
                        const uint4 u10 = *reinterpret_cast<const uint4*>(base + o10);
                        const uint4 u11 = *reinterpret_cast<const uint4*>(base + o11);
                        float v[16], p00[16], p01[16], p10[16], p11[16];
                        if (F8) {
                            unpack16q(u00, p00);
                            unpack16q(u01, p01);
                            unpack16q(u10, p10);
                            unpack16q(u11, p11);
                        } else {
                            unpack8h(u00, p00);
                            unpack8h(u01, p01);
                            unpack8h(u10, p10);
                            unpack8h(u11, p11);
                        }
#pragma unroll
                        for (int j = 0; j < CPC; ++j) {
                            const float top = fmaf(fx, p01[j] - p00[j], p00[j]);
                            const float bot = fmaf(fx, p11[j] - p10[j], p10[j]);
                            v[j] = fmaf(fy, bot - top, top);
                        }
                        *reinterpret_cast<uint4*>(dst) = F8 ? pack16q(v) : pack8h(v);
                    }
                }
            }
        }
        if (EPI == TEPI_HEADKP) {   // sparse R, G, B, M around the tile (2-pixel margin)
            const long long plane = (long long)im.H0 * im.W0;
            for (int i = tid; i < (TR + 4) * (TW + 4); i += kThreads) {
                const int r = i / (TW + 4), q = i - r * (TW + 4);
                const int gy = y0 + r - 2, gx = x0 + q - 2;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gy >= 0 && gx >= 0 && gy < im.H0 && gx < im.W0) {
                    const float* p = im.rgbam + (long long)gy * im.W0 + gx;
                    v = make_float4(__ldg(p), __ldg(p + plane), __ldg(p + 2 * plane), __ldg(p + 4 * plane));
                }
                sSP[i] = v;
            }
        }
    };

    int buf = 0;
    int tile = blockIdx.x;
    if (tile < a.ntiles) {
        stage(tile, 0);
        cp_wait_all();
        tc::fence_async_smem();
        __syncthreads();
    }
    for (; tile < a.ntiles && !failed; tile += gridDim.x) {
        const TcImg& im = a.img[find_img(a, tile)];
        const int ltile = tile - im.tile0;
        const int ty = ltile / im.tiles_x, tx = ltile - ty * im.tiles_x;
        const int y0 = ty * TR, x0 = tx * TW;
        const int next = tile + gridDim.x;
        const float4* sSP = reinterpret_cast<const float4*>(smem + L::sp_off + (size_t)buf * L::sp1_bytes);

        // ---- tensor-core main loop: one elected thread issues every MMA ----
        if (tid == 0) {
            tc::fence_after_sync();
            // descriptors differ only in their start address (bits 0-13, in
            // 16-byte units, far from overflowing below 228 KB of shared memory)
            const uint64_t a0 = tc::smem_desc(sH_u + (uint32_t)(buf * L::halo_bytes), HY * HXW * 16, 128);
            const uint64_t b0 = tc::smem_desc(sW_u, COUT * 16, 128);
#pragma unroll 1
            for (int r = 0; r < TR; ++r) {
                const uint32_t d = tmem + (uint32_t)(r * COUT);
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                    for (int kc = 0; kc < CH / 2; ++kc) {
                        const uint64_t ad = a0 + (uint64_t)(((2 * kc) * HY + r + dy) * HXW + dx);
                        const uint64_t bd = b0 + (uint64_t)((tap * CH + 2 * kc) * COUT);
                        if (F8) tc::mma_e4m3(d, ad, bd, idesc, (tap | kc) != 0);
                        else tc::mma_f16(d, ad, bd, idesc, (tap | kc) != 0);
                    }
                }
            }
            tc::mma_commit(bar);
        }
        // stage the next tile into the other buffer while the MMAs run
        if (L::NBUF == 2 && next < a.ntiles) stage(next, buf ^ 1);
        if (!tc::mbar_wait(bar, phase, kWaitLimit)) {
            failed = true;
            if (tid == 0) atomicExch(a.error, 1);
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();

        // ---- epilogue: one pixel per thread --------------------------------
        const int px = (warp & 3) * 32 + lane;   // TMEM lane = pixel within the tile row
        const int x = x0 + px;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        // warp group g = warp / 4 handles rows [2g, 2g + 2): the row pairs of the pooling
        const int r_lo = (warp >> 2) * 2, r_hi = min(TR, r_lo + 2);
        if (EPI != TEPI_HEADKP) {
            float prev[COUT];                    // row r - 1 (pooling pairs rows 2k, 2k+1)
#pragma unroll 1
            for (int r = r_lo; r < r_hi; ++r) {
                const int y = y0 + r;
                float v[COUT];
#pragma unroll
                for (int c = 0; c < COUT; c += 16) tc::tmem_ld16(tmem + lane_base + r * COUT + c, v + c);
#pragma unroll
                for (int c = 0; c < COUT; ++c) v[c] = fmaxf(fmaf(v[c], sScale[c], sBias[c]), 0.f);
                if (y < im.Hl && x < im.Wl)
                    store_pixel<COUT, F8>(im.out, (long long)im.Hl * im.Wl, (long long)y * im.Wl + x, v, a.out_q);
                if (EPI == TEPI_POOL) {
                    if (r & 1) {
                        float s[COUT];
#pragma unroll
                        for (int c = 0; c < COUT; ++c) {
                            s[c] = prev[c] + v[c];
                            s[c] += __shfl_xor_sync(0xffffffffu, s[c], 1);
                            s[c] *= 0.25f;
                        }
                        if ((lane & 1) == 0 && y < im.Hl && x < im.Wl)
                            store_pixel<COUT, F8>(im.pooled, (long long)(im.Hl >> 1) * (im.Wl >> 1),
                                                  (long long)(y >> 1) * (im.Wl >> 1) + (x >> 1), s, a.pool_q);
                    } else {
#pragma unroll
                        for (int c = 0; c < COUT; ++c) prev[c] = v[c];
                    }
                }
            }
        } else {
            // activations (scale, bias, ReLU, FP16) -> shared memory as the head's A operand
#pragma unroll 1
            for (int r = r_lo; r < r_hi; ++r) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + r * COUT, v);
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = fmaxf(fmaf(v[c], sScale[c], sBias[c]), 0.f);
                *reinterpret_cast<uint4*>(sHA + ((r * 2 + 0) * TW + px) * 16) = pack8h(v);
                *reinterpret_cast<uint4*>(sHA + ((r * 2 + 1) * TW + px) * 16) = pack8h(v + 8);
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                constexpr uint32_t hdesc = tc::idesc_f16(128, 32);
                const uint64_t bd = tc::smem_desc(tc::smem_addr(sHB), 32 * 16, 128);
                for (int r = 0; r < TR; ++r) {
                    const uint64_t ad = tc::smem_desc(tc::smem_addr(sHA + r * 2 * TW * 16), TW * 16, 128);
                    tc::mma_f16(tmem + (uint32_t)(r * 32), ad, bd, hdesc, 0);
                }
                tc::mma_commit(bar);
            }
            if (!tc::mbar_wait(bar, phase, kWaitLimit)) {
                failed = true;
                if (tid == 0) atomicExch(a.error, 1);
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            const long long plane = (long long)im.H0 * im.W0;
#pragma unroll 1
            for (int r = r_lo; r < r_hi; ++r) {
                const int y = y0 + r;
                float hd[32];
                tc::tmem_ld16(tmem + lane_base + r * 32, hd);
                tc::tmem_ld16(tmem + lane_base + r * 32 + 16, hd + 16);
#pragma unroll
                for (int j = 0; j < 29; ++j) hd[j] += sBias[COUT + j];
                float mx = hd[3];
#pragma unroll
                for (int q = 1; q < 25; ++q) mx = fmaxf(mx, hd[3 + q]);
                // one pass with the unnormalised softmax weights e_q: the
                // normalisation cancels in num / den, and den / sum(e) is the
                // normalised sampled weight the 1e-12 test is defined on
                float es = 0.f, den = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
                for (int q = 0; q < 25; ++q) {
                    const float e = expf(hd[3 + q] - mx);
                    const float4 s = sSP[(r + q / 5) * (TW + 4) + px + q % 5];
                    const float wm = e * s.w;
                    es += e;
                    den += wm;
                    n0 = fmaf(wm, s.x, n0);
                    n1 = fmaf(wm, s.y, n1);
                    n2 = fmaf(wm, s.z, n2);
                }
                float k0 = hd[0], k1 = hd[1], k2 = hd[2];
                if (den >= 1e-12f * es) {
                    k0 = n0 / den;
                    k1 = n1 / den;
                    k2 = n2 / den;
                }
                const float al = 1.0f / (1.0f + expf(-hd[28]));
                if (y < im.H0 && x < im.W0) {
                    float* o = im.rgb + (long long)y * im.W0 + x;
                    o[0] = fmaf(al, k0 - hd[0], hd[0]);
                    o[plane] = fmaf(al, k1 - hd[1], hd[1]);
                    o[2 * plane] = fmaf(al, k2 - hd[2], hd[2]);
                }
            }
        }
        // ---- make the next tile's halo ready --------------------------------
        tc::fence_before_sync();
        if (L::NBUF == 1) {
            __syncthreads();   // the epilogue is done with shared memory and TMEM
            if (next < a.ntiles) stage(next, 0);
        }
        cp_wait_all();
        tc::fence_async_smem();
        __syncthreads();
        tc::fence_after_sync();
        buf ^= L::NBUF - 1;
    }
    cp_wait_all();   // no copy may still target shared memory when the CTA exits
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, L::tmem_cols);
    }
}

// amax of a non-negative FP16 tensor (calibration of the FP8 scales)
__global__ void amax_f16_kernel(const __half* __restrict__ x, long long n, float* __restrict__ out) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__half2float(x[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

}  // namespace

}  // namespace fvn

#include "conv_ws.cuh"
#include "conv_ks.cuh"

namespace fvn {

// Launch with programmatic stream serialisation: the kernel may start (and
// run its prologue) while the previous kernel in the stream finishes; it
// waits for that kernel (griddepcontrol.wait) before touching activations.
template <typename Arg>
static cudaError_t launch_pdl(void (*kern)(Arg), dim3 grid, dim3 block, size_t smem, cudaStream_t st, const Arg& arg) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

template <int CIN, int CG, int COUT, int TR, int MODE, int EPI, int CUP, bool F8>
static fvn_status launch_tc(fvn_ctx* ctx, TcArgs& a, cudaStream_t st) {
    using L = TcLayout<CIN, CG, COUT, TR, MODE, EPI, CUP, F8>;
    auto kern = conv3x3_tc_kernel<CIN, CG, COUT, TR, MODE, EPI, CUP, F8>;
    static std::atomic<unsigned long long> configured{0};
    FVN_CUDA(ctx, opt_in_smem(ctx, kern, (int)L::bytes, configured));
    // CTAs per SM from the shared-memory budget (1 KB reserved per CTA) and
    // the 512 TMEM columns, so that no CTA ever waits in tcgen05.alloc.
    int smem_sm = 0;
    FVN_CUDA(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    int per_sm = smem_sm / (int)(L::bytes + 1024);
    per_sm = std::min(per_sm, (int)(512 / L::tmem_cols));
    per_sm = std::min(per_sm, 2048 / kThreads);
    if (per_sm < 1) return set_error(ctx, FVN_ERR_CUDA, "tensor-core conv kernel does not fit on an SM");
    int ntiles = 0;
    for (int i = 0; i < a.nimg; ++i) {
        TcImg& m = a.img[i];
        m.tiles_x = (m.Wl + TW - 1) / TW;
        m.tile0 = ntiles;
        ntiles += m.tiles_x * ((m.Hl + TR - 1) / TR);
    }
    a.ntiles = ntiles;
    const int grid = std::min(a.ntiles, ctx->num_sms * per_sm);
    a.error = ctx->d_error;
    if (grid > 0) {
        FVN_CUDA(ctx, launch_pdl(kern, dim3(grid), dim3(kThreads), L::bytes, st, a));
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

// ---- TMA tensor maps and the warp-specialised launches ---------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (the runtime is linked, not libcuda).
static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return static_cast<EncodeTiledFn>(nullptr);
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Map of a chunk-planar tensor [C / chunk][H][W][16 B] (FP16, or FP8 as
// bytes) seen as 8-byte elements, whose box is one chunk plane's 128 pixels
// (256 elements, 2048 contiguous bytes) x hy rows: one plane of a stage.
static fvn_status make_map(fvn_ctx* ctx, CUtensorMap* m, const void* base, int C, int W, int H, int hy, bool f8,
                           int box_px = ws::kHXW) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return set_error(ctx, FVN_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t cpc = f8 ? 16 : 8;
    const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)C / cpc};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)W * H * 16};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * box_px), (cuuint32_t)hy, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(ctx, FVN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for a %d x %d x %d tensor", (int)r, H,
                         W, C);
    return FVN_OK;
}

// One image of a warp-specialised layer: source 0 (c0 channels) and source 1
// (c1 channels, may be absent), outputs, size.
struct WsSpec {
    const void* in0;
    int c0;
    const void* in1;
    int c1;
    void* out;
    void* pooled;
    int Hl, Wl;
};

// Stages of the shared-memory ring that fit next to the resident weights.
template <int CIN, int COUT, int TR, bool F8, bool FUSE, int UPC = 0, bool CB1 = false>
constexpr int ws_stages() {
    using L1 = ws::Layout<CIN, COUT, TR, 1, F8, FUSE, UPC, CB1>;
    const long long per = (long long)L1::stage + (CB1 ? 0 : L1::coarse) + 8 * (UPC ? 3 : 2);   // bytes of one stage
    const long long budget = 227 * 1024 - (long long)L1::bytes + per;             // bytes for the stages
    const long long ns = budget / per;
    return ns >= 4 ? 4 : (ns < 1 ? 1 : (int)ns);
}

// A warp-specialised layer; UPC > 0: source 0 is the coarse level, whose
// bilinear x2 up-sampling (UPC chunks) the kernel computes itself.
template <int CIN, int CHG, int CH0, int COUT, int TR, bool POOL, bool F8, bool FUSE = false, int UPC = 0>
static fvn_status launch_ws(fvn_ctx* ctx, const WsSpec* spec, int n, const ConvW& w, float out_q, float pool_q,
                            cudaStream_t st) {
    // an up-sampled layer left with a single stage by a coarse buffer per
    // stage shares one coarse buffer among the stages instead, where that
    // makes room for a second stage
    constexpr int NS_PER = ws_stages<CIN, COUT, TR, F8, FUSE, UPC>();
    constexpr int NS_ONE = UPC > 0 ? ws_stages<CIN, COUT, TR, F8, FUSE, UPC, (UPC > 0)>() : 0;
    constexpr bool CB1 = NS_PER == 1 && NS_ONE > 1;
    constexpr int NS = CB1 ? NS_ONE : NS_PER;
    using L = ws::Layout<CIN, COUT, TR, NS, F8, FUSE, UPC, CB1>;
    static_assert(L::bytes <= 227 * 1024, "stage ring does not fit in shared memory");
    static_assert(sizeof(ws::Args) <= 32764, "kernel arguments exceed the parameter space");
    auto kern = ws::conv3x3_ws_kernel<CIN, CHG, CH0, COUT, TR, NS, POOL, F8, FUSE, UPC, CB1>;
    static std::atomic<unsigned long long> configured{0};
    FVN_CUDA(ctx, opt_in_smem(ctx, kern, (int)L::bytes, configured));
    int smem_sm = 0;
    FVN_CUDA(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    int per_sm = smem_sm / (int)(L::bytes + 1024);
    per_sm = std::min(per_sm, (int)(512 / L::tmem_cols));
    per_sm = std::min(per_sm, 2048 / L::threads);
    if (per_sm < 1) return set_error(ctx, FVN_ERR_CUDA, "warp-specialised conv kernel does not fit on an SM");
    constexpr int CPC = L::CPC;
    ws::Args a{};
    a.w = F8 ? static_cast<const void*>(w.w8) : static_cast<const void*>(w.w16);
    a.bias = w.bias;
    a.wscale = w.scale8;
    a.out_q = out_q;
    a.pool_q = pool_q;
    a.nimg = n;
    a.error = ctx->d_error;
    int ntiles = 0;
    for (int i = 0; i < n; ++i) {
        const WsSpec& sp = spec[i];
        ws::Img& m = a.img[i];
        if (sp.c0 != CH0 * CPC || sp.c0 + sp.c1 != CHG * CPC)
            return set_error(ctx, FVN_ERR_ARG, "conv layer channels %d + %d do not match the kernel", sp.c0, sp.c1);
        fvn_status s = UPC ? make_map(ctx, &m.map0, sp.in0, sp.c0, sp.Wl / 2, sp.Hl / 2, L::CR, F8, L::CC)
                           : make_map(ctx, &m.map0, sp.in0, sp.c0, sp.Wl, sp.Hl, L::HY, F8);
        if (s != FVN_OK) return s;
        if (sp.c1 > 0) {
            if ((s = make_map(ctx, &m.map1, sp.in1, sp.c1, sp.Wl, sp.Hl, L::HY, F8)) != FVN_OK) return s;
        } else {
            m.map1 = m.map0;
        }
        m.out = sp.out;
        m.pooled = sp.pooled;
        m.Hl = sp.Hl;
        m.Wl = sp.Wl;
        m.tiles_x = (sp.Wl + ws::kTO - 1) / ws::kTO;
        m.tile0 = ntiles;
        ntiles += m.tiles_x * ((sp.Hl + TR - 1) / TR);
    }
    a.ntiles = ntiles;
    const int grid = std::min(ntiles, ctx->num_sms * per_sm);
    if (grid > 0) {
        FVN_CUDA(ctx, launch_pdl(kern, dim3(grid), dim3(L::threads), L::bytes, st, a));
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

// Map of the sparse frame [5][H0][W0] float32 whose box is 136 columns x
// rows rows of one plane (the kernel-prediction window of a tile).
static fvn_status make_sparse_map(fvn_ctx* ctx, CUtensorMap* m, const float* base, int W0, int H0, int rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return set_error(ctx, FVN_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)W0, (cuuint64_t)H0, 5};
    const cuuint64_t strides[2] = {(cuuint64_t)W0 * 4, (cuuint64_t)W0 * H0 * 4};
    const cuuint32_t box[3] = {(cuuint32_t)ws::kSpW, (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(ctx, FVN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for a %d x %d sparse frame", (int)r,
                         H0, W0);
    return FVN_OK;
}

// Last layer + head + kernel prediction + blend, warp-specialised (frame
// widths that are multiples of 4, so the sparse frame's rows are 16-byte
// aligned for TMA).
template <bool F8>
static fvn_status launch_ws_headkp(fvn_ctx* ctx, const ReconView* views, int n, cudaStream_t st) {
    constexpr int CIN = F8 ? 32 : 16, CPC = F8 ? 16 : 8, TR = 4, NS = 4;
    using L = ws::HkLayout<CIN, TR, NS, F8>;
    static_assert(L::bytes <= 227 * 1024, "head / kernel-prediction kernel does not fit in shared memory");
    static_assert(sizeof(ws::HkArgs) <= 32764, "kernel arguments exceed the parameter space");
    auto kern = ws::conv3x3_ws_headkp_kernel<CIN, 16 / CPC, TR, NS, F8>;
    static std::atomic<unsigned long long> configured{0};
    FVN_CUDA(ctx, opt_in_smem(ctx, kern, (int)L::bytes, configured));
    const ConvW& w = ctx->layers[9];
    ws::HkArgs h{};
    ws::Args& a = h.conv;
    a.w = F8 ? static_cast<const void*>(w.w8) : static_cast<const void*>(w.w16);
    a.bias = w.bias;
    a.wscale = w.scale8;
    a.nimg = n;
    a.error = ctx->d_error;
    h.head_w = ctx->head_w16;
    h.head_b = ctx->head_b32;
    int ntiles = 0;
    for (int i = 0; i < n; ++i) {
        const ReconView& v = views[i];
        const int Wl = (v.w + 3) & ~3, Hl = (v.h + 3) & ~3;
        ws::Img& m = a.img[i];
        fvn_status s = make_map(ctx, &m.map0, v.plan.d0a, 16, Wl, Hl, TR + 2, F8);
        if (s != FVN_OK) return s;
        m.map1 = m.map0;
        if ((s = make_sparse_map(ctx, &h.sp[i], v.rgbam, v.w, v.h, TR + 4)) != FVN_OK) return s;
        h.rgb[i] = v.rgb;
        h.H0[i] = v.h;
        h.W0[i] = v.w;
        m.Hl = Hl;
        m.Wl = Wl;
        m.tiles_x = (Wl + ws::kTO - 1) / ws::kTO;
        m.tile0 = ntiles;
        ntiles += m.tiles_x * ((Hl + TR - 1) / TR);
    }
    a.ntiles = ntiles;
    int smem_sm = 0;
    FVN_CUDA(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    int per_sm = std::min(smem_sm / (int)(L::bytes + 1024), (int)(512 / L::tmem_cols));
    if (per_sm < 1) return set_error(ctx, FVN_ERR_CUDA, "head / kernel-prediction kernel does not fit on an SM");
    const int grid = std::min(ntiles, ctx->num_sms * per_sm);
    if (grid > 0) {
        FVN_CUDA(ctx, launch_pdl(kern, dim3(grid), dim3(ws::kHkThreads), L::bytes, st, h));
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

// Bilinear x2 up-sampling of the coarse level of every view (one launch, one
// block per pair of fine rows of one chunk plane of one view).
struct UpArgs {
    int n, chunks;
    struct {
        const void* coarse;
        void* fine;
        int Hl, Wl;
        int row0;                     // first block of this view
    } im[kMaxViews];
};

template <bool F8>
__global__ void __launch_bounds__(256) upsample2_views_kernel(const __grid_constant__ UpArgs u) {
    tc::grid_dep_wait();
    tc::grid_dep_launch();
    int i = 0;
    while (i + 1 < u.n && (int)blockIdx.x >= u.im[i + 1].row0) ++i;
    const int hp = u.im[i].Hl >> 1;                 // fine row pairs per chunk plane
    const int r = blockIdx.x - u.im[i].row0;        // chunk * hp + pair
    const int c = r / hp, my = r - c * hp;
    ws::upsample2_rowpair<F8>(u.im[i].coarse, u.im[i].fine, u.im[i].Hl, u.im[i].Wl, c, my);
}

template <bool F8>
static fvn_status upsample_views(fvn_ctx* ctx, const void* const* coarse, void* const* fine, const int* Hl,
                                 const int* Wl, int n, int channels, cudaStream_t st) {
    UpArgs u{};
    u.n = n;
    u.chunks = channels / (F8 ? 16 : 8);
    long long rows = 0;
    for (int i = 0; i < n; ++i) {
        u.im[i].coarse = coarse[i];
        u.im[i].fine = fine[i];
        u.im[i].Hl = Hl[i];
        u.im[i].Wl = Wl[i];
        u.im[i].row0 = (int)rows;
        rows += (long long)u.chunks * (Hl[i] >> 1);   // one block per pair of fine rows (Hl is even)
    }
    if (rows >= (1ll << 31)) return set_error(ctx, FVN_ERR_ARG, "up-sampling grid too large");
    if (rows > 0) {
        FVN_CUDA(ctx, launch_pdl(upsample2_views_kernel<F8>, dim3((unsigned)rows), dim3(256), 0, st, u));
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

// Tensors and sizes of layer l (0..9) of the network for one view.
static TcImg layer_img(int l, const ReconView& v) {
    const ReconPlan& B = v.plan;
    const int W4 = (v.w + 3) & ~3, H4 = (v.h + 3) & ~3;
    TcImg m{};
    switch (l) {
        case 0:
            m.rgbam = v.rgbam; m.prev = v.prev; m.H0 = v.h; m.W0 = v.w; m.out = B.e0a; m.Hl = H4; m.Wl = W4;
            break;
        case 1: m.in = B.e0a; m.out = B.e0; m.pooled = B.p0; m.Hl = H4; m.Wl = W4; break;
        case 2: m.in = B.p0; m.out = B.e1a; m.Hl = H4 / 2; m.Wl = W4 / 2; break;
        case 3: m.in = B.e1a; m.out = B.e1; m.pooled = B.p1; m.Hl = H4 / 2; m.Wl = W4 / 2; break;
        case 4: m.in = B.p1; m.out = B.ba; m.Hl = H4 / 4; m.Wl = W4 / 4; break;
        case 5: m.in = B.ba; m.out = B.bt; m.Hl = H4 / 4; m.Wl = W4 / 4; break;
        case 6: m.in = B.bt; m.skip = B.e1; m.out = B.d1a; m.Hl = H4 / 2; m.Wl = W4 / 2; break;
        case 7: m.in = B.d1a; m.out = B.d1; m.Hl = H4 / 2; m.Wl = W4 / 2; break;
        case 8: m.in = B.d1; m.skip = B.e0; m.out = B.d0a; m.Hl = H4; m.Wl = W4; break;
        default:
            m.in = B.d0a; m.rgbam = v.rgbam; m.H0 = v.h; m.W0 = v.w; m.rgb = v.rgb; m.Hl = H4; m.Wl = W4;
            break;
    }
    return m;
}

// The launches of the network over every view at once (one launch per layer
// covers the tiles of all views).  FP16 operands, or FP8 operands with the
// calibrated scales; FP8 tensors use half of each FP16 buffer.  The first
// layer (reading the planar sparse frame) and the last (head, kernel
// prediction, blend) run conv3x3_tc_kernel; the eight in between run the
// warp-specialised TMA kernel, the two decoder layers on an up-sampled copy
// of the coarse level.
template <bool F8>
static fvn_status run_tc(fvn_ctx* ctx, const ReconView* views, int n, cudaStream_t st) {
    const ConvW* L = ctx->layers;
    const float* q = ctx->fp8_inv_scale;   // 1 / s per activation tensor
    constexpr int CPC = F8 ? 16 : 8;
    constexpr int K16 = F8 ? 32 : 16;      // K per tap of the 16-channel layers (FP8 MMA K = 32)
    TcArgs a;
    auto prep = [&](int l) {
        a = TcArgs{};
        a.nimg = n;
        for (int i = 0; i < n; ++i) a.img[i] = layer_img(l, views[i]);
        a.w = F8 ? static_cast<const void*>(L[l].w8) : static_cast<const void*>(L[l].w16);
        a.bias = L[l].bias;
        a.wscale = L[l].scale8;
    };
    WsSpec sp[kMaxViews];
    int Hh[kMaxViews], Wh[kMaxViews], Hf[kMaxViews], Wf[kMaxViews];
    for (int i = 0; i < n; ++i) {
        Wf[i] = (views[i].w + 3) & ~3;
        Hf[i] = (views[i].h + 3) & ~3;
        Wh[i] = Wf[i] / 2;
        Hh[i] = Hf[i] / 2;
    }
    // spec of layer l for view i: sources, outputs, level size
    auto spec = [&](const void* in0, int c0, const void* in1, int c1, void* out, void* pooled, int H, int W) {
        return WsSpec{in0, c0, in1, c1, out, pooled, H, W};
    };
    fvn_status s;
    prep(0);
    a.in_q = q[FP8_RGBAM]; a.out_q = q[FP8_E0A];
    if ((s = launch_tc<K16, 16, 16, 4, TIN_RGBAM, TEPI_STORE, 0, F8>(ctx, a, st)) != FVN_OK) return s;
    // enc0b (+ pool)
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.e0a, 16, nullptr, 0, B.e0, B.p0, Hf[i], Wf[i]);
    }
    if ((s = launch_ws<K16, 16 / CPC, 16 / CPC, 16, 4, true, F8, true>(ctx, sp, n, L[1], q[FP8_E0], q[FP8_P0], st)) !=
        FVN_OK)
        return s;
    // enc1a, enc1b (+ pool)
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.p0, 16, nullptr, 0, B.e1a, nullptr, Hh[i], Wh[i]);
    }
    s = ctx->conv_rows_half == 2
            ? launch_ws<K16, 16 / CPC, 16 / CPC, 32, 2, false, F8>(ctx, sp, n, L[2], q[FP8_E1A], 0.f, st)
            : launch_ws<K16, 16 / CPC, 16 / CPC, 32, 4, false, F8>(ctx, sp, n, L[2], q[FP8_E1A], 0.f, st);
    if (s != FVN_OK)
        return s;
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.e1a, 32, nullptr, 0, B.e1, B.p1, Hh[i], Wh[i]);
    }
    s = ctx->conv_rows_half == 2
            ? launch_ws<32, 32 / CPC, 32 / CPC, 32, 2, true, F8>(ctx, sp, n, L[3], q[FP8_E1], q[FP8_P1], st)
            : launch_ws<32, 32 / CPC, 32 / CPC, 32, 4, true, F8>(ctx, sp, n, L[3], q[FP8_E1], q[FP8_P1], st);
    if (s != FVN_OK)
        return s;
    // bottleneck
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.p1, 32, nullptr, 0, B.ba, nullptr, Hf[i] / 4, Wf[i] / 4);
    }
    s = ctx->conv_rows_quarter == 1
            ? launch_ws<32, 32 / CPC, 32 / CPC, 64, 1, false, F8>(ctx, sp, n, L[4], q[FP8_BA], 0.f, st)
            : ctx->conv_rows_quarter == 4
                  ? launch_ws<32, 32 / CPC, 32 / CPC, 64, 4, false, F8>(ctx, sp, n, L[4], q[FP8_BA], 0.f, st)
                  : launch_ws<32, 32 / CPC, 32 / CPC, 64, 2, false, F8>(ctx, sp, n, L[4], q[FP8_BA], 0.f, st);
    if (s != FVN_OK)
        return s;
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.ba, 64, nullptr, 0, B.bt, nullptr, Hf[i] / 4, Wf[i] / 4);
    }
    s = ctx->conv_rows_quarter == 1
            ? launch_ws<64, 64 / CPC, 64 / CPC, 64, 1, false, F8>(ctx, sp, n, L[5], q[FP8_BT], 0.f, st)
            : ctx->conv_rows_quarter == 4
                  ? launch_ws<64, 64 / CPC, 64 / CPC, 64, 4, false, F8>(ctx, sp, n, L[5], q[FP8_BT], 0.f, st)
                  : launch_ws<64, 64 / CPC, 64 / CPC, 64, 2, false, F8>(ctx, sp, n, L[5], q[FP8_BT], 0.f, st);
    if (s != FVN_OK)
        return s;
    // dec1a on [up(bt), e1]: the up-sampling of bt in its own pass, or
    // inside the convolution (FVN_OPT_CONV_FUSE_UP_DEC1), then dec1b
    if (ctx->conv_fuse_up_dec1) {
        for (int i = 0; i < n; ++i) {
            const ReconPlan& B = views[i].plan;
            sp[i] = spec(B.bt, 64, B.e1, 32, B.d1a, nullptr, Hh[i], Wh[i]);
        }
        s = ctx->conv_rows_dec1 == 2
                ? launch_ws<96, 96 / CPC, 64 / CPC, 32, 2, false, F8, false, 64 / CPC>(ctx, sp, n, L[6],
                                                                                    q[FP8_D1A], 0.f, st)
                : launch_ws<96, 96 / CPC, 64 / CPC, 32, 1, false, F8, false, 64 / CPC>(ctx, sp, n, L[6],
                                                                                    q[FP8_D1A], 0.f, st);
    } else {
        const void* c[kMaxViews];
        void* f[kMaxViews];
        for (int i = 0; i < n; ++i) {
            c[i] = views[i].plan.bt;
            f[i] = views[i].plan.u1;
        }
        if ((s = upsample_views<F8>(ctx, c, f, Hh, Wh, n, 64, st)) != FVN_OK) return s;
        for (int i = 0; i < n; ++i) {
            const ReconPlan& B = views[i].plan;
            sp[i] = spec(B.u1, 64, B.e1, 32, B.d1a, nullptr, Hh[i], Wh[i]);
        }
        s = ctx->conv_rows_dec1 == 2
                ? launch_ws<96, 96 / CPC, 64 / CPC, 32, 2, false, F8>(ctx, sp, n, L[6], q[FP8_D1A], 0.f, st)
                : launch_ws<96, 96 / CPC, 64 / CPC, 32, 1, false, F8>(ctx, sp, n, L[6], q[FP8_D1A], 0.f, st);
    }
    if (s != FVN_OK) return s;
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.d1a, 32, nullptr, 0, B.d1, nullptr, Hh[i], Wh[i]);
    }
    s = ctx->conv_rows_half == 2
            ? launch_ws<32, 32 / CPC, 32 / CPC, 32, 2, false, F8>(ctx, sp, n, L[7], q[FP8_D1], 0.f, st)
            : launch_ws<32, 32 / CPC, 32 / CPC, 32, 4, false, F8>(ctx, sp, n, L[7], q[FP8_D1], 0.f, st);
    if (s != FVN_OK)
        return s;
    // dec0a on [up(d1), e0], the up-sampling computed inside the layer from d1
    for (int i = 0; i < n; ++i) {
        const ReconPlan& B = views[i].plan;
        sp[i] = spec(B.d1, 32, B.e0, 16, B.d0a, nullptr, Hf[i], Wf[i]);
    }
    if ((s = launch_ws<F8 ? 64 : 48, 48 / CPC, 32 / CPC, 16, 4, false, F8, true, 32 / CPC>(
             ctx, sp, n, L[8], q[FP8_D0A], 0.f, st)) != FVN_OK)
        return s;
    // dec0b + head + kernel prediction + blend: the warp-specialised kernel for
    // views whose width is a multiple of 4 (TMA rows of the sparse frame), the
    // staged kernel for the others -- each view always takes the same kernel
    ReconView al[kMaxViews], un[kMaxViews];
    int na = 0, nu = 0;
    for (int i = 0; i < n; ++i) {
        if (views[i].w % 4 == 0) al[na++] = views[i];
        else un[nu++] = views[i];
    }
    if (na > 0 && (s = launch_ws_headkp<F8>(ctx, al, na, st)) != FVN_OK) return s;
    if (nu == 0) return FVN_OK;
    a = TcArgs{};
    a.nimg = nu;
    for (int i = 0; i < nu; ++i) a.img[i] = layer_img(9, un[i]);
    a.w = F8 ? static_cast<const void*>(L[9].w8) : static_cast<const void*>(L[9].w16);
    a.bias = L[9].bias;
    a.wscale = L[9].scale8;
    a.head_w = ctx->head_w16;
    a.head_b = ctx->head_b32;
    return launch_tc<K16, 16, 16, 4, TIN_ACT, TEPI_HEADKP, 0, F8>(ctx, a, st);
}

fvn_status reconstruct_tc_views(fvn_ctx* ctx, const ReconView* views, int n, int precision, cudaStream_t st) {
    if (n < 1 || n > kMaxViews) return set_error(ctx, FVN_ERR_ARG, "%d views (1..%d)", n, kMaxViews);
    return precision == FVN_PREC_FP8 ? run_tc<true>(ctx, views, n, st) : run_tc<false>(ctx, views, n, st);
}

fvn_status reconstruct_tc(fvn_ctx* ctx, const ReconPlan& B, const float* rgbam, const float* prev, int w, int h,
                          float* rgb, cudaStream_t st) {
    const ReconView v{B, rgbam, w, h, rgb, prev};
    return run_tc<false>(ctx, &v, 1, st);
}

fvn_status reconstruct_tc_fp8(fvn_ctx* ctx, const ReconPlan& B, const float* rgbam, const float* prev, int w,
                              int h, float* rgb, cudaStream_t st) {
    const ReconView v{B, rgbam, w, h, rgb, prev};
    return run_tc<true>(ctx, &v, 1, st);
}

// Reduce the amax of every calibrated activation tensor of the FP16 network
// into d_amax[FP8_NT] (running maximum).
fvn_status calibrate_amax(fvn_ctx* ctx, const ReconPlan& B, int w, int h, float* d_amax, cudaStream_t st) {
    const long long W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    const long long n0 = W4 * H4, n1 = n0 / 4, n2 = n0 / 16;
    struct T {
        const __half* p;
        long long n;
        int slot;
    } t[] = {{B.e0a, n0 * 16, FP8_E0A}, {B.e0, n0 * 16, FP8_E0},  {B.p0, n1 * 16, FP8_P0},
             {B.e1a, n1 * 32, FP8_E1A}, {B.e1, n1 * 32, FP8_E1},  {B.p1, n2 * 32, FP8_P1},
             {B.ba, n2 * 64, FP8_BA},   {B.bt, n2 * 64, FP8_BT},  {B.d1a, n1 * 32, FP8_D1A},
             {B.d1, n1 * 32, FP8_D1},   {B.d0a, n0 * 16, FP8_D0A}};
    for (const auto& x : t) {
        const int grid = (int)std::min<long long>((x.n + 255) / 256, 8LL * ctx->num_sms);
        amax_f16_kernel<<<grid, 256, 0, st>>>(x.p, x.n, d_amax + x.slot);
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

// ---------------------------------------------------------------------------
// K-streamed layers (conv_ks.cuh)
// ---------------------------------------------------------------------------

// Stages of the ring that fit in shared memory (at most 4).
template <int COUTP, int TR, bool K1, bool UP>
constexpr int ks_stages() {
    using L1 = ks::Layout<COUTP, TR, 1, K1, UP>;
    const long long per = (long long)L1::stage + 16;
    const long long ns = (227 * 1024 - (long long)L1::bytes + per) / per;
    return ns >= 4 ? 4 : (ns < 1 ? 1 : (int)ns);
}

template <int COUTP, int TR, bool K1, bool UP>
static fvn_status launch_ks(fvn_ctx* ctx, const KsConv& c, cudaStream_t st) {
    constexpr int NS = ks_stages<COUTP, TR, K1, UP>();
    using L = ks::Layout<COUTP, TR, NS, K1, UP>;
    static_assert(L::bytes <= 227 * 1024, "stage ring does not fit in shared memory");
    auto kern = ks::conv_ks_kernel<COUTP, TR, NS, K1, UP>;
    static std::atomic<unsigned long long> configured{0};
    FVN_CUDA(ctx, opt_in_smem(ctx, kern, (int)L::bytes, configured));
    ks::Args a{};
    fvn_status s = UP ? make_map(ctx, &a.map0, c.in0, 8 * c.ch0, c.W / 2, c.H / 2, L::CR, false, L::CC)
                      : make_map(ctx, &a.map0, c.in0, 8 * c.ch0, c.W, c.H, L::HY, false);
    if (s != FVN_OK) return s;
    if (c.ch1 > 0) {
        if ((s = make_map(ctx, &a.map1, c.in1, 8 * c.ch1, c.W, c.H, L::HY, false)) != FVN_OK) return s;
    } else {
        a.map1 = a.map0;
    }
    a.ch0 = c.ch0;
    a.has1 = c.ch1 > 0;
    a.groups = (c.ch0 + c.ch1 + 1) / 2;
    a.w = static_cast<const uint4*>(c.wpk);
    a.bias = c.bias;
    a.out = static_cast<uint4*>(c.out);
    a.out_chunks = (c.cout + 7) / 8;
    a.out32 = c.out32;
    a.cout = c.cout;
    a.relu = c.relu;
    a.H = c.H;
    a.W = c.W;
    a.tiles_x = (c.W + L::TO - 1) / L::TO;
    a.ntiles = a.tiles_x * ((c.H + TR - 1) / TR);
    a.Hc = c.H / 2;
    a.Wc = c.W / 2;
    a.error = ctx->d_error;
    const int grid = std::max(1, std::min(a.ntiles, ctx->num_sms > 0 ? ctx->num_sms : 148));
    kern<<<grid, L::threads, L::bytes, st>>>(a);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

int ks_coutp(int cout) { return (cout + 15) / 16 * 16; }

fvn_status ks_conv(fvn_ctx* ctx, const KsConv& c, cudaStream_t st) {
    FVN_CHECK_ARG(ctx, c.in0 && c.wpk && c.bias && (c.out || c.out32) && (c.ch1 == 0 || c.in1), "null tensor");
    FVN_CHECK_ARG(ctx, c.ch0 >= 1 && c.ch1 >= 0 && c.H >= 1 && c.W >= 1 && (c.k == 1 || c.k == 3), "bad layer");
    FVN_CHECK_ARG(ctx, !c.up || (c.ch0 % 2 == 0 && c.H % 2 == 0 && c.W % 2 == 0 && c.H >= 2 && c.W >= 2),
                  "an up-sampled source needs an even chunk count and an even frame");
    const int cp = ks_coutp(c.cout);
    const bool k1 = c.k == 1;
#define FVN_KS(CP, TR)                                                                                           \
    if (cp == CP) {                                                                                              \
        if (c.up) return k1 ? launch_ks<CP, TR, true, true>(ctx, c, st) : launch_ks<CP, TR, false, true>(ctx, c, st); \
        return k1 ? launch_ks<CP, TR, true, false>(ctx, c, st) : launch_ks<CP, TR, false, false>(ctx, c, st);       \
    }
    FVN_KS(16, 4)
    FVN_KS(32, 4)
    FVN_KS(48, 4)
    FVN_KS(64, 4)
    FVN_KS(80, 2)
    FVN_KS(96, 2)
    FVN_KS(112, 2)
    FVN_KS(128, 2)
#undef FVN_KS
    return set_error(ctx, FVN_ERR_UNSUPPORTED, "no K-streamed convolution for %d output channels", c.cout);
}

}  // namespace fvn

namespace fvn {

// The error path of every bounded tensor-core wait, on its own: an mbarrier
// that nothing completes, polled `limit` times by one thread, which then
// records the give-up in the context's error flag and returns.
__global__ void selftest_wait_kernel(int* error, unsigned limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit)) atomicExch(error, 2);
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_selftest_wait_timeout(fvn_ctx* ctx, unsigned limit, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, limit >= 1 && limit <= (1u << 20), "limit %u outside [1, 2^20]", limit);
    selftest_wait_kernel<<<1, 32, 0, as_stream(stream)>>>(ctx->d_error, limit);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}
