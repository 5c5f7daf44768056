// Reconstruction network inference (paper: "Reconstruction Network", Fig.
// "network architecture"; "Model Precision & Optimization": weights truncated
// to 16 bit).  Slim U-Net of 16/32/64 channels, then the 1x1 head, the 5x5
// kernel prediction on the sparse samples and the blend.
//
// Layout: activations are NHWC FP16 ("channels innermost"), per resolution
// level of the frame padded to a multiple of 4.  Every 3x3 convolution is an
// implicit GEMM on the tensor cores (FP16 operands, FP32 accumulation):
// M = output pixels, N = output channels, K = 9 taps x input channels.
//
// Conv kernel: persistent CTAs keep the layer's weights in shared memory and
// loop over output tiles of 4 rows x 64 pixels.  Each tile stages its input
// halo (6 x 66 pixels) in shared memory as planes of 8 channels x 16 bytes
// per pixel, so that any 8 consecutive pixels of one channel group are one
// contiguous 128-byte block: ldmatrix reads them without bank conflicts and
// the tap shift (dy, dx) is only an address offset.  Fusions: the first layer
// converts the FP32 planar sparse frame on load; decoder layers compute the
// bilinear x2 up-sampling of the coarser level and the skip concatenation on
// load; the second conv of each encoder level also writes the 2x2 average
// pooled tensor of the next level from its accumulators.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_fp8.h>

#include "common.cuh"

namespace fvn {

// ---------------------------------------------------------------------------
// layer table (flat weight order of fvn_load_weights)
// ---------------------------------------------------------------------------
struct LayerSpec {
    int cin, cout, k;
};
static const LayerSpec kLayers[kNumLayers] = {
    {5, 16, 3},  {16, 16, 3}, {16, 32, 3}, {32, 32, 3}, {32, 64, 3}, {64, 64, 3},
    {96, 32, 3}, {32, 32, 3}, {48, 16, 3}, {16, 16, 3}, {16, 29, 1},
};
constexpr int kHeadC = 29;

// Layer li of the plain network, or of the recurrent one (paper:
// "Recurrence": the previous output enters the first layer as three more
// input channels).
static LayerSpec layer_spec(bool recurrent, int li) {
    LayerSpec s = kLayers[li];
    if (li == 0 && recurrent) s.cin = 8;
    return s;
}

static size_t weight_count(bool recurrent = false) {
    size_t n = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec l = layer_spec(recurrent, li);
        n += (size_t)l.cout * l.cin * l.k * l.k + l.cout;
    }
    return n;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                            uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_f16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint4 pack8(const float* v) {
    uint4 r;
    __half2 h0 = __floats2half2_rn(v[0], v[1]);
    __half2 h1 = __floats2half2_rn(v[2], v[3]);
    __half2 h2 = __floats2half2_rn(v[4], v[5]);
    __half2 h3 = __floats2half2_rn(v[6], v[7]);
    r.x = *reinterpret_cast<uint32_t*>(&h0);
    r.y = *reinterpret_cast<uint32_t*>(&h1);
    r.z = *reinterpret_cast<uint32_t*>(&h2);
    r.w = *reinterpret_cast<uint32_t*>(&h3);
    return r;
}

__device__ __forceinline__ void unpack8(uint4 u, float* v) {
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __half22float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// ---------------------------------------------------------------------------
// conv3x3 + bias + ReLU (+ fused 2x2 average pool), FP16 tensor cores
// ---------------------------------------------------------------------------
enum { IN_NHWC = 0, IN_RGBAM = 1, IN_UPCAT = 2 };

constexpr int TR = 4;            // output rows per tile
constexpr int TW = 64;           // output pixels per row per tile
constexpr int HY = TR + 2, HX = TW + 2;

struct ConvArgs {
    const __half* in;            // IN_NHWC: [Hl][Wl][CIN]; IN_UPCAT: coarse [Hl/2][Wl/2][CUP]
    const __half* skip;          // IN_UPCAT: [Hl][Wl][CIN - CUP]
    const float* rgbam;          // IN_RGBAM: [5][H0][W0] planar FP32
    const float* prev;           // IN_RGBAM, recurrent model: previous output [3][H0][W0] (NULL: zeros)
    int H0, W0;                  // IN_RGBAM: unpadded frame
    const __half* w;             // [9][CIN/8][COUT][8]
    const float* bias;           // [COUT]
    __half* out;                 // [Hl][Wl][COUT]
    __half* pooled;              // POOL: [Hl/2][Wl/2][COUT]
    int Hl, Wl;                  // this level's frame
    int tiles_x, ntiles;
};

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int CH = CIN / 8;
    static constexpr size_t w_bytes = (size_t)9 * CIN * COUT * 2;
    static constexpr size_t halo_bytes = (size_t)CH * HY * HX * 16;
    static constexpr size_t bytes = w_bytes + halo_bytes + COUT * 4;
};

template <int CIN, int COUT, int MODE, bool POOL, int CUP>
__global__ void __launch_bounds__(COUT == 64 ? 256 : 128) conv3x3_f16_kernel(ConvArgs a) {
    constexpr int CH = CIN / 8;
    constexpr int NW = COUT < 32 ? COUT : 32;       // output channels per warp
    constexpr int NT = NW / 8;                       // n-tiles per warp
    constexpr int WN = COUT / NW;                    // warps along N
    constexpr int NTHREADS = 4 * WN * 32;            // 2 row pairs x 2 pixel halves x WN
    static_assert(CIN % 16 == 0, "CIN must be a multiple of 16");
    extern __shared__ __align__(128) unsigned char smem[];
    __half* sW = reinterpret_cast<__half*>(smem);
    unsigned char* sH = smem + ConvSmem<CIN, COUT>::w_bytes;
    float* sB = reinterpret_cast<float*>(sH + ConvSmem<CIN, COUT>::halo_bytes);

    const int tid = threadIdx.x;
    {   // weights and bias stay resident for every tile of this CTA
        const uint4* src = reinterpret_cast<const uint4*>(a.w);
        uint4* dst = reinterpret_cast<uint4*>(sW);
        constexpr int n16 = (int)(ConvSmem<CIN, COUT>::w_bytes / 16);
        for (int i = tid; i < n16; i += NTHREADS) dst[i] = __ldg(src + i);
        for (int i = tid; i < COUT; i += NTHREADS) sB[i] = __ldg(a.bias + i);
    }
    const int warp = tid >> 5, lane = tid & 31;
    const int wn = warp % WN;                        // channel block
    const int wx = (warp / WN) & 1;                  // pixel half (32 px)
    const int wr = warp / (2 * WN);                  // row pair
    const int g = lane >> 2, t = lane & 3;
    const uint32_t sW_u = smem_u32(sW), sH_u = smem_u32(sH);

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
        const int y0 = ty * TR, x0 = tx * TW;
        __syncthreads();   // previous tile's reads of the halo are done
        // ---- stage the input halo -------------------------------------
        if (MODE == IN_RGBAM) {
            const long long plane = (long long)a.H0 * a.W0;
            for (int i = tid; i < HY * HX; i += NTHREADS) {
                const int hy = i / HX, hx = i - hy * HX;
                const int gy = y0 + hy - 1, gx = x0 + hx - 1;
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gy >= 0 && gx >= 0 && gy < a.H0 && gx < a.W0) {
                    const float* p = a.rgbam + (long long)gy * a.W0 + gx;
#pragma unroll
                    for (int c = 0; c < 5; ++c) v[c] = __ldg(p + c * plane);
                    if (a.prev) {   // the previous output, clamped to [0, 1], as channels 5..7
                        const float* q = a.prev + (long long)gy * a.W0 + gx;
#pragma unroll
                        for (int c = 0; c < 3; ++c) v[5 + c] = __saturatef(__ldg(q + c * plane));
                    }
                }
                uint4* d0 = reinterpret_cast<uint4*>(sH + ((0 * HY + hy) * HX + hx) * 16);
                *d0 = pack8(v);
#pragma unroll
                for (int c = 1; c < CH; ++c)
                    *reinterpret_cast<uint4*>(sH + ((c * HY + hy) * HX + hx) * 16) = make_uint4(0, 0, 0, 0);
            }
        } else {
            for (int i = tid; i < CH * HY * HX; i += NTHREADS) {
                const int c = i / (HY * HX);
                const int rem = i - c * (HY * HX);
                const int hy = rem / HX, hx = rem - hy * HX;
                const int gy = y0 + hy - 1, gx = x0 + hx - 1;
                unsigned char* dst = sH + ((c * HY + hy) * HX + hx) * 16;
                const bool inside = gy >= 0 && gx >= 0 && gy < a.Hl && gx < a.Wl;
                if (!inside) {
                    *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
                } else if (MODE == IN_NHWC) {
                    cp_async16(smem_u32(dst), a.in + ((long long)gy * a.Wl + gx) * CIN + c * 8);
                } else if (c >= CUP / 8) {   // skip connection channels
                    constexpr int CS = CIN - CUP;
                    cp_async16(smem_u32(dst), a.skip + ((long long)gy * a.Wl + gx) * CS + (c - CUP / 8) * 8);
                } else {                     // bilinear x2 up-sampling of the coarse level
                    const int Hc = a.Hl >> 1, Wc = a.Wl >> 1;
                    const float sy = fmaxf((gy + 0.5f) * 0.5f - 0.5f, 0.f);
                    const float sx = fmaxf((gx + 0.5f) * 0.5f - 0.5f, 0.f);
                    const int iy0 = (int)sy, ix0 = (int)sx;
                    const float fy = sy - iy0, fx = sx - ix0;
                    const int iy1 = min(iy0 + 1, Hc - 1), ix1 = min(ix0 + 1, Wc - 1);
                    const __half* base = a.in + c * 8;
                    float p00[8], p01[8], p10[8], p11[8], v[8];
                    unpack8(__ldg(reinterpret_cast<const uint4*>(base + ((long long)iy0 * Wc + ix0) * CUP)), p00);
                    unpack8(__ldg(reinterpret_cast<const uint4*>(base + ((long long)iy0 * Wc + ix1) * CUP)), p01);
                    unpack8(__ldg(reinterpret_cast<const uint4*>(base + ((long long)iy1 * Wc + ix0) * CUP)), p10);
                    unpack8(__ldg(reinterpret_cast<const uint4*>(base + ((long long)iy1 * Wc + ix1) * CUP)), p11);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float top = fmaf(fx, p01[j] - p00[j], p00[j]);
                        const float bot = fmaf(fx, p11[j] - p10[j], p10[j]);
                        v[j] = fmaf(fy, bot - top, top);
                    }
                    *reinterpret_cast<uint4*>(dst) = pack8(v);
                }
            }
            if (MODE != IN_RGBAM) cp_async_wait_all();
        }
        __syncthreads();

        // ---- implicit GEMM main loop ----------------------------------
        float acc[2][2][NT][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[rr][mt][nt][e] = 0.f;

        const int lj = lane >> 3, li = lane & 7;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
            for (int kc = 0; kc < CH / 2; ++kc) {
                uint32_t b[NT][2];
#pragma unroll
                for (int jj = 0; jj < NT / 2; ++jj) {
                    const int ntile = wn * NT + 2 * jj + (lj >> 1);
                    const int chunk = 2 * kc + (lj & 1);
                    const uint32_t addr = sW_u + (((tap * CH + chunk) * COUT + ntile * 8 + li) * 16);
                    ldmatrix_x4(addr, b[2 * jj][0], b[2 * jj][1], b[2 * jj + 1][0], b[2 * jj + 1][1]);
                }
                if (NT == 1) {   // 8-channel warp slice (COUT = 8 is not used; kept for completeness)
                }
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int hy = wr * 2 + rr + dy;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        const int px = wx * 32 + mt * 16 + (lj & 1) * 8 + li + dx;
                        const int chunk = 2 * kc + (lj >> 1);
                        uint32_t af[4];
                        ldmatrix_x4(sH_u + ((chunk * HY + hy) * HX + px) * 16, af[0], af[1], af[2], af[3]);
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) mma_f16(acc[rr][mt][nt], af, b[nt][0], b[nt][1]);
                    }
                }
            }
        }

        // ---- epilogue: bias, ReLU, FP16 store, fused 2x2 average pool --
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int ch = (wn * NT + nt) * 8 + 2 * t;
                const float b0 = sB[ch], b1 = sB[ch + 1];
                float v[2][2][2];   // [row][pixel g / g+8][channel pair]
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    v[rr][0][0] = fmaxf(acc[rr][mt][nt][0] + b0, 0.f);
                    v[rr][0][1] = fmaxf(acc[rr][mt][nt][1] + b1, 0.f);
                    v[rr][1][0] = fmaxf(acc[rr][mt][nt][2] + b0, 0.f);
                    v[rr][1][1] = fmaxf(acc[rr][mt][nt][3] + b1, 0.f);
                    const int y = y0 + wr * 2 + rr;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int x = x0 + wx * 32 + mt * 16 + hh * 8 + g;
                        if (y < a.Hl && x < a.Wl)
                            *reinterpret_cast<__half2*>(a.out + ((long long)y * a.Wl + x) * COUT + ch) =
                                __floats2half2_rn(v[rr][hh][0], v[rr][hh][1]);
                    }
                }
                if (POOL) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        float s0 = v[0][hh][0] + v[1][hh][0];
                        float s1 = v[0][hh][1] + v[1][hh][1];
                        s0 += __shfl_xor_sync(0xffffffffu, s0, 4);
                        s1 += __shfl_xor_sync(0xffffffffu, s1, 4);
                        const int y = y0 + wr * 2;
                        const int x = x0 + wx * 32 + mt * 16 + hh * 8 + g;
                        if ((g & 1) == 0 && y < a.Hl && x < a.Wl)
                            *reinterpret_cast<__half2*>(a.pooled +
                                                        ((long long)(y >> 1) * (a.Wl >> 1) + (x >> 1)) * COUT + ch) =
                                __floats2half2_rn(0.25f * s0, 0.25f * s1);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// head (1x1, 16 -> 29) + softmax 5x5 kernel prediction on the sparse samples
// + sigmoid blend, FP32 (paper: "Kernel Prediction")
// ---------------------------------------------------------------------------
constexpr int KP_BX = 32, KP_BY = 8, KP_R = 2;
constexpr int KP_HX = KP_BX + 2 * KP_R, KP_HY = KP_BY + 2 * KP_R;

__global__ void __launch_bounds__(KP_BX* KP_BY) head_kp_kernel(const __half* __restrict__ feat, int W4,
                                                               const float* __restrict__ headw,
                                                               const float* __restrict__ rgbam, int H, int W,
                                                               float* __restrict__ rgb) {
    __shared__ float sw[kHeadC * 16 + kHeadC];
    __shared__ float4 sn[KP_HY][KP_HX];     // sparse R, G, B, M of the window
    const int tid = threadIdx.y * KP_BX + threadIdx.x;
    for (int i = tid; i < kHeadC * 17; i += KP_BX * KP_BY) sw[i] = __ldg(headw + i);
    const int bx0 = blockIdx.x * KP_BX, by0 = blockIdx.y * KP_BY;
    const long long plane = (long long)H * W;
    for (int i = tid; i < KP_HY * KP_HX; i += KP_BX * KP_BY) {
        const int hy = i / KP_HX, hx = i - hy * KP_HX;
        const int gy = by0 + hy - KP_R, gx = bx0 + hx - KP_R;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gy >= 0 && gx >= 0 && gy < H && gx < W) {
            const float* p = rgbam + (long long)gy * W + gx;
            v = make_float4(__ldg(p), __ldg(p + plane), __ldg(p + 2 * plane), __ldg(p + 4 * plane));
        }
        sn[hy][hx] = v;
    }
    __syncthreads();
    const int x = bx0 + threadIdx.x, y = by0 + threadIdx.y;
    if (x >= W || y >= H) return;
    float f[16];
    const uint4* fp = reinterpret_cast<const uint4*>(feat + ((long long)y * W4 + x) * 16);
    unpack8(__ldg(fp), f);
    unpack8(__ldg(fp + 1), f + 8);
    float hd[kHeadC];
#pragma unroll
    for (int j = 0; j < kHeadC; ++j) {
        float s = sw[kHeadC * 16 + j];
#pragma unroll
        for (int c = 0; c < 16; ++c) s = fmaf(sw[j * 16 + c], f[c], s);
        hd[j] = s;
    }
    float mx = hd[3];
#pragma unroll
    for (int q = 1; q < 25; ++q) mx = fmaxf(mx, hd[3 + q]);
    float e[25], esum = 0.f;
#pragma unroll
    for (int q = 0; q < 25; ++q) {
        e[q] = expf(hd[3 + q] - mx);
        esum += e[q];
    }
    const float inv = 1.0f / esum;
    float den = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
    for (int q = 0; q < 25; ++q) {
        const float4 s = sn[threadIdx.y + q / 5][threadIdx.x + q % 5];
        const float wm = e[q] * inv * s.w;
        den += wm;
        n0 = fmaf(wm, s.x, n0);
        n1 = fmaf(wm, s.y, n1);
        n2 = fmaf(wm, s.z, n2);
    }
    float k0 = hd[0], k1 = hd[1], k2 = hd[2];
    if (den >= 1e-12f) {
        k0 = n0 / den;
        k1 = n1 / den;
        k2 = n2 / den;
    }
    const float al = 1.0f / (1.0f + expf(-hd[28]));
    float* o = rgb + (long long)y * W + x;
    o[0] = fmaf(al, k0 - hd[0], hd[0]);
    o[plane] = fmaf(al, k1 - hd[1], hd[1]);
    o[2 * plane] = fmaf(al, k2 - hd[2], hd[2]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int MODE, bool POOL, int CUP>
static fvn_status launch_conv(fvn_ctx* ctx, ConvArgs a, cudaStream_t st) {
    auto kern = conv3x3_f16_kernel<CIN, COUT, MODE, POOL, CUP>;
    constexpr size_t smem = ConvSmem<CIN, COUT>::bytes;
    constexpr int nthreads = 4 * (COUT / (COUT < 32 ? COUT : 32)) * 32;
    static bool configured = false;
    if (!configured) {
        FVN_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    int per_sm = 0;
    FVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem));
    if (per_sm < 1) return set_error(ctx, FVN_ERR_CUDA, "conv kernel does not fit on an SM");
    a.tiles_x = (a.Wl + TW - 1) / TW;
    a.ntiles = a.tiles_x * ((a.Hl + TR - 1) / TR);
    const int grid = std::min(a.ntiles, ctx->num_sms * per_sm);
    kern<<<grid, nthreads, smem, st>>>(a);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

// separate_up: give the up-sampled decoder inputs buffers of their own
// (FP8 calibration reads every activation after the pass).
static size_t plan_buffers(int W4, int H4, ReconPlan* b, char* base, bool separate_up = false) {
    const size_t n0 = (size_t)W4 * H4, n1 = n0 / 4, n2 = n0 / 16;
    const size_t sizes[12] = {n0 * 16, n0 * 16, n1 * 16, n1 * 32, n1 * 32, n2 * 32,
                              n2 * 64, n2 * 64, n1 * 32, n1 * 32, n0 * 16, n0 * 16};
    __half** ptrs[12] = {&b->e0a, &b->e0, &b->p0, &b->e1a, &b->e1, &b->p1,
                         &b->ba,  &b->bt, &b->d1a, &b->d1, &b->d0a, &b->d0};
    size_t off = 0;
    for (int i = 0; i < 12; ++i) {
        if (base) *ptrs[i] = reinterpret_cast<__half*>(base + off);
        off += (sizes[i] * sizeof(__half) + 255) & ~(size_t)255;
    }
    // up-sampled decoder inputs on dead buffers: u1 (n1 x 64) on e0a (n0 x 16,
    // dead after the second layer); u0 (n0 x 32) from p0 on, over p0, e1a,
    // e1, p1, ba, bt, d1a (n0 x 38 in total, all dead once d1 is written)
    if (separate_up) {
        if (base) {
            b->u1 = reinterpret_cast<__half*>(base + off);
            b->u0 = reinterpret_cast<__half*>(base + off + ((n1 * 64 * sizeof(__half) + 255) & ~(size_t)255));
        }
        return off + ((n1 * 64 * sizeof(__half) + 255) & ~(size_t)255) + ((n0 * 32 * sizeof(__half) + 255) & ~(size_t)255);
    }
    if (base) {
        b->u1 = b->e0a;
        b->u0 = b->p0;
    }
    return off;
}

size_t recon_workspace_bytes(int w, int h) {
    return plan_buffers((w + 3) & ~3, (h + 3) & ~3, nullptr, nullptr);
}

size_t plan_view(int w, int h, ReconPlan* plan, char* base) {
    ReconPlan tmp;
    return plan_buffers((w + 3) & ~3, (h + 3) & ~3, plan ? plan : &tmp, base);
}

fvn_status reconstruct_impl(fvn_ctx* ctx, const float* rgbam, const float* prev, int w, int h, int precision,
                            float* rgb, cudaStream_t st) {
    if (precision == FVN_PREC_FP8 && !ctx->has_fp8)
        return set_error(ctx, FVN_ERR_STATE, "FP8 needs calibrated scales (call fvn_calibrate_fp8 first)");
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    ReconWorkspace& ws = ctx->recon_ws;
    if (ws.w != W4 || ws.h != H4) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(ws.base);
        ws = ReconWorkspace();
        size_t bytes = plan_buffers(W4, H4, nullptr, nullptr);
        FVN_CUDA(ctx, cudaMalloc(&ws.base, bytes));
        ws.bytes = bytes;
        ws.w = W4;
        ws.h = H4;
    }
    return reconstruct_on(ctx, ws.base, rgbam, prev, w, h, precision, rgb, st);
}

fvn_status reconstruct_on(fvn_ctx* ctx, void* workspace, const float* rgbam, const float* prev, int w, int h,
                          int precision, float* rgb, cudaStream_t st) {
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    ReconPlan B;
    plan_buffers(W4, H4, &B, static_cast<char*>(workspace));
    if (precision == FVN_PREC_FP8) {
        if (!ctx->has_fp8)
            return set_error(ctx, FVN_ERR_STATE, "FP8 needs calibrated scales (call fvn_calibrate_fp8 first)");
        return reconstruct_tc_fp8(ctx, B, rgbam, prev, w, h, rgb, st);
    }
    if (ctx->conv_impl == CONV_TCGEN05) return reconstruct_tc(ctx, B, rgbam, prev, w, h, rgb, st);
    const ConvW* L = ctx->layers;
    fvn_status s;
    ConvArgs a{};
    // level 0: enc0a (sparse frame -> 16), enc0b (16 -> 16, + pool)
    a = ConvArgs{};
    a.rgbam = rgbam; a.prev = prev; a.H0 = h; a.W0 = w; a.w = L[0].w16; a.bias = L[0].bias; a.out = B.e0a;
    a.Hl = H4; a.Wl = W4;
    if ((s = launch_conv<16, 16, IN_RGBAM, false, 0>(ctx, a, st)) != FVN_OK) return s;
    a = ConvArgs{};
    a.in = B.e0a; a.w = L[1].w16; a.bias = L[1].bias; a.out = B.e0; a.pooled = B.p0; a.Hl = H4; a.Wl = W4;
    if ((s = launch_conv<16, 16, IN_NHWC, true, 0>(ctx, a, st)) != FVN_OK) return s;
    // level 1: enc1a, enc1b (+ pool)
    a = ConvArgs{};
    a.in = B.p0; a.w = L[2].w16; a.bias = L[2].bias; a.out = B.e1a; a.Hl = H4 / 2; a.Wl = W4 / 2;
    if ((s = launch_conv<16, 32, IN_NHWC, false, 0>(ctx, a, st)) != FVN_OK) return s;
    a = ConvArgs{};
    a.in = B.e1a; a.w = L[3].w16; a.bias = L[3].bias; a.out = B.e1; a.pooled = B.p1; a.Hl = H4 / 2; a.Wl = W4 / 2;
    if ((s = launch_conv<32, 32, IN_NHWC, true, 0>(ctx, a, st)) != FVN_OK) return s;
    // level 2: bottleneck
    a = ConvArgs{};
    a.in = B.p1; a.w = L[4].w16; a.bias = L[4].bias; a.out = B.ba; a.Hl = H4 / 4; a.Wl = W4 / 4;
    if ((s = launch_conv<32, 64, IN_NHWC, false, 0>(ctx, a, st)) != FVN_OK) return s;
    a = ConvArgs{};
    a.in = B.ba; a.w = L[5].w16; a.bias = L[5].bias; a.out = B.bt; a.Hl = H4 / 4; a.Wl = W4 / 4;
    if ((s = launch_conv<64, 64, IN_NHWC, false, 0>(ctx, a, st)) != FVN_OK) return s;
    // level 1 decoder: up(bt) ++ e1 -> dec1a, dec1b
    a = ConvArgs{};
    a.in = B.bt; a.skip = B.e1; a.w = L[6].w16; a.bias = L[6].bias; a.out = B.d1a; a.Hl = H4 / 2; a.Wl = W4 / 2;
    if ((s = launch_conv<96, 32, IN_UPCAT, false, 64>(ctx, a, st)) != FVN_OK) return s;
    a = ConvArgs{};
    a.in = B.d1a; a.w = L[7].w16; a.bias = L[7].bias; a.out = B.d1; a.Hl = H4 / 2; a.Wl = W4 / 2;
    if ((s = launch_conv<32, 32, IN_NHWC, false, 0>(ctx, a, st)) != FVN_OK) return s;
    // level 0 decoder: up(d1) ++ e0 -> dec0a, dec0b
    a = ConvArgs{};
    a.in = B.d1; a.skip = B.e0; a.w = L[8].w16; a.bias = L[8].bias; a.out = B.d0a; a.Hl = H4; a.Wl = W4;
    if ((s = launch_conv<48, 16, IN_UPCAT, false, 32>(ctx, a, st)) != FVN_OK) return s;
    a = ConvArgs{};
    a.in = B.d0a; a.w = L[9].w16; a.bias = L[9].bias; a.out = B.d0; a.Hl = H4; a.Wl = W4;
    if ((s = launch_conv<16, 16, IN_NHWC, false, 0>(ctx, a, st)) != FVN_OK) return s;
    // head + kernel prediction + blend
    dim3 grid((w + KP_BX - 1) / KP_BX, (h + KP_BY - 1) / KP_BY);
    head_kp_kernel<<<grid, dim3(KP_BX, KP_BY), 0, st>>>(B.d0, W4, ctx->head_w, rgbam, h, w, rgb);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

}  // namespace fvn

using namespace fvn;

extern "C" size_t fvn_weight_count(void) { return weight_count(false); }

extern "C" size_t fvn_weight_count_recurrent(void) { return weight_count(true); }

extern "C" fvn_status fvn_load_weights(fvn_ctx* ctx, const float* host_w, size_t n) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, host_w != nullptr, "weights pointer is NULL");
    FVN_CHECK_ARG(ctx, n == weight_count(false) || n == weight_count(true),
                  "weight vector has %zu entries, expected %zu (or %zu for the recurrent network)", n,
                  weight_count(false), weight_count(true));
    const bool recurrent = n == weight_count(true);
    for (size_t i = 0; i < n; ++i)
        FVN_CHECK_ARG(ctx, isfinite(host_w[i]), "weight %zu is not finite", i);
    FVN_CUDA(ctx, cudaDeviceSynchronize());
    ctx->host_weights.assign(host_w, host_w + n);
    ctx->has_fp8 = false;   // FP8 weights follow the FP32 weights: calibrate again
    ctx->has_weights = false;
    size_t off = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec sp = layer_spec(recurrent, li);
        const float* W = host_w + off;
        const float* b = W + (size_t)sp.cout * sp.cin * sp.k * sp.k;
        off += (size_t)sp.cout * sp.cin * sp.k * sp.k + sp.cout;
        ConvW& L = ctx->layers[li];
        L.cin = sp.cin;
        L.cout = sp.cout;
        L.k = sp.k;
        if (sp.k == 1) {   // head: FP32 [29][16] then bias [29]
            std::vector<float> hw((size_t)kHeadC * 17);
            for (int o = 0; o < kHeadC; ++o)
                for (int c = 0; c < 16; ++c) hw[o * 16 + c] = W[o * sp.cin + c];
            for (int o = 0; o < kHeadC; ++o) hw[kHeadC * 16 + o] = b[o];
            if (!ctx->head_w) FVN_CUDA(ctx, cudaMalloc(&ctx->head_w, hw.size() * sizeof(float)));
            FVN_CUDA(ctx, cudaMemcpy(ctx->head_w, hw.data(), hw.size() * sizeof(float), cudaMemcpyHostToDevice));
            // tensor-core operand: [k chunk 2][n 32][8], output rows 29..31 zero
            std::vector<__half> h16(2 * 32 * 8, __float2half(0.f));
            std::vector<float> hb(32, 0.f);
            for (int o = 0; o < kHeadC; ++o) {
                for (int c = 0; c < 16; ++c) h16[((c / 8) * 32 + o) * 8 + (c % 8)] = __float2half(W[o * sp.cin + c]);
                hb[o] = b[o];
            }
            if (!ctx->head_w16) FVN_CUDA(ctx, cudaMalloc(&ctx->head_w16, h16.size() * sizeof(__half)));
            if (!ctx->head_b32) FVN_CUDA(ctx, cudaMalloc(&ctx->head_b32, hb.size() * sizeof(float)));
            FVN_CUDA(ctx, cudaMemcpy(ctx->head_w16, h16.data(), h16.size() * sizeof(__half), cudaMemcpyHostToDevice));
            FVN_CUDA(ctx, cudaMemcpy(ctx->head_b32, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice));
            continue;
        }
        const int cp = (sp.cin + 15) & ~15;
        L.cin_pad = cp;
        const int chunks = cp / 8;
        std::vector<__half> w16((size_t)9 * cp * sp.cout, __float2half(0.f));
        for (int o = 0; o < sp.cout; ++o)
            for (int c = 0; c < sp.cin; ++c)
                for (int tap = 0; tap < 9; ++tap) {
                    const float v = W[((size_t)o * sp.cin + c) * 9 + tap];
                    w16[(((size_t)tap * chunks + c / 8) * sp.cout + o) * 8 + (c % 8)] = __float2half(v);
                }
        if (!L.w16) FVN_CUDA(ctx, cudaMalloc(&L.w16, w16.size() * sizeof(__half)));
        if (!L.bias) FVN_CUDA(ctx, cudaMalloc(&L.bias, sp.cout * sizeof(float)));
        FVN_CUDA(ctx, cudaMemcpy(L.w16, w16.data(), w16.size() * sizeof(__half), cudaMemcpyHostToDevice));
        FVN_CUDA(ctx, cudaMemcpy(L.bias, b, sp.cout * sizeof(float), cudaMemcpyHostToDevice));
    }
    ctx->recurrent = recurrent;
    ctx->has_weights = true;
    return FVN_OK;
}

static fvn_status reconstruct_entry(fvn_ctx* ctx, const float* rgbam, const float* prev, int w, int h,
                                    int precision, float* rgb, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam && rgb, "rgbam and rgb must be device pointers");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    FVN_CHECK_ARG(ctx, precision == FVN_PREC_FP16 || precision == FVN_PREC_FP8, "unknown precision %d", precision);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    if (prev && !ctx->recurrent)
        return set_error(ctx, FVN_ERR_STATE, "a previous frame needs the recurrent network's weights");
    return reconstruct_impl(ctx, rgbam, prev, w, h, precision, rgb, as_stream(stream));
}

extern "C" fvn_status fvn_reconstruct(fvn_ctx* ctx, const float* rgbam, int w, int h, int precision, float* rgb,
                                      void* stream) {
    return reconstruct_entry(ctx, rgbam, nullptr, w, h, precision, rgb, stream);
}

extern "C" fvn_status fvn_reconstruct_recurrent(fvn_ctx* ctx, const float* rgbam, const float* prev_rgb, int w,
                                                int h, int precision, float* rgb, void* stream) {
    return reconstruct_entry(ctx, rgbam, prev_rgb, w, h, precision, rgb, stream);
}

namespace fvn {

// Input tensor of every input channel of a layer, and the layer's output /
// pooled tensor (FP8 scales; see conv_tc.cu).
static void fp8_tensors(int layer, int c, int* in_t) {
    static const int single[kNumLayers] = {FP8_RGBAM, FP8_E0A, FP8_P0, FP8_E1A, FP8_P1, FP8_BA,
                                           -1,        FP8_D1A, -1,     FP8_D0A, -1};
    if (layer == 6) *in_t = c < 64 ? FP8_BT : FP8_E1;          // [up(bt), e1]
    else if (layer == 8) *in_t = c < 32 ? FP8_D1 : FP8_E0;     // [up(d1), e0]
    else *in_t = single[layer];
}

// Quantise every 3x3 layer to E4M3 with the activation scales folded in:
// w' = w s_in(c); s_w[o] = max |w'| / 448; q = e4m3(w' / s_w[o]).  Layout
// [tap][cin_pad / 16][cout][16 bytes] (cin padded to a multiple of 32).
static fvn_status build_fp8_weights(fvn_ctx* ctx) {
    const float* hw = ctx->host_weights.data();
    float s[FP8_NT];
    for (int t = 0; t < FP8_NT; ++t) {
        const float amax = t == FP8_RGBAM ? 1.0f : ctx->fp8_amax[t];
        s[t] = amax > 0.f ? amax / 448.0f : 1.0f;
        ctx->fp8_inv_scale[t] = 1.0f / s[t];
    }
    size_t off = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec sp = layer_spec(ctx->recurrent, li);
        const float* W = hw + off;
        off += (size_t)sp.cout * sp.cin * sp.k * sp.k + sp.cout;
        if (sp.k != 3) continue;
        const int cp = (sp.cin + 31) & ~31;
        std::vector<float> wf((size_t)sp.cout * sp.cin * 9);
        std::vector<float> sw(sp.cout, 1.0f);
        for (int o = 0; o < sp.cout; ++o) {
            float m = 0.f;
            for (int c = 0; c < sp.cin; ++c) {
                int t;
                fp8_tensors(li, c, &t);
                for (int tap = 0; tap < 9; ++tap) {
                    const size_t i = ((size_t)o * sp.cin + c) * 9 + tap;
                    wf[i] = W[i] * s[t];
                    m = std::max(m, std::fabs(wf[i]));
                }
            }
            sw[o] = m > 0.f ? m / 448.0f : 1.0f;
        }
        std::vector<uint8_t> q((size_t)9 * cp * sp.cout, 0);
        for (int o = 0; o < sp.cout; ++o)
            for (int c = 0; c < sp.cin; ++c)
                for (int tap = 0; tap < 9; ++tap) {
                    const float v = wf[((size_t)o * sp.cin + c) * 9 + tap] / sw[o];
                    q[(((size_t)tap * (cp / 16) + c / 16) * sp.cout + o) * 16 + (c % 16)] =
                        (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
                }
        ConvW& L = ctx->layers[li];
        if (!L.w8) FVN_CUDA(ctx, cudaMalloc(&L.w8, q.size()));
        if (!L.scale8) FVN_CUDA(ctx, cudaMalloc(&L.scale8, sp.cout * sizeof(float)));
        FVN_CUDA(ctx, cudaMemcpy(L.w8, q.data(), q.size(), cudaMemcpyHostToDevice));
        FVN_CUDA(ctx, cudaMemcpy(L.scale8, sw.data(), sp.cout * sizeof(float), cudaMemcpyHostToDevice));
    }
    ctx->has_fp8 = true;
    return FVN_OK;
}

}  // namespace fvn

extern "C" fvn_status fvn_calibrate_fp8(fvn_ctx* ctx, const float* rgbam, int w, int h, int reset, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam != nullptr, "rgbam must be a device pointer");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    cudaStream_t st = as_stream(stream);
    // run the FP16 tensor-core network on this frame into a workspace where
    // no activation is overwritten, then reduce every activation's amax
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    float* out = nullptr;
    char* wsp = nullptr;
    FVN_CUDA(ctx, cudaMalloc(&out, sizeof(float) * 3 * (size_t)w * h));
    if (cudaMalloc(&wsp, plan_buffers(W4, H4, nullptr, nullptr, true)) != cudaSuccess) {
        cudaFree(out);
        return set_error(ctx, FVN_ERR_OOM, "no memory for the calibration workspace");
    }
    ReconView v;
    plan_buffers(W4, H4, &v.plan, wsp, true);
    v.rgbam = rgbam;
    v.w = w;
    v.h = h;
    v.rgb = out;
    fvn_status s = reconstruct_tc_views(ctx, &v, 1, FVN_PREC_FP16, st);
    if (s == FVN_OK && !ctx->d_amax && cudaMalloc(&ctx->d_amax, FP8_NT * sizeof(float)) != cudaSuccess)
        s = set_error(ctx, FVN_ERR_OOM, "no memory for the amax accumulators");
    if (s == FVN_OK && cudaMemsetAsync(ctx->d_amax, 0, FP8_NT * sizeof(float), st) != cudaSuccess)
        s = set_error(ctx, FVN_ERR_CUDA, "cudaMemsetAsync failed");
    if (s == FVN_OK) s = calibrate_amax(ctx, v.plan, w, h, ctx->d_amax, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaFree(out);
    cudaFree(wsp);
    if (s != FVN_OK) return s;
    if (se != cudaSuccess) return set_error(ctx, FVN_ERR_CUDA, "calibration pass failed: %s", cudaGetErrorString(se));
    float amax[FP8_NT];
    FVN_CUDA(ctx, cudaMemcpy(amax, ctx->d_amax, sizeof amax, cudaMemcpyDeviceToHost));
    for (int t = 0; t < FP8_NT; ++t) ctx->fp8_amax[t] = reset ? amax[t] : std::max(ctx->fp8_amax[t], amax[t]);
    return build_fp8_weights(ctx);
}
