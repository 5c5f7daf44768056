// Tensor-core convolutions of the training step (paper: "Training" and
// "Model Precision & Optimization": the network is trained with FP32 master
// weights; here its 3x3 layers' forward pass, data gradient and weight
// gradient run as GEMMs on the 5th-generation tensor cores).
//
// The training pass keeps FP32 NCHW tensors ([N][C][H][W]).  A CTA stages a
// tile's input halo (TR + 2 rows x 130 pixels) into shared memory as BF16
// chunk planes (8 channels = 16 bytes per pixel: the K-major core-matrix
// layout, so a tap is only a descriptor start address), rounding the FP32
// values to BF16 on the way -- BF16 keeps FP32's exponent range, so the
// data gradients need no loss scaling -- and issues, per output row, one
// tcgen05.mma (kind::f16 with BF16 operands, M = 128 pixels, N = output
// channels, K = 16) per tap and channel pair into an FP32 TMEM accumulator.
// The weights are read from the FP32 master copy and converted in the
// prologue: as they are for the forward pass, transposed (input <-> output
// channel) and flipped (tap 8 - t) for the data gradient, which is the
// convolution of the output gradient with them.  The data gradient's input
// is the output gradient times the layer's ReLU mask (saved output > 0),
// applied while staging.  Epilogue: bias and ReLU (forward), FP32 stores of
// one pixel per thread, channel by channel (coalesced along x); the data
// gradient's channels go to the two tensors of a concatenated input.  The
// CTAs are persistent, as many per SM as registers and shared memory allow;
// an instance double-buffers its halo (staging the next tile while the MMAs
// run) only where that costs no CTAs per SM.
//
// The weight gradient is a GEMM over the pixels (see conv3x3_wgrad_kernel).
//
// Every mbarrier wait has an iteration limit; a wait that gives up sets the
// error flag the caller passed and the CTA leaves its loop.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace fvn {
namespace ttc {

constexpr int TW = 128;                 // output pixels per tile row = MMA M
constexpr int HXW = TW + 2;             // halo pixels per row
constexpr int kThreads = 256;
constexpr uint32_t kLimit = 1u << 26;
constexpr size_t kSmemSM = 233472;      // shared memory of an SM (228 KB)

struct Args {
    const float* src0;                  // input channels [0, c0): [N][c0][H][W]
    const float* src1;                  // input channels [c0, cin): [N][cin - c0][H][W] (NULL when cin == c0)
    const float* mask;                  // data gradient: src0 is used where mask > 0 (same layout), else NULL
    int c0, cin, cout;
    const float* w;                     // the layer's FP32 weights [cout_layer][cin_layer][3][3]
    const float* bias;                  // forward: [cout] (NULL: none)
    int dgrad;                          // 1: weights transposed and flipped (data gradient)
    int relu;
    float* out0;                        // output channels [0, o0): [N][o0][H][W] (NULL: not written)
    float* out1;                        // output channels [o0, cout): [N][cout - o0][H][W] (NULL: not written)
    int o0;
    int n, H, W;
    int tiles_x, tiles_img, ntiles;
    int* error;
};

// Shared-memory layout of an instance: CINP input channels (multiple of 16),
// COUTP output channels (multiple of 16), TR output rows per tile.
template <int CINP, int COUTP, int TR>
struct Layout {
    static constexpr int CH = CINP / 8;                                    // chunk planes
    static constexpr int HY = TR + 2;
    static constexpr size_t w_bytes = 9ull * CINP * COUTP * 2;             // [tap][CH][COUTP][8] BF16
    static constexpr size_t halo = (size_t)CH * HY * HXW * 16 + 32;        // one halo buffer (+ MMA over-read)
    static constexpr size_t halo_r = (halo + 127) / 128 * 128;
    static constexpr size_t w_off = 0;
    static constexpr size_t halo_off = (w_bytes + 1023) / 1024 * 1024;
    // two halo buffers (staging overlaps the MMAs) unless that costs CTAs per
    // SM (several CTAs also overlap one another's staging; registers cap an
    // SM at 3 of them)
    static constexpr size_t bytes1 = halo_off + 1 * halo_r + COUTP * 4 + 16;
    static constexpr size_t bytes2 = halo_off + 2 * halo_r + COUTP * 4 + 16;
    static constexpr int ctas1 = (int)(kSmemSM / (bytes1 + 1024)), ctas2 = (int)(kSmemSM / (bytes2 + 1024));
    static constexpr int NBUF = bytes2 <= 220 * 1024 && ctas2 >= (ctas1 < 3 ? ctas1 : 3) ? 2 : 1;
    static constexpr int ctas = NBUF == 2 ? ctas2 : ctas1;                 // CTAs one SM holds by shared memory
    static constexpr int min_blocks = ctas >= 3 ? 3 : ctas >= 2 ? 2 : 1;   // the register budget follows
    static constexpr size_t bias_off = halo_off + NBUF * halo_r;
    static constexpr size_t bar_off = bias_off + COUTP * 4;
    static constexpr size_t bytes = bar_off + 16;
    static constexpr uint32_t acc_cols = TR * COUTP;
    static constexpr uint32_t tmem_cols = acc_cols <= 32 ? 32 : acc_cols <= 64 ? 64 : acc_cols <= 128 ? 128
                                        : acc_cols <= 256 ? 256 : 512;
    static_assert(acc_cols <= 512, "accumulators exceed the TMEM");
    static_assert(COUTP % 16 == 0 && COUTP <= 256 && CINP % 16 == 0, "unsupported shape");
    static_assert(bytes <= 227 * 1024, "shared memory");
};

// BF16 instruction descriptor of kind::f16: FP32 accumulator, A and B BF16,
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint4 pack8bf(const float* v) {
    uint4 r;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
    r.x = *reinterpret_cast<uint32_t*>(&h0);
    r.y = *reinterpret_cast<uint32_t*>(&h1);
    r.z = *reinterpret_cast<uint32_t*>(&h2);
    r.w = *reinterpret_cast<uint32_t*>(&h3);
    return r;
}

template <int CINP, int COUTP, int TR>
__global__ void __launch_bounds__(kThreads, (Layout<CINP, COUTP, TR>::min_blocks))
    conv3x3_train_kernel(const __grid_constant__ Args a) {
    using L = Layout<CINP, COUTP, TR>;
    constexpr int CH = L::CH, HY = L::HY;
    static_assert(TR % 2 == 0, "the two warp groups of the epilogue split the rows");
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sBias = reinterpret_cast<float*>(smem + L::bias_off);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::bar_off + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {   // this GEMM's weights as BF16 chunks [tap][CH][COUTP][8], zero beyond cin / cout: one
        // 16-byte chunk per item, its 8 input channels gathered by independent loads
        for (int i = tid; i < COUTP; i += kThreads) sBias[i] = (a.bias && i < a.cout) ? __ldg(a.bias + i) : 0.f;
        uint4* wz = reinterpret_cast<uint4*>(smem + L::w_off);
        constexpr int items = 9 * CH * COUTP;
#pragma unroll 4
        for (int i = tid; i < items; i += kThreads) {
            const int co = i % COUTP, t = i / COUTP, ch = t % CH, tap = t / CH;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ci = ch * 8 + j;
                const bool ok = ci < a.cin && co < a.cout;
                // forward: the layer is [cout][cin][tap]; data gradient: [cin][cout][8 - tap]
                const size_t off = a.dgrad ? ((size_t)min(ci, a.cin - 1) * a.cout + min(co, a.cout - 1)) * 9 + (8 - tap)
                                           : ((size_t)min(co, a.cout - 1) * a.cin + min(ci, a.cin - 1)) * 9 + tap;
                const float w = __ldg(a.w + off);
                v[j] = ok ? w : 0.f;
            }
            wz[i] = pack8bf(v);
        }
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, L::tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t sW_u = tc::smem_addr(smem + L::w_off), sH_u = tc::smem_addr(smem + L::halo_off);
    constexpr uint32_t idesc = idesc_bf16(128, COUTP);
    const size_t plane = (size_t)a.H * a.W;

    // the input halo of a tile as BF16 chunk planes [CH][HY][HXW][8], one
    // 16-byte chunk (8 channels of a pixel) per item, consecutive items along x
    auto stage = [&](int tile, int buf) {
        const int img = tile / a.tiles_img, lt = tile - img * a.tiles_img;
        const int ty = lt / a.tiles_x, tx = lt - ty * a.tiles_x;
        const int y0 = ty * TR, x0 = tx * TW;
        const float* s0 = a.src0 + (size_t)img * a.c0 * plane;
        const float* s1 = a.src1 ? a.src1 + (size_t)img * (a.cin - a.c0) * plane : nullptr;
        const float* mk = a.mask ? a.mask + (size_t)img * a.c0 * plane : nullptr;
        unsigned char* sH = smem + L::halo_off + (size_t)buf * L::halo_r;
        // chunks never straddle the two sources nor run past cin: one base
        // pointer per chunk, one add per channel
        const bool aligned = a.c0 % 8 == 0 && a.cin % 8 == 0;
        for (int i = tid; i < HY * HXW; i += kThreads) {   // one halo pixel, all its chunks
            const int hy = i / HXW, hx = i - hy * HXW;
            const int gy = y0 + hy - 1, gx = x0 + hx - 1;
            // every load issued without a branch (addresses clamped into the
            // tensors, the values outside the frame / channels zeroed after)
            const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
            const size_t p = (size_t)min(max(gy, 0), a.H - 1) * a.W + min(max(gx, 0), a.W - 1);
            unsigned char* dst = sH + (size_t)i * 16;
#pragma unroll 4
            for (int ch = 0; ch < CH; ++ch) {
                float v[8], m[8];
                if (aligned) {
                    const int c = min(ch * 8, a.cin - 8);
                    const float* src = (c < a.c0 ? s0 + (size_t)c * plane : s1 + (size_t)(c - a.c0) * plane) + p;
                    const float* ms = mk ? mk + (size_t)min(c, a.c0 - 8) * plane + p : nullptr;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v[j] = __ldg(src + (size_t)j * plane);
                        m[j] = ms ? __ldg(ms + (size_t)j * plane) : 1.f;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int c = min(ch * 8 + j, a.cin - 1);
                        const float* src = c < a.c0 ? s0 + (size_t)c * plane : s1 + (size_t)(c - a.c0) * plane;
                        v[j] = __ldg(src + p);
                        m[j] = mk ? __ldg(mk + (size_t)min(ch * 8 + j, a.c0 - 1) * plane + p) : 1.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = (in && ch * 8 + j < a.cin && m[j] > 0.f) ? v[j] : 0.f;
                *reinterpret_cast<uint4*>(dst + (size_t)ch * HY * HXW * 16) = pack8bf(v);
            }
        }
    };

    uint32_t phase = 0;
    bool failed = false;
    int buf = 0;
    int tile = blockIdx.x;
    if (tile < a.ntiles) {
        stage(tile, 0);
        tc::fence_async_smem();
        __syncthreads();
    }
    for (; tile < a.ntiles; tile += gridDim.x) {
        const int img = tile / a.tiles_img, lt = tile - img * a.tiles_img;
        const int ty = lt / a.tiles_x, tx = lt - ty * a.tiles_x;
        const int y0 = ty * TR, x0 = tx * TW;
        const int next = tile + gridDim.x;
        if (tid == 0) {   // one thread issues every MMA of the tile
            tc::fence_after_sync();
            const uint64_t a0 = tc::smem_desc(sH_u + (uint32_t)(buf * L::halo_r), HY * HXW * 16, 128);
            const uint64_t b0 = tc::smem_desc(sW_u, COUTP * 16, 128);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                for (int kc = 0; kc < CH / 2; ++kc) {
                    const uint64_t bd = b0 + (uint64_t)((tap * CH + 2 * kc) * COUTP);
#pragma unroll
                    for (int r = 0; r < TR; ++r) {
                        const uint64_t ad = a0 + (uint64_t)(((2 * kc) * HY + r + dy) * HXW + dx);
                        tc::mma_f16(tmem + (uint32_t)(r * COUTP), ad, bd, idesc, (tap | kc) != 0);
                    }
                }
            }
            tc::mma_commit(bar);
        }
        if (L::NBUF == 2 && next < a.ntiles) stage(next, buf ^ 1);   // overlaps the MMAs
        if (!tc::mbar_wait(bar, phase, kLimit)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // ---- epilogue: one pixel per thread; warp group warp / 4 takes half the rows
        const int q = warp & 3, px = q * 32 + lane, x = x0 + px;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        constexpr int RG = TR / 2;
        const int r_lo = (warp >> 2) * RG;
#pragma unroll 1
        for (int r = r_lo; r < r_lo + RG; ++r) {
            const int y = y0 + r;
            const bool inside = y < a.H && x < a.W;
#pragma unroll 1
            for (int cb = 0; cb < COUTP; cb += 16) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + (uint32_t)(r * COUTP + cb), v);   // the whole warp
                if (inside) {
                    const size_t pix = (size_t)y * a.W + x;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = cb + j;
                        if (c >= a.cout) break;
                        float o = v[j] + sBias[c];
                        if (a.relu) o = fmaxf(o, 0.f);
                        if (c < a.o0) {
                            if (a.out0) a.out0[((size_t)img * a.o0 + c) * plane + pix] = o;
                        } else if (a.out1) {
                            a.out1[((size_t)img * (a.cout - a.o0) + (c - a.o0)) * plane + pix] = o;
                        }
                    }
                }
            }
        }
        if (L::NBUF == 1 && next < a.ntiles) stage(next, 0);   // the MMAs are done with the buffer
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();                                        // TMEM read, next tile staged
        buf ^= L::NBUF - 1;
    }
    if (failed) atomicExch(a.error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, L::tmem_cols);
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: dL/dW[co][ci][t] =
// sum over images and pixels p of dz[co](p) x[ci](p + shift(t)), with dz the
// output gradient times the ReLU mask, and dL/db[co] = sum of dz[co].  As a
// GEMM: rows R = 9 ci + t (and one more row of ones, R = 9 cin, for the
// bias; R is then the flat index of W[co] itself), columns co, K = pixels.
// A CTA owns 128 rows (an M block: at most 16 input channels) and a range of
// K tiles -- 128-pixel segments of image rows, y fastest, so that the CTA
// walks down a column of segments -- and accumulates D[R][co] in TMEM
// (M = 128, N = COUTP, K = 16 per MMA, BF16 operands, both K-major).
// Per K tile the needed input rows and dz are stored coalesced into FP32
// shared memory (a rolling window of three input rows: one new row per tile
// down the column) from registers loaded during the previous tile, and the
// BF16 operands are built from there: row R of A is the segment of x[ci]
// shifted by tap t, B is dz with the ReLU mask applied.  The next tile's
// loads are in flight while a tile is built.  At the end the CTA adds D to the
// FP32 gradients with atomics (the M blocks and K ranges of the grid
// partition the sum).
struct WgArgs {
    const float* xa;                    // layer input channels [0, ca): [N][ca][H][W]
    const float* xb;                    // [ca, cin): [N][cin - ca][H][W] (NULL when cin == ca)
    const float* gy;                    // [N][cout][H][W]
    const float* y;                     // ReLU output of the layer (NULL: no ReLU)
    int ca, cin, cout;
    float* gw;                          // [cout][cin][3][3], accumulated into (zeroed by the caller)
    float* gb;                          // [cout], accumulated into
    int n, H, W;
    int segs_x, ktiles, kper;           // row segments per image row, K tiles, K tiles per CTA
    int* error;
};

constexpr int kWgRS = 132;              // FP32 row stride of the staged dz (16-byte rows for float4 reads)
constexpr int kWgXS = 131;              // FP32 row stride of the staged input rows (130 used: x0 - 1 .. x0 + 128);
                                        // odd, so the 32 rows R = 9 ci + t of a warp fall in distinct banks
constexpr int kWgCh = 16;               // input channels 128 consecutive rows R = 9 ci + t touch at most

template <int COUTP>
struct WgLayout {
    static constexpr size_t a_bytes = 16ull * 128 * 16;                 // [16 chunks][128 rows][8 px] BF16
    static constexpr size_t b_bytes = 16ull * COUTP * 16;               // [16 chunks][COUTP][8 px]
    static constexpr size_t x_off = a_bytes + b_bytes;                  // [kWgCh][3 slots][kWgXS] FP32
    static constexpr size_t g_off = (x_off + 4ull * kWgCh * 3 * kWgXS + 15) / 16 * 16;   // dz: [COUTP][kWgRS] FP32
    static constexpr size_t bar_off = g_off + 4ull * COUTP * kWgRS;
    static constexpr size_t bytes = bar_off + 16;
    static constexpr uint32_t tmem_cols = COUTP <= 32 ? 32 : COUTP <= 64 ? 64 : COUTP <= 128 ? 128 : 256;
    static constexpr int row_per = (kWgCh * 130 + kThreads - 1) / kThreads;   // row values per thread
    static constexpr int dz_per = COUTP * 128 / kThreads;                    // dz values per thread
};

template <int COUTP>
__global__ void __launch_bounds__(kThreads, COUTP <= 32 ? 3 : COUTP <= 64 ? 2 : 1)
conv3x3_wgrad_kernel(const __grid_constant__ WgArgs a) {
    using L = WgLayout<COUTP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::bar_off + 8);
    unsigned char* sA = smem;
    unsigned char* sB = smem + L::a_bytes;
    float* xs = reinterpret_cast<float*>(smem + L::x_off);
    float* gs = reinterpret_cast<float*>(smem + L::g_off);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mblock = blockIdx.y;
    const int rows = 9 * a.cin + 1;                      // weight rows + the bias row
    const int ci_lo = min(mblock * 128 / 9, a.cin);
    const int nch = min(a.cin, (mblock * 128 + 127) / 9 + 1) - ci_lo;   // 0 .. kWgCh
    const size_t plane = (size_t)a.H * a.W;
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, L::tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int k0 = blockIdx.x * a.kper, k1 = min(a.ktiles, k0 + a.kper);

    // Registers that carry one tile's global loads to the next iteration's
    // shared-memory stores: one input row of this M block's channels
    // (segment x0 - 1 .. x0 + 128) and the tile's dz (ReLU mask applied).
    float rv[L::row_per], gv[L::dz_per];
    auto coords = [&](int kt, int& img, int& x0, int& y) {
        y = kt % a.H;
        const int r = kt / a.H;
        x0 = (r % a.segs_x) * 128;
        img = r / a.segs_x;
    };
    auto load_row = [&](int img, int x0, int yy) {      // zero outside the image
        const bool row_in = yy >= 0 && yy < a.H;
        const size_t roff = (size_t)min(max(yy, 0), a.H - 1) * a.W;
#pragma unroll
        for (int k = 0; k < L::row_per; ++k) {
            const int i = tid + k * kThreads;
            rv[k] = 0.f;
            if (i < nch * 130) {
                const int cl = i / 130, px = i - cl * 130;
                const int ci = ci_lo + cl, xx = x0 - 1 + px;
                const float* src = ci < a.ca ? a.xa + ((size_t)img * a.ca + ci) * plane
                                             : a.xb + ((size_t)img * (a.cin - a.ca) + (ci - a.ca)) * plane;
                if (row_in && xx >= 0 && xx < a.W) rv[k] = __ldg(src + roff + xx);   // predicated: no wait here
            }
        }
    };
    auto store_row = [&](int yy) {                      // into slot (yy + 3) % 3
        const int slot = (yy + 3) % 3;
#pragma unroll
        for (int k = 0; k < L::row_per; ++k) {
            const int i = tid + k * kThreads;
            if (i < nch * 130) {
                const int cl = i / 130, px = i - cl * 130;
                xs[(cl * 3 + slot) * kWgXS + px] = rv[k];
            }
        }
    };
    float mv[L::dz_per];
    auto load_dz = [&](int img, int x0, int y) {        // zero past the edge and for padded channels
        const size_t goff = ((size_t)img * a.cout * a.H + y) * a.W;
#pragma unroll
        for (int k = 0; k < L::dz_per; ++k) {
            const int i = tid + k * kThreads, co = i >> 7, px = i & 127;
            const size_t off = goff + (size_t)co * plane + (x0 + px);
            gv[k] = 0.f;
            mv[k] = 1.f;
            if (co < a.cout && x0 + px < a.W) {         // predicated: no wait here
                gv[k] = __ldg(a.gy + off);
                if (a.y) mv[k] = __ldg(a.y + off);
            }
        }
    };
    auto store_dz = [&]() {                             // the ReLU mask applied
#pragma unroll
        for (int k = 0; k < L::dz_per; ++k) {
            const int i = tid + k * kThreads;
            gs[(i >> 7) * kWgRS + (i & 127)] = mv[k] > 0.f ? gv[k] : 0.f;
        }
    };

    // The A build: thread tid always fills row r = tid % 128 (chunks tid / 128
    // + 2 k), so its (ci, tap) decomposition is fixed; the bias row of ones
    // and the zero rows past it never change and are written once here.
    static_assert(kThreads == 256, "the A build gives each thread one row and every other chunk");
    const int r_own = tid & 127, c_own = tid >> 7;
    const int R_own = mblock * 128 + r_own;
    const bool weight_row = R_own < rows - 1;
    int ty_own = 0;
    const float* xrow = xs;
    if (weight_row) {
        const int ci = R_own / 9, t = R_own - ci * 9;
        ty_own = t / 3;
        xrow = xs + (ci - ci_lo) * 3 * kWgXS + (t - ty_own * 3);
    } else {
        float v[8];
        const float one = R_own == rows - 1 ? 1.f : 0.f;   // dz is zero past the edge
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = one;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            *reinterpret_cast<uint4*>(sA + ((size_t)(c_own + 2 * k) * 128 + r_own) * 16) = pack8bf(v);
    }

    constexpr uint32_t idesc = idesc_bf16(128, COUTP);
    uint32_t phase = 0;
    bool failed = false;
    int img = 0, x0 = 0, y = 0;
    bool rolled = false;                                 // rv holds row y + 1 of this tile
    if (k0 < k1) {
        coords(k0, img, x0, y);
        load_dz(img, x0, y);
    }
    for (int kt = k0; kt < k1; ++kt) {
        // ---- this tile's rows and dz into shared memory (the previous tile's build is done with them)
        store_dz();
        if (rolled) {
            store_row(y + 1);                            // the window moves down one row
        } else {
            for (int d = -1; d <= 1; ++d) {
                load_row(img, x0, y + d);
                store_row(y + d);
            }
        }
        // the previous tile's MMAs must be done with the BF16 operands before they are rebuilt
        if (kt > k0) {
            if (!tc::mbar_wait(bar, phase, kLimit)) failed = true;
            phase ^= 1u;
        }
        if (__syncthreads_or(failed)) break;
        // ---- the next tile's loads, in flight while this one is built
        int nimg = img, nx0 = x0, ny = y;
        rolled = false;
        if (kt + 1 < k1) {
            coords(kt + 1, nimg, nx0, ny);
            rolled = nimg == img && nx0 == x0 && ny == y + 1;
            if (rolled) load_row(nimg, nx0, ny + 1);
            load_dz(nimg, nx0, ny);
        }
        // ---- BF16 operands: A row R = x[ci] shifted by tap t; B = dz
        if (weight_row) {   // row R of A: x[ci] of image row y + ty - 1 (window slot (y + ty + 2) % 3), shifted by tx
            const float* src = xrow + ((y + ty_own + 2) % 3) * kWgXS;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = c_own + 2 * k;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = src[c * 8 + j];
                *reinterpret_cast<uint4*>(sA + ((size_t)c * 128 + r_own) * 16) = pack8bf(v);
            }
        }
        for (int i = tid; i < COUTP * 16; i += kThreads) {   // (output channel co, chunk c), co fastest
            const int c = i / COUTP, co = i - c * COUTP;
            const float4 p = *reinterpret_cast<const float4*>(gs + co * kWgRS + c * 8);
            const float4 q = *reinterpret_cast<const float4*>(gs + co * kWgRS + c * 8 + 4);
            const float v[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
            *reinterpret_cast<uint4*>(sB + ((size_t)c * COUTP + co) * 16) = pack8bf(v);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sA), 128 * 16, 128);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sB), COUTP * 16, 128);
#pragma unroll
            for (int s = 0; s < 8; ++s)   // K = 16 pixels = chunks 2s, 2s + 1
                tc::mma_f16(tmem, ad + (uint64_t)(2 * s * 128), bd + (uint64_t)(2 * s * COUTP), idesc,
                            (kt > k0 || s > 0) ? 1u : 0u);
            tc::mma_commit(bar);
        }
        img = nimg, x0 = nx0, y = ny;
    }
    if (!failed && k0 < k1 && !tc::mbar_wait(bar, phase, kLimit)) failed = true;   // the last tile's MMAs
    tc::fence_after_sync();
    // ---- D[R][co] -> the gradients: warps 0-3, one TMEM lane (row) per thread
    if (!__syncthreads_or(failed) && k0 < k1 && warp < 4) {
        const int r = warp * 32 + lane, R = mblock * 128 + r;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int cb = 0; cb < COUTP; cb += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)cb, v);
            if (R < rows) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int co = cb + j;
                    if (co >= a.cout) break;
                    if (R == rows - 1) atomicAdd(a.gb + co, v[j]);
                    else atomicAdd(a.gw + (size_t)co * (rows - 1) + R, v[j]);   // W[co] flat = 9 ci + t
                }
            }
        }
    }
    if (failed) atomicExch(a.error, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, L::tmem_cols);
    }
}

}  // namespace ttc
}  // namespace fvn

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace fvn {
namespace {

int g_error_dev = -1;          // device of the error flag below
int* g_error = nullptr;        // set by a kernel whose bounded wait gave up

fvn_status error_flag(int** out) {
    int dev = 0;
    FVN_CUDA(nullptr, cudaGetDevice(&dev));
    if (!g_error || g_error_dev != dev) {
        int* p = nullptr;
        FVN_CUDA(nullptr, cudaMalloc(&p, sizeof(int)));
        FVN_CUDA(nullptr, cudaMemset(p, 0, sizeof(int)));
        g_error = p;   // one flag per process and device in use (the previous device's flag is kept)
        g_error_dev = dev;
    }
    *out = g_error;
    return FVN_OK;
}

// Shared memory opted in and the largest shared-memory carveout preferred,
// once per device: the occupancy query (and the launch) then count every CTA
// that the SM's shared memory holds, not only those of the default L1 split.
template <typename K>
cudaError_t configure_train(int dev, K kern, int bytes, std::atomic<unsigned long long>& done) {
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return opt_in_smem(dev, kern, bytes, done);
}

// CTAs of `kern` (kThreads threads, `bytes` of dynamic shared memory) one SM
// holds at once, from its registers and shared memory (the largest carveout,
// which the launch takes; the occupancy query counts the default split).
template <typename K>
cudaError_t resident_ctas(int dev, K kern, int bytes, int& per_sm) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    int smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return e;
    const int warps = ttc::kThreads / 32;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;       // allocated per warp in 256-register units
    const int by_smem = smem_sm / std::max(1, bytes + (int)fa.sharedSizeBytes + reserved);
    const int by_regs = regs_sm / std::max(1, warp_regs * warps);
    per_sm = std::min({by_smem, by_regs, threads_sm / ttc::kThreads});
    return cudaSuccess;
}

template <int CINP, int COUTP, int TR>
fvn_status launch_train(ttc::Args a, cudaStream_t st) {
    using L = ttc::Layout<CINP, COUTP, TR>;
    auto kern = ttc::conv3x3_train_kernel<CINP, COUTP, TR>;
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    FVN_CUDA(nullptr, cudaGetDevice(&dev));
    FVN_CUDA(nullptr, configure_train(dev, kern, (int)L::bytes, configured));
    int sms = 0;
    FVN_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;   // CTAs resident at once (registers, shared memory), within the TMEM
    FVN_CUDA(nullptr, resident_ctas(dev, kern, (int)L::bytes, per_sm));
    per_sm = std::min(per_sm, (int)(512 / L::tmem_cols));
    if (per_sm < 1) return set_error(nullptr, FVN_ERR_CUDA, "training conv kernel does not fit on an SM");
    a.tiles_x = (a.W + ttc::TW - 1) / ttc::TW;
    a.tiles_img = a.tiles_x * ((a.H + TR - 1) / TR);
    const long long nt = (long long)a.tiles_img * a.n;
    if (nt >= (1ll << 31)) return set_error(nullptr, FVN_ERR_ARG, "too many tiles");
    a.ntiles = (int)nt;
    fvn_status s = error_flag(&a.error);
    if (s != FVN_OK) return s;
    const int grid = (int)std::min<long long>(nt, (long long)sms * per_sm);
    kern<<<grid, ttc::kThreads, L::bytes, st>>>(a);
    FVN_LAUNCH_CHECK(nullptr);
    return FVN_OK;
}

// The instance for a GEMM of cin -> cout channels (padded to multiples of 16).
fvn_status dispatch(const ttc::Args& a, cudaStream_t st) {
    const int ci = (a.cin + 15) & ~15, co = (a.cout + 15) & ~15;
#define FVN_TTC(CI, CO, TR) \
    if (ci == CI && co == CO) return launch_train<CI, CO, TR>(a, st);
    FVN_TTC(16, 16, 4)
    FVN_TTC(16, 32, 4)
    FVN_TTC(16, 48, 4)
    FVN_TTC(32, 16, 4)
    FVN_TTC(32, 32, 4)
    FVN_TTC(32, 64, 4)
    FVN_TTC(32, 96, 4)
    FVN_TTC(48, 16, 2)
    FVN_TTC(64, 32, 2)
    FVN_TTC(64, 64, 2)
    FVN_TTC(96, 32, 2)
#undef FVN_TTC
    return set_error(nullptr, FVN_ERR_UNSUPPORTED, "no tensor-core training convolution for %d -> %d channels",
                     a.cin, a.cout);
}

template <int COUTP>
fvn_status launch_wgrad(ttc::WgArgs a, cudaStream_t st) {
    using L = ttc::WgLayout<COUTP>;
    auto kern = ttc::conv3x3_wgrad_kernel<COUTP>;
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    FVN_CUDA(nullptr, cudaGetDevice(&dev));
    FVN_CUDA(nullptr, configure_train(dev, kern, (int)L::bytes, configured));
    int sms = 0, per_sm = 0;
    FVN_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FVN_CUDA(nullptr, resident_ctas(dev, kern, (int)L::bytes, per_sm));
    per_sm = std::min(per_sm, (int)(512 / L::tmem_cols));
    if (per_sm < 1) return set_error(nullptr, FVN_ERR_CUDA, "weight-gradient kernel does not fit on an SM");
    a.segs_x = (a.W + 127) / 128;
    const long long kt = (long long)a.n * a.H * a.segs_x;
    if (kt >= (1ll << 31)) return set_error(nullptr, FVN_ERR_ARG, "too many pixels");
    a.ktiles = (int)kt;
    const int mb = (9 * a.cin + 1 + 127) / 128;
    // split K so that the grid fills the resident CTAs once
    const int splits = (int)std::max(1ll, std::min(kt, (long long)sms * per_sm / mb));
    a.kper = (int)((kt + splits - 1) / splits);
    const int gx = (int)((kt + a.kper - 1) / a.kper);
    fvn_status s = error_flag(&a.error);
    if (s != FVN_OK) return s;
    FVN_CUDA(nullptr, cudaMemsetAsync(a.gw, 0, sizeof(float) * 9 * (size_t)a.cin * a.cout, st));
    FVN_CUDA(nullptr, cudaMemsetAsync(a.gb, 0, sizeof(float) * (size_t)a.cout, st));
    kern<<<dim3(gx, mb), ttc::kThreads, L::bytes, st>>>(a);
    FVN_LAUNCH_CHECK(nullptr);
    return FVN_OK;
}

}  // namespace
}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_conv3x3_wgrad_bf16(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                             const float* gy, const float* y_relu, int cout, float* gw, float* gb,
                                             void* stream) {
    FVN_CHECK_ARG(nullptr, xa && gy && gw && gb && (cb == 0 || xb), "null tensor");
    FVN_CHECK_ARG(nullptr, ca >= 1 && cb >= 0 && n >= 1 && h >= 1 && w_ >= 1 && cout >= 1, "bad sizes");
    ttc::WgArgs a{};
    a.xa = xa;
    a.xb = cb ? xb : nullptr;
    a.gy = gy;
    a.y = y_relu;
    a.ca = ca;
    a.cin = ca + cb;
    a.cout = cout;
    a.gw = gw;
    a.gb = gb;
    a.n = n;
    a.H = h;
    a.W = w_;
    const int cp = (cout + 15) & ~15;
    cudaStream_t st = as_stream(stream);
    if (cp == 16) return launch_wgrad<16>(a, st);
    if (cp == 32) return launch_wgrad<32>(a, st);
    if (cp == 48) return launch_wgrad<48>(a, st);
    if (cp == 64) return launch_wgrad<64>(a, st);
    if (cp == 96) return launch_wgrad<96>(a, st);
    return set_error(nullptr, FVN_ERR_UNSUPPORTED, "no tensor-core weight gradient for %d output channels", cout);
}

extern "C" fvn_status fvn_conv3x3_fwd_bf16(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                           const float* w, const float* b, int cout, int relu, float* y,
                                           void* stream) {
    FVN_CHECK_ARG(nullptr, xa && w && y && (cb == 0 || xb), "null tensor");
    FVN_CHECK_ARG(nullptr, ca >= 1 && cb >= 0 && n >= 1 && h >= 1 && w_ >= 1 && cout >= 1, "bad sizes");
    ttc::Args a{};
    a.src0 = xa;
    a.c0 = ca;
    a.src1 = cb ? xb : nullptr;
    a.cin = ca + cb;
    a.cout = cout;
    a.w = w;
    a.bias = b;
    a.relu = relu != 0;
    a.out0 = y;
    a.o0 = cout;
    a.n = n;
    a.H = h;
    a.W = w_;
    return dispatch(a, as_stream(stream));
}

extern "C" fvn_status fvn_conv3x3_dgrad_bf16(const float* gy, const float* y_relu, int cout, int n, int h, int w_,
                                             const float* w, int ca, int cb, float* gxa, float* gxb, void* stream) {
    FVN_CHECK_ARG(nullptr, gy && w && (gxa || gxb), "null tensor");
    FVN_CHECK_ARG(nullptr, ca >= 1 && cb >= 0 && n >= 1 && h >= 1 && w_ >= 1 && cout >= 1, "bad sizes");
    FVN_CHECK_ARG(nullptr, cb > 0 || gxb == nullptr, "gxb without second input channels");
    ttc::Args a{};
    a.src0 = gy;
    a.c0 = cout;
    a.mask = y_relu;
    a.cin = cout;            // this GEMM runs from the layer's output channels ...
    a.cout = ca + cb;        // ... to its input channels
    a.w = w;
    a.dgrad = 1;
    a.out0 = gxa;
    a.out1 = gxb;
    a.o0 = ca;
    a.n = n;
    a.H = h;
    a.W = w_;
    return dispatch(a, as_stream(stream));
}

extern "C" fvn_status fvn_train_device_status(void) {
    if (!g_error) return FVN_OK;
    FVN_CUDA(nullptr, cudaDeviceSynchronize());
    int flag = 0;
    FVN_CUDA(nullptr, cudaMemcpy(&flag, g_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        FVN_CUDA(nullptr, cudaMemset(g_error, 0, sizeof(int)));
        return set_error(nullptr, FVN_ERR_TIMEOUT, "a training convolution gave up waiting for the tensor cores");
    }
    return FVN_OK;
}
