// Two-stage reconstruction network (paper: "Reconstruction Network", Fig.
// "network architecture", "Model Configuration"): a U-Net D of 3x3
// convolutions predicts a coarse image O_d and keeps its decoder's states;
// a U-Net K of 1x1 convolutions predicts, per block, a 3x3 kernel per pixel
// (and, in its decoder blocks, a blend weight) and passes O_d through those
// kernels in sequence: filtered by the encoder blocks with pooling between
// scales, by the coarsest block, then joined to each scale's encoder image
// (X = J + sigmoid(z) up(Y - pool J)) and filtered by the decoder blocks.
//
// FP32, NCHW.  The convolutions, pooling and up-sampling are the FP32
// training kernels; this file adds the per-pixel filter, the join (forward
// and backward) and the whole-frame forward pass behind
// fvn_reconstruct_wnet.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "resample.cuh"

namespace fvn {
namespace {

constexpr int kTaps = 9;
constexpr int kMaxWidth = 256;

int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 148;
    }();
    return n;
}

int grid_of(long long total) {
    return (int)std::max(1LL, std::min((total + 255) / 256, 16LL * sm_count()));
}

__device__ __forceinline__ bool tap_inside(int q, int y, int x, int h, int w) {
    const int yy = y + q / 3 - 1, xx = x + q % 3 - 1;
    return yy >= 0 && yy < h && xx >= 0 && xx < w;
}

// Softmax of the 9 logits at pixel (y, x) over the taps inside the frame;
// lg points at logit 0 of the pixel, logits are hw apart.
__device__ __forceinline__ void tap_weights(const float* __restrict__ lg, long long hw, int h, int w, int y, int x,
                                            float wq[kTaps]) {
    float m = -INFINITY;
#pragma unroll
    for (int q = 0; q < kTaps; ++q) {
        wq[q] = tap_inside(q, y, x, h, w) ? __ldg(lg + q * hw) : 0.f;
        if (tap_inside(q, y, x, h, w)) m = fmaxf(m, wq[q]);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kTaps; ++q) {
        wq[q] = tap_inside(q, y, x, h, w) ? expf(wq[q] - m) : 0.f;
        s += wq[q];
    }
    const float inv = 1.f / s;   // s >= 1: the largest in-frame term is exp(0)
#pragma unroll
    for (int q = 0; q < kTaps; ++q) wq[q] *= inv;
}

// The image-path kernels of the forward pass run on a (column block, row,
// image) grid of kRowThreads-pixel row segments: the pixel comes from the
// block and thread indices, with no division.
constexpr int kRowThreads = 128;

dim3 row_grid(int w, int h, int n) { return dim3((unsigned)((w + kRowThreads - 1) / kRowThreads), (unsigned)h, (unsigned)n); }

__global__ void __launch_bounds__(kRowThreads) filter3_fwd_kernel(const float* __restrict__ img,
                                                                   const float* __restrict__ logits, int n, int h,
                                                                   int w, float* __restrict__ out) {
    const int x = blockIdx.x * kRowThreads + threadIdx.x, y = blockIdx.y, b = blockIdx.z;
    if (x >= w) return;
    const long long hw = (long long)h * w, p = (long long)y * w + x;
    float wq[kTaps];
    tap_weights(logits + b * kTaps * hw + p, hw, h, w, y, x, wq);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* im = img + (b * 3 + c) * hw + p;
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < kTaps; ++q)
            if (tap_inside(q, y, x, h, w)) acc = fmaf(wq[q], __ldg(im + (q / 3 - 1) * w + (q % 3 - 1)), acc);
        out[(b * 3 + c) * hw + p] = acc;
    }
}

// dL/dlogit_q(p) = w_q (sum_c g_c(p) (img_c(p + q) - out_c(p))), zero outside
__global__ void filter3_bwd_logits_kernel(const float* __restrict__ img, const float* __restrict__ logits, int n,
                                          int h, int w, const float* __restrict__ gout, float* __restrict__ glog) {
    const long long hw = (long long)h * w, total = n * hw;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / hw, p = i - b * hw;
        const int y = (int)(p / w), x = (int)(p - (long long)y * w);
        float wq[kTaps], d[kTaps];
        tap_weights(logits + b * kTaps * hw + p, hw, h, w, y, x, wq);
#pragma unroll
        for (int q = 0; q < kTaps; ++q) d[q] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* im = img + (b * 3 + c) * hw + p;
            float v[kTaps], o = 0.f;
#pragma unroll
            for (int q = 0; q < kTaps; ++q) {
                v[q] = tap_inside(q, y, x, h, w) ? __ldg(im + (q / 3 - 1) * w + (q % 3 - 1)) : 0.f;
                o = fmaf(wq[q], v[q], o);
            }
            const float g = __ldg(gout + (b * 3 + c) * hw + p);
#pragma unroll
            for (int q = 0; q < kTaps; ++q) d[q] = fmaf(g, v[q] - o, d[q]);
        }
#pragma unroll
        for (int q = 0; q < kTaps; ++q)
            glog[(b * kTaps + q) * hw + p] = tap_inside(q, y, x, h, w) ? wq[q] * d[q] : 0.f;
    }
}

// dL/dimg_c(r) = sum over taps q with p = r - q in the frame of w_q(p) g_c(p)
__global__ void filter3_bwd_img_kernel(const float* __restrict__ logits, int n, int h, int w,
                                       const float* __restrict__ gout, float* __restrict__ gimg) {
    const long long hw = (long long)h * w, total = n * hw;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / hw, r = i - b * hw;
        const int ry = (int)(r / w), rx = (int)(r - (long long)ry * w);
        float acc[3] = {0.f, 0.f, 0.f};
        for (int q = 0; q < kTaps; ++q) {
            const int py = ry - (q / 3 - 1), px = rx - (q % 3 - 1);
            if (py < 0 || py >= h || px < 0 || px >= w) continue;
            const long long p = (long long)py * w + px;
            float wq[kTaps];
            tap_weights(logits + b * kTaps * hw + p, hw, h, w, py, px, wq);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] = fmaf(wq[q], __ldg(gout + (b * 3 + c) * hw + p), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) gimg[(b * 3 + c) * hw + r] = acc[c];
    }
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// up(Y - pool J) at fine pixel (y, x) of channel plane jc / yc
__device__ __forceinline__ float join_detail(const float* __restrict__ jc, const float* __restrict__ yc, int w,
                                             int hc, int wc, int y, int x) {
    int y0, y1, x0, x1;
    float ty, tx;
    up_src(y, hc, y0, y1, ty);
    up_src(x, wc, x0, x1, tx);
    auto d = [&](int cy, int cx) {
        const float* q = jc + (long long)(2 * cy) * w + 2 * cx;
        return __ldg(yc + (long long)cy * wc + cx) - 0.25f * (__ldg(q) + __ldg(q + 1) + __ldg(q + w) + __ldg(q + w + 1));
    };
    const float top = (1.f - tx) * d(y0, x0) + tx * d(y0, x1);
    const float bot = (1.f - tx) * d(y1, x0) + tx * d(y1, x1);
    return (1.f - ty) * top + ty * bot;
}

__global__ void __launch_bounds__(kRowThreads) join_fwd_kernel(const float* __restrict__ j,
                                                                const float* __restrict__ yv,
                                                                const float* __restrict__ z, int n, int h, int w,
                                                                float* __restrict__ xo) {
    const int x = blockIdx.x * kRowThreads + threadIdx.x, y = blockIdx.y, b = blockIdx.z;
    if (x >= w) return;
    const long long hw = (long long)h * w, p = (long long)y * w + x;
    const int hc = h / 2, wc = w / 2;
    const long long hwc = (long long)hc * wc;
    const float a = sigmoidf_(__ldg(z + b * hw + p));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* jc = j + (b * 3 + c) * hw;
        const float u = join_detail(jc, yv + (b * 3 + c) * hwc, w, hc, wc, y, x);
        xo[(b * 3 + c) * hw + p] = __ldg(jc + p) + a * u;
    }
}

// The join of the tensor-core pass in two steps: the coarse difference
// y - pool(j) once per coarse pixel (the term join_detail recomputes for
// each fine pixel it feeds), then x = j + sigmoid(z) up(d); one image, the
// same expressions as join_fwd_kernel.
__global__ void __launch_bounds__(kRowThreads) join_diff_kernel(const float* __restrict__ j,
                                                                 const float* __restrict__ yv, int h, int w,
                                                                 float* __restrict__ d) {
    const int cx = blockIdx.x * kRowThreads + threadIdx.x, cy = blockIdx.y, c = blockIdx.z;
    const int hc = h / 2, wc = w / 2;
    if (cx >= wc) return;
    const float* q = j + (long long)c * h * w + (long long)(2 * cy) * w + 2 * cx;
    const long long o = ((long long)c * hc + cy) * wc + cx;
    d[o] = __ldg(yv + o) - 0.25f * (__ldg(q) + __ldg(q + 1) + __ldg(q + w) + __ldg(q + w + 1));
}

__global__ void __launch_bounds__(kRowThreads) join_up_kernel(const float* __restrict__ j,
                                                               const float* __restrict__ d,
                                                               const float* __restrict__ z, int h, int w,
                                                               float* __restrict__ xo) {
    const int x = blockIdx.x * kRowThreads + threadIdx.x, y = blockIdx.y;
    if (x >= w) return;
    const int hc = h / 2, wc = w / 2;
    const long long hw = (long long)h * w, p = (long long)y * w + x;
    int y0, y1, x0, x1;
    float ty, tx;
    up_src(y, hc, y0, y1, ty);
    up_src(x, wc, x0, x1, tx);
    const float a = sigmoidf_(__ldg(z + p));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* dc = d + (long long)c * hc * wc;
        const float top = (1.f - tx) * __ldg(dc + (long long)y0 * wc + x0) + tx * __ldg(dc + (long long)y0 * wc + x1);
        const float bot = (1.f - tx) * __ldg(dc + (long long)y1 * wc + x0) + tx * __ldg(dc + (long long)y1 * wc + x1);
        xo[c * hw + p] = __ldg(j + c * hw + p) + a * ((1.f - ty) * top + ty * bot);
    }
}

// dL/dY = up^T(sigmoid(z) gx) at every coarse pixel (the up-sampling's adjoint)
__global__ void join_bwd_coarse_kernel(const float* __restrict__ z, const float* __restrict__ gx, int n, int h,
                                       int w, float* __restrict__ gy) {
    const int hc = h / 2, wc = w / 2;
    const long long hw = (long long)h * w, hwc = (long long)hc * wc, total = n * 3 * hwc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long bc = i / hwc, r = i - bc * hwc;
        const long long b = bc / 3;
        const int iy = (int)(r / wc), ix = (int)(r - (long long)iy * wc);
        const float* g = gx + bc * hw;
        const float* zb = z + b * hw;
        float s = 0.f;
        for (int oy = max(2 * iy - 1, 0); oy <= min(2 * iy + 2, h - 1); ++oy) {
            const float wy = up_weight(oy, iy, hc);
            if (wy == 0.f) continue;
            for (int ox = max(2 * ix - 1, 0); ox <= min(2 * ix + 2, w - 1); ++ox) {
                const float wx = up_weight(ox, ix, wc);
                if (wx == 0.f) continue;
                const long long o = (long long)oy * w + ox;
                s += wy * wx * sigmoidf_(__ldg(zb + o)) * __ldg(g + o);
            }
        }
        gy[i] = s;
    }
}

// dL/dJ = gx - pool^T(dL/dY);  dL/dz = sigmoid'(z) sum_c gx_c up(Y - pool J)_c
__global__ void join_bwd_fine_kernel(const float* __restrict__ j, const float* __restrict__ yv,
                                     const float* __restrict__ z, int n, int h, int w, const float* __restrict__ gx,
                                     const float* __restrict__ gy, float* __restrict__ gj, float* __restrict__ gz) {
    const long long hw = (long long)h * w, total = n * hw;
    const int hc = h / 2, wc = w / 2;
    const long long hwc = (long long)hc * wc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / hw, p = i - b * hw;
        const int y = (int)(p / w), x = (int)(p - (long long)y * w);
        const float a = sigmoidf_(__ldg(z + b * hw + p));
        float sz = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long bc = b * 3 + c;
            const float g = __ldg(gx + bc * hw + p);
            const float u = join_detail(j + bc * hw, yv + bc * hwc, w, hc, wc, y, x);
            sz = fmaf(g, u, sz);
            gj[bc * hw + p] = g - 0.25f * __ldg(gy + bc * hwc + (long long)(y / 2) * wc + x / 2);
        }
        gz[b * hw + p] = sz * a * (1.f - a);
    }
}

// dst[c][y][x] = src[c][y][x] inside src's sw x sh frame, 0 outside; dst is dw x dh
__global__ void __launch_bounds__(kRowThreads) window_copy_kernel(const float* __restrict__ src, int sw, int sh,
                                                                   float* __restrict__ dst, int dw, int dh, int nc) {
    const int x = blockIdx.x * kRowThreads + threadIdx.x, y = blockIdx.y, c = blockIdx.z;
    if (x >= dw) return;
    dst[((long long)c * dh + y) * dw + x] = (y < sh && x < sw) ? __ldg(src + ((long long)c * sh + y) * sw + x) : 0.f;
}

// ---------------------------------------------------------------------------
// layer table (the flat weight order of fvn_wnet_weight_count)
// ---------------------------------------------------------------------------
struct WLayer {
    int cin, cout, k;
    size_t off;   // W[cout][cin][k][k] at off, bias after it
};

struct WTable {
    int d_enc_a[FVN_WNET_MAX_LEVELS], d_enc_b[FVN_WNET_MAX_LEVELS], d_bot_a, d_bot_b;
    int d_dec_a[FVN_WNET_MAX_LEVELS], d_dec_b[FVN_WNET_MAX_LEVELS], d_out;
    int k_enc[FVN_WNET_MAX_LEVELS], k_enc_taps[FVN_WNET_MAX_LEVELS], k_bot, k_bot_taps;
    int k_dec[FVN_WNET_MAX_LEVELS], k_dec_taps[FVN_WNET_MAX_LEVELS], k_dec_blend[FVN_WNET_MAX_LEVELS];
    std::vector<WLayer> L;
    size_t total = 0;

    int add(int cin, int cout, int k) {
        L.push_back({cin, cout, k, total});
        total += (size_t)cout * cin * k * k + cout;
        return (int)L.size() - 1;
    }
};

bool config_ok(const fvn_wnet_config* c) {
    if (!c || c->levels < 1 || c->levels > FVN_WNET_MAX_LEVELS) return false;
    if (c->bot < 1 || c->bot > kMaxWidth) return false;
    for (int s = 0; s < c->levels; ++s)
        if (c->enc[s] < 1 || c->enc[s] > kMaxWidth || c->dec[s] < 1 || c->dec[s] > kMaxWidth) return false;
    return true;
}

WTable make_table(const fvn_wnet_config& c) {
    WTable t;
    const int L = c.levels;
    int ci = 5;
    for (int s = 0; s < L; ++s) {
        t.d_enc_a[s] = t.add(ci, c.enc[s], 3);
        t.d_enc_b[s] = t.add(c.enc[s], c.enc[s], 3);
        ci = c.enc[s];
    }
    t.d_bot_a = t.add(c.enc[L - 1], c.bot, 3);
    t.d_bot_b = t.add(c.bot, c.bot, 3);
    int prev = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        t.d_dec_a[s] = t.add(prev + c.enc[s], c.dec[s], 3);
        t.d_dec_b[s] = t.add(c.dec[s], c.dec[s], 3);
        prev = c.dec[s];
    }
    t.d_out = t.add(c.dec[0], 3, 1);
    for (int s = 0; s < L; ++s) {
        t.k_enc[s] = t.add((s ? c.enc[s - 1] : 0) + c.dec[s], c.enc[s], 1);
        t.k_enc_taps[s] = t.add(c.enc[s], kTaps, 1);
    }
    t.k_bot = t.add(c.enc[L - 1] + c.bot, c.bot, 1);
    t.k_bot_taps = t.add(c.bot, kTaps, 1);
    prev = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        t.k_dec[s] = t.add(prev + c.dec[s], c.dec[s], 1);
        t.k_dec_taps[s] = t.add(c.dec[s], kTaps, 1);
        t.k_dec_blend[s] = t.add(c.dec[s], 1, 1);
        prev = c.dec[s];
    }
    return t;
}

// ---------------------------------------------------------------------------
// activation buffers of one frame (padded to a multiple of 2^levels)
// ---------------------------------------------------------------------------
struct WPlan {
    float* x;                                        // [5] padded sparse frame
    float *T[FVN_WNET_MAX_LEVELS], *E[FVN_WNET_MAX_LEVELS], *U[FVN_WNET_MAX_LEVELS];
    float *UPD[FVN_WNET_MAX_LEVELS], *P[FVN_WNET_MAX_LEVELS + 1];
    float *G[FVN_WNET_MAX_LEVELS], *PG[FVN_WNET_MAX_LEVELS + 1], *LE[FVN_WNET_MAX_LEVELS];
    float *GD[FVN_WNET_MAX_LEVELS], *UPK[FVN_WNET_MAX_LEVELS], *LD[FVN_WNET_MAX_LEVELS], *ZD[FVN_WNET_MAX_LEVELS];
    float *I[FVN_WNET_MAX_LEVELS + 1], *J[FVN_WNET_MAX_LEVELS], *X[FVN_WNET_MAX_LEVELS];
    float *Y[FVN_WNET_MAX_LEVELS + 1];
    float *TB, *B, *GB, *LB;
};

// Carve the buffers from base (nullptr: size only); returns the bytes used.
size_t plan_wnet(const fvn_wnet_config& c, int Wp, int Hp, WPlan* pl, char* base) {
    size_t off = 0;
    auto take = [&](int ch, int s) -> float* {
        const size_t bytes = ((size_t)ch * (size_t)(Hp >> s) * (size_t)(Wp >> s) * sizeof(float) + 255) & ~(size_t)255;
        float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
        off += bytes;
        return p;
    };
    const int L = c.levels;
    pl->x = take(5, 0);
    for (int s = 0; s < L; ++s) {
        const int up = s == L - 1 ? c.bot : c.dec[s + 1];
        pl->T[s] = take(std::max(c.enc[s], c.dec[s]), s);
        pl->E[s] = take(c.enc[s], s);
        pl->U[s] = take(c.dec[s], s);
        pl->UPD[s] = take(up, s);
        pl->G[s] = take(c.enc[s], s);
        pl->LE[s] = take(kTaps, s);
        pl->GD[s] = take(c.dec[s], s);
        pl->UPK[s] = take(up, s);
        pl->LD[s] = take(kTaps, s);
        pl->ZD[s] = take(1, s);
        pl->I[s] = take(3, s);
        pl->J[s] = take(3, s);
        pl->X[s] = take(3, s);
        pl->Y[s] = take(3, s);
    }
    for (int s = 1; s <= L; ++s) {
        pl->P[s] = take(c.enc[s - 1], s);
        pl->PG[s] = take(c.enc[s - 1], s);
    }
    pl->I[L] = take(3, L);
    pl->Y[L] = take(3, L);
    pl->TB = take(c.bot, L);
    pl->B = take(c.bot, L);
    pl->GB = take(c.bot, L);
    pl->LB = take(kTaps, L);
    return off;
}

// ---------------------------------------------------------------------------
// tensor-core path (FVN_OPT_WNET_TENSOR_CORES): the convolutions' tensors are
// FP16 chunk-planar ([C / 8][H][W][8 halves]) and every convolution is the
// K-streamed tcgen05 kernel; the 3-channel image path, the tap logits and
// the blend logits stay FP32 planar.
// ---------------------------------------------------------------------------

// the sparse frame (FP32 [5][h][w]) as chunk 0 of a Wp x Hp chunk-planar
// tensor: zero outside the frame and in lanes 5..7
__global__ void cp_frame_kernel(const float* __restrict__ rgbam, int w, int h, uint4* __restrict__ out, int Wp,
                                int Hp) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Wp * Hp) return;
    const int y = r / Wp, x = r - y * Wp;
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (x < w && y < h)
#pragma unroll
        for (int c = 0; c < 5; ++c) f[c] = __ldg(rgbam + ((long long)c * h + y) * w + x);
    out[r] = f_to_h8(f);
}

// 2 x 2 average of every chunk plane (H, W even); blockIdx.y = chunk
__global__ void cp_pool2_kernel(const uint4* __restrict__ in, int H, int W, uint4* __restrict__ out) {
    const int ho = H / 2, wo = W / 2, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ho * wo) return;
    const int y = r / wo, x = r - y * wo;
    const uint4* p = in + (long long)blockIdx.y * H * W + (long long)(2 * y) * W + 2 * x;
    float a[8], b[8], s[8];
    h8_to_f(__ldg(p), s);
    h8_to_f(__ldg(p + 1), a);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] += a[j];
    h8_to_f(__ldg(p + W), a);
    h8_to_f(__ldg(p + W + 1), b);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = 0.25f * (s[j] + a[j] + b[j]);
    out[(long long)blockIdx.y * ho * wo + r] = f_to_h8(s);
}

// bilinear x2 up-sampling of every chunk plane (half-pixel centres, edge
// clamp): h x w -> 2h x 2w; blockIdx.y = chunk.  A thread takes fine rows
// 2m and 2m + 1 of one column: from m = 1 on they share their middle
// coarse row, whose x interpolation is done once (the arithmetic of each
// output is that of a single bilinear sample).
__global__ void cp_up2_kernel(const uint4* __restrict__ in, int h, int w, uint4* __restrict__ out) {
    const int W2 = 2 * w, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= h * W2) return;
    const int m = r / W2, ox = r - m * W2;
    int x0, x1, y0e, y1e, y0o, y1o;
    float tx, tye, tyo;
    up_src(ox, w, x0, x1, tx);
    up_src(2 * m, h, y0e, y1e, tye);
    up_src(2 * m + 1, h, y0o, y1o, tyo);
    const uint4* p = in + (long long)blockIdx.y * h * w;
    auto xlerp = [&](int y, float* o) {   // x interpolation of coarse row y
        up_xlerp8(__ldg(p + y * w + x0), __ldg(p + y * w + x1), tx, o);
    };
    float te[8], be[8], to[8], bo[8];
    xlerp(y0e, te);
    xlerp(y1e, be);
    if (y0o == y1e) {
#pragma unroll
        for (int j = 0; j < 8; ++j) to[j] = be[j];
    } else {
        xlerp(y0o, to);
    }
    xlerp(y1o, bo);
    uint4* q = out + (long long)blockIdx.y * (2 * h) * W2 + (long long)(2 * m) * W2 + ox;
    q[0] = up_ylerp8(te, be, tye);
    q[W2] = up_ylerp8(to, bo, tyo);
}

bool tc_widths_ok(const fvn_wnet_config& c) {
    auto ok = [](int v) { return v % 8 == 0 && v <= 128; };
    if (!ok(c.bot)) return false;
    for (int s = 0; s < c.levels; ++s)
        if (!ok(c.enc[s]) || !ok(c.dec[s])) return false;
    return true;
}

// Every layer's weights packed for the K-streamed convolution: FP16
// [group][tap][2 chunks][coutp][8], input channel (2 group + chunk) 8 + lane
// (the concatenated inputs of a layer meet on a chunk boundary: every width
// is a multiple of 8), zero past cin / cout; biases zero padded to coutp.
// One layer's weights (FP32 [cout][cin][k][k], bias [cout]) appended to the
// packed arrays; returns its offsets (halves, floats).
void pack_one(const float* w, const float* b, int cin, int cout, int k, std::vector<__half>& wp,
              std::vector<float>& bp, size_t* woff, size_t* boff) {
    const int coutp = ks_coutp(cout), chunks = (cin + 7) / 8, groups = (chunks + 1) / 2, taps = k * k;
    *woff = wp.size();
    *boff = bp.size();
    wp.resize(wp.size() + (size_t)groups * taps * 2 * coutp * 8, __float2half(0.f));
    bp.resize(bp.size() + coutp, 0.f);
    __half* dst = wp.data() + *woff;
    for (int g = 0; g < groups; ++g)
        for (int tp = 0; tp < taps; ++tp)
            for (int kk = 0; kk < 2; ++kk)
                for (int co = 0; co < cout; ++co)
                    for (int j = 0; j < 8; ++j) {
                        const int ci = (2 * g + kk) * 8 + j;
                        if (ci < cin)
                            dst[((((size_t)g * taps + tp) * 2 + kk) * coutp + co) * 8 + j] =
                                __float2half(w[((size_t)co * cin + ci) * taps + tp]);
                    }
    for (int co = 0; co < cout; ++co) bp[*boff + co] = b[co];
}

// Every layer's weights packed for the K-streamed convolution: FP16
// [group][tap][2 chunks][coutp][8], input channel (2 group + chunk) 8 + lane
// (the concatenated inputs of a layer meet on a chunk boundary: every width
// is a multiple of 8), zero past cin / cout; biases zero padded to coutp.
// Each K decoder level's tap head (9 outputs) and blend head (1) are also
// packed together as one 10-output layer.
void pack_tc(const WTable& t, const fvn_wnet_config& c, const float* host_w, std::vector<__half>& wp,
             std::vector<float>& bp, WnetState& S) {
    wp.clear();
    bp.clear();
    for (size_t li = 0; li < t.L.size(); ++li) {
        const WLayer& l = t.L[li];
        const float* w = host_w + l.off;
        pack_one(w, w + (size_t)l.cout * l.cin * l.k * l.k, l.cin, l.cout, l.k, wp, bp, &S.wpk_off[li],
                 &S.bpk_off[li]);
    }
    for (int s = 0; s < c.levels; ++s) {
        const WLayer& lt = t.L[t.k_dec_taps[s]];
        const WLayer& lb = t.L[t.k_dec_blend[s]];
        std::vector<float> w((size_t)(kTaps + 1) * lt.cin), b(kTaps + 1);
        const float* wt = host_w + lt.off;
        const float* wb = host_w + lb.off;
        std::copy(wt, wt + (size_t)kTaps * lt.cin, w.begin());
        std::copy(wb, wb + lb.cin, w.begin() + (size_t)kTaps * lt.cin);
        std::copy(wt + (size_t)kTaps * lt.cin, wt + (size_t)kTaps * lt.cin + kTaps, b.begin());
        b[kTaps] = wb[lb.cin];
        pack_one(w.data(), b.data(), lt.cin, kTaps + 1, 1, wp, bp, &S.wpk_tb_off[s], &S.bpk_tb_off[s]);
    }
}

// activation buffers of the tensor-core path (chunk-planar FP16 for the
// convolutions' tensors, FP32 planar for the image path and the heads)
struct TPlan {
    uint4* x;                                        // the sparse frame, one chunk
    uint4 *T[FVN_WNET_MAX_LEVELS], *E[FVN_WNET_MAX_LEVELS], *U[FVN_WNET_MAX_LEVELS], *UPD[FVN_WNET_MAX_LEVELS];
    uint4 *P[FVN_WNET_MAX_LEVELS + 1], *G[FVN_WNET_MAX_LEVELS], *PG[FVN_WNET_MAX_LEVELS + 1];
    uint4 *GD[FVN_WNET_MAX_LEVELS], *UPK[FVN_WNET_MAX_LEVELS];
    uint4 *TB, *B, *GB;
    float *LE[FVN_WNET_MAX_LEVELS], *LD[FVN_WNET_MAX_LEVELS], *ZD[FVN_WNET_MAX_LEVELS];
    float *I[FVN_WNET_MAX_LEVELS + 1], *J[FVN_WNET_MAX_LEVELS], *X[FVN_WNET_MAX_LEVELS], *Y[FVN_WNET_MAX_LEVELS + 1];
    float* LB;
    float* D[FVN_WNET_MAX_LEVELS + 1];               // coarse differences of the joins (3 planes at level s)
};

size_t plan_wnet_tc(const fvn_wnet_config& c, int Wp, int Hp, TPlan* pl, char* base) {
    size_t off = 0;
    auto bytes_at = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    auto half = [&](int ch, int s) {   // ch channels as chunk planes at level s
        return reinterpret_cast<uint4*>(bytes_at((size_t)((ch + 7) / 8) * (Hp >> s) * (Wp >> s) * 16));
    };
    auto f32 = [&](int ch, int s) {
        return reinterpret_cast<float*>(bytes_at((size_t)ch * (Hp >> s) * (Wp >> s) * sizeof(float)));
    };
    const int L = c.levels;
    pl->x = half(8, 0);
    for (int s = 0; s < L; ++s) {
        const int up = s == L - 1 ? c.bot : c.dec[s + 1];
        pl->T[s] = half(std::max(c.enc[s], c.dec[s]), s);
        pl->E[s] = half(c.enc[s], s);
        pl->U[s] = half(c.dec[s], s);
        pl->UPD[s] = half(up, s);
        pl->G[s] = half(c.enc[s], s);
        pl->GD[s] = half(c.dec[s], s);
        pl->UPK[s] = half(up, s);
        pl->LE[s] = f32(kTaps, s);
        pl->LD[s] = f32(kTaps + 1, s);   // the tap logits, then the blend logit (one head launch)
        pl->ZD[s] = base ? pl->LD[s] + (size_t)kTaps * (Hp >> s) * (Wp >> s) : nullptr;
        pl->I[s] = f32(3, s);
        pl->J[s] = f32(3, s);
        pl->X[s] = f32(3, s);
        pl->Y[s] = f32(3, s);
    }
    for (int s = 1; s <= L; ++s) {
        pl->P[s] = half(c.enc[s - 1], s);
        pl->PG[s] = half(c.enc[s - 1], s);
    }
    pl->I[L] = f32(3, L);
    pl->Y[L] = f32(3, L);
    pl->TB = half(c.bot, L);
    pl->B = half(c.bot, L);
    pl->GB = half(c.bot, L);
    pl->LB = f32(kTaps, L);
    for (int s = 1; s <= L; ++s) pl->D[s] = f32(3, s);
    return off;
}

dim3 cp_grid(long long plane, int chunks) { return dim3((unsigned)((plane + 255) / 256), (unsigned)chunks); }

#define WK(call)                                        \
    do {                                                \
        const fvn_status s_ = (call);                   \
        if (s_ != FVN_OK) return s_;                    \
    } while (0)
#define WQ(call)                                                                       \
    do {                                                                               \
        const fvn_status s_ = (call);                                                  \
        if (s_ != FVN_OK) return set_error(ctx, s_, "%s", fvn_last_error(nullptr));    \
    } while (0)

// The forward pass of fvn_reconstruct_wnet on the tensor cores: the same
// layers, in the same order, as the FP32 pass.
fvn_status wnet_forward_tc(fvn_ctx* ctx, const float* rgbam, int w, int h, float* rgb, void* stream) {
    WnetState& S = ctx->wnet;
    const fvn_wnet_config& c = S.cfg;
    const int L = c.levels, m = 1 << L;
    const int Wp = (w + m - 1) / m * m, Hp = (h + m - 1) / m * m;
    cudaStream_t st = as_stream(stream);
    if (S.tws_w != Wp || S.tws_h != Hp) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(S.tws);
        S.tws = nullptr;
        S.tws_w = S.tws_h = 0;
        TPlan tmp;
        const size_t bytes = plan_wnet_tc(c, Wp, Hp, &tmp, nullptr);
        FVN_CUDA(ctx, cudaMalloc(&S.tws, bytes));
        S.tws_bytes = bytes;
        S.tws_w = Wp;
        S.tws_h = Hp;
    }
    TPlan B;
    plan_wnet_tc(c, Wp, Hp, &B, static_cast<char*>(S.tws));
    const WTable t = make_table(c);
    auto hs = [&](int s) { return Hp >> s; };
    auto ws = [&](int s) { return Wp >> s; };
    // upx: xa is the level below (coarse), up-sampled inside the convolution
    auto convx = [&](const uint4* xa, int ca, const uint4* xb, int cb, int s, int li, int relu, uint4* y, float* y32,
                     bool upx) {
        KsConv k{};
        k.up = upx;
        k.in0 = xa;
        k.ch0 = (ca + 7) / 8;
        k.in1 = xb;
        k.ch1 = xb ? (cb + 7) / 8 : 0;
        k.H = hs(s);
        k.W = ws(s);
        // li < 0: the tap + blend heads of K decoder level -1 - li
        k.wpk = static_cast<const __half*>(S.d_wpk) + (li >= 0 ? S.wpk_off[li] : S.wpk_tb_off[-1 - li]);
        k.bias = S.d_bpk + (li >= 0 ? S.bpk_off[li] : S.bpk_tb_off[-1 - li]);
        k.cout = li >= 0 ? t.L[li].cout : kTaps + 1;
        k.k = li >= 0 ? t.L[li].k : 1;
        k.relu = relu;
        k.out = y;
        k.out32 = y32;
        return ks_conv(ctx, k, st);
    };
    auto conv = [&](const uint4* xa, int ca, const uint4* xb, int cb, int s, int li, int relu, uint4* y, float* y32) {
        return convx(xa, ca, xb, cb, s, li, relu, y, y32, false);
    };
    auto pool = [&](const uint4* x, int ch, int s, uint4* y) {   // level s -> s + 1
        cp_pool2_kernel<<<cp_grid((long long)hs(s + 1) * ws(s + 1), (ch + 7) / 8), 256, 0, st>>>(x, hs(s), ws(s), y);
        return cudaGetLastError() == cudaSuccess ? FVN_OK : set_error(ctx, FVN_ERR_CUDA, "pooling launch failed");
    };
    auto up = [&](const uint4* x, int ch, int s, uint4* y) {     // level s + 1 -> s
        cp_up2_kernel<<<cp_grid((long long)hs(s + 1) * ws(s), (ch + 7) / 8), 256, 0, st>>>(x, hs(s + 1), ws(s + 1), y);
        return cudaGetLastError() == cudaSuccess ? FVN_OK : set_error(ctx, FVN_ERR_CUDA, "up-sampling launch failed");
    };
    // a decoder level's first layer on [up(x), skip]: up-sampled inside the
    // convolution where the chunks of x form whole groups, else by a pass
    auto conv_up = [&](const uint4* x, int ch, const uint4* skip, int cs, int s, int li, uint4* upbuf, uint4* y) {
        if (S.fuse_up && ((ch + 7) / 8) % 2 == 0) return convx(x, ch, skip, cs, s, li, 1, y, nullptr, true);
        const fvn_status us = up(x, ch, s, upbuf);
        return us != FVN_OK ? us : conv(upbuf, ch, skip, cs, s, li, 1, y, nullptr);
    };

    cp_frame_kernel<<<(Wp * Hp + 255) / 256, 256, 0, st>>>(rgbam, w, h, B.x, Wp, Hp);
    FVN_LAUNCH_CHECK(ctx);
    // D: encoder, coarsest block, decoder, output layer
    const uint4* in = B.x;
    int cin = 5;
    for (int s = 0; s < L; ++s) {
        WK(conv(in, cin, nullptr, 0, s, t.d_enc_a[s], 1, B.T[s], nullptr));
        WK(conv(B.T[s], c.enc[s], nullptr, 0, s, t.d_enc_b[s], 1, B.E[s], nullptr));
        WK(pool(B.E[s], c.enc[s], s, B.P[s + 1]));
        in = B.P[s + 1];
        cin = c.enc[s];
    }
    WK(conv(B.P[L], c.enc[L - 1], nullptr, 0, L, t.d_bot_a, 1, B.TB, nullptr));
    WK(conv(B.TB, c.bot, nullptr, 0, L, t.d_bot_b, 1, B.B, nullptr));
    const uint4* prev = B.B;
    int pc = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        WK(conv_up(prev, pc, B.E[s], c.enc[s], s, t.d_dec_a[s], B.UPD[s], B.T[s]));
        WK(conv(B.T[s], c.dec[s], nullptr, 0, s, t.d_dec_b[s], 1, B.U[s], nullptr));
        prev = B.U[s];
        pc = c.dec[s];
    }
    WK(conv(B.U[0], c.dec[0], nullptr, 0, 0, t.d_out, 0, nullptr, B.I[0]));
    // K: encoder blocks, coarsest block, decoder blocks (features and heads)
    for (int s = 0; s < L; ++s) {
        if (s == 0) {
            WK(conv(B.U[0], c.dec[0], nullptr, 0, 0, t.k_enc[0], 1, B.G[0], nullptr));
        } else {
            WK(pool(B.G[s - 1], c.enc[s - 1], s - 1, B.PG[s]));
            WK(conv(B.PG[s], c.enc[s - 1], B.U[s], c.dec[s], s, t.k_enc[s], 1, B.G[s], nullptr));
        }
        WK(conv(B.G[s], c.enc[s], nullptr, 0, s, t.k_enc_taps[s], 0, nullptr, B.LE[s]));
    }
    WK(pool(B.G[L - 1], c.enc[L - 1], L - 1, B.PG[L]));
    WK(conv(B.PG[L], c.enc[L - 1], B.B, c.bot, L, t.k_bot, 1, B.GB, nullptr));
    WK(conv(B.GB, c.bot, nullptr, 0, L, t.k_bot_taps, 0, nullptr, B.LB));
    const uint4* kprev = B.GB;
    pc = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        WK(conv_up(kprev, pc, B.U[s], c.dec[s], s, t.k_dec[s], B.UPK[s], B.GD[s]));
        WK(conv(B.GD[s], c.dec[s], nullptr, 0, s, -1 - s, 0, nullptr, B.LD[s]));   // taps + blend: LD, ZD
        kprev = B.GD[s];
        pc = c.dec[s];
    }
    // image path (FP32): O_d through the encoder kernels, the coarsest, then
    // the decoder joins and kernels
    for (int s = 0; s < L; ++s) {
        WQ(fvn_filter3_fwd(B.I[s], B.LE[s], 1, hs(s), ws(s), B.J[s], stream));
        WQ(fvn_avgpool2_fwd(B.J[s], 3, hs(s), ws(s), B.I[s + 1], stream));
    }
    WQ(fvn_filter3_fwd(B.I[L], B.LB, 1, hs(L), ws(L), B.Y[L], stream));
    for (int s = L - 1; s >= 0; --s) {
        join_diff_kernel<<<row_grid(ws(s + 1), hs(s + 1), 3), kRowThreads, 0, st>>>(B.J[s], B.Y[s + 1], hs(s), ws(s),
                                                                                 B.D[s + 1]);
        FVN_LAUNCH_CHECK(ctx);
        join_up_kernel<<<row_grid(ws(s), hs(s), 1), kRowThreads, 0, st>>>(B.J[s], B.D[s + 1], B.ZD[s], hs(s), ws(s),
                                                                          B.X[s]);
        FVN_LAUNCH_CHECK(ctx);
        WQ(fvn_filter3_fwd(B.X[s], B.LD[s], 1, hs(s), ws(s), B.Y[s], stream));
    }
    window_copy_kernel<<<row_grid(w, h, 3), kRowThreads, 0, st>>>(B.Y[0], Wp, Hp, rgb, w, h, 3);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

}  // namespace
}  // namespace fvn

using namespace fvn;

// error text of a context-free call, moved to the context
#define WN(call)                                                                       \
    do {                                                                               \
        const fvn_status s_ = (call);                                                  \
        if (s_ != FVN_OK) return set_error(ctx, s_, "%s", fvn_last_error(nullptr));    \
    } while (0)

extern "C" size_t fvn_wnet_weight_count(const fvn_wnet_config* cfg) {
    return config_ok(cfg) ? make_table(*cfg).total : 0;
}

extern "C" fvn_status fvn_load_wnet_weights(fvn_ctx* ctx, const fvn_wnet_config* cfg, const float* host_w,
                                            size_t n) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, config_ok(cfg), "invalid two-stage configuration (levels 1..%d, widths 1..%d)",
                  FVN_WNET_MAX_LEVELS, kMaxWidth);
    FVN_CHECK_ARG(ctx, host_w != nullptr, "weights pointer is NULL");
    const size_t want = make_table(*cfg).total;
    FVN_CHECK_ARG(ctx, n == want, "weight vector has %zu entries, expected %zu", n, want);
    for (size_t i = 0; i < n; ++i) FVN_CHECK_ARG(ctx, isfinite(host_w[i]), "weight %zu is not finite", i);
    FVN_CUDA(ctx, cudaDeviceSynchronize());
    WnetState& S = ctx->wnet;
    S.loaded = false;                  // until the new set is complete
    if (S.cap < n) {
        cudaFree(S.d_w);
        S.d_w = nullptr;
        S.cap = 0;
        FVN_CUDA(ctx, cudaMalloc(&S.d_w, n * sizeof(float)));
        S.cap = n;
    }
    FVN_CUDA(ctx, cudaMemcpy(S.d_w, host_w, n * sizeof(float), cudaMemcpyHostToDevice));
    S.n = n;
    if (memcmp(&S.cfg, cfg, sizeof(*cfg)) != 0) {   // buffers are planned for the widths
        cudaFree(S.ws);
        S.ws = nullptr;
        S.ws_bytes = 0;
        S.ws_w = S.ws_h = 0;
        cudaFree(S.tws);
        S.tws = nullptr;
        S.tws_bytes = 0;
        S.tws_w = S.tws_h = 0;
    }
    S.cfg = *cfg;
    // the tensor-core path's packed weights
    S.tc_ok = tc_widths_ok(*cfg);
    if (S.tc_ok) {
        const WTable t = make_table(*cfg);
        std::vector<__half> wp;
        std::vector<float> bp;
        pack_tc(t, *cfg, host_w, wp, bp, S);
        cudaFree(S.d_wpk);
        cudaFree(S.d_bpk);
        S.d_wpk = nullptr;
        S.d_bpk = nullptr;
        FVN_CUDA(ctx, cudaMalloc(&S.d_wpk, wp.size() * sizeof(__half)));
        FVN_CUDA(ctx, cudaMalloc(&S.d_bpk, bp.size() * sizeof(float)));
        FVN_CUDA(ctx, cudaMemcpy(S.d_wpk, wp.data(), wp.size() * sizeof(__half), cudaMemcpyHostToDevice));
        FVN_CUDA(ctx, cudaMemcpy(S.d_bpk, bp.data(), bp.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    S.loaded = true;
    return FVN_OK;
}

extern "C" fvn_status fvn_reconstruct_wnet(fvn_ctx* ctx, const float* rgbam, int w, int h, float* rgb,
                                           void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam && rgb, "null buffer");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "bad frame size %d x %d", w, h);
    WnetState& S = ctx->wnet;
    if (!S.loaded) return set_error(ctx, FVN_ERR_STATE, "no two-stage weights (call fvn_load_wnet_weights first)");
    if (S.tc) {
        if (!S.tc_ok)
            return set_error(ctx, FVN_ERR_UNSUPPORTED,
                             "the tensor-core two-stage path needs every width a multiple of 8 and at most 128");
        return wnet_forward_tc(ctx, rgbam, w, h, rgb, stream);
    }
    const fvn_wnet_config& c = S.cfg;
    const int L = c.levels, m = 1 << L;
    const int Wp = (w + m - 1) / m * m, Hp = (h + m - 1) / m * m;
    cudaStream_t st = as_stream(stream);
    if (S.ws_w != Wp || S.ws_h != Hp) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(S.ws);
        S.ws = nullptr;
        S.ws_w = S.ws_h = 0;
        WPlan tmp;
        const size_t bytes = plan_wnet(c, Wp, Hp, &tmp, nullptr);
        FVN_CUDA(ctx, cudaMalloc(&S.ws, bytes));
        S.ws_bytes = bytes;
        S.ws_w = Wp;
        S.ws_h = Hp;
    }
    WPlan B;
    plan_wnet(c, Wp, Hp, &B, static_cast<char*>(S.ws));
    const WTable t = make_table(c);
    auto Wt = [&](int li) { return S.d_w + t.L[li].off; };
    auto Bs = [&](int li) { return S.d_w + t.L[li].off + (size_t)t.L[li].cout * t.L[li].cin * t.L[li].k * t.L[li].k; };
    auto conv = [&](const float* xa, int ca, const float* xb, int cb, int s, int li, int relu, float* y) {
        return fvn_conv_fwd(xa, ca, xb, cb, 1, Hp >> s, Wp >> s, Wt(li), Bs(li), t.L[li].cout, t.L[li].k, relu, y,
                            stream);
    };
    auto hs = [&](int s) { return Hp >> s; };
    auto ws = [&](int s) { return Wp >> s; };

    window_copy_kernel<<<row_grid(Wp, Hp, 5), kRowThreads, 0, st>>>(rgbam, w, h, B.x, Wp, Hp, 5);
    FVN_LAUNCH_CHECK(ctx);
    // D: encoder, coarsest block, decoder, output layer
    const float* in = B.x;
    int cin = 5;
    for (int s = 0; s < L; ++s) {
        WN(conv(in, cin, nullptr, 0, s, t.d_enc_a[s], 1, B.T[s]));
        WN(conv(B.T[s], c.enc[s], nullptr, 0, s, t.d_enc_b[s], 1, B.E[s]));
        WN(fvn_avgpool2_fwd(B.E[s], c.enc[s], hs(s), ws(s), B.P[s + 1], stream));
        in = B.P[s + 1];
        cin = c.enc[s];
    }
    WN(conv(B.P[L], c.enc[L - 1], nullptr, 0, L, t.d_bot_a, 1, B.TB));
    WN(conv(B.TB, c.bot, nullptr, 0, L, t.d_bot_b, 1, B.B));
    const float* prev = B.B;
    int pc = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        WN(fvn_upsample2_fwd(prev, pc, hs(s + 1), ws(s + 1), B.UPD[s], stream));
        WN(conv(B.UPD[s], pc, B.E[s], c.enc[s], s, t.d_dec_a[s], 1, B.T[s]));
        WN(conv(B.T[s], c.dec[s], nullptr, 0, s, t.d_dec_b[s], 1, B.U[s]));
        prev = B.U[s];
        pc = c.dec[s];
    }
    WN(conv(B.U[0], c.dec[0], nullptr, 0, 0, t.d_out, 0, B.I[0]));
    // K: encoder blocks, coarsest block, decoder blocks (features and heads)
    for (int s = 0; s < L; ++s) {
        if (s == 0) {
            WN(conv(B.U[0], c.dec[0], nullptr, 0, 0, t.k_enc[0], 1, B.G[0]));
        } else {
            WN(fvn_avgpool2_fwd(B.G[s - 1], c.enc[s - 1], hs(s - 1), ws(s - 1), B.PG[s], stream));
            WN(conv(B.PG[s], c.enc[s - 1], B.U[s], c.dec[s], s, t.k_enc[s], 1, B.G[s]));
        }
        WN(conv(B.G[s], c.enc[s], nullptr, 0, s, t.k_enc_taps[s], 0, B.LE[s]));
    }
    WN(fvn_avgpool2_fwd(B.G[L - 1], c.enc[L - 1], hs(L - 1), ws(L - 1), B.PG[L], stream));
    WN(conv(B.PG[L], c.enc[L - 1], B.B, c.bot, L, t.k_bot, 1, B.GB));
    WN(conv(B.GB, c.bot, nullptr, 0, L, t.k_bot_taps, 0, B.LB));
    prev = B.GB;
    pc = c.bot;
    for (int s = L - 1; s >= 0; --s) {
        WN(fvn_upsample2_fwd(prev, pc, hs(s + 1), ws(s + 1), B.UPK[s], stream));
        WN(conv(B.UPK[s], pc, B.U[s], c.dec[s], s, t.k_dec[s], 1, B.GD[s]));
        WN(conv(B.GD[s], c.dec[s], nullptr, 0, s, t.k_dec_taps[s], 0, B.LD[s]));
        WN(conv(B.GD[s], c.dec[s], nullptr, 0, s, t.k_dec_blend[s], 0, B.ZD[s]));
        prev = B.GD[s];
        pc = c.dec[s];
    }
    // image path: O_d through the encoder kernels, the coarsest, then the
    // decoder joins and kernels
    for (int s = 0; s < L; ++s) {
        WN(fvn_filter3_fwd(B.I[s], B.LE[s], 1, hs(s), ws(s), B.J[s], stream));
        WN(fvn_avgpool2_fwd(B.J[s], 3, hs(s), ws(s), B.I[s + 1], stream));
    }
    WN(fvn_filter3_fwd(B.I[L], B.LB, 1, hs(L), ws(L), B.Y[L], stream));
    for (int s = L - 1; s >= 0; --s) {
        WN(fvn_wnet_join_fwd(B.J[s], B.Y[s + 1], B.ZD[s], 1, hs(s), ws(s), B.X[s], stream));
        WN(fvn_filter3_fwd(B.X[s], B.LD[s], 1, hs(s), ws(s), B.Y[s], stream));
    }
    window_copy_kernel<<<row_grid(w, h, 3), kRowThreads, 0, st>>>(B.Y[0], Wp, Hp, rgb, w, h, 3);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_filter3_fwd(const float* img, const float* logits, int n, int h, int w_, float* out,
                                      void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, img && logits && out && n >= 1 && h >= 1 && w_ >= 1, "bad filter arguments");
    FVN_CHECK_ARG(ctx, h <= 65535 && n <= 65535, "bad filter arguments");
    filter3_fwd_kernel<<<row_grid(w_, h, n), kRowThreads, 0, as_stream(stream)>>>(img, logits, n, h, w_, out);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_filter3_bwd(const float* img, const float* logits, int n, int h, int w_,
                                      const float* gout, float* gimg, float* glogits, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, img && logits && gout && gimg && glogits && n >= 1 && h >= 1 && w_ >= 1,
                  "bad filter arguments");
    const int g = grid_of((long long)n * h * w_);
    filter3_bwd_logits_kernel<<<g, 256, 0, as_stream(stream)>>>(img, logits, n, h, w_, gout, glogits);
    FVN_LAUNCH_CHECK(ctx);
    filter3_bwd_img_kernel<<<g, 256, 0, as_stream(stream)>>>(logits, n, h, w_, gout, gimg);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_wnet_join_fwd(const float* j, const float* y, const float* z, int n, int h, int w_,
                                        float* x, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, j && y && z && x && n >= 1 && h >= 2 && w_ >= 2 && h % 2 == 0 && w_ % 2 == 0,
                  "bad join arguments");
    FVN_CHECK_ARG(ctx, h <= 65535 && n <= 65535, "bad join arguments");
    join_fwd_kernel<<<row_grid(w_, h, n), kRowThreads, 0, as_stream(stream)>>>(j, y, z, n, h, w_, x);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_wnet_join_bwd(const float* j, const float* y, const float* z, int n, int h, int w_,
                                        const float* gx, float* gj, float* gy, float* gz, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, j && y && z && gx && gj && gy && gz && n >= 1 && h >= 2 && w_ >= 2 && h % 2 == 0 &&
                           w_ % 2 == 0,
                  "bad join arguments");
    join_bwd_coarse_kernel<<<grid_of((long long)n * 3 * (h / 2) * (w_ / 2)), 256, 0, as_stream(stream)>>>(
        z, gx, n, h, w_, gy);
    FVN_LAUNCH_CHECK(ctx);
    join_bwd_fine_kernel<<<grid_of((long long)n * h * w_), 256, 0, as_stream(stream)>>>(j, y, z, n, h, w_, gx, gy,
                                                                                        gj, gz);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}
