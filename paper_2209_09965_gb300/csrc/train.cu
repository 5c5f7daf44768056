// Training kernels of the reconstruction network, FP32 (paper: "Training",
// "Loss", "Model Precision & Optimization": the network is trained in full
// 32-bit precision).  NCHW tensors with a batch dimension.  These are the
// forward / backward pieces called by the Python autograd functions.
//
//  - conv (k = 1 or 3, zero padding k/2) with bias and optional ReLU, whose
//    input may be the channel concatenation of two tensors (skip
//    connections without a copy);
//  - its data gradient (the same kernel with flipped, transposed weights and
//    the ReLU mask applied to the incoming gradient on load) and its weight /
//    bias gradient (per-CTA partial sums over a pixel range, FP32 atomics);
//  - 2x2 average pooling, bilinear x2 up-sampling and their adjoints;
//  - the kernel-prediction blend forward / backward;
//  - the L1 + image-gradient loss and Adam.
// The same convolutions run the two-stage network's inference pass
// (fvn_reconstruct_wnet, wnet.cu).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "resample.cuh"

namespace fvn {

constexpr int CT = 16;          // output-pixel tile side of the conv kernels
constexpr int CO_T = 16;        // output channels per CTA

// y[n][co][p] (+)= sum_ci sum_tap W(co, ci, tap) x[n][ci][p + tap - r]
// FWD:  W(co, ci, tap) = w[co][ci][tap], x = xa ++ xb, epilogue bias / ReLU.
// DGRAD: x = gy masked by (y_relu > 0), W(co', ci', tap) = w[ci'][co'][flip(tap)],
//        output split into gxa / gxb.
// A CTA computes a TH x TW pixel tile for CO_T output channels; each thread
// four consecutive pixels of one row for all CO_T channels, so every weight
// read from shared memory (a broadcast) feeds four FMAs and every input read
// sixteen.  Input channels are staged CI_T at a time; the forward pass
// copies the next group asynchronously (cp.async, double-buffered) while
// it computes on the current one.
constexpr int TH = 16, TW = 64, CI_T = 4;
constexpr int TWS = TW + 4;     // staged row stride: 16-byte aligned rows

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int K, bool DGRAD>
__global__ void __launch_bounds__(256, 2) conv_f32_kernel(const float* __restrict__ xa, int ca,
                                                          const float* __restrict__ xb, int cb,
                                                          const float* __restrict__ mask_src, int n_in, int h,
                                                          int w_, const float* __restrict__ wt,
                                                          const float* __restrict__ bias, int n_out, int relu,
                                                          float* __restrict__ ya, int ya_c, float* __restrict__ yb,
                                                          int tiles_x) {
    constexpr int R = K / 2, HH = TH + 2 * R, HW = TW + 2 * R, KK = K * K;
    __shared__ __align__(16) float s_in[2][CI_T][HH][TWS];
    __shared__ __align__(16) float s_w[2][CI_T][KK][CO_T];
    const int tile = blockIdx.x;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int co0 = blockIdx.y * CO_T;
    const int n = blockIdx.z;
    const int tc = threadIdx.x % (TW / 4), tr = threadIdx.x / (TW / 4);
    const int y = ty * TH + tr, x0 = tx * TW + 4 * tc;
    const long long hw = (long long)h * w_;
    float acc[4][CO_T];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int j = 0; j < CO_T; ++j) acc[p][j] = 0.f;

    auto accumulate = [&](int buf) {
#pragma unroll
        for (int c = 0; c < CI_T; ++c) {
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
                float v[4 + 2 * R];
                const float4 a = *reinterpret_cast<const float4*>(&s_in[buf][c][tr + ky][4 * tc]);
                v[0] = a.x;
                v[1] = a.y;
                v[2] = a.z;
                v[3] = a.w;
                if constexpr (R > 0) {
                    const float2 b = *reinterpret_cast<const float2*>(&s_in[buf][c][tr + ky][4 * tc + 4]);
                    v[4] = b.x;
                    v[5] = b.y;
                }
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const float4* wp = reinterpret_cast<const float4*>(&s_w[buf][c][ky * K + kx][0]);
#pragma unroll
                    for (int q = 0; q < CO_T / 4; ++q) {
                        const float4 wv = wp[q];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float xv = v[p + kx];
                            acc[p][4 * q + 0] = fmaf(wv.x, xv, acc[p][4 * q + 0]);
                            acc[p][4 * q + 1] = fmaf(wv.y, xv, acc[p][4 * q + 1]);
                            acc[p][4 * q + 2] = fmaf(wv.z, xv, acc[p][4 * q + 2]);
                            acc[p][4 * q + 3] = fmaf(wv.w, xv, acc[p][4 * q + 3]);
                        }
                    }
                }
            }
        }
    };

    if constexpr (!DGRAD) {
        // zero-filled copies read nothing; their source is any valid address
        auto stage = [&](int buf, int ci0) {
            // each thread copies fixed tile positions of all CI_T channels:
            // the position arithmetic is done once per position
            const float* plane[CI_T];
#pragma unroll
            for (int c = 0; c < CI_T; ++c) {
                const int ci = ci0 + c;
                plane[c] = ci >= n_in ? nullptr
                           : ci < ca  ? xa + ((long long)n * ca + ci) * hw
                                      : xb + ((long long)n * cb + (ci - ca)) * hw;
            }
            for (int pos = threadIdx.x; pos < HH * HW; pos += 256) {
                const int hy = pos / HW, hx = pos - hy * HW;
                const int gy = ty * TH + hy - R, gx = tx * TW + hx - R;
                const bool in = gy >= 0 && gx >= 0 && gy < h && gx < w_;
                const long long off = in ? (long long)gy * w_ + gx : 0;
#pragma unroll
                for (int c = 0; c < CI_T; ++c) {
                    const bool ok = in && plane[c] != nullptr;
                    cp_async4(&s_in[buf][c][hy][hx], ok ? plane[c] + off : xa, ok);
                }
            }
            for (int i = threadIdx.x; i < CI_T * KK * CO_T; i += 256) {
                const int c = i / (KK * CO_T), r = i - c * (KK * CO_T);
                const int tap = r / CO_T, j = r - tap * CO_T;
                const int ci = ci0 + c, co = co0 + j;
                const bool ok = ci < n_in && co < n_out;
                cp_async4(&s_w[buf][c][tap][j], ok ? wt + ((long long)co * n_in + ci) * KK + tap : wt, ok);
            }
        };
        const int nch = (n_in + CI_T - 1) / CI_T;
        stage(0, 0);
        cp_async_commit();
        for (int k = 0; k < nch; ++k) {
            if (k + 1 < nch) stage((k + 1) & 1, (k + 1) * CI_T);
            cp_async_commit();
            cp_async_wait_1();          // this thread's copies of group k have landed
            __syncthreads();            // ... and every thread's
            accumulate(k & 1);
            __syncthreads();            // buffer k & 1 is free for group k + 2
        }
    } else {
        for (int ci0 = 0; ci0 < n_in; ci0 += CI_T) {
            __syncthreads();
            for (int pos = threadIdx.x; pos < HH * HW; pos += 256) {
                const int hy = pos / HW, hx = pos - hy * HW;
                const int gy = ty * TH + hy - R, gx = tx * TW + hx - R;
                const bool in = gy >= 0 && gx >= 0 && gy < h && gx < w_;
                const long long off = (long long)gy * w_ + gx;
                float v[CI_T];
#pragma unroll
                for (int c = 0; c < CI_T; ++c) {
                    const int ci = ci0 + c;
                    v[c] = 0.f;
                    if (in && ci < n_in) {
                        const long long base = ((long long)n * n_in + ci) * hw + off;
                        v[c] = __ldg(xa + base);
                        if (mask_src && !(__ldg(mask_src + base) > 0.f)) v[c] = 0.f;
                    }
                }
#pragma unroll
                for (int c = 0; c < CI_T; ++c) s_in[0][c][hy][hx] = v[c];
            }
            for (int i = threadIdx.x; i < CI_T * KK * CO_T; i += 256) {
                const int c = i / (KK * CO_T), r = i - c * (KK * CO_T);
                const int tap = r / CO_T, j = r - tap * CO_T;
                const int ci = ci0 + c, co = co0 + j;
                s_w[0][c][tap][j] = (ci < n_in && co < n_out)
                                        ? __ldg(wt + ((long long)ci * n_out + co) * KK + (KK - 1 - tap))
                                        : 0.f;
            }
            __syncthreads();
            accumulate(0);
        }
    }
    if (y >= h) return;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int x = x0 + p;
        if (x >= w_) break;
        const long long pix = (long long)y * w_ + x;
#pragma unroll
        for (int j = 0; j < CO_T; ++j) {
            const int co = co0 + j;
            if (co >= n_out) break;
            float v = acc[p][j];
            if (!DGRAD) {
                v += __ldg(bias + co);
                if (relu) v = fmaxf(v, 0.f);
                ya[((long long)n * n_out + co) * hw + pix] = v;
            } else {
                if (co < ya_c) {
                    if (ya) ya[((long long)n * ya_c + co) * hw + pix] = v;
                } else if (yb) {
                    yb[((long long)n * (n_out - ya_c) + (co - ya_c)) * hw + pix] = v;
                }
            }
        }
    }
}

// 1x1 convolution (FWD / DGRAD as above with K = 1) as a skinny GEMM over
// pixel strips: a CTA takes PW x 128 consecutive pixels of one image and up
// to 8 groups of 16 output channels (blockIdx.z selects the groups when
// there are more), so each input value is read from memory once per 128
// output channels; warp w handles sub-strip w / ncog (128 pixels, 4 per
// lane) and group w % ncog.  Input channels are staged P1_CI at a time; the
// forward pass on 16-byte aligned planes copies the next group with cp.async
// into a second buffer while it computes on the current one.
constexpr int P1_CI = 8;

__global__ void __launch_bounds__(256) conv1x1_f32_kernel(const float* __restrict__ xa, int ca,
                                                          const float* __restrict__ xb, int cb,
                                                          const float* __restrict__ mask_src, int n_in, long long hw,
                                                          const float* __restrict__ wt,
                                                          const float* __restrict__ bias, int n_out, int relu,
                                                          float* __restrict__ ya, int ya_c, float* __restrict__ yb,
                                                          int ncog, int pw, bool dgrad) {
    extern __shared__ __align__(16) float smem1[];
    const int px = 128 * pw;                           // pixels of the strip
    const int cop = ncog * CO_T;
    float* s_in = smem1;                               // [2][P1_CI][px]
    float* s_w = smem1 + 2 * P1_CI * px;               // [2][P1_CI][cop]
    const int co_base = blockIdx.z * cop;
    const long long p0 = (long long)blockIdx.x * px;
    const int n = blockIdx.y;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int sub = warp / ncog, cog = warp - sub * ncog;
    const int lp = sub * 128 + 4 * lane;               // first pixel of this lane within the strip
    float acc[4][CO_T];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int j = 0; j < CO_T; ++j) acc[p][j] = 0.f;
    auto accumulate = [&](int buf) {
        if (sub >= pw) return;
        const float* si = s_in + buf * P1_CI * px;
        const float* sw = s_w + buf * P1_CI * cop;
#pragma unroll
        for (int c = 0; c < P1_CI; ++c) {
            const float4 xv = *reinterpret_cast<const float4*>(si + c * px + lp);
            const float x4[4] = {xv.x, xv.y, xv.z, xv.w};
            const float4* wp = reinterpret_cast<const float4*>(sw + c * cop + cog * CO_T);
#pragma unroll
            for (int q = 0; q < CO_T / 4; ++q) {
                const float4 wv = wp[q];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    acc[p][4 * q + 0] = fmaf(wv.x, x4[p], acc[p][4 * q + 0]);
                    acc[p][4 * q + 1] = fmaf(wv.y, x4[p], acc[p][4 * q + 1]);
                    acc[p][4 * q + 2] = fmaf(wv.z, x4[p], acc[p][4 * q + 2]);
                    acc[p][4 * q + 3] = fmaf(wv.w, x4[p], acc[p][4 * q + 3]);
                }
            }
        }
    };
    // planes whose length is a multiple of 4 (and 16-byte aligned tensors)
    // are staged with 16-byte copies
    const bool vec = (hw & 3) == 0 && ((reinterpret_cast<uintptr_t>(xa) | reinterpret_cast<uintptr_t>(xb) |
                                        reinterpret_cast<uintptr_t>(mask_src)) & 15) == 0;
    if (!dgrad && vec) {
        // forward: the next channel group is copied asynchronously
        // (double-buffered) while the current one is used
        auto stage = [&](int buf, int ci0) {
            float* si = s_in + buf * P1_CI * px;
            for (int i = threadIdx.x; i < P1_CI * px / 4; i += blockDim.x) {
                const int c = (4 * i) / px, q = 4 * i - c * px;
                const int ci = ci0 + c;
                const long long pix = p0 + q;
                const bool ok = ci < n_in && pix < hw;
                const float* src = xa;
                if (ok)
                    src = (ci < ca ? xa + ((long long)n * ca + ci) * hw : xb + ((long long)n * cb + (ci - ca)) * hw) +
                          pix;
                cp_async16(si + 4 * i, src, ok);
            }
            float* sw = s_w + buf * P1_CI * cop;
            for (int i = threadIdx.x; i < P1_CI * cop; i += blockDim.x) {
                const int c = i / cop, co = co_base + (i - c * cop);
                const int ci = ci0 + c;
                const bool ok = ci < n_in && co < n_out;
                cp_async4(sw + i, ok ? wt + (long long)co * n_in + ci : wt, ok);
            }
        };
        const int nch = (n_in + P1_CI - 1) / P1_CI;
        stage(0, 0);
        cp_async_commit();
        for (int k = 0; k < nch; ++k) {
            if (k + 1 < nch) stage((k + 1) & 1, (k + 1) * P1_CI);
            cp_async_commit();
            cp_async_wait_1();
            __syncthreads();
            accumulate(k & 1);
            __syncthreads();
        }
    } else {
        for (int ci0 = 0; ci0 < n_in; ci0 += P1_CI) {
            __syncthreads();
            if (vec) {
#pragma unroll 8
                for (int i = threadIdx.x; i < P1_CI * px / 4; i += blockDim.x) {
                    const int c = (4 * i) / px, q = 4 * i - c * px;
                    const int ci = ci0 + c;
                    const long long pix = p0 + q;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ci < n_in && pix < hw) {
                        const long long o = ((long long)n * n_in + ci) * hw + pix;
                        v = __ldg(reinterpret_cast<const float4*>(xa + o));
                        if (mask_src) {
                            const float4 m = __ldg(reinterpret_cast<const float4*>(mask_src + o));
                            v.x = m.x > 0.f ? v.x : 0.f;
                            v.y = m.y > 0.f ? v.y : 0.f;
                            v.z = m.z > 0.f ? v.z : 0.f;
                            v.w = m.w > 0.f ? v.w : 0.f;
                        }
                    }
                    *reinterpret_cast<float4*>(s_in + 4 * i) = v;
                }
            } else {
                for (int i = threadIdx.x; i < P1_CI * px; i += blockDim.x) {
                    const int c = i / px, q = i - c * px;
                    const int ci = ci0 + c;
                    const long long pix = p0 + q;
                    float v = 0.f;
                    if (ci < n_in && pix < hw) {
                        if (!dgrad) {
                            const float* src = ci < ca ? xa + ((long long)n * ca + ci) * hw
                                                       : xb + ((long long)n * cb + (ci - ca)) * hw;
                            v = __ldg(src + pix);
                        } else {
                            const long long o = ((long long)n * n_in + ci) * hw + pix;
                            v = __ldg(xa + o);
                            if (mask_src && !(__ldg(mask_src + o) > 0.f)) v = 0.f;
                        }
                    }
                    s_in[i] = v;
                }
            }
            for (int i = threadIdx.x; i < P1_CI * cop; i += blockDim.x) {
                const int c = i / cop, co = co_base + (i - c * cop);
                const int ci = ci0 + c;
                float v = 0.f;
                if (ci < n_in && co < n_out)
                    v = dgrad ? __ldg(wt + (long long)ci * n_out + co) : __ldg(wt + (long long)co * n_in + ci);
                s_w[i] = v;
            }
            __syncthreads();
            accumulate(0);
        }
    }
    if (sub >= pw) return;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const long long pix = p0 + lp + p;
        if (pix >= hw) break;
#pragma unroll
        for (int j = 0; j < CO_T; ++j) {
            const int co = co_base + cog * CO_T + j;
            if (co >= n_out) break;
            float v = acc[p][j];
            if (!dgrad) {
                v += __ldg(bias + co);
                if (relu) v = fmaxf(v, 0.f);
                ya[((long long)n * n_out + co) * hw + pix] = v;
            } else if (co < ya_c) {
                if (ya) ya[((long long)n * ya_c + co) * hw + pix] = v;
            } else if (yb) {
                yb[((long long)n * (n_out - ya_c) + (co - ya_c)) * hw + pix] = v;
            }
        }
    }
}

// launch shape of conv1x1_f32_kernel for n_out output channels: groups of
// 16 channels per CTA (at most 8), CTAs over the groups (nz), sub-strips
struct Conv1Shape {
    int ncog, nz, pw, threads;
    size_t smem;
};
inline Conv1Shape conv1_shape(int n_out) {
    Conv1Shape s;
    const int groups = (n_out + CO_T - 1) / CO_T;
    s.nz = (groups + 7) / 8;
    s.ncog = (groups + s.nz - 1) / s.nz;
    s.pw = std::max(1, std::min(4, 8 / s.ncog));
    s.threads = 32 * s.ncog * s.pw;
    s.smem = sizeof(float) * 2 * (size_t)P1_CI * (128 * s.pw + s.ncog * CO_T);   // two buffers
    return s;
}

// dL/dw[co][ci][tap] and dL/db[co]: each CTA reduces a 16 x 16 (co, ci) block
// over a range of 16 x 16 pixel tiles and adds its partial sums atomically.
// Thread t takes output channels 4 (t >> 6) .. + 3, input channel (t >> 2) & 15
// and the tile rows r = 4 i + (t & 3); per step four pixels of a row: four
// 16-byte loads of dL/dy and one 16- and one 8-byte load per tap row of x
// feed 4 x 4 x K^2 FMAs.  The four row subsets of a (co, ci) pair sit in
// consecutive lanes and are summed by shuffles before the atomics.
constexpr int WG_XS = CT + 4;   // staged x row stride (16-byte aligned rows)

template <int K>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const float* __restrict__ xa, int ca,
                                                         const float* __restrict__ xb, int cb,
                                                         const float* __restrict__ gy,
                                                         const float* __restrict__ y_relu, int n, int h, int w_,
                                                         int cout, float* __restrict__ gw, float* __restrict__ gb,
                                                         int tiles_x, int tiles_per_img, int tiles_per_cta) {
    constexpr int R = K / 2, HT = CT + 2 * R, KK = K * K;
    __shared__ __align__(16) float s_g[16][CT * CT];
    __shared__ __align__(16) float s_x[16][HT][WG_XS];
    const int cin = ca + cb;
    const int co0 = blockIdx.x * 16, ci0 = blockIdx.y * 16;
    const int cg = threadIdx.x >> 6, tci = (threadIdx.x >> 2) & 15, sub = threadIdx.x & 3;
    const long long hw = (long long)h * w_;
    float acc[4][KK];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < KK; ++i) acc[j][i] = 0.f;
    float accb[4] = {0.f, 0.f, 0.f, 0.f};
    const int total_tiles = n * tiles_per_img;
    const int t_begin = blockIdx.z * tiles_per_cta;
    const int t_end = std::min(total_tiles, t_begin + tiles_per_cta);
    for (int tt = t_begin; tt < t_end; ++tt) {
        const int img = tt / tiles_per_img, tl = tt - img * tiles_per_img;
        const int ty = tl / tiles_x, tx = tl - ty * tiles_x;
        __syncthreads();
        for (int i = threadIdx.x; i < 16 * CT * CT; i += 256) {
            const int j = i / (CT * CT), pp = i - j * CT * CT;
            const int yy = ty * CT + pp / CT, xx = tx * CT + pp % CT;
            const int co = co0 + j;
            float v = 0.f;
            if (co < cout && yy < h && xx < w_) {
                const long long o = ((long long)img * cout + co) * hw + (long long)yy * w_ + xx;
                v = __ldg(gy + o);
                if (y_relu && !(__ldg(y_relu + o) > 0.f)) v = 0.f;
            }
            s_g[j][pp] = v;
        }
        for (int i = threadIdx.x; i < 16 * HT * HT; i += 256) {
            const int j = i / (HT * HT), pp = i - j * HT * HT;
            const int hy = pp / HT, hx = pp - hy * HT;
            const int yy = ty * CT + hy - R, xx = tx * CT + hx - R;
            const int ci = ci0 + j;
            float v = 0.f;
            if (ci < cin && yy >= 0 && xx >= 0 && yy < h && xx < w_) {
                const float* src = ci < ca ? xa + ((long long)img * ca + ci) * hw
                                           : xb + ((long long)img * cb + (ci - ca)) * hw;
                v = __ldg(src + (long long)yy * w_ + xx);
            }
            s_x[j][hy][hx] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int rr = 0; rr < CT / 4; ++rr) {
            const int r = 4 * rr + sub;
#pragma unroll
            for (int k4 = 0; k4 < CT / 4; ++k4) {
                float g[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 gv = *reinterpret_cast<const float4*>(&s_g[4 * cg + j][r * CT + 4 * k4]);
                    g[j][0] = gv.x;
                    g[j][1] = gv.y;
                    g[j][2] = gv.z;
                    g[j][3] = gv.w;
                    accb[j] += (gv.x + gv.y) + (gv.z + gv.w);
                }
#pragma unroll
                for (int ky = 0; ky < K; ++ky) {
                    float xv[4 + 2 * R];
                    const float4 a = *reinterpret_cast<const float4*>(&s_x[tci][r + ky][4 * k4]);
                    xv[0] = a.x;
                    xv[1] = a.y;
                    xv[2] = a.z;
                    xv[3] = a.w;
                    if constexpr (R > 0) {
                        const float2 b = *reinterpret_cast<const float2*>(&s_x[tci][r + ky][4 * k4 + 4]);
                        xv[4] = b.x;
                        xv[5] = b.y;
                    }
#pragma unroll
                    for (int kx = 0; kx < K; ++kx)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int p = 0; p < 4; ++p)
                                acc[j][ky * K + kx] = fmaf(g[j][p], xv[p + kx], acc[j][ky * K + kx]);
                }
            }
        }
    }
    // sum the four row subsets (consecutive lanes), then one atomic per entry
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int i = 0; i < KK; ++i) {
            acc[j][i] += __shfl_xor_sync(0xffffffffu, acc[j][i], 1);
            acc[j][i] += __shfl_xor_sync(0xffffffffu, acc[j][i], 2);
        }
        accb[j] += __shfl_xor_sync(0xffffffffu, accb[j], 1);
        accb[j] += __shfl_xor_sync(0xffffffffu, accb[j], 2);
    }
    const int ci = ci0 + tci;
    if (sub == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int co = co0 + 4 * cg + j;
            if (co < cout && ci < cin) {
#pragma unroll
                for (int i = 0; i < KK; ++i) atomicAdd(gw + ((long long)co * cin + ci) * KK + i, acc[j][i]);
            }
            if (blockIdx.y == 0 && tci == 0 && co < cout) atomicAdd(gb + co, accb[j]);
        }
    }
}

// The resampling kernels run on a 2-D grid: blockIdx.y walks the planes
// (image x channel), blockIdx.x x 256 + threadIdx.x the pixels of one plane,
// so the index arithmetic stays 32-bit and one division per element.
// VEC: the fine tensor is 8-byte aligned (w_ is even, so every pixel pair
// 2 xx, 2 xx + 1 is too) and is accessed as float2
template <bool VEC>
__global__ void avgpool2_fwd_kernel(const float* __restrict__ x, long long nc, int h, int w_, float* __restrict__ y) {
    const int ho = h / 2, wo = w_ / 2, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ho * wo) return;
    const int yy = r / wo, xx = r - yy * wo;
#pragma unroll 4
    for (long long c = blockIdx.y; c < nc; c += gridDim.y) {
        const float* p = x + c * h * w_ + (long long)(2 * yy) * w_ + 2 * xx;
        float2 a, b;
        if (VEC) {
            a = __ldg(reinterpret_cast<const float2*>(p));
            b = __ldg(reinterpret_cast<const float2*>(p + w_));
        } else {
            a = make_float2(__ldg(p), __ldg(p + 1));
            b = make_float2(__ldg(p + w_), __ldg(p + w_ + 1));
        }
        y[c * ho * wo + r] = 0.25f * (a.x + a.y + b.x + b.y);
    }
}

template <bool VEC>
__global__ void avgpool2_bwd_kernel(const float* __restrict__ gy, long long nc, int h, int w_, float* __restrict__ gx) {
    const int ho = h / 2, wo = w_ / 2, r = blockIdx.x * blockDim.x + threadIdx.x;   // one coarse pixel
    if (r >= ho * wo) return;
    const int yy = r / wo, xx = r - yy * wo;
#pragma unroll 4
    for (long long c = blockIdx.y; c < nc; c += gridDim.y) {
        const float v = 0.25f * __ldg(gy + c * ho * wo + r);
        float* q = gx + c * h * w_ + (long long)(2 * yy) * w_ + 2 * xx;
        if (VEC) {
            *reinterpret_cast<float2*>(q) = make_float2(v, v);
            *reinterpret_cast<float2*>(q + w_) = make_float2(v, v);
        } else {
            q[0] = q[1] = q[w_] = q[w_ + 1] = v;
        }
    }
}

__global__ void upsample2_fwd_kernel(const float* __restrict__ x, long long nc, int h, int w_, float* __restrict__ y) {
    const int H2 = 2 * h, W2 = 2 * w_, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H2 * W2) return;
    const int oy = r / W2, ox = r - oy * W2;
    int y0, y1, x0, x1;
    float ty, tx;
    up_src(oy, h, y0, y1, ty);
    up_src(ox, w_, x0, x1, tx);
#pragma unroll 4
    for (long long c = blockIdx.y; c < nc; c += gridDim.y) {
        const float* p = x + c * h * w_;
        const float top = (1.f - tx) * __ldg(p + y0 * w_ + x0) + tx * __ldg(p + y0 * w_ + x1);
        const float bot = (1.f - tx) * __ldg(p + y1 * w_ + x0) + tx * __ldg(p + y1 * w_ + x1);
        y[c * H2 * W2 + r] = (1.f - ty) * top + ty * bot;
    }
}

__global__ void upsample2_bwd_kernel(const float* __restrict__ gy, long long nc, int h, int w_, float* __restrict__ gx) {
    const int H2 = 2 * h, W2 = 2 * w_, r = blockIdx.x * blockDim.x + threadIdx.x;   // one coarse pixel
    if (r >= h * w_) return;
    const int iy = r / w_, ix = r - iy * w_;
    const int oy0 = max(2 * iy - 1, 0), oy1 = min(2 * iy + 2, H2 - 1);
    const int ox0 = max(2 * ix - 1, 0), ox1 = min(2 * ix + 2, W2 - 1);
    float wy[4], wx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        wy[k] = oy0 + k <= oy1 ? up_weight(oy0 + k, iy, h) : 0.f;
        wx[k] = ox0 + k <= ox1 ? up_weight(ox0 + k, ix, w_) : 0.f;
    }
#pragma unroll 4
    for (long long c = blockIdx.y; c < nc; c += gridDim.y) {
        const float* g = gy + c * H2 * W2;
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (wy[a] == 0.f) continue;
            const float* row = g + (long long)(oy0 + a) * W2;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (wx[b] != 0.f) s += wy[a] * wx[b] * __ldg(row + ox0 + b);
        }
        gx[c * h * w_ + r] = s;
    }
}

// kernel prediction + blend, per pixel (see the inference head kernel)
template <bool BWD>
__global__ void kp_blend_kernel(const float* __restrict__ head, const float* __restrict__ sparse, int n, int h,
                                int w_, const float* __restrict__ gout, float* __restrict__ out) {
    const long long hw = (long long)h * w_;
    const long long total = (long long)n * hw;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long img = i / hw;
        const int r = (int)(i - img * hw);
        const int y = r / w_, x = r - y * w_;
        const float* hd = head + img * 29 * hw + r;
        const float* sp = sparse + img * 5 * hw;
        float lg[25], mx = -INFINITY;
#pragma unroll
        for (int q = 0; q < 25; ++q) {
            lg[q] = hd[(3 + q) * hw];
            mx = fmaxf(mx, lg[q]);
        }
        float es = 0.f;
#pragma unroll
        for (int q = 0; q < 25; ++q) {
            lg[q] = expf(lg[q] - mx);
            es += lg[q];
        }
        const float inv = 1.f / es;
        float m[25], c[25][3];
        float den = 0.f, num[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 25; ++q) {
            lg[q] *= inv;   // softmax weight w_q
            const int yy = y + q / 5 - 2, xx = x + q % 5 - 2;
            m[q] = 0.f;
            c[q][0] = c[q][1] = c[q][2] = 0.f;
            if (yy >= 0 && xx >= 0 && yy < h && xx < w_) {
                const long long o = (long long)yy * w_ + xx;
                m[q] = sp[4 * hw + o];
                c[q][0] = sp[o];
                c[q][1] = sp[hw + o];
                c[q][2] = sp[2 * hw + o];
            }
            const float wm = lg[q] * m[q];
            den += wm;
            num[0] = fmaf(wm, c[q][0], num[0]);
            num[1] = fmaf(wm, c[q][1], num[1]);
            num[2] = fmaf(wm, c[q][2], num[2]);
        }
        const bool valid = den >= 1e-12f;
        float rd[3] = {hd[0], hd[hw], hd[2 * hw]};
        float kp[3];
        for (int ch = 0; ch < 3; ++ch) kp[ch] = valid ? num[ch] / den : rd[ch];
        const float z = hd[28 * hw];
        const float a = 1.f / (1.f + expf(-z));
        if (!BWD) {
            float* o = out + img * 3 * hw + r;
            for (int ch = 0; ch < 3; ++ch) o[ch * hw] = a * kp[ch] + (1.f - a) * rd[ch];
        } else {
            const float* go = gout + img * 3 * hw + r;
            float* gh = out + img * 29 * hw + r;
            float g[3] = {go[0], go[hw], go[2 * hw]};
            float ga = 0.f;
            for (int ch = 0; ch < 3; ++ch) {
                ga += g[ch] * (kp[ch] - rd[ch]);
                gh[ch * hw] = g[ch] * (1.f - a) + (valid ? 0.f : g[ch] * a);
            }
            gh[28 * hw] = ga * a * (1.f - a);
            float dw[25], sdw = 0.f;
#pragma unroll
            for (int q = 0; q < 25; ++q) {
                float s = 0.f;
                if (valid)
                    for (int ch = 0; ch < 3; ++ch) s += g[ch] * a * m[q] * (c[q][ch] - kp[ch]);
                dw[q] = valid ? s / den : 0.f;
                sdw += lg[q] * dw[q];
            }
#pragma unroll
            for (int q = 0; q < 25; ++q) gh[(3 + q) * hw] = lg[q] * (dw[q] - sdw);
        }
    }
}

// L1 + lam (L1 of forward differences), gradient and loss.  Blocks walk the
// image rows (grid-stride), threads the pixels of a row; the loss is reduced
// in the block and added with one atomic per block.
__global__ void loss_kernel(const float* __restrict__ p, const float* __restrict__ t, long long nc, int h, int w_,
                            float lam, float* __restrict__ loss, float* __restrict__ g) {
    __shared__ float red[32];
    const long long rows = nc * h;
    const double n1 = (double)rows * w_, nx = (double)rows * (w_ - 1), ny = (double)nc * (h - 1) * w_;
    const float i1 = (float)(1.0 / n1), ix = nx > 0 ? (float)(lam / nx) : 0.f, iy = ny > 0 ? (float)(lam / ny) : 0.f;
    auto sgn = [](float v) { return (float)((v > 0.f) - (v < 0.f)); };
    float part = 0.f;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (int)(row % h);
        for (int x = threadIdx.x; x < w_; x += blockDim.x) {
            const long long i = row * w_ + x;
            const float d = __ldg(p + i) - __ldg(t + i);
            float gi = sgn(d) * i1;
            part += fabsf(d) * i1;
            if (x + 1 < w_) {
                const float dx = (__ldg(p + i + 1) - __ldg(t + i + 1)) - d;
                gi -= sgn(dx) * ix;
                part += fabsf(dx) * ix;
            }
            if (x > 0) gi += sgn(d - (__ldg(p + i - 1) - __ldg(t + i - 1))) * ix;
            if (y + 1 < h) {
                const float dy = (__ldg(p + i + w_) - __ldg(t + i + w_)) - d;
                gi -= sgn(dy) * iy;
                part += fabsf(dy) * iy;
            }
            if (y > 0) gi += sgn(d - (__ldg(p + i - w_) - __ldg(t + i - w_))) * iy;
            g[i] = gi;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = part;
    __syncthreads();
    if (warp == 0) {
        part = (int)threadIdx.x < nw ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) atomicAdd(loss, part);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Adam with the step count read from device memory (a step replayed from a
// CUDA graph): the bias corrections 1 - beta^step in double, as on the host.
__global__ void adam_dev_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, size_t n, const int* __restrict__ step, float lr, float b1,
                                float b2, float eps) {
    const int t = max(__ldg(step), 1);
    const float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// grid of the resampling kernels: pixels of a plane x planes, about 8192
// CTAs in all -- each thread loops over the planes gridDim.y apart, so that
// the CTAs are not so small that their scheduling is the limit
static dim3 plane_grid(long long plane, long long nc) {
    const long long gx = (plane + 255) / 256;
    const long long gy = std::max(1LL, std::min(nc, 8192 / std::max(1LL, gx)));
    return dim3((unsigned)gx, (unsigned)std::min(gy, 65535LL));
}

static int grid_for(fvn_ctx* ctx, long long total) {
    long long g = (total + 255) / 256;
    const long long cap = 32LL * (ctx->num_sms > 0 ? ctx->num_sms : 148);
    return (int)std::max(1LL, std::min(g, cap));
}

}  // namespace fvn

using namespace fvn;

namespace {
fvn_ctx* train_ctx() {
    // Training kernels are context-free; a process-wide descriptor carries the
    // SM count used for grid sizing and the error text.
    static fvn_ctx* c = [] {
        fvn_ctx* x = new fvn_ctx();
        cudaGetDevice(&x->device);
        cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, x->device);
        return x;
    }();
    return c;
}
}  // namespace

extern "C" fvn_status fvn_conv_fwd(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                   const float* w, const float* b, int cout, int k, int relu, float* y, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, xa && w && b && y && (cb == 0 || xb), "null tensor");
    FVN_CHECK_ARG(ctx, ca >= 1 && cb >= 0 && n >= 1 && h >= 1 && w_ >= 1 && cout >= 1, "bad sizes");
    FVN_CHECK_ARG(ctx, k == 1 || k == 3, "k must be 1 or 3");
    const int tiles_x = (w_ + TW - 1) / TW;
    dim3 grid(tiles_x * ((h + TH - 1) / TH), (cout + CO_T - 1) / CO_T, n);
    if (k == 3) {
        conv_f32_kernel<3, false><<<grid, 256, 0, as_stream(stream)>>>(xa, ca, xb, cb, nullptr, ca + cb, h, w_, w,
                                                                       b, cout, relu, y, cout, nullptr, tiles_x);
    } else {
        const Conv1Shape sh = conv1_shape(cout);
        const long long hw = (long long)h * w_;
        dim3 g1((unsigned)((hw + 128 * sh.pw - 1) / (128 * sh.pw)), n, sh.nz);
        conv1x1_f32_kernel<<<g1, sh.threads, sh.smem, as_stream(stream)>>>(xa, ca, xb, cb, nullptr, ca + cb, hw, w, b,
                                                                          cout, relu, y, cout, nullptr, sh.ncog,
                                                                          sh.pw, false);
    }
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_conv_bwd(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                   const float* w, int cout, int k, const float* gy, const float* y_relu, float* gxa,
                                   float* gxb, float* gw, float* gb, void* stream) {
    fvn_ctx* ctx = nullptr;
    cudaStream_t st = as_stream(stream);
    FVN_CHECK_ARG(ctx, xa && w && gy && (cb == 0 || xb), "null tensor");
    FVN_CHECK_ARG(ctx, (gw == nullptr) == (gb == nullptr), "gw and gb must both be set or both NULL");
    FVN_CHECK_ARG(ctx, ca >= 1 && cb >= 0 && n >= 1 && h >= 1 && w_ >= 1 && cout >= 1, "bad sizes");
    FVN_CHECK_ARG(ctx, k == 1 || k == 3, "k must be 1 or 3");
    const int cin = ca + cb;
    const int tiles_x = (w_ + CT - 1) / CT;            // wgrad tiles
    const int tiles = tiles_x * ((h + CT - 1) / CT);
    if (gxa || gxb) {
        const int dtx = (w_ + TW - 1) / TW;
        dim3 grid(dtx * ((h + TH - 1) / TH), (cin + CO_T - 1) / CO_T, n);
        if (k == 3) {
            conv_f32_kernel<3, true><<<grid, 256, 0, st>>>(gy, cout, nullptr, 0, y_relu, cout, h, w_, w, nullptr,
                                                           cin, 0, gxa, ca, gxb, dtx);
        } else {
            const Conv1Shape sh = conv1_shape(cin);
            const long long hw = (long long)h * w_;
            dim3 g1((unsigned)((hw + 128 * sh.pw - 1) / (128 * sh.pw)), n, sh.nz);
            conv1x1_f32_kernel<<<g1, sh.threads, sh.smem, st>>>(gy, cout, nullptr, 0, y_relu, cout, hw, w, nullptr, cin,
                                                               0, gxa, ca, gxb, sh.ncog, sh.pw, true);
        }
        FVN_LAUNCH_CHECK(ctx);
    }
    if (gw) {
        FVN_CUDA(ctx, cudaMemsetAsync(gw, 0, sizeof(float) * (size_t)cout * cin * k * k, st));
        FVN_CUDA(ctx, cudaMemsetAsync(gb, 0, sizeof(float) * (size_t)cout, st));
        const int gco = (cout + 15) / 16, gci = (cin + 15) / 16;
        const long long total_tiles = (long long)n * tiles;
        const int sms = train_ctx()->num_sms > 0 ? train_ctx()->num_sms : 148;
        long long parts = std::max(1LL, (4LL * sms) / (gco * gci));
        parts = std::min(parts, total_tiles);
        const int per = (int)((total_tiles + parts - 1) / parts);
        parts = (total_tiles + per - 1) / per;
        dim3 grid(gco, gci, (unsigned)parts);
        if (k == 3)
            conv_wgrad_kernel<3><<<grid, 256, 0, st>>>(xa, ca, xb, cb, gy, y_relu, n, h, w_, cout, gw, gb, tiles_x,
                                                       tiles, per);
        else
            conv_wgrad_kernel<1><<<grid, 256, 0, st>>>(xa, ca, xb, cb, gy, y_relu, n, h, w_, cout, gw, gb, tiles_x,
                                                       tiles, per);
        FVN_LAUNCH_CHECK(ctx);
    }
    return FVN_OK;
}

extern "C" fvn_status fvn_avgpool2_fwd(const float* x, int nc, int h, int w_, float* y, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, x && y && nc >= 1 && h >= 2 && w_ >= 2 && h % 2 == 0 && w_ % 2 == 0, "bad pool arguments");
    const dim3 grid = plane_grid((long long)(h / 2) * (w_ / 2), nc);
    if (((uintptr_t)x & 7) == 0) avgpool2_fwd_kernel<true><<<grid, 256, 0, as_stream(stream)>>>(x, nc, h, w_, y);
    else avgpool2_fwd_kernel<false><<<grid, 256, 0, as_stream(stream)>>>(x, nc, h, w_, y);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_avgpool2_bwd(const float* gy, int nc, int h, int w_, float* gx, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, gx && gy && nc >= 1 && h >= 2 && w_ >= 2 && h % 2 == 0 && w_ % 2 == 0, "bad pool arguments");
    const dim3 grid = plane_grid((long long)(h / 2) * (w_ / 2), nc);
    if (((uintptr_t)gx & 7) == 0) avgpool2_bwd_kernel<true><<<grid, 256, 0, as_stream(stream)>>>(gy, nc, h, w_, gx);
    else avgpool2_bwd_kernel<false><<<grid, 256, 0, as_stream(stream)>>>(gy, nc, h, w_, gx);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_upsample2_fwd(const float* x, int nc, int h, int w_, float* y, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, x && y && nc >= 1 && h >= 1 && w_ >= 1, "bad upsample arguments");
    upsample2_fwd_kernel<<<plane_grid(4ll * h * w_, nc), 256, 0, as_stream(stream)>>>(x, nc, h, w_, y);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_upsample2_bwd(const float* gy, int nc, int h, int w_, float* gx, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, gx && gy && nc >= 1 && h >= 1 && w_ >= 1, "bad upsample arguments");
    upsample2_bwd_kernel<<<plane_grid((long long)h * w_, nc), 256, 0, as_stream(stream)>>>(gy, nc, h, w_, gx);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_kp_blend_fwd(const float* head, const float* sparse, int n, int h, int w_, float* out,
                                       void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, head && sparse && out && n >= 1 && h >= 1 && w_ >= 1, "bad kp arguments");
    kp_blend_kernel<false><<<grid_for(train_ctx(), (long long)n * h * w_), 256, 0, as_stream(stream)>>>(
        head, sparse, n, h, w_, nullptr, out);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_kp_blend_bwd(const float* head, const float* sparse, const float* gout, int n, int h,
                                       int w_, float* ghead, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, head && sparse && gout && ghead && n >= 1 && h >= 1 && w_ >= 1, "bad kp arguments");
    kp_blend_kernel<true><<<grid_for(train_ctx(), (long long)n * h * w_), 256, 0, as_stream(stream)>>>(
        head, sparse, n, h, w_, gout, ghead);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_loss_l1grad(const float* pred, const float* target, int nc, int h, int w_, float lam,
                                      float* loss, float* gpred, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, pred && target && loss && gpred && nc >= 1 && h >= 1 && w_ >= 1, "bad loss arguments");
    FVN_CUDA(ctx, cudaMemsetAsync(loss, 0, sizeof(float), as_stream(stream)));
    const fvn_ctx* tc = train_ctx();
    const long long rows = (long long)nc * h;
    const int grid = (int)std::min<long long>(rows, 4LL * (tc->num_sms > 0 ? tc->num_sms : 148));
    loss_kernel<<<grid, 256, 0, as_stream(stream)>>>(pred, target, nc, h, w_, lam, loss, gpred);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_adam_step(float* p, const float* g, float* m, float* v, size_t n, int step, float lr,
                                    float beta1, float beta2, float eps, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, p && g && m && v && n >= 1 && step >= 1, "bad adam arguments");
    const float c1 = (float)(1.0 - pow((double)beta1, step));
    const float c2 = (float)(1.0 - pow((double)beta2, step));
    adam_kernel<<<grid_for(train_ctx(), (long long)n), 256, 0, as_stream(stream)>>>(p, g, m, v, n, lr, beta1, beta2,
                                                                                    eps, c1, c2);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

extern "C" fvn_status fvn_adam_step_dev(float* p, const float* g, float* m, float* v, size_t n, const int* step,
                                        float lr, float beta1, float beta2, float eps, void* stream) {
    fvn_ctx* ctx = nullptr;
    FVN_CHECK_ARG(ctx, p && g && m && v && step && n >= 1, "bad adam arguments");
    adam_dev_kernel<<<grid_for(train_ctx(), (long long)n), 256, 0, as_stream(stream)>>>(p, g, m, v, n, step, lr,
                                                                                        beta1, beta2, eps);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}
