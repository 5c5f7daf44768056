// The training step's output stage, fused: the 1x1 head convolution (16 ->
// 29 channels: direct RGB, 25 kernel logits, blend logit) and the kernel
// prediction + blend of the paper's "Kernel Prediction" subsection (one 5x5
// softmax kernel over the sparse samples, normalised by the mask it covers,
// blended with the direct prediction by a sigmoid weight).
//
// Forward, per pixel: head = W x + b from the 16 decoder channels, written
// out for the backward pass, and the blended RGB.
// Backward, per pixel: dL/dhead from dL/dout, dL/dx = W^T dL/dhead, and the
// head's weight and bias gradients -- sum over pixels of dL/dhead x^T --
// accumulated as register-blocked outer products: each warp owns 32 staged
// pixels of a 256-pixel tile, lane (cb, kb) a 4 x 4 block of (output,
// input) channels; at the end the CTA's warps are summed in shared memory
// and added to the FP32 gradients with one atomic per weight per CTA.
// dL/dhead itself never reaches memory.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace fvn {
namespace {

constexpr int kHeadIn = 16;    // decoder channels
constexpr int kHeadOut = 29;   // 3 direct RGB + 25 kernel logits + 1 blend logit
constexpr int kHeadThreads = 256;

// Mask and sparse colour of tap q of pixel (y, x); zero outside the frame.
__device__ __forceinline__ float kp_tap(const float* sp, long long hw, int h, int w_, int y, int x, int q, float c[3]) {
    const int yy = y + q / 5 - 2, xx = x + q % 5 - 2;
    c[0] = c[1] = c[2] = 0.f;
    if (yy < 0 || xx < 0 || yy >= h || xx >= w_) return 0.f;
    const long long o = (long long)yy * w_ + xx;
    c[0] = __ldg(sp + o);
    c[1] = __ldg(sp + hw + o);
    c[2] = __ldg(sp + 2 * hw + o);
    return __ldg(sp + 4 * hw + o);
}

// Softmax kernel weights over the 25 taps (from the logits hv[3 .. 27]), the
// normaliser den = sum_q w_q M_q and the filtered colour kp = num / den
// (the direct prediction hv[0 .. 2] where den < 1e-12).
struct KpPixel {
    float w[25];
    float den, kp[3];
    bool valid;
};

__device__ __forceinline__ void kp_pixel(const float* hv, const float* sp, long long hw, int h, int w_, int y, int x,
                                         KpPixel& k) {
    float mx = -INFINITY;
#pragma unroll
    for (int q = 0; q < 25; ++q) mx = fmaxf(mx, hv[3 + q]);
    float es = 0.f;
#pragma unroll
    for (int q = 0; q < 25; ++q) {
        k.w[q] = expf(hv[3 + q] - mx);
        es += k.w[q];
    }
    const float inv = 1.f / es;
    float num[3] = {0.f, 0.f, 0.f};
    k.den = 0.f;
#pragma unroll
    for (int q = 0; q < 25; ++q) {
        k.w[q] *= inv;
        float c[3];
        const float wm = k.w[q] * kp_tap(sp, hw, h, w_, y, x, q, c);
        k.den += wm;
        num[0] = fmaf(wm, c[0], num[0]);
        num[1] = fmaf(wm, c[1], num[1]);
        num[2] = fmaf(wm, c[2], num[2]);
    }
    k.valid = k.den >= 1e-12f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) k.kp[ch] = k.valid ? num[ch] / k.den : hv[ch];
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + expf(-z)); }

// head = W x + b (written for the backward pass) and out = a kp + (1 - a) rd
__global__ void __launch_bounds__(kHeadThreads)
    head_kp_fwd_kernel(const float* __restrict__ x, long long n, int h, int w_, const float* __restrict__ wt,
                       const float* __restrict__ bias, const float* __restrict__ sparse, float* __restrict__ head,
                       float* __restrict__ out) {
    __shared__ float sw[kHeadOut * kHeadIn], sb[kHeadOut];
    for (int i = threadIdx.x; i < kHeadOut * kHeadIn; i += blockDim.x) sw[i] = wt[i];
    if (threadIdx.x < kHeadOut) sb[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const long long hw = (long long)h * w_, total = n * hw;
    for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < total;
         P += (long long)gridDim.x * blockDim.x) {
        const long long img = P / hw;
        const int r = (int)(P - img * hw), y = r / w_, xq = r - y * w_;
        float xv[kHeadIn], hv[kHeadOut];
#pragma unroll
        for (int ci = 0; ci < kHeadIn; ++ci) xv[ci] = __ldg(x + (img * kHeadIn + ci) * hw + r);
#pragma unroll
        for (int co = 0; co < kHeadOut; ++co) {
            float s = sb[co];
#pragma unroll
            for (int ci = 0; ci < kHeadIn; ++ci) s = fmaf(sw[co * kHeadIn + ci], xv[ci], s);
            hv[co] = s;
            head[(img * kHeadOut + co) * hw + r] = s;
        }
        KpPixel k;
        kp_pixel(hv, sparse + img * 5 * hw, hw, h, w_, y, xq, k);
        const float a = sigmoidf(hv[28]);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) out[(img * 3 + ch) * hw + r] = a * k.kp[ch] + (1.f - a) * hv[ch];
    }
}

// shared memory of the backward kernel
constexpr size_t kBwdDh = (size_t)kHeadThreads * 32 * 4;   // dL/dhead of the tile, [pixel][32] (29 used)
constexpr size_t kBwdX = (size_t)kHeadThreads * 16 * 4;    // the tile's input, [pixel][16]
constexpr size_t kBwdBytes = kBwdDh + kBwdX + kHeadOut * kHeadIn * 4;

__global__ void __launch_bounds__(kHeadThreads, 2)
    head_kp_bwd_kernel(const float* __restrict__ x, const float* __restrict__ head, const float* __restrict__ sparse,
                       const float* __restrict__ wt, const float* __restrict__ gout, long long n, int h, int w_,
                       float* __restrict__ gx, float* __restrict__ gw, float* __restrict__ gb) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4* sdh = reinterpret_cast<float4*>(smem);                 // [256][8]
    float4* sx = reinterpret_cast<float4*>(smem + kBwdDh);         // [256][4]
    float* sw = reinterpret_cast<float*>(smem + kBwdDh + kBwdX);   // [29][16]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cb = lane >> 2, kb = lane & 3;   // this lane's output channels 4 cb .., input channels 4 kb ..
    for (int i = tid; i < kHeadOut * kHeadIn; i += blockDim.x) sw[i] = wt[i];
    __syncthreads();
    const long long hw = (long long)h * w_, total = n * hw;
    float acc[4][4] = {}, accb[4] = {};
    for (long long T = (long long)blockIdx.x * kHeadThreads; T < total; T += (long long)gridDim.x * kHeadThreads) {
        const long long P = T + tid;
        float dh[32] = {}, xv[kHeadIn] = {};
        if (P < total) {
            const long long img = P / hw;
            const int r = (int)(P - img * hw), y = r / w_, xq = r - y * w_;
            const float* sp = sparse + img * 5 * hw;
            float hv[kHeadOut];
#pragma unroll
            for (int co = 0; co < kHeadOut; ++co) hv[co] = __ldg(head + (img * kHeadOut + co) * hw + r);
            KpPixel k;
            kp_pixel(hv, sp, hw, h, w_, y, xq, k);
            const float a = sigmoidf(hv[28]);
            float g[3], ga = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                g[ch] = __ldg(gout + (img * 3 + ch) * hw + r);
                ga += g[ch] * (k.kp[ch] - hv[ch]);
                dh[ch] = g[ch] * (1.f - a) + (k.valid ? 0.f : g[ch] * a);
            }
            dh[28] = ga * a * (1.f - a);
            // d out / d w_q through kp = num / den, then through the softmax
            float dw[25], sdw = 0.f;
#pragma unroll
            for (int q = 0; q < 25; ++q) {
                dw[q] = 0.f;
                if (k.valid) {
                    float c[3];
                    const float m = kp_tap(sp, hw, h, w_, y, xq, q, c);
                    float s = 0.f;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) s += g[ch] * (c[ch] - k.kp[ch]);
                    dw[q] = a * m * s / k.den;
                }
                sdw += k.w[q] * dw[q];
            }
#pragma unroll
            for (int q = 0; q < 25; ++q) dh[3 + q] = k.w[q] * (dw[q] - sdw);
            // dL/dx = W^T dL/dhead
#pragma unroll
            for (int ci = 0; ci < kHeadIn; ++ci) {
                xv[ci] = __ldg(x + (img * kHeadIn + ci) * hw + r);
                float s = 0.f;
#pragma unroll
                for (int co = 0; co < kHeadOut; ++co) s = fmaf(sw[co * kHeadIn + ci], dh[co], s);
                gx[(img * kHeadIn + ci) * hw + r] = s;
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) sdh[tid * 8 + j] = make_float4(dh[4 * j], dh[4 * j + 1], dh[4 * j + 2], dh[4 * j + 3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) sx[tid * 4 + j] = make_float4(xv[4 * j], xv[4 * j + 1], xv[4 * j + 2], xv[4 * j + 3]);
        __syncthreads();
        // this warp's 32 pixels into the lane's 4 x 4 block (and the bias sums)
#pragma unroll 4
        for (int p = warp * 32; p < warp * 32 + 32; ++p) {
            const float4 d4 = sdh[p * 8 + cb], x4 = sx[p * 4 + kb];
            const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, xw[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                accb[i] += dv[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], xw[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    // the warps' blocks summed in shared memory, one atomic per weight
    float* red = reinterpret_cast<float*>(smem);   // [8 warps][32 lanes][20]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(warp * 32 + lane) * 20 + i * 4 + j] = acc[i][j];
        red[(warp * 32 + lane) * 20 + 16 + i] = accb[i];
    }
    __syncthreads();
    for (int o = tid; o < kHeadOut * kHeadIn + kHeadOut; o += blockDim.x) {
        int L, e;
        if (o < kHeadOut * kHeadIn) {
            const int co = o / kHeadIn, ci = o - co * kHeadIn;
            L = (co >> 2) * 4 + (ci >> 2);
            e = (co & 3) * 4 + (ci & 3);
        } else {
            const int co = o - kHeadOut * kHeadIn;
            L = (co >> 2) * 4;
            e = 16 + (co & 3);
        }
        float s = 0.f;
        for (int w = 0; w < kHeadThreads / 32; ++w) s += red[(w * 32 + L) * 20 + e];
        atomicAdd(o < kHeadOut * kHeadIn ? gw + o : gb + (o - kHeadOut * kHeadIn), s);
    }
}

}  // namespace
}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_head_kp_fwd(const float* x, int n, int h, int w_, const float* w, const float* b,
                                      const float* sparse, float* head, float* out, void* stream) {
    FVN_CHECK_ARG(nullptr, x && w && b && sparse && head && out, "null tensor");
    FVN_CHECK_ARG(nullptr, n >= 1 && h >= 1 && w_ >= 1, "bad sizes");
    int dev = 0, sms = 0;
    FVN_CUDA(nullptr, cudaGetDevice(&dev));
    FVN_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long total = (long long)n * h * w_;
    const int grid = (int)std::max(1LL, std::min((total + kHeadThreads - 1) / kHeadThreads, 16LL * sms));
    head_kp_fwd_kernel<<<grid, kHeadThreads, 0, as_stream(stream)>>>(x, n, h, w_, w, b, sparse, head, out);
    FVN_LAUNCH_CHECK(nullptr);
    return FVN_OK;
}

extern "C" fvn_status fvn_head_kp_bwd(const float* x, const float* head, const float* sparse, const float* w,
                                      const float* gout, int n, int h, int w_, float* gx, float* gw, float* gb,
                                      void* stream) {
    FVN_CHECK_ARG(nullptr, x && head && sparse && w && gout && gx && gw && gb, "null tensor");
    FVN_CHECK_ARG(nullptr, n >= 1 && h >= 1 && w_ >= 1, "bad sizes");
    static std::atomic<unsigned long long> configured{0};
    int dev = 0, sms = 0, per_sm = 0;
    FVN_CUDA(nullptr, cudaGetDevice(&dev));
    FVN_CUDA(nullptr, opt_in_smem(dev, head_kp_bwd_kernel, (int)kBwdBytes, configured));
    FVN_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FVN_CUDA(nullptr, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, head_kp_bwd_kernel, kHeadThreads,
                                                                     kBwdBytes));
    const long long total = (long long)n * h * w_;
    // persistent: every CTA adds its weight-gradient partial sums once
    const int grid = (int)std::max(1LL, std::min((total + kHeadThreads - 1) / kHeadThreads,
                                                  (long long)sms * std::max(1, per_sm)));
    cudaStream_t st = as_stream(stream);
    FVN_CUDA(nullptr, cudaMemsetAsync(gw, 0, sizeof(float) * kHeadOut * kHeadIn, st));
    FVN_CUDA(nullptr, cudaMemsetAsync(gb, 0, sizeof(float) * kHeadOut, st));
    head_kp_bwd_kernel<<<grid, kHeadThreads, kBwdBytes, st>>>(x, head, sparse, w, gout, n, h, w_, gx, gw, gb);
    FVN_LAUNCH_CHECK(nullptr);
    return FVN_OK;
}
