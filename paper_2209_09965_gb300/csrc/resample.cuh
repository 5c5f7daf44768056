// x2 bilinear up-sampling with half-pixel centres: the coarse neighbours of a
// fine sample and their weights (shared by the FP32 training kernels and the
// two-stage network's join).
#pragma once

#include <cuda_fp16.h>

namespace fvn {

// coarse neighbours i0, i1 and the weight t of i1 for fine sample o of a side
// of n coarse samples (source (o + 0.5)/2 - 0.5 clamped at 0, upper
// neighbour clamped to n - 1)
__device__ __forceinline__ void up_src(int o, int n, int& i0, int& i1, float& t) {
    float s = fmaxf((o + 0.5f) * 0.5f - 0.5f, 0.f);
    i0 = (int)s;
    t = s - i0;
    i1 = min(i0 + 1, n - 1);
}

// weight of coarse index i in fine sample o
__device__ __forceinline__ float up_weight(int o, int i, int n) {
    int i0, i1;
    float t;
    up_src(o, n, i0, i1, t);
    return (i0 == i ? 1.f - t : 0.f) + (i1 == i ? t : 0.f);
}

// FP16 chunk (8 channels) <-> FP32
__device__ __forceinline__ void h8_to_f(uint4 u, float* f) {
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __half22float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 f_to_h8(const float* f) {
    uint4 u;
    __half2* h = reinterpret_cast<__half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

// (1 - t) a + t b, rounded as written (no contraction into an FMA), so that
// every kernel that up-samples FP16 chunks gets the same bits
__device__ __forceinline__ float up_lerp(float a, float b, float t) {
    return __fadd_rn(__fmul_rn(1.f - t, a), __fmul_rn(t, b));
}

// x interpolation of one coarse FP16 chunk pair (8 channels)
__device__ __forceinline__ void up_xlerp8(uint4 u0, uint4 u1, float t, float* o) {
    float a[8], b[8];
    h8_to_f(u0, a);
    h8_to_f(u1, b);
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = up_lerp(a[j], b[j], t);
}

// y interpolation of two x-interpolated rows, packed to an FP16 chunk
__device__ __forceinline__ uint4 up_ylerp8(const float* top, const float* bot, float t) {
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = up_lerp(top[j], bot[j], t);
    return f_to_h8(o);
}

}  // namespace fvn
