// x2 bilinear up-sampling with half-pixel centres: the coarse neighbours of a
// fine sample and their weights (shared by the FP32 training kernels and the
// two-stage network's join).
#pragma once

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

}  // namespace fvn
