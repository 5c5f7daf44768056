// Foveated sample mask and stream compaction (paper: "Sample Maps", Eq. 1-2,
// and "Stream Compaction").
//
// M(x, y) = 1 iff N(x, y) < tau(x, y).  N is the top 24 bits of a nested
// 32-bit PCG-style integer hash of (seed, frame, y, x) (the "pcg" hash of
// Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 2020).  tau
// comes from a 16384-entry table of floor(tau 2^24) indexed by the squared
// half-pixel distance to the focal point shifted right so the largest
// distance of the frame fits; the table is built on the host in float64 from
// Eq. 1-2 (fovea of radius r0 with tau = 1, Gaussian falloff of width s to
// the periphery density P_b; distances in units of the half diagonal), so the
// per-pixel decision is integer-only and bit-exact.
//
// One fused kernel: each 256-thread block covers a 32 x 8 pixel tile, writes
// the mask bytes, counts its sampled pixels with warp ballots, reserves a
// range of the id list with one atomic and writes the ids.
#include <math.h>

#include "common.cuh"

namespace fvn {

__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

__global__ void __launch_bounds__(256) mask_compact_kernel(int W, int H, uint32_t key, int f2x, int f2y,
                                                           int shift, const uint32_t* __restrict__ lut,
                                                           uint8_t* __restrict__ mask, int32_t* __restrict__ ids,
                                                           int32_t* __restrict__ count) {
    __shared__ int warp_off[8];
    __shared__ int block_base;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane, y = blockIdx.y * 8 + wy;
    const bool valid = x < W && y < H;
    bool m = false;
    if (valid) {
        const uint32_t h = pcg_hash((uint32_t)x + pcg_hash((uint32_t)y + key));
        const int dx = 2 * x + 1 - f2x, dy = 2 * y + 1 - f2y;
        const uint32_t q = (uint32_t)(dx * dx) + (uint32_t)(dy * dy);
        m = (h >> 8) < __ldg(lut + (q >> shift));
        mask[(size_t)y * W + x] = (uint8_t)m;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) warp_off[wy] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int i = 0; i < 8; ++i) {
            int c = warp_off[i];
            warp_off[i] = tot;
            tot += c;
        }
        block_base = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    if (m) ids[block_base + warp_off[wy] + __popc(bal & ((1u << lane) - 1u))] = y * W + x;
}

static int lut_shift(int W, int H) {
    const uint64_t qmax = 4ull * (uint64_t)W * W + 4ull * (uint64_t)H * H;
    int s = 0;
    while ((qmax >> s) >= (uint64_t)kLutBins) ++s;
    return s;
}

// Eq. 2 with the falloff of Eq. 1 read as a Gaussian of the distance beyond
// the fovea; d in units of the half diagonal.
static double tau_at(double d, double r0, double s, double pb) {
    double pf;
    if (d <= r0) pf = 1.0;
    else if (s <= 0.0) pf = 0.0;
    else {
        double z = (d - r0) / s;
        pf = exp(-0.5 * z * z);
    }
    return (1.0 - pb) * pf + pb;
}

static void fill_lut(uint32_t* t, int W, int H, int shift, double r0, double s, double pb) {
    const double big_r = 0.5 * sqrt((double)W * W + (double)H * H);
    const double one24 = 16777216.0;
    for (int b = 0; b < kLutBins; ++b) {
        double qc = ((double)b + 0.5) * (double)(1u << shift);
        double d = sqrt(qc) * 0.5 / big_r;
        double tau = tau_at(d, r0, s, pb);
        uint32_t v;
        if (tau >= 1.0) v = 1u << 24;
        else if (tau <= 0.0) v = 0;
        else v = (uint32_t)floor(tau * one24);
        t[b] = v;
    }
}

static fvn_status get_lut(fvn_ctx* ctx, int W, int H, float r0, float s, float pb, cudaStream_t st,
                          const LutEntry** out) {
    ++ctx->lut_clock;
    LutEntry* slot = nullptr;
    for (auto& e : ctx->lut)
        if (e.valid && e.w == W && e.h == H && e.r0 == r0 && e.s == s && e.pb == pb) {
            e.last_use = ctx->lut_clock;
            *out = &e;
            return FVN_OK;
        }
    for (auto& e : ctx->lut)
        if (!e.valid) { slot = &e; break; }
    if (!slot) {
        // Evict the least recently used profile; kernels already queued may
        // still read it, so wait for the device first.
        slot = &ctx->lut[0];
        for (auto& e : ctx->lut)
            if (e.last_use < slot->last_use) slot = &e;
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        slot->valid = false;
    }
    if (!slot->d_lut) FVN_CUDA(ctx, cudaMalloc(&slot->d_lut, kLutBins * sizeof(uint32_t)));
    if (!slot->h_lut) FVN_CUDA(ctx, cudaMallocHost(&slot->h_lut, kLutBins * sizeof(uint32_t)));
    slot->shift = lut_shift(W, H);
    fill_lut(slot->h_lut, W, H, slot->shift, r0, s, pb);
    FVN_CUDA(ctx, cudaMemcpyAsync(slot->d_lut, slot->h_lut, kLutBins * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    slot->w = W;
    slot->h = H;
    slot->r0 = r0;
    slot->s = s;
    slot->pb = pb;
    slot->valid = true;
    slot->last_use = ctx->lut_clock;
    *out = slot;
    return FVN_OK;
}

fvn_status make_mask_impl(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, uint8_t* mask, int32_t* ids,
                          int32_t* count, cudaStream_t st) {
    const LutEntry* lut = nullptr;
    fvn_status s = get_lut(ctx, w, h, fov->fovea_radius, fov->falloff_sigma, fov->p_base, st, &lut);
    if (s != FVN_OK) return s;
    int f2x = (int)floor(2.0 * (double)fov->focal_px[0] + 0.5);
    int f2y = (int)floor(2.0 * (double)fov->focal_px[1] + 0.5);
    f2x = f2x < 0 ? 0 : (f2x > 2 * w ? 2 * w : f2x);
    f2y = f2y < 0 ? 0 : (f2y > 2 * h ? 2 * h : f2y);
    const uint32_t key = pcg_hash(fov->frame + pcg_hash(fov->seed));
    FVN_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int32_t), st));
    dim3 grid((w + 31) / 32, (h + 7) / 8);
    mask_compact_kernel<<<grid, 256, 0, st>>>(w, h, key, f2x, f2y, lut->shift, lut->d_lut, mask, ids, count);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_make_mask(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, uint8_t* mask,
                                    int32_t* ids, int32_t* count, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, fov != nullptr, "foveation is NULL");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    FVN_CHECK_ARG(ctx, mask && ids && count, "mask, ids and count must be device pointers");
    FVN_CHECK_ARG(ctx, isfinite(fov->focal_px[0]) && isfinite(fov->focal_px[1]), "focal point is not finite");
    FVN_CHECK_ARG(ctx, fov->fovea_radius >= 0.f && fov->falloff_sigma >= 0.f && fov->p_base >= 0.f &&
                           fov->p_base <= 1.f && isfinite(fov->fovea_radius) && isfinite(fov->falloff_sigma),
                  "foveation radius / falloff must be >= 0 and p_base in [0, 1]");
    return make_mask_impl(ctx, fov, w, h, mask, ids, count, as_stream(stream));
}
