// Foveated sample mask and stream compaction (paper: "Sample Maps", Eq. 1-2,
// and "Stream Compaction").
//
// M(x, y) = 1 iff N(x, y) < tau(x, y).  N is the top 24 bits of a nested
// 32-bit PCG-style integer hash of (seed, frame, y, x) (the "pcg" hash of
// Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 2020), or,
// once the caller has installed a looping series of noise tiles
// (fvn_set_noise_tiles; the paper's "Noise Patterns" use 64 pre-computed
// spatio-temporal blue-noise tiles), tile[frame mod K][y mod T][x mod T].  tau
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

#include <algorithm>

#include "common.cuh"

namespace fvn {

__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

// Compact Morton (Z-order) index -> 2-D tile coordinates.
__device__ __forceinline__ void morton_decode(uint32_t m, int& tx, int& ty) {
    uint32_t x = m & 0x55555555u, y = (m >> 1) & 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    y = (y | (y >> 1)) & 0x33333333u;
    y = (y | (y >> 2)) & 0x0F0F0F0Fu;
    y = (y | (y >> 4)) & 0x00FF00FFu;
    y = (y | (y >> 8)) & 0x0000FFFFu;
    tx = (int)x;
    ty = (int)y;
}

// Each block covers a 16 x 16 pixel tile (tiles in Z-order of the block
// number, so that consecutive blocks are neighbours on screen), each warp an
// 8 x 4 sub-tile: the id list comes out in compact screen regions, which keeps
// the 32 rays of a march packet close together.
__device__ __forceinline__ void mask_tile(uint32_t block, int W, int H, uint32_t key, int f2x, int f2y, int shift,
                                          const uint32_t* __restrict__ lut, const uint32_t* __restrict__ noise,
                                          int nlog2, uint8_t* __restrict__ mask, int32_t* __restrict__ ids,
                                          int32_t* __restrict__ count) {
    __shared__ int warp_off[8];
    __shared__ int block_base;
    int tx, ty;
    morton_decode(block, tx, ty);
    if (tx * 16 >= W || ty * 16 >= H) return;   // uniform per block: the Z-order domain is a square
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x = tx * 16 + (wy & 1) * 8 + (lane & 7), y = ty * 16 + (wy >> 1) * 4 + (lane >> 3);
    const bool valid = x < W && y < H;
    bool m = false;
    if (valid) {
        const int tmask = (1 << nlog2) - 1;
        const uint32_t n24 = noise ? __ldg(noise + ((y & tmask) << nlog2) + (x & tmask))
                                   : pcg_hash((uint32_t)x + pcg_hash((uint32_t)y + key)) >> 8;
        const int dx = 2 * x + 1 - f2x, dy = 2 * y + 1 - f2y;
        const uint32_t q = (uint32_t)(dx * dx) + (uint32_t)(dy * dy);
        m = n24 < __ldg(lut + (q >> shift));
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

__global__ void __launch_bounds__(256) mask_compact_kernel(int W, int H, uint32_t key, int f2x, int f2y,
                                                           int shift, const uint32_t* __restrict__ lut,
                                                           const uint32_t* __restrict__ noise, int nlog2,
                                                           uint8_t* __restrict__ mask, int32_t* __restrict__ ids,
                                                           int32_t* __restrict__ count) {
    mask_tile(blockIdx.x, W, H, key, f2x, f2y, shift, lut, noise, nlog2, mask, ids, count);
}

// Several views in one launch: view i owns blocks [block0, next view's block0).
struct MaskView {
    int W, H;
    uint32_t key;
    int f2x, f2y, shift;
    const uint32_t* lut;
    const uint32_t* noise;   // this frame's noise tile, or NULL for the hash
    int nlog2;               // log2 of the tile side
    uint8_t* mask;
    int32_t* ids;
    int32_t* count;
    uint32_t block0;
};
struct MaskBatch {
    int n;
    MaskView v[kMaxViews];
};
static_assert(sizeof(MaskBatch) <= 4096, "batched mask arguments exceed the 4 KB parameter space");

__global__ void __launch_bounds__(256) mask_compact_batch_kernel(const __grid_constant__ MaskBatch b) {
    int i = 0;
    while (i + 1 < b.n && blockIdx.x >= b.v[i + 1].block0) ++i;
    const MaskView& m = b.v[i];
    mask_tile(blockIdx.x - m.block0, m.W, m.H, m.key, m.f2x, m.f2y, m.shift, m.lut, m.noise, m.nlog2, m.mask, m.ids,
              m.count);
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

// Per-view launch parameters: threshold table, focal point in half pixels,
// hash key and the side of the Z-ordered square of 16 x 16 tiles.
static fvn_status mask_view(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, cudaStream_t st, MaskView* mv,
                            int* side_out) {
    const LutEntry* lut = nullptr;
    fvn_status s = get_lut(ctx, w, h, fov->fovea_radius, fov->falloff_sigma, fov->p_base, st, &lut);
    if (s != FVN_OK) return s;
    int f2x = (int)floor(2.0 * (double)fov->focal_px[0] + 0.5);
    int f2y = (int)floor(2.0 * (double)fov->focal_px[1] + 0.5);
    mv->f2x = f2x < 0 ? 0 : (f2x > 2 * w ? 2 * w : f2x);
    mv->f2y = f2y < 0 ? 0 : (f2y > 2 * h ? 2 * h : f2y);
    mv->key = pcg_hash(fov->frame + pcg_hash(fov->seed));
    mv->W = w;
    mv->H = h;
    mv->shift = lut->shift;
    mv->lut = lut->d_lut;
    mv->noise = nullptr;
    mv->nlog2 = 0;
    if (ctx->d_noise) {
        mv->nlog2 = ctx->noise_log2;
        mv->noise = ctx->d_noise + ((size_t)(fov->frame % (uint32_t)ctx->noise_frames) << (2 * ctx->noise_log2));
    }
    const int tiles = std::max((w + 15) / 16, (h + 15) / 16);
    int side = 1;
    while (side < tiles) side <<= 1;
    *side_out = side;
    return FVN_OK;
}

fvn_status make_mask_impl(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, uint8_t* mask, int32_t* ids,
                          int32_t* count, cudaStream_t st) {
    MaskView mv{};
    int side = 0;
    fvn_status s = mask_view(ctx, fov, w, h, st, &mv, &side);
    if (s != FVN_OK) return s;
    FVN_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int32_t), st));
    // Z-order over a power-of-two square of 16 x 16 tiles covering the frame
    mask_compact_kernel<<<side * side, 256, 0, st>>>(w, h, mv.key, mv.f2x, mv.f2y, mv.shift, mv.lut, mv.noise,
                                                     mv.nlog2, mask, ids, count);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

fvn_status make_mask_batch_impl(fvn_ctx* ctx, const fvn_foveation* const* fov, const int* w, const int* h,
                                uint8_t* const* mask, int32_t* const* ids, int32_t* counts, int n,
                                cudaStream_t st) {
    if (n < 1 || n > kMaxViews) return set_error(ctx, FVN_ERR_ARG, "%d views (1..%d)", n, kMaxViews);
    MaskBatch b{};
    b.n = n;
    unsigned long long blocks = 0;
    for (int i = 0; i < n; ++i) {
        int side = 0;
        fvn_status s = mask_view(ctx, fov[i], w[i], h[i], st, &b.v[i], &side);
        if (s != FVN_OK) return s;
        b.v[i].mask = mask[i];
        b.v[i].ids = ids[i];
        b.v[i].count = counts + i;
        b.v[i].block0 = (uint32_t)blocks;
        blocks += (unsigned long long)side * side;
    }
    if (blocks >= (1ull << 31)) return set_error(ctx, FVN_ERR_ARG, "batch too large for one mask launch");
    FVN_CUDA(ctx, cudaMemsetAsync(counts, 0, n * sizeof(int32_t), st));
    mask_compact_batch_kernel<<<(unsigned)blocks, 256, 0, st>>>(b);
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

extern "C" fvn_status fvn_set_noise_tiles(fvn_ctx* ctx, const uint32_t* tiles, int tile, int frames) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    if (!tiles) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());   // masks already queued may still read the tiles
        cudaFree(ctx->d_noise);
        ctx->d_noise = nullptr;
        ctx->noise_log2 = ctx->noise_frames = 0;
        return FVN_OK;
    }
    int lg = 0;
    while ((1 << lg) < tile && lg < 30) ++lg;
    FVN_CHECK_ARG(ctx, tile >= 16 && tile <= 256 && (1 << lg) == tile, "tile side %d: a power of two in [16, 256]",
                  tile);
    FVN_CHECK_ARG(ctx, frames >= 1 && frames <= 256, "%d tiles (1..256)", frames);
    const size_t n = (size_t)frames * tile * tile;
    for (size_t i = 0; i < n; ++i)
        FVN_CHECK_ARG(ctx, tiles[i] < (1u << 24), "noise value %u at %zu is not below 2^24", tiles[i], i);
    FVN_CUDA(ctx, cudaDeviceSynchronize());
    cudaFree(ctx->d_noise);
    ctx->d_noise = nullptr;
    ctx->noise_log2 = ctx->noise_frames = 0;
    uint32_t* d = nullptr;
    FVN_CUDA(ctx, cudaMalloc(&d, n * sizeof(uint32_t)));
    const cudaError_t e = cudaMemcpy(d, tiles, n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return set_error(ctx, FVN_ERR_CUDA, "copying the noise tiles: %s", cudaGetErrorString(e));
    }
    ctx->d_noise = d;
    ctx->noise_log2 = lg;
    ctx->noise_frames = frames;
    return FVN_OK;
}

// ---------------------------------------------------------------------------
// Error estimate for the denser-mask fallback (not in the paper).  A sparse
// probe set -- pixels whose second hash falls below 1/256 and that the mask
// left out -- is ray-marched as well; the reconstruction's error at those
// pixels estimates the frame's PSNR.  When the estimate is below a threshold
// the frame is rendered again with the periphery density doubled.
// ---------------------------------------------------------------------------
namespace fvn {

constexpr uint32_t kProbeSalt = 0x9E3779B9u;     // second, independent hash key
constexpr uint32_t kProbeThreshold = 1u << 16;   // N2 < 2^24 / 256

__global__ void __launch_bounds__(256) probe_compact_kernel(int W, int H, uint32_t key2,
                                                            const uint8_t* __restrict__ mask,
                                                            int32_t* __restrict__ ids, int32_t* __restrict__ count) {
    __shared__ int warp_off[8];
    __shared__ int block_base;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane, y = blockIdx.y * 8 + wy;
    bool m = false;
    if (x < W && y < H) {
        const uint32_t h = pcg_hash((uint32_t)x + pcg_hash((uint32_t)y + key2));
        m = (h >> 8) < kProbeThreshold && mask[(size_t)y * W + x] == 0;
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

// sum over the probes of the squared error of the clamped RGB (double)
__global__ void probe_error_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ count,
                                   const float* __restrict__ rgb, const float* __restrict__ probe, long long plane,
                                   double* __restrict__ acc) {
    const int n = *count;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = ids[i];
        for (int c = 0; c < 3; ++c) {
            const float d = __saturatef(rgb[c * plane + p]) - __saturatef(probe[c * plane + p]);
            s += (double)d * d;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(acc, s);
}

uint32_t probe_key(const fvn_foveation* f) { return pcg_hash(f->frame + pcg_hash(f->seed ^ kProbeSalt)); }

fvn_status probe_compact(fvn_ctx* ctx, int w, int h, uint32_t key2, const uint8_t* mask, int32_t* ids,
                         int32_t* count, cudaStream_t st) {
    dim3 grid((w + 31) / 32, (h + 7) / 8);
    probe_compact_kernel<<<grid, 256, 0, st>>>(w, h, key2, mask, ids, count);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

fvn_status probe_error(fvn_ctx* ctx, const int32_t* ids, const int32_t* count, const float* rgb, const float* probe,
                       long long plane, double* acc, cudaStream_t st) {
    probe_error_kernel<<<4 * ctx->num_sms, 256, 0, st>>>(ids, count, rgb, probe, plane, acc);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_render_adaptive(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf,
                                          const fvn_camera* cam, const fvn_foveation* fov,
                                          const fvn_march_params* mp, int precision, float min_psnr_db,
                                          int max_levels, float* rgb, int* level_out, float* psnr_out,
                                          void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, fov != nullptr && cam != nullptr && rgb != nullptr, "null argument");
    FVN_CHECK_ARG(ctx, max_levels >= 0 && max_levels <= 8, "max_levels must be in [0, 8]");
    FVN_CHECK_ARG(ctx, cam->width >= 1 && cam->height >= 1 && cam->width <= kMaxSide && cam->height <= kMaxSide,
                  "camera size outside [1, %d]", kMaxSide);
    cudaStream_t st = as_stream(stream);
    const int w = cam->width, h = cam->height;
    const size_t npix = (size_t)w * h;
    ProbeWorkspace& pw = ctx->probe_ws;
    if (pw.w != w || pw.h != h) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(pw.ids);
        cudaFree(pw.count);
        cudaFree(pw.rgbam);
        cudaFree(pw.acc);
        pw = ProbeWorkspace();
        FVN_CUDA(ctx, cudaMalloc(&pw.ids, npix * sizeof(int32_t)));
        FVN_CUDA(ctx, cudaMalloc(&pw.count, sizeof(int32_t)));
        FVN_CUDA(ctx, cudaMalloc(&pw.rgbam, 5 * npix * sizeof(float)));
        FVN_CUDA(ctx, cudaMalloc(&pw.acc, sizeof(double)));
        pw.w = w;
        pw.h = h;
    }
    fvn_foveation f = *fov;
    const uint32_t key2 = probe_key(fov);
    float est = 0.f;
    int level = 0;
    for (;; ++level) {
        fvn_status s = fvn_render(ctx, vol, tf, cam, &f, mp, precision, rgb, nullptr, stream);
        if (s != FVN_OK) return s;
        // probes: outside this level's mask
        FVN_CUDA(ctx, cudaMemsetAsync(pw.count, 0, sizeof(int32_t), st));
        FVN_CUDA(ctx, cudaMemsetAsync(pw.acc, 0, sizeof(double), st));
        if ((s = probe_compact(ctx, w, h, key2, ctx->render_ws.mask, pw.ids, pw.count, st)) != FVN_OK) return s;
        if ((s = march_impl(ctx, vol, tf, cam, mp, pw.ids, pw.count, pw.rgbam, nullptr, st)) != FVN_OK) return s;
        if ((s = probe_error(ctx, pw.ids, pw.count, rgb, pw.rgbam, (long long)npix, pw.acc, st)) != FVN_OK) return s;
        double sum = 0.0;
        int n = 0;
        FVN_CUDA(ctx, cudaMemcpyAsync(&sum, pw.acc, sizeof(double), cudaMemcpyDeviceToHost, st));
        FVN_CUDA(ctx, cudaMemcpyAsync(&n, pw.count, sizeof(int), cudaMemcpyDeviceToHost, st));
        FVN_CUDA(ctx, cudaStreamSynchronize(st));
        est = (n == 0 || sum == 0.0) ? 99.0f : (float)(-10.0 * log10(sum / (3.0 * n)));
        if (est >= min_psnr_db || level >= max_levels || f.p_base >= 1.0f) break;
        f.p_base = std::min(1.0f, 2.0f * f.p_base);
    }
    if (level_out) *level_out = level;
    if (psnr_out) *psnr_out = est;
    return FVN_OK;
}
