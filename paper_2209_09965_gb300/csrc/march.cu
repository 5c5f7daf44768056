// Emission-absorption ray march, dense or through the compacted pixel list
// (paper: "Foveated Rendering" and "Rendering": one ray per valid pixel of the
// compacted buffer, results written back to their full-frame positions).
//
// Persistent kernel: every warp repeatedly takes a packet of 32 rays from a
// global ticket counter, so lanes stay busy however uneven the ray lengths
// and however sparse the mask.  Dense rays are numbered in 8 x 4 pixel
// blocks, sparse rays follow the id list (written tile by tile by the mask
// kernel), so the 32 rays of a packet are neighbours on screen and their
// trilinear gathers share cache lines.  The transfer function sits in shared
// memory; the volume is read through the read-only data path (a 256^3 float
// volume is 64 MiB and stays resident in the 126 MB L2).
//
// Per sample (FP32): trilinear fetch between voxel centres with clamp to
// edge, TF lookup at v (n - 1), optional Phong headlight shading from central
// differences at +-1 voxel (only for samples with alpha > 0, which are the
// only ones that contribute), C += (1 - A) a c, A += (1 - A) a, stop once
// A >= term_alpha.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace fvn {

struct MarchArgs {
    const void* vol;
    int nx, ny, nz;
    int ntf;
    const float4* tf;
    float ox, oy, oz;                 // eye in voxel units
    float fx, fy, fz, rx, ry, rz, ux, uy, uz;
    float tan_x, tan_y;               // tan(fov/2) * W/H, tan(fov/2)
    float two_over_w, two_over_h;
    int W, H;
    float dt, term;
    float bg0, bg1, bg2;
    const int32_t* ids;
    const int32_t* count;
    int n_dense;                      // rays of the dense numbering (multiple of 32)
    int tiles_x;                      // 8-pixel-wide blocks per row (dense numbering)
    float* rgbam;
    long long plane;
    unsigned long long* nsamples;
    int* ticket;
};

template <typename T>
__device__ __forceinline__ float load_norm(const T* p);
template <>
__device__ __forceinline__ float load_norm<float>(const float* p) {
    return __saturatef(__ldg(p));
}
template <>
__device__ __forceinline__ float load_norm<uint8_t>(const uint8_t* p) {
    return (float)__ldg(p) * (1.0f / 255.0f);
}
template <>
__device__ __forceinline__ float load_norm<uint16_t>(const uint16_t* p) {
    return (float)__ldg(p) * (1.0f / 65535.0f);
}
template <>
__device__ __forceinline__ float load_norm<__half>(const __half* p) {
    return __saturatef(__half2float(__ldg(p)));
}

template <typename T, typename I>
__device__ __forceinline__ float trilinear(const T* __restrict__ v, int nx, int ny, int nz, float x, float y,
                                           float z) {
    const float ux = x - 0.5f, uy = y - 0.5f, uz = z - 0.5f;
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    const float tx = ux - fx, ty = uy - fy, tz = uz - fz;
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const int x0 = min(max(ix, 0), nx - 1), x1 = min(max(ix + 1, 0), nx - 1);
    const int y0 = min(max(iy, 0), ny - 1), y1 = min(max(iy + 1, 0), ny - 1);
    const int z0 = min(max(iz, 0), nz - 1), z1 = min(max(iz + 1, 0), nz - 1);
    const I r00 = ((I)z0 * ny + y0) * nx, r01 = ((I)z0 * ny + y1) * nx;
    const I r10 = ((I)z1 * ny + y0) * nx, r11 = ((I)z1 * ny + y1) * nx;
    const float v000 = load_norm(v + r00 + x0), v001 = load_norm(v + r00 + x1);
    const float v010 = load_norm(v + r01 + x0), v011 = load_norm(v + r01 + x1);
    const float v100 = load_norm(v + r10 + x0), v101 = load_norm(v + r10 + x1);
    const float v110 = load_norm(v + r11 + x0), v111 = load_norm(v + r11 + x1);
    const float a00 = fmaf(tx, v001 - v000, v000), a01 = fmaf(tx, v011 - v010, v010);
    const float a10 = fmaf(tx, v101 - v100, v100), a11 = fmaf(tx, v111 - v110, v110);
    const float b0 = fmaf(ty, a01 - a00, a00), b1 = fmaf(ty, a11 - a10, a10);
    return fmaf(tz, b1 - b0, b0);
}

template <typename T, typename I, bool SHADE>
__global__ void __launch_bounds__(128) march_kernel(MarchArgs a) {
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < a.ntf; i += blockDim.x) s_tf[i] = a.tf[i];
    __syncthreads();
    const T* __restrict__ vol = static_cast<const T*>(a.vol);
    const int lane = threadIdx.x & 31;
    const int npix = a.W * a.H;
    // the id list never holds more than one entry per pixel
    const int nrays = a.ids ? min(max(*a.count, 0), npix) : a.n_dense;
    const float fnx = (float)a.nx, fny = (float)a.ny, fnz = (float)a.nz;
    const float tfmax = (float)(a.ntf - 1);
    unsigned long long my_samples = 0;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.ticket, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nrays) break;
        const int r = base + lane;
        int pix = -1, px = 0, py = 0;
        if (a.ids) {
            if (r < nrays) {
                pix = __ldg(a.ids + r);
                if ((unsigned)pix >= (unsigned)npix) pix = -1;   // ignore ids outside the frame
                py = pix / a.W;
                px = pix - py * a.W;
            }
        } else {
            const int tile = r >> 5;
            const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
            px = tx * 8 + (lane & 7);
            py = ty * 4 + (lane >> 3);
            if (px < a.W && py < a.H) pix = py * a.W + px;
        }
        if (pix < 0) continue;

        const float sx = ((px + 0.5f) * a.two_over_w - 1.0f) * a.tan_x;
        const float sy = (1.0f - (py + 0.5f) * a.two_over_h) * a.tan_y;
        float dx = a.fx + sx * a.rx + sy * a.ux;
        float dy = a.fy + sx * a.ry + sy * a.uy;
        float dz = a.fz + sx * a.rz + sy * a.uz;
        const float len = sqrtf(dx * dx + dy * dy + dz * dz);
        dx /= len;
        dy /= len;
        dz /= len;

        float tn = -INFINITY, tfar = INFINITY;
        bool miss = false;
        {
            const float o[3] = {a.ox, a.oy, a.oz};
            const float d[3] = {dx, dy, dz};
            const float n[3] = {fnx, fny, fnz};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (d[ax] == 0.0f) {
                    if (o[ax] < 0.0f || o[ax] > n[ax]) miss = true;
                } else {
                    float t0 = (0.0f - o[ax]) / d[ax];
                    float t1 = (n[ax] - o[ax]) / d[ax];
                    if (t0 > t1) {
                        const float s = t0;
                        t0 = t1;
                        t1 = s;
                    }
                    tn = fmaxf(tn, t0);
                    tfar = fminf(tfar, t1);
                }
            }
        }
        const float tnear = fmaxf(tn, 0.0f);
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
        int k = 0;
        if (!miss && tnear < tfar) {
            for (;; ++k) {
                const float t = fmaf((float)k, a.dt, tnear);
                if (t >= tfar) break;
                const float x = fmaf(t, dx, a.ox), y = fmaf(t, dy, a.oy), z = fmaf(t, dz, a.oz);
                const float v = trilinear<T, I>(vol, a.nx, a.ny, a.nz, x, y, z);
                const float xi = v * tfmax;
                int i = (int)floorf(xi);
                i = min(max(i, 0), a.ntf - 2);
                const float fr = xi - (float)i;
                const float4 c0 = s_tf[i], c1 = s_tf[i + 1];
                const float al = fmaf(fr, c1.w - c0.w, c0.w);
                if (al > 0.0f) {
                    float cr = fmaf(fr, c1.x - c0.x, c0.x);
                    float cg = fmaf(fr, c1.y - c0.y, c0.y);
                    float cb = fmaf(fr, c1.z - c0.z, c0.z);
                    if (SHADE) {
                        const float gx = 0.5f * (trilinear<T, I>(vol, a.nx, a.ny, a.nz, x + 1.f, y, z) -
                                                 trilinear<T, I>(vol, a.nx, a.ny, a.nz, x - 1.f, y, z));
                        const float gy = 0.5f * (trilinear<T, I>(vol, a.nx, a.ny, a.nz, x, y + 1.f, z) -
                                                 trilinear<T, I>(vol, a.nx, a.ny, a.nz, x, y - 1.f, z));
                        const float gz = 0.5f * (trilinear<T, I>(vol, a.nx, a.ny, a.nz, x, y, z + 1.f) -
                                                 trilinear<T, I>(vol, a.nx, a.ny, a.nz, x, y, z - 1.f));
                        const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
                        if (gn >= 1e-6f) {
                            const float ndl = fabsf(gx * dx + gy * dy + gz * dz) / gn;
                            float sp = ndl * ndl;   // ndl^32 by five squarings
                            sp *= sp;
                            sp *= sp;
                            sp *= sp;
                            sp *= sp;
                            const float diff = 0.2f + 0.7f * ndl;
                            cr = __saturatef(fmaf(cr, diff, 0.3f * sp));
                            cg = __saturatef(fmaf(cg, diff, 0.3f * sp));
                            cb = __saturatef(fmaf(cb, diff, 0.3f * sp));
                        }
                    }
                    const float w = (1.0f - A) * al;
                    C0 = fmaf(w, cr, C0);
                    C1 = fmaf(w, cg, C1);
                    C2 = fmaf(w, cb, C2);
                    A += w;
                }
                if (A >= a.term) {
                    ++k;
                    break;
                }
            }
        }
        my_samples += (unsigned long long)k;
        const float ta = 1.0f - A;
        float* out = a.rgbam + pix;
        out[0] = fmaf(ta, a.bg0, C0);
        out[a.plane] = fmaf(ta, a.bg1, C1);
        out[2 * a.plane] = fmaf(ta, a.bg2, C2);
        out[3 * a.plane] = A;
        out[4 * a.plane] = 1.0f;
    }
    if (a.nsamples) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
        if (lane == 0 && my_samples) atomicAdd(a.nsamples, my_samples);
    }
}

template <typename T, typename I>
static fvn_status launch_typed(fvn_ctx* ctx, const MarchArgs& a, bool shade, cudaStream_t st) {
    const size_t smem = (size_t)a.ntf * sizeof(float4);
    auto kern = shade ? march_kernel<T, I, true> : march_kernel<T, I, false>;
    if (smem > 48 * 1024)
        FVN_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = ctx->num_sms * per_sm;
    kern<<<grid, 128, smem, st>>>(a);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

fvn_status march_impl(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                      const fvn_march_params* mp, const int32_t* ids, const int32_t* count, float* rgbam,
                      unsigned long long* nsamples, cudaStream_t st) {
    MarchArgs a{};
    a.vol = vol->data;
    a.nx = vol->nx;
    a.ny = vol->ny;
    a.nz = vol->nz;
    a.ntf = tf->n;
    a.tf = reinterpret_cast<const float4*>(tf->rgba);
    const int nmax = std::max(vol->nx, std::max(vol->ny, vol->nz));
    double o[3], f[3], r[3], u[3];
    const int n[3] = {vol->nx, vol->ny, vol->nz};
    for (int i = 0; i < 3; ++i) {
        o[i] = (double)cam->eye[i] * nmax + 0.5 * n[i];
        f[i] = (double)cam->target[i] - (double)cam->eye[i];
    }
    double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double& x : f) x /= fl;
    const double up[3] = {cam->up[0], cam->up[1], cam->up[2]};
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (double& x : r) x /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double th = tan((double)cam->fov_y_deg * M_PI / 360.0);
    a.ox = (float)o[0];
    a.oy = (float)o[1];
    a.oz = (float)o[2];
    a.fx = (float)f[0];
    a.fy = (float)f[1];
    a.fz = (float)f[2];
    a.rx = (float)r[0];
    a.ry = (float)r[1];
    a.rz = (float)r[2];
    a.ux = (float)u[0];
    a.uy = (float)u[1];
    a.uz = (float)u[2];
    a.tan_y = (float)th;
    a.tan_x = (float)(th * cam->width / cam->height);
    a.two_over_w = (float)(2.0 / cam->width);
    a.two_over_h = (float)(2.0 / cam->height);
    a.W = cam->width;
    a.H = cam->height;
    a.dt = mp->step_vox;
    a.term = mp->term_alpha;
    a.bg0 = mp->bg[0];
    a.bg1 = mp->bg[1];
    a.bg2 = mp->bg[2];
    a.ids = ids;
    a.count = count;
    a.tiles_x = (a.W + 7) / 8;
    a.n_dense = a.tiles_x * ((a.H + 3) / 4) * 32;
    a.rgbam = rgbam;
    a.plane = (long long)a.W * a.H;
    a.nsamples = nsamples;
    a.ticket = ctx->d_ticket + (ctx->ticket_ring++ & 63);
    if (ids) FVN_CUDA(ctx, cudaMemsetAsync(rgbam, 0, 5 * sizeof(float) * (size_t)a.plane, st));
    FVN_CUDA(ctx, cudaMemsetAsync(a.ticket, 0, sizeof(int), st));
    const bool big = (unsigned long long)vol->nx * vol->ny * vol->nz >= (1ull << 31);
    const bool shade = mp->shading != 0;
    switch (vol->dtype) {
        case FVN_U8:
            return big ? launch_typed<uint8_t, long long>(ctx, a, shade, st)
                       : launch_typed<uint8_t, int>(ctx, a, shade, st);
        case FVN_U16:
            return big ? launch_typed<uint16_t, long long>(ctx, a, shade, st)
                       : launch_typed<uint16_t, int>(ctx, a, shade, st);
        case FVN_F16:
            return big ? launch_typed<__half, long long>(ctx, a, shade, st)
                       : launch_typed<__half, int>(ctx, a, shade, st);
        default:
            return big ? launch_typed<float, long long>(ctx, a, shade, st)
                       : launch_typed<float, int>(ctx, a, shade, st);
    }
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_march(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                                const fvn_march_params* mp, const int32_t* ids, const int32_t* count,
                                float* rgbam, unsigned long long* nsamples, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    fvn_status st;
    if ((st = validate_volume(ctx, vol)) != FVN_OK) return st;
    if ((st = validate_camera(ctx, cam)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, tf && tf->rgba && tf->n >= 2 && tf->n <= 4096, "transfer function needs 2..4096 entries");
    FVN_CHECK_ARG(ctx, ((uintptr_t)tf->rgba & 15) == 0, "transfer function must be 16-byte aligned");
    FVN_CHECK_ARG(ctx, mp != nullptr, "march parameters are NULL");
    FVN_CHECK_ARG(ctx, mp->step_vox > 0.f && isfinite(mp->step_vox), "step_vox must be > 0");
    FVN_CHECK_ARG(ctx, mp->term_alpha > 0.f && mp->term_alpha <= 1.f, "term_alpha must be in (0, 1]");
    FVN_CHECK_ARG(ctx, rgbam != nullptr, "rgbam output is NULL");
    FVN_CHECK_ARG(ctx, (ids == nullptr) == (count == nullptr), "ids and count must both be set or both NULL");
    return march_impl(ctx, vol, tf, cam, mp, ids, count, rgbam, nsamples, as_stream(stream));
}
