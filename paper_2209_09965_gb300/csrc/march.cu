// Emission-absorption ray march, dense or through the compacted pixel list
// (paper: "Foveated Rendering" and "Rendering": one ray per valid pixel of the
// compacted buffer, results written back to their full-frame positions).
//
// Persistent kernel: warps take rays from a global ticket counter; a lane
// whose ray ends goes idle and the idle lanes of a warp refill together once
// fewer than a tuned number of lanes are busy (1 = whole 32-ray packets), so
// lanes stay busy however uneven the ray lengths.  Dense rays are numbered in
// 8 x 4 pixel blocks, sparse rays follow the id list (written in Z-ordered
// 16 x 16 tiles of 8 x 4 sub-tiles by the mask kernel), so the rays of a warp
// are neighbours on screen and their gathers share cache lines.  The
// transfer function sits in shared memory; the volume is read through the
// read-only path from a copy with a 2-voxel clamp-to-edge border (a 256^3
// float volume and its copy stay in the 126 MB L2), so the per-sample code
// has no boundary branches.
//
// Per sample (FP32): trilinear value between voxel centres (clamp to edge),
// TF lookup at v (n - 1), optional shading from central differences at
// +-1 voxel (only for samples with alpha > 0, which are the only ones that
// contribute) -- Phong with a headlight, or, as in the paper's renderer,
// Phong lit by a directional light whose transmittance a shadow ray towards
// the light measures at a quarter of the sample rate -- then
// C += (1 - A) a c, A += (1 - A) a, stop once A >= term_alpha.  The 32 voxels a shaded sample needs are loaded in one
// batch, and two consecutive samples are loaded before the first is
// composited: the latency chain of a long ray, which bounds sparse frames,
// is a quarter of the naive one.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace fvn {

// The march reads a copy of the volume with kPad voxels of clamp-to-edge
// border on every side: every index of the 32-voxel stencil of a sample in
// the box is then inside the copy, so the per-sample code has no clamping
// and no divergent boundary path.
constexpr int kPad = 2;

struct MarchArgs {
    const void* vol;
    const void* pvol;                 // padded copy, (nx + 4) x (ny + 4) x (nz + 4)
    const void* svol;                 // shading 2: shadow-ray cells over the padded box (Quad<T> each)
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
    int refill_below;                 // refill idle lanes once fewer than this many are busy
    int coop_below;                   // finish the rays cooperatively once at most this many are busy (0 = never)
    const uint8_t* reject;            // dense numbering: skip pixels whose mask byte is 0
};

// Shading 2: the directional light and the shadow-ray step (the same for
// every view of a batch: world and voxel space share directions).
struct Light {
    float lx, ly, lz;                 // unit direction towards the light
    float ilx, ily, ilz;              // 1 / l per axis (1 where l = 0)
    float ds, inv_ds;                 // shadow step (shadow_rate * dt) and its reciprocal
    int srate;                        // shadow_rate
    int count;                        // add the shadow rays' samples to the sample counter
};

// A shadow ray stops once the light's transmittance falls below this; the
// light it could still carry changes no output channel by as much.
constexpr float kShadowCutoff = 1.0f / 16384.0f;

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

// The march's copies of the volume (padded copy, shadow-ray cells) hold
// float and half voxels already clamped to [0, 1], so their loads skip the
// clamp load_norm applies to the caller's volume (the same values).
template <typename T>
__device__ __forceinline__ T prenorm(T v) {
    return v;
}
template <>
__device__ __forceinline__ float prenorm<float>(float v) {
    return __saturatef(v);
}
template <>
__device__ __forceinline__ __half prenorm<__half>(__half v) {
    return __float2half_rn(__saturatef(__half2float(v)));   // exact: a half in [0, 1] converts back unchanged
}

// Normalised value of a voxel of a copy written through prenorm.
template <typename T>
__device__ __forceinline__ float load_pre(const T* p) {
    return load_norm(p);
}
template <>
__device__ __forceinline__ float load_pre<float>(const float* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float load_pre<__half>(const __half* p) {
    return __half2float(__ldg(p));
}

// Shadow-ray cells (shading 2): per padded voxel (x, y, z) the 2 x 2 block
// (v(x, y), v(x + 1, y), v(x, y + 1), v(x + 1, y + 1)) at z, in the voxel type,
// so the 8 voxels of a shadow sample are two vector loads (the cells at z
// and z + 1) instead of eight scalar ones.
template <typename T>
struct Quad;
template <>
struct Quad<float> {
    using type = float4;
    __device__ static __forceinline__ type make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
    __device__ static __forceinline__ void norm(const type& q, float& a, float& b, float& c, float& d) {
        a = q.x;   // clamped when the cells were written
        b = q.y;
        c = q.z;
        d = q.w;
    }
};
template <>
struct Quad<uint16_t> {
    using type = ushort4;
    __device__ static __forceinline__ type make(uint16_t a, uint16_t b, uint16_t c, uint16_t d) {
        return make_ushort4(a, b, c, d);
    }
    __device__ static __forceinline__ void norm(const type& q, float& a, float& b, float& c, float& d) {
        a = (float)q.x * (1.0f / 65535.0f);
        b = (float)q.y * (1.0f / 65535.0f);
        c = (float)q.z * (1.0f / 65535.0f);
        d = (float)q.w * (1.0f / 65535.0f);
    }
};
template <>
struct Quad<uint8_t> {
    using type = uchar4;
    __device__ static __forceinline__ type make(uint8_t a, uint8_t b, uint8_t c, uint8_t d) {
        return make_uchar4(a, b, c, d);
    }
    __device__ static __forceinline__ void norm(const type& q, float& a, float& b, float& c, float& d) {
        a = (float)q.x * (1.0f / 255.0f);
        b = (float)q.y * (1.0f / 255.0f);
        c = (float)q.z * (1.0f / 255.0f);
        d = (float)q.w * (1.0f / 255.0f);
    }
};
template <>
struct Quad<__half> {
    using type = uint2;   // four halves
    __device__ static __forceinline__ type make(__half a, __half b, __half c, __half d) {
        const __half2 lo = __halves2half2(a, b), hi = __halves2half2(c, d);
        return make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
    __device__ static __forceinline__ void norm(const type& q, float& a, float& b, float& c, float& d) {
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&q.x));   // clamped when written
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        a = lo.x;
        b = lo.y;
        c = hi.x;
        d = hi.y;
    }
};

// floor without conversion instructions (|x| < 2^22): returns i with
// x - i in [0, 1] (either neighbour at an exact integer, where the trilinear
// weights make both choices give the same value).
__device__ __forceinline__ int floor_frac(float x, float& frac) {
    const float M = 12582912.0f;   // 1.5 * 2^23: adding it rounds to an integer
    const float r = __fadd_rn(__fadd_rn(x, -0.5f), M);
    frac = __fadd_rn(x, -__fadd_rn(r, -M));
    return __float_as_int(r) - 0x4B400000;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Packed FP32 pairs (the f32x2 instructions of this architecture): one
// instruction computes both lanes with the same IEEE operations as two
// scalar ones, so lerp2 gives bit for bit the two lerpf results.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n.reg .b64 ra, rb, rc, rd;\n"
        "mov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\nmov.b64 rc, {%6, %7};\n"
        "fma.rn.f32x2 rd, ra, rb, rc;\nmov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 ra, rb, rd;\n"
        "mov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
        "sub.rn.f32x2 rd, ra, rb;\nmov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 t) { return fma2(t, sub2(b, a), a); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }

// Ray state of one lane.
struct Ray {
    int pix;                     // pixel id, < 0 when the lane is idle
    float dx, dy, dz, tnear, tfar, kf;
    float C0, C1, C2, A;
};

// Set up ray number r (dense: 8 x 4 pixel blocks; sparse: the id list).
// Returns false when r names no pixel.  A ray that misses the box is written
// out at once and leaves the lane idle.
__device__ __forceinline__ bool start_ray(const MarchArgs& a, int r, int npix, Ray& s) {
    int pix, px, py;
    if (a.ids) {
        pix = __ldg(a.ids + r);
        if ((unsigned)pix >= (unsigned)npix) return false;   // ignore ids outside the frame
        py = pix / a.W;
        px = pix - py * a.W;
    } else {
        const int tile = r >> 5, q = r & 31;
        const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
        px = tx * 8 + (q & 7);
        py = ty * 4 + (q >> 3);
        if (px >= a.W || py >= a.H) return false;
        pix = py * a.W + px;
        if (a.reject && __ldg(a.reject + pix) == 0) return false;   // naive rejection: skip in place
    }
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
    const float o[3] = {a.ox, a.oy, a.oz};
    const float d[3] = {dx, dy, dz};
    const float n[3] = {(float)a.nx, (float)a.ny, (float)a.nz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0f) {
            if (o[ax] < 0.0f || o[ax] > n[ax]) miss = true;
        } else {
            float t0 = (0.0f - o[ax]) / d[ax];
            float t1 = (n[ax] - o[ax]) / d[ax];
            if (t0 > t1) {
                const float t = t0;
                t0 = t1;
                t1 = t;
            }
            tn = fmaxf(tn, t0);
            tfar = fminf(tfar, t1);
        }
    }
    const float tnear = fmaxf(tn, 0.0f);
    s.pix = pix;
    s.dx = dx;
    s.dy = dy;
    s.dz = dz;
    s.tnear = tnear;
    s.tfar = (miss || !(tnear < tfar)) ? -INFINITY : tfar;   // no sample when missed
    s.kf = 0.f;
    s.C0 = s.C1 = s.C2 = s.A = 0.f;
    return true;
}

__device__ __forceinline__ void finish_ray(const MarchArgs& a, const Ray& s) {
    const float ta = 1.0f - s.A;
    float* out = a.rgbam + s.pix;
    out[0] = fmaf(ta, a.bg0, s.C0);
    out[a.plane] = fmaf(ta, a.bg1, s.C1);
    out[2 * a.plane] = fmaf(ta, a.bg2, s.C2);
    out[3 * a.plane] = s.A;
    out[4 * a.plane] = 1.0f;
}

// The 32 voxels one shaded sample reads: the trilinear cell c[z][y][x] and
// the two extra rows each central difference needs, all loaded at once so a
// sample costs one round trip to the memory system.
struct Stencil {
    float c[2][2][2];
    float xm[2][2], xp[2][2];   // x = -1, +2 at (y, z) of the cell, [z][y]
    float ym[2][2], yp[2][2];   // y = -1, +2 at (x, z), [z][x]
    float zm[2][2], zp[2][2];   // z = -1, +2 at (x, y), [y][x]
    float tx, ty, tz;
};

// Cell of a sample position (voxel-centre coordinates): fractions into S
// and the offset of the cell's first voxel in the padded copy.
template <typename I>
__device__ __forceinline__ I cell_base(const MarchArgs& a, I sy, I sz, float ux, float uy, float uz, float& tx,
                                       float& ty, float& tz) {
    int i = floor_frac(ux, tx), j = floor_frac(uy, ty), k = floor_frac(uz, tz);
    // samples lie in the box, so i is in [-1, n - 1]; the clamp only guards
    // against rounding and keeps every stencil index inside the padded copy
    i = min(max(i, -1), a.nx - 1);
    j = min(max(j, -1), a.ny - 1);
    k = min(max(k, -1), a.nz - 1);
    return (I)(k + kPad) * sz + (I)(j + kPad) * sy + (i + kPad);
}

template <typename I>
__device__ __forceinline__ I stencil_cell(const MarchArgs& a, I sy, I sz, float ux, float uy, float uz, Stencil& S) {
    return cell_base<I>(a, sy, sz, ux, uy, uz, S.tx, S.ty, S.tz);
}

// The trilinear cell of a shadow sample (values only).
struct Cell {
    float c[2][2][2];
    float tx, ty, tz;
};

__device__ __forceinline__ float cell_value(const Cell& C) {
    float rows[2][2];
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y) rows[z][y] = lerpf(C.c[z][y][0], C.c[z][y][1], C.tx);
    return lerpf(lerpf(rows[0][0], rows[0][1], C.ty), lerpf(rows[1][0], rows[1][1], C.ty), C.tz);
}

// The voxels of the stencil whose cell starts at vol + b.
template <typename T, typename I, bool SHADE>
__device__ __forceinline__ void stencil_fetch(const T* __restrict__ vol, I b0, I sy, I sz, Stencil& S) {
    const T* b = vol + b0;
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const T* r = b + (I)z * sz + (I)y * sy;
            S.c[z][y][0] = load_pre(r);
            S.c[z][y][1] = load_pre(r + 1);
            if (SHADE) {
                S.xm[z][y] = load_pre(r - 1);
                S.xp[z][y] = load_pre(r + 2);
            }
        }
    if (SHADE) {
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                S.ym[z][x] = load_pre(b + (I)z * sz - sy + x);
                S.yp[z][x] = load_pre(b + (I)z * sz + 2 * sy + x);
            }
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                S.zm[y][x] = load_pre(b - sz + (I)y * sy + x);
                S.zp[y][x] = load_pre(b + 2 * sz + (I)y * sy + x);
            }
    }
}

// The 32 voxels one shaded sample reads, loaded at once so a sample costs one
// round trip to the memory system.
template <typename T, typename I, bool SHADE>
__device__ __forceinline__ void load_stencil(const MarchArgs& a, const T* __restrict__ vol, I sy, I sz, float ux,
                                             float uy, float uz, Stencil& S) {
    const I b = stencil_cell<I>(a, sy, sz, ux, uy, uz, S);
    stencil_fetch<T, I, SHADE>(vol, b, sy, sz, S);
}

// TF entry below value v and the fraction towards the next one.
__device__ __forceinline__ int tf_index(const MarchArgs& a, float tfmax, float v, float& fr) {
    const float xi = v * tfmax;
    int ti = floor_frac(xi, fr);
    if (ti > a.ntf - 2) {
        fr += (float)(ti - (a.ntf - 2));
        ti = a.ntf - 2;
    }
    if (ti < 0) {
        fr += (float)ti;
        ti = 0;
    }
    return ti;
}

// TF opacity at value v, from the table of opacity pairs (a_i, a_i+1) that
// shadowed marches keep in shared memory right after the TF (one 8-byte
// read with few bank conflicts, where the .w of two float4 entries would be
// two reads over a quarter of the banks).
__device__ __forceinline__ float tf_alpha(const MarchArgs& a, const float4* s_tf, float tfmax, float v) {
    float fr;
    const int ti = tf_index(a, tfmax, v, fr);
    const float2 p = reinterpret_cast<const float2*>(s_tf + a.ntf + 1)[ti];
    return fmaf(fr, p.y - p.x, p.x);
}

// Shared-memory slots (float4) of a TF of n entries: the entries and a copy
// of the last one (so an index at the top end needs no clamp), and for
// shadowed marches the opacity pairs after them.
__host__ __device__ __forceinline__ int tf_slots(int n, int shade) {
    return shade == 2 ? n + 1 + (n + 1) / 2 : n + 1;
}

// Copy a TF of n entries (and its last entry once more) into shared memory
// at s, and for shadowed marches its opacity pairs; the block's threads
// share the work.
template <int SHADE>
__device__ __forceinline__ void load_tf(float4* s, const float4* __restrict__ tf, int n) {
    for (int i = threadIdx.x; i <= n; i += blockDim.x) s[i] = tf[min(i, n - 1)];
    if (SHADE == 2) {
        float2* p = reinterpret_cast<float2*>(s + n + 1);
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = make_float2(tf[i].w, tf[min(i + 1, n - 1)].w);
    }
}

// TF lookup at value v: returns the opacity and, when it is > 0, the colour.
__device__ __forceinline__ float tf_lookup(const MarchArgs& a, const float4* s_tf, float tfmax, float v, float& cr,
                                           float& cg, float& cb) {
    float fr;
    const int ti = tf_index(a, tfmax, v, fr);
    const float4 c0 = s_tf[ti], c1 = s_tf[ti + 1];
    const float al = fmaf(fr, c1.w - c0.w, c0.w);
    if (al > 0.0f) {
        cr = fmaf(fr, c1.x - c0.x, c0.x);
        cg = fmaf(fr, c1.y - c0.y, c0.y);
        cb = fmaf(fr, c1.z - c0.z, c0.z);
    }
    return al;
}

// Phong with a headlight from the gradient (gx, gy, gz) and the ray
// direction; no shading where |g| < 1e-6.
__device__ __forceinline__ void phong(float gx, float gy, float gz, float dx, float dy, float dz, float& cr, float& cg,
                                      float& cb) {
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    if (g2 >= 1e-12f) {   // |g| >= 1e-6: shade, otherwise keep the TF colour
        const float ndl = fabsf(fmaf(gx, dx, fmaf(gy, dy, gz * dz))) * rsqrtf(g2);
        float sp = ndl * ndl;   // ndl^32 by five squarings
        sp *= sp;
        sp *= sp;
        sp *= sp;
        sp *= sp;
        const float diff = fmaf(0.7f, ndl, 0.2f);
        const float spec = 0.3f * sp;
        cr = __saturatef(fmaf(cr, diff, spec));
        cg = __saturatef(fmaf(cg, diff, spec));
        cb = __saturatef(fmaf(cb, diff, spec));
    }
}

// Phong lit by the directional light l, attenuated by the shadow
// transmittance tr: c' = clamp(c (0.2 + 0.7 tr |n.l|) + 0.3 tr |n.h|^32) with
// h = |l - dir|; where |g| < 1e-6, c' = clamp(c (0.2 + 0.7 tr)).
__device__ __forceinline__ void phong_lit(const Light& a, float gx, float gy, float gz, float dx, float dy,
                                          float dz, float tr, float& cr, float& cg, float& cb) {
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    float diff, spec = 0.0f;
    if (g2 >= 1e-12f) {
        const float ig = rsqrtf(g2);
        const float ndl = fabsf(fmaf(gx, a.lx, fmaf(gy, a.ly, gz * a.lz))) * ig;
        const float hx = a.lx - dx, hy = a.ly - dy, hz = a.lz - dz;
        const float h2 = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
        if (h2 >= 1e-24f) {   // no half vector when the light shines straight back along the ray
            float sp = fabsf(fmaf(gx, hx, fmaf(gy, hy, gz * hz))) * ig * rsqrtf(h2);
            sp *= sp;   // ndh^32 by five squarings
            sp *= sp;
            sp *= sp;
            sp *= sp;
            sp *= sp;
            spec = 0.3f * tr * sp;
        }
        diff = fmaf(0.7f * tr, ndl, 0.2f);
    } else {
        diff = fmaf(0.7f, tr, 0.2f);
    }
    cr = __saturatef(fmaf(cr, diff, spec));
    cg = __saturatef(fmaf(cg, diff, spec));
    cb = __saturatef(fmaf(cb, diff, spec));
}

// The voxel-centre coordinate of the face a shadow ray along l leaves the
// box [0, n] by (1e30 where l = 0: that axis never bounds it).
__device__ __forceinline__ float exit_face(float l, int n) {
    return l > 0.0f ? (float)n - 0.5f : (l < 0.0f ? -0.5f : 1e30f);
}

// Light reaching a sample: the shadow ray from the sample point u
// (voxel-centre coordinates) towards the light, with samples at j ds,
// j = 1, 2, ..., while inside the box.  Each multiplies the transmittance by
// (1 - a)^shadow_rate, the last one by the power for the part of its step
// left inside the box (so the result is continuous in the exit distance);
// the ray stops once the transmittance falls below kShadowCutoff.  The loads
// of kG consecutive samples are issued before any is used.
template <typename Src, typename I>
__device__ __forceinline__ float shadow_ray(const MarchArgs& a, const Light& lt,
                                            const typename Src::V* __restrict__ vol, const float4* s_tf, float tfmax,
                                            I sy, I sz, float ux, float uy, float uz, unsigned& nsh) {
    constexpr int kG = 4;   // samples whose loads are in flight together
    const float se = fminf(fminf((exit_face(lt.lx, a.nx) - ux) * lt.ilx, (exit_face(lt.ly, a.ny) - uy) * lt.ily),
                           (exit_face(lt.lz, a.nz) - uz) * lt.ilz);
    float tr = 1.0f;
    for (float j = 1.0f;; j += (float)kG) {
        if (!(j * lt.ds < se)) break;
        Cell C[kG];
        float sj[kG];
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            sj[q] = (j + (float)q) * lt.ds;
            const float sc = sj[q] < se ? sj[q] : j * lt.ds;   // past the exit: reload the first (unused)
            Src::template load_cell<I>(a, vol, sy, sz, fmaf(sc, lt.lx, ux), fmaf(sc, lt.ly, uy), fmaf(sc, lt.lz, uz),
                                       C[q]);
        }
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            if (!(sj[q] < se)) return tr;
            ++nsh;
            const float al = tf_alpha(a, s_tf, tfmax, cell_value(C[q]));
            if (al > 0.0f) {
                const float base = 1.0f - al;
                const float e = (se - sj[q]) * lt.inv_ds;   // steps left inside the box
                float f = base;
                if (e >= 1.0f) {
                    if (lt.srate == 4) {
                        f *= f;
                        f *= f;
                    } else {
                        for (int i = 1; i < lt.srate; ++i) f *= base;
                    }
                } else {
                    f = base > 0.0f ? exp2f((float)lt.srate * e * log2f(base)) : 0.0f;
                }
                tr *= f;
            }
            if (tr < kShadowCutoff) return tr;
        }
    }
    return tr;
}

// The voxel rows of a stencil interpolated along x, and the trilinear value.
__device__ __forceinline__ float stencil_value(const Stencil& S, float (&rows)[2][2]) {
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y) rows[z][y] = lerpf(S.c[z][y][0], S.c[z][y][1], S.tx);
    return lerpf(lerpf(rows[0][0], rows[0][1], S.ty), lerpf(rows[1][0], rows[1][1], S.ty), S.tz);
}

// Central differences at +-1 voxel of the trilinear field.
__device__ __forceinline__ void stencil_gradient(const Stencil& S, const float (&rows)[2][2], float& gx, float& gy,
                                                 float& gz) {
    float d[2][2];
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y)
            d[z][y] = lerpf(S.c[z][y][1], S.xp[z][y], S.tx) - lerpf(S.xm[z][y], S.c[z][y][0], S.tx);
    gx = 0.5f * lerpf(lerpf(d[0][0], d[0][1], S.ty), lerpf(d[1][0], d[1][1], S.ty), S.tz);
    float ym[2], yp[2], zm[2], zp[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        ym[q] = lerpf(S.ym[q][0], S.ym[q][1], S.tx);
        yp[q] = lerpf(S.yp[q][0], S.yp[q][1], S.tx);
        zm[q] = lerpf(S.zm[q][0], S.zm[q][1], S.tx);
        zp[q] = lerpf(S.zp[q][0], S.zp[q][1], S.tx);
    }
    gy = 0.5f * lerpf(lerpf(rows[0][1], yp[0], S.ty) - lerpf(ym[0], rows[0][0], S.ty),
                      lerpf(rows[1][1], yp[1], S.ty) - lerpf(ym[1], rows[1][0], S.ty), S.tz);
    gz = 0.5f * lerpf(lerpf(rows[1][0], zp[0], S.tz) - lerpf(zm[0], rows[0][0], S.tz),
                      lerpf(rows[1][1], zp[1], S.tz) - lerpf(zm[1], rows[0][1], S.tz), S.ty);
}

// Shade a classified sample (al > 0) from its gradient: SHADE 1 headlight,
// SHADE 2 directional light with the shadow ray from u.
template <typename Src, int SHADE, typename I>
__device__ __forceinline__ void light_sample(const MarchArgs& a, const Light& lt,
                                             const typename Src::V* __restrict__ vol, const float4* s_tf, float tfmax,
                                             I sy, I sz, float gx, float gy, float gz, float ux, float uy, float uz,
                                             float dx, float dy, float dz, float& cr, float& cg, float& cb,
                                             unsigned& nsh) {
    if constexpr (SHADE == 1) {
        phong(gx, gy, gz, dx, dy, dz, cr, cg, cb);
    } else if constexpr (SHADE == 2) {
        const float tr = shadow_ray<Src, I>(a, lt, vol, s_tf, tfmax, sy, sz, ux, uy, uz, nsh);
        phong_lit(lt, gx, gy, gz, dx, dy, dz, tr, cr, cg, cb);
    }
}

// Sample source of the scalar padded copy: the 32-voxel stencil.
template <typename T>
struct ScalarSrc {
    using V = T;
    using St = Stencil;
    template <typename I, bool SHADE>
    __device__ static __forceinline__ void load(const MarchArgs& a, const V* __restrict__ vol, I sy, I sz, float ux,
                                                float uy, float uz, St& S) {
        load_stencil<T, I, SHADE>(a, vol, sy, sz, ux, uy, uz, S);
    }
    // the 8 voxels of a shadow sample: two cells of the shadow-ray cell volume
    template <typename I>
    __device__ static __forceinline__ void load_cell(const MarchArgs& a, const V* __restrict__, I sy, I sz, float ux,
                                                     float uy, float uz, Cell& C) {
        using Q = Quad<T>;
        const typename Q::type* b =
            static_cast<const typename Q::type*>(a.svol) + cell_base<I>(a, sy, sz, ux, uy, uz, C.tx, C.ty, C.tz);
        const typename Q::type q0 = __ldg(b), q1 = __ldg(b + sz);
        Q::norm(q0, C.c[0][0][0], C.c[0][0][1], C.c[0][1][0], C.c[0][1][1]);
        Q::norm(q1, C.c[1][0][0], C.c[1][0][1], C.c[1][1][0], C.c[1][1][1]);
    }
    // Classify and shade one loaded sample: returns its opacity al and, when
    // al > 0, its (clamped) shaded colour.
    template <int SHADE, typename I>
    __device__ static __forceinline__ float shade(const MarchArgs& a, const Light& lt, const V* __restrict__ vol,
                                                  const float4* s_tf, float tfmax, I sy, I sz, const St& S, float ux,
                                                  float uy, float uz, float dx, float dy, float dz, float& cr,
                                                  float& cg, float& cb, unsigned& nsh) {
        float rows[2][2];
        const float al = tf_lookup(a, s_tf, tfmax, stencil_value(S, rows), cr, cg, cb);
        if (SHADE != 0 && al > 0.0f) {
            float gx, gy, gz;
            stencil_gradient(S, rows, gx, gy, gz);
            light_sample<ScalarSrc<T>, SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, gx, gy, gz, ux, uy, uz, dx, dy,
                                                 dz, cr, cg, cb, nsh);
        }
        return al;
    }
};

// Sample source of the gradient volume: every padded voxel holds
// (v, Dx, Dy, Dz) with D = half the difference of its two neighbours along
// the axis (clamp to edge).  The central difference at +-1 voxel of the
// trilinear field equals the trilinear interpolation of D (both shifted
// fields use the sample's own weights), so a shaded sample is 8 float4
// loads instead of 32 scalar ones.
struct Stencil4 {
    float4 c[2][2][2];
    float tx, ty, tz;
};

struct Grad4Src {
    using V = float4;
    using St = Stencil4;
    template <typename I, bool SHADE>
    __device__ static __forceinline__ void load(const MarchArgs& a, const V* __restrict__ vol, I sy, I sz, float ux,
                                                float uy, float uz, St& S) {
        const V* b = vol + cell_base<I>(a, sy, sz, ux, uy, uz, S.tx, S.ty, S.tz);
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                const V* r = b + (I)z * sz + (I)y * sy;
                S.c[z][y][0] = __ldg(r);
                S.c[z][y][1] = __ldg(r + 1);
            }
    }
    // The trilinear interpolation of all four channels (value and the three
    // half differences) as packed pairs, in the order of the scalar
    // definition (x, then y, then z); the TF colour and opacity likewise.  No
    // branch depends on the sample, so the two samples of a step interleave.
    template <int SHADE, typename I>
    __device__ static __forceinline__ float shade(const MarchArgs& a, const Light& lt, const V* __restrict__ vol,
                                                  const float4* s_tf, float tfmax, I sy, I sz, const St& S, float ux,
                                                  float uy, float uz, float dx, float dy, float dz, float& cr,
                                                  float& cg, float& cb, unsigned& nsh) {
        const float2 tx = make_float2(S.tx, S.tx), ty = make_float2(S.ty, S.ty), tz = make_float2(S.tz, S.tz);
        float2 lo[2][2], hi[2][2];
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                lo[z][y] = lerp2(lo2(S.c[z][y][0]), lo2(S.c[z][y][1]), tx);   // (v, Dx)
                hi[z][y] = lerp2(hi2(S.c[z][y][0]), hi2(S.c[z][y][1]), tx);   // (Dy, Dz)
            }
        const float2 vx = lerp2(lerp2(lo[0][0], lo[0][1], ty), lerp2(lo[1][0], lo[1][1], ty), tz);
        const float2 yz = lerp2(lerp2(hi[0][0], hi[0][1], ty), lerp2(hi[1][0], hi[1][1], ty), tz);
        // v is in [0, 1] up to rounding (the copy holds clamped values): the
        // entry below v (n - 1) needs only a floor at 0 and a cap at n - 1,
        // the padded last entry covers ti + 1 = n
        float fr;
        const int ti = min(floor_frac(fmaxf(vx.x * tfmax, 0.0f), fr), a.ntf - 1);
        const float4 c0 = s_tf[ti], c1 = s_tf[ti + 1];
        const float2 f2 = make_float2(fr, fr);
        const float2 rg = lerp2(lo2(c0), lo2(c1), f2), ba = lerp2(hi2(c0), hi2(c1), f2);
        cr = rg.x;
        cg = rg.y;
        cb = ba.x;
        if constexpr (SHADE == 1) {
            phong(vx.y, yz.x, yz.y, dx, dy, dz, cr, cg, cb);
        } else if constexpr (SHADE != 0) {
            if (ba.y > 0.0f)
                light_sample<Grad4Src, SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, vx.y, yz.x, yz.y, ux, uy, uz, dx,
                                                 dy, dz, cr, cg, cb, nsh);
        }
        return ba.y;
    }
};

// Composite one classified sample (opacity al, shaded colour c); returns
// true once the ray is opaque enough to stop.
__device__ __forceinline__ bool composite(const MarchArgs& a, float al, float cr, float cg, float cb, Ray& s) {
    if (al > 0.0f) {
        const float w = (1.0f - s.A) * al;
        s.C0 = fmaf(w, cr, s.C0);
        s.C1 = fmaf(w, cg, s.C1);
        s.C2 = fmaf(w, cb, s.C2);
        s.A += w;
    }
    return s.A >= a.term;
}

// Classify, shade and composite one loaded sample; returns true once the ray
// is opaque enough to stop.
template <typename Src, int SHADE, typename I>
__device__ __forceinline__ bool composite_sample(const MarchArgs& a, const Light& lt,
                                                 const typename Src::V* __restrict__ vol, const float4* s_tf,
                                                 float tfmax, I sy, I sz, const typename Src::St& S, float ux,
                                                 float uy, float uz, Ray& s, unsigned& nsh) {
    float cr, cg, cb;
    const float al = Src::template shade<SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, S, ux, uy, uz, s.dx, s.dy, s.dz,
                                                   cr, cg, cb, nsh);
    return composite(a, al, cr, cg, cb, s);
}

// Up to two samples of the ray with both samples' loads issued before either
// is composited (the loads do not depend on the compositing), which halves
// the latency chain a long ray walks.  Returns true when the ray is finished.
template <typename Src, typename I, int SHADE>
__device__ __forceinline__ bool ray_step(const MarchArgs& a, const Light& lt, const typename Src::V* __restrict__ vol,
                                         const float4* s_tf, I sy, I sz, float ux0, float uy0, float uz0,
                                         float tfmax, Ray& s, unsigned& nsh) {
    const float t0 = fmaf(s.kf, a.dt, s.tnear);
    if (!(t0 < s.tfar)) return true;
    if constexpr (SHADE == 2) {
        // a shadowed sample's time goes into its shadow ray: one sample per
        // step, so no second stencil stays live across it
        typename Src::St S0;
        const float px0 = fmaf(t0, s.dx, ux0), py0 = fmaf(t0, s.dy, uy0), pz0 = fmaf(t0, s.dz, uz0);
        Src::template load<I, true>(a, vol, sy, sz, px0, py0, pz0, S0);
        s.kf += 1.0f;
        return composite_sample<Src, SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, S0, px0, py0, pz0, s, nsh);
    }
    const float t1 = fmaf(s.kf + 1.0f, a.dt, s.tnear);
    const bool has1 = t1 < s.tfar;
    const float t1c = has1 ? t1 : t0;
    typename Src::St S0, S1;
    const float px0 = fmaf(t0, s.dx, ux0), py0 = fmaf(t0, s.dy, uy0), pz0 = fmaf(t0, s.dz, uz0);
    const float px1 = fmaf(t1c, s.dx, ux0), py1 = fmaf(t1c, s.dy, uy0), pz1 = fmaf(t1c, s.dz, uz0);
    Src::template load<I, SHADE != 0>(a, vol, sy, sz, px0, py0, pz0, S0);
    Src::template load<I, SHADE != 0>(a, vol, sy, sz, px1, py1, pz1, S1);
    // both samples are classified and shaded before either is composited
    // (independent work the scheduler can interleave; the second is wasted
    // only on a ray's last step)
    float r0, g0, b0, r1, g1, b1;
    const float al0 = Src::template shade<SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, S0, px0, py0, pz0, s.dx, s.dy,
                                                    s.dz, r0, g0, b0, nsh);
    const float al1 = Src::template shade<SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, S1, px1, py1, pz1, s.dx, s.dy,
                                                    s.dz, r1, g1, b1, nsh);
    s.kf += 1.0f;
    if (composite(a, al0, r0, g0, b0, s)) return true;
    if (!has1) return true;
    s.kf += 1.0f;
    return composite(a, al1, r1, g1, b1, s);
}

// Cooperative march of one ray by the whole warp, for the last few rays of a
// warp (which otherwise walk their long latency chains with the other lanes
// idle).  In each chunk lane j takes sample kf + j; the chunk is composited
// front to back as a product scan of the transmittances (1 - A) over the
// lanes -- the same recurrence as the sequential march, evaluated in a
// different order -- and the ray stops at the first sample whose opacity
// reaches term_alpha, or where it leaves the box.  `r` is the same on every
// lane on entry and on return.
template <typename Src, typename I, int SHADE>
__device__ __forceinline__ void coop_ray(const MarchArgs& a, const Light& lt, const typename Src::V* __restrict__ vol,
                                         const float4* s_tf, I sy, I sz, float ux0, float uy0, float uz0, float tfmax,
                                         Ray& r, unsigned& nsh) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        const float t = fmaf(r.kf + (float)lane, a.dt, r.tnear);
        const bool valid = t < r.tfar;          // a prefix of the lanes
        const unsigned vb = __ballot_sync(FULL, valid);
        if (vb == 0) return;
        float cr = 0.f, cg = 0.f, cb = 0.f, al = 0.f;
        if (valid) {
            typename Src::St S;
            const float px = fmaf(t, r.dx, ux0), py = fmaf(t, r.dy, uy0), pz = fmaf(t, r.dz, uz0);
            Src::template load<I, SHADE != 0>(a, vol, sy, sz, px, py, pz, S);
            al = Src::template shade<SHADE, I>(a, lt, vol, s_tf, tfmax, sy, sz, S, px, py, pz, r.dx, r.dy, r.dz, cr,
                                               cg, cb, nsh);
            if (!(al > 0.0f)) al = 0.0f;
        }
        // incl = prod_{i <= j} (1 - al_i), excl = prod_{i < j} (1 - al_i)
        float incl = 1.0f - al;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl *= v;
        }
        float excl = __shfl_up_sync(FULL, incl, 1);
        if (lane == 0) excl = 1.0f;
        const float tin = 1.0f - r.A;
        const float a_after = 1.0f - tin * incl;
        const unsigned stop = __ballot_sync(FULL, valid && a_after >= a.term);
        const int last = stop ? __ffs(stop) - 1 : 31 - __clz(vb);
        const float w = (lane <= last && al > 0.0f) ? tin * excl * al : 0.0f;
        float c0 = w * cr, c1 = w * cg, c2 = w * cb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_xor_sync(FULL, c0, o);
            c1 += __shfl_xor_sync(FULL, c1, o);
            c2 += __shfl_xor_sync(FULL, c2, o);
        }
        r.C0 += c0;
        r.C1 += c1;
        r.C2 += c2;
        r.A = __shfl_sync(FULL, a_after, last);
        r.kf += (float)(last + 1);
        if (stop || last < 31) return;
    }
}

// The ray of lane `src` on every lane.
__device__ __forceinline__ Ray shfl_ray(const Ray& s, int src) {
    const unsigned FULL = 0xffffffffu;
    Ray r;
    r.pix = __shfl_sync(FULL, s.pix, src);
    r.dx = __shfl_sync(FULL, s.dx, src);
    r.dy = __shfl_sync(FULL, s.dy, src);
    r.dz = __shfl_sync(FULL, s.dz, src);
    r.tnear = __shfl_sync(FULL, s.tnear, src);
    r.tfar = __shfl_sync(FULL, s.tfar, src);
    r.kf = __shfl_sync(FULL, s.kf, src);
    r.C0 = __shfl_sync(FULL, s.C0, src);
    r.C1 = __shfl_sync(FULL, s.C1, src);
    r.C2 = __shfl_sync(FULL, s.C2, src);
    r.A = __shfl_sync(FULL, s.A, src);
    return r;
}

// Persistent kernel with per-lane ray refill: a lane whose ray finishes goes
// idle, and once fewer than `refill_below` lanes of the warp are busy the
// idle lanes take new rays from the global queue together (one atomic per
// warp), so warps neither wait for their longest ray nor for the slowest
// warp at the end of the queue.
// Shadowed marches spend their time in independent shadow-ray samples:
// registers are capped for five CTAs per SM (more warps to hide latency).
template <typename Src, typename I, int SHADE>
__global__ void __launch_bounds__(128, SHADE == 2 ? 5 : 1) march_kernel(MarchArgs a, Light lt) {
    extern __shared__ float4 s_tf[];
    load_tf<SHADE>(s_tf, a.tf, a.ntf);
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const typename Src::V* __restrict__ vol = static_cast<const typename Src::V*>(a.pvol);
    const int lane = threadIdx.x & 31;
    const int npix = a.W * a.H;
    // the id list never holds more than one entry per pixel
    const int nrays = a.ids ? min(max(*a.count, 0), npix) : a.n_dense;
    const float tfmax = (float)(a.ntf - 1);
    const I sy = (I)(a.nx + 2 * kPad), sz = sy * (I)(a.ny + 2 * kPad);   // padded strides
    // sample positions are handled in voxel-centre coordinates u = p - 0.5
    const float ux0 = a.ox - 0.5f, uy0 = a.oy - 0.5f, uz0 = a.oz - 0.5f;
    unsigned long long my_samples = 0;
    unsigned nsh = 0;                 // shadow-ray samples of this lane
    Ray s;
    s.pix = -1;
    if (a.coop_below >= 32) {
        // fully cooperative mode (few, long rays): a warp takes one ray at a
        // time and marches it with all 32 lanes
        for (;;) {
            int r = 0;
            if (lane == 0) r = atomicAdd(a.ticket, 1);
            r = __shfl_sync(FULL, r, 0);
            if (r >= nrays) break;
            if (!start_ray(a, r, npix, s)) continue;   // every lane sets up the same ray
            if (s.tfar > -INFINITY) coop_ray<Src, I, SHADE>(a, lt, vol, s_tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
            if (lane == 0) {
                my_samples += (unsigned long long)s.kf;
                finish_ray(a, s);
            }
        }
        s.pix = -1;
    }
    bool exhausted = a.coop_below >= 32;   // warp-uniform: the queue has run dry
    for (;;) {
        if (!exhausted) {
            const unsigned idle = __ballot_sync(FULL, s.pix < 0);
            if (idle) {
                const int nidle = __popc(idle);
                int base = 0;
                if (lane == 0) base = atomicAdd(a.ticket, nidle);
                base = __shfl_sync(FULL, base, 0);
                if (base + nidle >= nrays) exhausted = true;
                if (s.pix < 0) {
                    const int r = base + __popc(idle & ((1u << lane) - 1u));
                    if (r < nrays && start_ray(a, r, npix, s) && !(s.tfar > -INFINITY)) {
                        finish_ray(a, s);   // missed the box: background, no sample
                        s.pix = -1;
                    }
                }
            }
        }
        unsigned busy = __ballot_sync(FULL, s.pix >= 0);
        if (busy == 0) {
            if (exhausted) break;
            continue;
        }
        while (busy != 0 && (exhausted || __popc(busy) >= a.refill_below)) {
            if (__popc(busy) <= a.coop_below) {
                // the warp's last few rays: march each with all 32 lanes
                do {
                    const int src = __ffs(busy) - 1;
                    Ray r = shfl_ray(s, src);
                    coop_ray<Src, I, SHADE>(a, lt, vol, s_tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
                    if (lane == src) {
                        s = r;
                        my_samples += (unsigned long long)s.kf;
                        finish_ray(a, s);
                        s.pix = -1;
                    }
                    busy &= busy - 1u;
                } while (busy != 0);
                break;
            }
            if (s.pix >= 0 && ray_step<Src, I, SHADE>(a, lt, vol, s_tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh)) {
                my_samples += (unsigned long long)s.kf;
                finish_ray(a, s);
                s.pix = -1;
            }
            busy = __ballot_sync(FULL, s.pix >= 0);
        }
        if (exhausted && busy == 0) break;
    }
    if (a.nsamples) {
        if (SHADE == 2 && lt.count) my_samples += nsh;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(FULL, my_samples, o);
        if (lane == 0 && my_samples) atomicAdd(a.nsamples, my_samples);
    }
}

// ---------------------------------------------------------------------------
// Batched march: the rays of several views (each with its own camera, frame,
// compacted id list, output, volume of any voxel type and transfer function)
// in one persistent launch.  Tickets run over the concatenation of the views'
// id lists, so a warp takes rays of one view except where two lists meet;
// per ray the arithmetic is exactly that of march_kernel.

struct MarchBatchView {
    MarchArgs a;                      // per-view fields (pvol = padded copy of its volume)
    int dtype;                        // fvn_dtype of the volume
    int tf_off;                       // first entry of its transfer function in shared memory
};

struct MarchBatch {
    Light light;
    int nviews;
    int ntfs;                         // distinct transfer functions
    const float4* tf[kMaxViews];
    int tf_n[kMaxViews], tf_off[kMaxViews];
    unsigned long long* nsamples;
    int* ticket;
    int refill_below;
    int coop_below;
    MarchBatchView v[kMaxViews];
};
static_assert(sizeof(MarchBatch) <= 4096, "batched march arguments exceed the 4 KB parameter space");

// Volume kinds of a batch view: the fvn_dtype of a scalar padded copy, or
// kGrad4 for a gradient volume.
constexpr int kGrad4 = 16;

template <typename I, int SHADE>
__device__ __forceinline__ bool batch_step(const MarchBatchView& bv, const Light& lt, const float4* s_tf, Ray& s,
                                           unsigned& nsh) {
    const MarchArgs& a = bv.a;
    const I sy = (I)(a.nx + 2 * kPad), sz = sy * (I)(a.ny + 2 * kPad);
    const float ux0 = a.ox - 0.5f, uy0 = a.oy - 0.5f, uz0 = a.oz - 0.5f;
    const float tfmax = (float)(a.ntf - 1);
    const float4* tf = s_tf + bv.tf_off;
    switch (bv.dtype) {
        case kGrad4:   // never with shading 2 (shadowed marches read the padded copy and the cells)
            if constexpr (SHADE == 2) {
                return true;
            } else {
                const float4* v = static_cast<const float4*>(a.pvol);
                return ray_step<Grad4Src, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
            }
        case FVN_U8: {
            const uint8_t* v = static_cast<const uint8_t*>(a.pvol);
            return ray_step<ScalarSrc<uint8_t>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
        }
        case FVN_U16: {
            const uint16_t* v = static_cast<const uint16_t*>(a.pvol);
            return ray_step<ScalarSrc<uint16_t>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
        }
        case FVN_F16: {
            const __half* v = static_cast<const __half*>(a.pvol);
            return ray_step<ScalarSrc<__half>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
        }
        default: {
            const float* v = static_cast<const float*>(a.pvol);
            return ray_step<ScalarSrc<float>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, s, nsh);
        }
    }
}

template <typename I, int SHADE>
__device__ __forceinline__ void batch_coop(const MarchBatchView& bv, const Light& lt, const float4* s_tf, Ray& r,
                                           unsigned& nsh) {
    const MarchArgs& a = bv.a;
    const I sy = (I)(a.nx + 2 * kPad), sz = sy * (I)(a.ny + 2 * kPad);
    const float ux0 = a.ox - 0.5f, uy0 = a.oy - 0.5f, uz0 = a.oz - 0.5f;
    const float tfmax = (float)(a.ntf - 1);
    const float4* tf = s_tf + bv.tf_off;
    switch (bv.dtype) {
        case kGrad4:
            if constexpr (SHADE != 2) {
                const float4* v = static_cast<const float4*>(a.pvol);
                coop_ray<Grad4Src, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
            }
            break;
        case FVN_U8: {
            const uint8_t* v = static_cast<const uint8_t*>(a.pvol);
            coop_ray<ScalarSrc<uint8_t>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
            break;
        }
        case FVN_U16: {
            const uint16_t* v = static_cast<const uint16_t*>(a.pvol);
            coop_ray<ScalarSrc<uint16_t>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
            break;
        }
        case FVN_F16: {
            const __half* v = static_cast<const __half*>(a.pvol);
            coop_ray<ScalarSrc<__half>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
            break;
        }
        default: {
            const float* v = static_cast<const float*>(a.pvol);
            coop_ray<ScalarSrc<float>, I, SHADE>(a, lt, v, tf, sy, sz, ux0, uy0, uz0, tfmax, r, nsh);
            break;
        }
    }
}

template <typename I, int SHADE>
__global__ void __launch_bounds__(128, SHADE == 2 ? 5 : 1)
    march_batch_kernel(const __grid_constant__ MarchBatch b) {
    extern __shared__ float4 s_tf[];
    __shared__ int s_start[kMaxViews + 1];   // first ticket of each view
    for (int k = 0; k < b.ntfs; ++k)
        load_tf<SHADE>(s_tf + b.tf_off[k], b.tf[k], b.tf_n[k]);
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int v = 0; v < b.nviews; ++v) {
            s_start[v] = acc;
            const MarchArgs& a = b.v[v].a;
            acc += min(max(*a.count, 0), a.W * a.H);
        }
        s_start[b.nviews] = acc;
    }
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nrays = s_start[b.nviews];
    unsigned long long my_samples = 0;
    unsigned nsh = 0;                 // shadow-ray samples of this lane
    Ray s;
    s.pix = -1;
    int view = 0;
    bool exhausted = false;
    for (;;) {
        if (!exhausted) {
            const unsigned idle = __ballot_sync(FULL, s.pix < 0);
            if (idle) {
                const int nidle = __popc(idle);
                int base = 0;
                if (lane == 0) base = atomicAdd(b.ticket, nidle);
                base = __shfl_sync(FULL, base, 0);
                if (base + nidle >= nrays) exhausted = true;
                if (s.pix < 0) {
                    const int r = base + __popc(idle & ((1u << lane) - 1u));
                    if (r < nrays) {
                        int v = 0;
                        while (v + 1 < b.nviews && r >= s_start[v + 1]) ++v;
                        view = v;
                        const MarchArgs& a = b.v[v].a;
                        if (start_ray(a, r - s_start[v], a.W * a.H, s) && !(s.tfar > -INFINITY)) {
                            finish_ray(a, s);   // missed the box: background, no sample
                            s.pix = -1;
                        }
                    }
                }
            }
        }
        unsigned busy = __ballot_sync(FULL, s.pix >= 0);
        if (busy == 0) {
            if (exhausted) break;
            continue;
        }
        while (busy != 0 && (exhausted || __popc(busy) >= b.refill_below)) {
            if (__popc(busy) <= b.coop_below) {
                do {
                    const int src = __ffs(busy) - 1;
                    Ray r = shfl_ray(s, src);
                    const int v = __shfl_sync(FULL, view, src);
                    batch_coop<I, SHADE>(b.v[v], b.light, s_tf, r, nsh);
                    if (lane == src) {
                        s = r;
                        my_samples += (unsigned long long)s.kf;
                        finish_ray(b.v[v].a, s);
                        s.pix = -1;
                    }
                    busy &= busy - 1u;
                } while (busy != 0);
                break;
            }
            if (s.pix >= 0 && batch_step<I, SHADE>(b.v[view], b.light, s_tf, s, nsh)) {
                my_samples += (unsigned long long)s.kf;
                finish_ray(b.v[view].a, s);
                s.pix = -1;
            }
            busy = __ballot_sync(FULL, s.pix >= 0);
        }
        if (exhausted && busy == 0) break;
    }
    if (b.nsamples) {
        if (SHADE == 2 && b.light.count) my_samples += nsh;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(FULL, my_samples, o);
        if (lane == 0 && my_samples) atomicAdd(b.nsamples, my_samples);
    }
}

// One warp per padded (y, z) row, eight rows per block: few, full blocks and
// coalesced row copies (clamp-to-edge in x, y and z).
template <typename T>
__global__ void __launch_bounds__(256) pad_volume_kernel(const T* __restrict__ src, int nx, int ny, int nz,
                                                         T* __restrict__ dst) {
    const int px = nx + 2 * kPad, py = ny + 2 * kPad, pz = nz + 2 * kPad;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= py * pz) return;
    const int z = row / py, y = row - z * py;
    const int sy = min(max(y - kPad, 0), ny - 1), sz = min(max(z - kPad, 0), nz - 1);
    const T* s = src + ((long long)sz * ny + sy) * nx;
    T* d = dst + (long long)row * px;
#pragma unroll 4
    for (int x = threadIdx.x & 31; x < px; x += 32) d[x] = prenorm(s[min(max(x - kPad, 0), nx - 1)]);
}

template <typename T>
static fvn_status pad_volume(fvn_ctx* ctx, const void* vol, int nx, int ny, int nz, void* pvol, cudaStream_t st) {
    const long long rows = (long long)(ny + 2 * kPad) * (nz + 2 * kPad);
    pad_volume_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(static_cast<const T*>(vol), nx, ny, nz,
                                                                       static_cast<T*>(pvol));
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

__device__ __forceinline__ int clampi(int v, int n) { return min(max(v, 0), n - 1); }

// Gradient volume over the padded box: (v, Dx, Dy, Dz) per voxel with
// D = (v[+1] - v[-1]) / 2 along each axis (clamp to edge).  One warp per
// padded (y, z) row, eight rows per block.
template <typename T>
__global__ void __launch_bounds__(256) grad4_volume_kernel(const T* __restrict__ src, int nx, int ny, int nz,
                                                           float4* __restrict__ dst) {
    const int px = nx + 2 * kPad, py = ny + 2 * kPad, pz = nz + 2 * kPad;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= py * pz) return;
    const int z = row / py, y = row - z * py;
    const int j = y - kPad, k = z - kPad;
    const long long sxy = (long long)nx * ny;
    const T* r0 = src + clampi(k, nz) * sxy + (long long)clampi(j, ny) * nx;
    const T* rym = src + clampi(k, nz) * sxy + (long long)clampi(j - 1, ny) * nx;
    const T* ryp = src + clampi(k, nz) * sxy + (long long)clampi(j + 1, ny) * nx;
    const T* rzm = src + clampi(k - 1, nz) * sxy + (long long)clampi(j, ny) * nx;
    const T* rzp = src + clampi(k + 1, nz) * sxy + (long long)clampi(j, ny) * nx;
    float4* d = dst + (long long)row * px;
    for (int x = threadIdx.x & 31; x < px; x += 32) {
        const int i = x - kPad;
        const int ic = clampi(i, nx), im = clampi(i - 1, nx), ip = clampi(i + 1, nx);
        d[x] = make_float4(load_norm(r0 + ic), 0.5f * (load_norm(r0 + ip) - load_norm(r0 + im)),
                           0.5f * (load_norm(ryp + ic) - load_norm(rym + ic)),
                           0.5f * (load_norm(rzp + ic) - load_norm(rzm + ic)));
    }
}

template <typename T>
static fvn_status grad4_volume(fvn_ctx* ctx, const void* vol, int nx, int ny, int nz, void* gvol, cudaStream_t st) {
    const long long rows = (long long)(ny + 2 * kPad) * (nz + 2 * kPad);
    grad4_volume_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(static_cast<const T*>(vol), nx, ny, nz,
                                                                          static_cast<float4*>(gvol));
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

// Shadow-ray cells over the padded box: cell (x, y, z) holds the padded
// voxels (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1) at z (clamp to edge).
// One warp per padded (y, z) row, eight rows per block.
template <typename T>
__global__ void __launch_bounds__(256) cell_volume_kernel(const T* __restrict__ src, int nx, int ny, int nz,
                                                          typename Quad<T>::type* __restrict__ dst) {
    const int px = nx + 2 * kPad, py = ny + 2 * kPad, pz = nz + 2 * kPad;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= py * pz) return;
    const int z = row / py, y = row - z * py;
    const long long zo = (long long)clampi(z - kPad, nz) * ny;
    const T* r0 = src + (zo + clampi(y - kPad, ny)) * nx;
    const T* r1 = src + (zo + clampi(y + 1 - kPad, ny)) * nx;
    typename Quad<T>::type* d = dst + (long long)row * px;
    for (int x = threadIdx.x & 31; x < px; x += 32) {
        const int x0 = clampi(x - kPad, nx), x1 = clampi(x + 1 - kPad, nx);
        d[x] = Quad<T>::make(prenorm(r0[x0]), prenorm(r0[x1]), prenorm(r1[x0]), prenorm(r1[x1]));
    }
}

template <typename T>
static fvn_status cell_volume(fvn_ctx* ctx, const void* vol, int nx, int ny, int nz, void* cells, cudaStream_t st) {
    const long long rows = (long long)(ny + 2 * kPad) * (nz + 2 * kPad);
    cell_volume_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        static_cast<const T*>(vol), nx, ny, nz, static_cast<typename Quad<T>::type*>(cells));
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

template <typename Src, typename I, bool SHADOWS = true>
static fvn_status launch_march(fvn_ctx* ctx, const MarchArgs& a, const Light& lt, int shade, cudaStream_t st) {
    const size_t smem = (size_t)tf_slots(a.ntf, shade) * sizeof(float4);
    auto kern = shade == 1 ? march_kernel<Src, I, 1> : march_kernel<Src, I, 0>;
    if constexpr (SHADOWS) {
        if (shade == 2) kern = march_kernel<Src, I, 2>;
    }
    if (smem > 48 * 1024)
        FVN_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    const int bps = a.ids ? ctx->march_blocks_per_sm : ctx->march_blocks_per_sm_dense;
    if (bps > 0) per_sm = std::min(per_sm, bps);
    if (per_sm < 1) per_sm = 1;
    const int grid = ctx->num_sms * per_sm;
    kern<<<grid, 128, smem, st>>>(a, lt);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
}

static unsigned long long padded_voxels(const fvn_volume* vol) {
    return (unsigned long long)(vol->nx + 2 * kPad) * (vol->ny + 2 * kPad) * (vol->nz + 2 * kPad);
}

// The light of shading 2 (zero for the other modes).
static Light make_light(const fvn_ctx* ctx, const fvn_march_params* mp) {
    Light lt{};
    if (mp->shading != 2) return lt;
    lt.count = ctx->march_count_shadow;
    double l[3] = {mp->light_dir[0], mp->light_dir[1], mp->light_dir[2]};
    const double ll = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (double& x : l) x /= ll;
    lt.lx = (float)l[0];
    lt.ly = (float)l[1];
    lt.lz = (float)l[2];
    lt.ilx = l[0] != 0.0 ? (float)(1.0 / l[0]) : 1.0f;
    lt.ily = l[1] != 0.0 ? (float)(1.0 / l[1]) : 1.0f;
    lt.ilz = l[2] != 0.0 ? (float)(1.0 / l[2]) : 1.0f;
    lt.srate = mp->shadow_rate;
    lt.ds = (float)((double)mp->shadow_rate * mp->step_vox);
    lt.inv_ds = (float)(1.0 / ((double)mp->shadow_rate * mp->step_vox));
    return lt;
}

// Per-view fields of the march arguments: volume size, transfer function,
// camera basis in voxel units, frame size, step and background.
static MarchArgs view_args(const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                           const fvn_march_params* mp) {
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
    a.tiles_x = (a.W + 7) / 8;
    a.n_dense = a.tiles_x * ((a.H + 3) / 4) * 32;
    a.plane = (long long)a.W * a.H;
    return a;
}

static const void* march_cells(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp,
                               const void* buf);
static fvn_status launch_for(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, const MarchArgs& a,
                             cudaStream_t st);

fvn_status march_impl(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                      const fvn_march_params* mp, const int32_t* ids, const int32_t* count, float* rgbam,
                      unsigned long long* nsamples, cudaStream_t st, const uint8_t* reject) {
    MarchArgs a = view_args(vol, tf, cam, mp);
    a.ids = ids;
    a.count = count;
    a.rgbam = rgbam;
    a.nsamples = nsamples;
    a.refill_below = ids ? ctx->march_refill : ctx->march_refill_dense;
    a.coop_below = ids ? ctx->march_coop : ctx->march_coop_dense;
    a.ticket = ctx->d_ticket + (ctx->ticket_ring++ & 63);
    a.reject = ids ? nullptr : reject;
    if (ids || reject) FVN_CUDA(ctx, cudaMemsetAsync(rgbam, 0, 5 * sizeof(float) * (size_t)a.plane, st));
    FVN_CUDA(ctx, cudaMemsetAsync(a.ticket, 0, sizeof(int), st));
    stage_mark(ctx, TM_SETUP, st);
    const size_t bytes = march_volume_bytes(ctx, vol, mp);
    if (ctx->pad_bytes < bytes) {
        // growing the volume scratch is a synchronising step
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(ctx->pad_buf);
        ctx->pad_buf = nullptr;
        ctx->pad_bytes = 0;
        ctx->pad_key = PreparedKey();
        FVN_CUDA(ctx, cudaMalloc(&ctx->pad_buf, bytes));
        ctx->pad_bytes = bytes;
    }
    a.pvol = ctx->pad_buf;
    a.svol = march_cells(ctx, vol, mp, ctx->pad_buf);
    // one pass over the volume, skipped while a non-zero generation says the copy is current
    fvn_status ps = march_volume_prepare_cached(ctx, vol, mp, ctx->pad_buf, ctx->pad_key, st);
    if (ps != FVN_OK) return ps;
    stage_mark(ctx, TM_PREP, st);
    const fvn_status ls = launch_for(ctx, vol, mp, a, st);
    stage_mark(ctx, TM_MARCH, st);
    return ls;
}

// The march kernel for the volume's copy and voxel type.
static fvn_status launch_for(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, const MarchArgs& a,
                             cudaStream_t st) {
    const bool big = padded_voxels(vol) >= (1ull << 31);
    const int shade = mp->shading;
    const Light lt = make_light(ctx, mp);
    if (march_uses_grad4(ctx, vol, mp)) return launch_march<Grad4Src, int, false>(ctx, a, lt, shade, st);
    switch (vol->dtype) {
        case FVN_U8:
            return big ? launch_march<ScalarSrc<uint8_t>, long long>(ctx, a, lt, shade, st)
                       : launch_march<ScalarSrc<uint8_t>, int>(ctx, a, lt, shade, st);
        case FVN_U16:
            return big ? launch_march<ScalarSrc<uint16_t>, long long>(ctx, a, lt, shade, st)
                       : launch_march<ScalarSrc<uint16_t>, int>(ctx, a, lt, shade, st);
        case FVN_F16:
            return big ? launch_march<ScalarSrc<__half>, long long>(ctx, a, lt, shade, st)
                       : launch_march<ScalarSrc<__half>, int>(ctx, a, lt, shade, st);
        default:
            return big ? launch_march<ScalarSrc<float>, long long>(ctx, a, lt, shade, st)
                       : launch_march<ScalarSrc<float>, int>(ctx, a, lt, shade, st);
    }
}

// Shaded marches read a gradient volume (16 bytes per padded voxel) when the
// option allows it and it takes at most 4 GiB; the others a padded copy.
// Shadowed marches (shading 2) read the padded copy for their samples and
// the shadow-ray cells (4 voxels per padded voxel) for their shadow rays.
bool march_uses_grad4(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp) {
    return mp->shading == 1 && ctx->march_grad4 != 0 && padded_voxels(vol) * 16ull <= (4ull << 30);
}

static size_t voxel_bytes(const fvn_volume* vol) {
    return vol->dtype == FVN_U8 ? 1 : (vol->dtype == FVN_F32 ? 4 : 2);
}

// Offset of the shadow-ray cells after the padded copy.
static size_t cells_offset(const fvn_volume* vol) {
    return (voxel_bytes(vol) * (size_t)padded_voxels(vol) + 255) & ~(size_t)255;
}

// Shadowed marches read shadow-ray cells.
static bool uses_cells(const fvn_ctx*, const fvn_march_params* mp) { return mp->shading == 2; }

size_t march_volume_bytes(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp) {
    if (march_uses_grad4(ctx, vol, mp)) return 16 * (size_t)padded_voxels(vol);
    const size_t pad = voxel_bytes(vol) * (size_t)padded_voxels(vol);
    return uses_cells(ctx, mp) ? cells_offset(vol) + 4 * pad : pad;
}

// The shadow-ray cells inside a volume buffer (NULL when the march reads none).
static const void* march_cells(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp,
                               const void* buf) {
    return uses_cells(ctx, mp) ? static_cast<const char*>(buf) + cells_offset(vol) : nullptr;
}

template <typename T>
static fvn_status prepare_as(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, void* buf, bool g4,
                             cudaStream_t st) {
    if (g4) return grad4_volume<T>(ctx, vol->data, vol->nx, vol->ny, vol->nz, buf, st);
    fvn_status s = pad_volume<T>(ctx, vol->data, vol->nx, vol->ny, vol->nz, buf, st);
    if (s != FVN_OK || !uses_cells(ctx, mp)) return s;
    return cell_volume<T>(ctx, vol->data, vol->nx, vol->ny, vol->nz, static_cast<char*>(buf) + cells_offset(vol),
                          st);
}

fvn_status march_volume_prepare(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, void* buf,
                                cudaStream_t st) {
    const bool g4 = march_uses_grad4(ctx, vol, mp);
    switch (vol->dtype) {
        case FVN_U8: return prepare_as<uint8_t>(ctx, vol, mp, buf, g4, st);
        case FVN_U16: return prepare_as<uint16_t>(ctx, vol, mp, buf, g4, st);
        case FVN_F16: return prepare_as<__half>(ctx, vol, mp, buf, g4, st);
        default: return prepare_as<float>(ctx, vol, mp, buf, g4, st);
    }
}

// Kind of copy a march reads: 0 padded copy, 1 gradient volume, 2 padded
// copy + shadow cells.
static int volume_kind(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp) {
    return march_uses_grad4(ctx, vol, mp) ? 1 : (uses_cells(ctx, mp) ? 2 : 0);
}

fvn_status march_volume_prepare_cached(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, void* buf,
                                       PreparedKey& key, cudaStream_t st) {
    const int kind = volume_kind(ctx, vol, mp);
    if (key.matches(vol, kind)) return FVN_OK;
    key = PreparedKey();
    const fvn_status s = march_volume_prepare(ctx, vol, mp, buf, st);
    if (s != FVN_OK || vol->generation == 0) return s;
    key.data = vol->data;
    key.nx = vol->nx;
    key.ny = vol->ny;
    key.nz = vol->nz;
    key.dtype = vol->dtype;
    key.kind = kind;
    key.generation = vol->generation;
    return FVN_OK;
}

fvn_status march_batch_impl(fvn_ctx* ctx, const BatchMarchView* views, int n, const fvn_march_params* mp,
                            unsigned long long* nsamples, cudaStream_t st) {
    MarchBatch b{};
    b.light = make_light(ctx, mp);
    b.nviews = n;
    b.nsamples = nsamples;
    b.refill_below = ctx->march_refill;
    b.coop_below = ctx->march_coop;
    int tf_total = 0, tf_slots_total = 0;
    bool big = false;
    for (int i = 0; i < n; ++i) {
        const BatchMarchView& v = views[i];
        MarchBatchView& bv = b.v[i];
        bv.a = view_args(v.vol, v.tf, v.cam, mp);
        bv.a.pvol = v.pvol;
        bv.a.svol = march_cells(ctx, v.vol, mp, v.pvol);
        bv.a.ids = v.ids;
        bv.a.count = v.count;
        bv.a.rgbam = v.rgbam;
        bv.dtype = march_uses_grad4(ctx, v.vol, mp) ? kGrad4 : v.vol->dtype;
        big = big || padded_voxels(v.vol) >= (1ull << 31);
        int k = 0;   // transfer functions are shared by pointer
        while (k < b.ntfs && !(b.tf[k] == bv.a.tf && b.tf_n[k] == bv.a.ntf)) ++k;
        if (k == b.ntfs) {
            b.tf[k] = bv.a.tf;
            b.tf_n[k] = bv.a.ntf;
            b.tf_off[k] = tf_slots_total;
            tf_slots_total += tf_slots(bv.a.ntf, mp->shading);
            tf_total += bv.a.ntf;
            ++b.ntfs;
        }
        bv.tf_off = b.tf_off[k];
    }
    if (tf_total > 4096)
        return set_error(ctx, FVN_ERR_ARG, "the batch's transfer functions hold %d entries (at most 4096)", tf_total);
    b.ticket = ctx->d_ticket + (ctx->ticket_ring++ & 63);
    FVN_CUDA(ctx, cudaMemsetAsync(b.ticket, 0, sizeof(int), st));
    const int shade = mp->shading;
    auto kern = big ? (shade == 2 ? march_batch_kernel<long long, 2>
                                  : (shade == 1 ? march_batch_kernel<long long, 1> : march_batch_kernel<long long, 0>))
                    : (shade == 2 ? march_batch_kernel<int, 2>
                                  : (shade == 1 ? march_batch_kernel<int, 1> : march_batch_kernel<int, 0>));
    const size_t smem = (size_t)tf_slots_total * sizeof(float4);
    if (smem > 48 * 1024)
        FVN_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    if (ctx->march_blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->march_blocks_per_sm);
    if (per_sm < 1) per_sm = 1;
    kern<<<ctx->num_sms * per_sm, 128, smem, st>>>(b);
    FVN_LAUNCH_CHECK(ctx);
    return FVN_OK;
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
    if ((st = validate_march_params(ctx, mp)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, rgbam != nullptr, "rgbam output is NULL");
    FVN_CHECK_ARG(ctx, (ids == nullptr) == (count == nullptr), "ids and count must both be set or both NULL");
    return march_impl(ctx, vol, tf, cam, mp, ids, count, rgbam, nsamples, as_stream(stream));
}

extern "C" fvn_status fvn_march_masked(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf,
                                       const fvn_camera* cam, const fvn_march_params* mp, const uint8_t* mask,
                                       float* rgbam, unsigned long long* nsamples, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, mask != nullptr, "mask is NULL");
    fvn_status st;
    if ((st = validate_volume(ctx, vol)) != FVN_OK) return st;
    if ((st = validate_camera(ctx, cam)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, tf && tf->rgba && tf->n >= 2 && tf->n <= 4096, "transfer function needs 2..4096 entries");
    FVN_CHECK_ARG(ctx, ((uintptr_t)tf->rgba & 15) == 0, "transfer function must be 16-byte aligned");
    if ((st = validate_march_params(ctx, mp)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, rgbam != nullptr, "rgbam output is NULL");
    return march_impl(ctx, vol, tf, cam, mp, nullptr, nullptr, rgbam, nsamples, as_stream(stream), mask);
}
