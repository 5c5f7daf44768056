/*
 * Oracle: FP64 emission-absorption ray marcher (dense and masked).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code with the CUDA
 * path.
 *
 * What it computes (the paper's "Foveated Rendering" and "Rendering"
 * subsections describe a CUDA ray-marching DVR renderer but fix none of its
 * conventions; the readings below are this project's):
 *
 *  - Volume: nx*ny*nz voxels, x fastest, occupying the box [0,n] in voxel
 *    units; voxel centres at i + 0.5.  World space: the box is centred at the
 *    origin and scaled so its longest axis has length 1 (p_vox = p_w / s + n/2
 *    with s = 1 / max(n)).
 *  - Values are normalised per voxel to [0,1]: u8 / 255, u16 / 65535, f16 and
 *    f32 clamped to [0,1].  Trilinear interpolation between voxel centres,
 *    clamp-to-edge.
 *  - Camera: pinhole, forward f = |target - eye|, right r = |f x up|,
 *    u = r x f; pixel (x, y) (y = 0 at the top) looks along
 *    |f + sx r + sy u| with sx = (2(x+.5)/W - 1) tan(fov/2) W/H,
 *    sy = (1 - 2(y+.5)/H) tan(fov/2).
 *  - Ray / box slab test; t_near = max(t_enter, 0); samples at
 *    t_k = t_near + k dt for every k >= 0 with t_k < t_far (strict).
 *  - 1-D RGBA transfer function of ntf entries: continuous index v (ntf - 1),
 *    linear between entries.
 *  - shading 1, Phong with a headlight (L = V = -dir, so H = L): gradient by
 *    central differences of the trilinear field at +-1 voxel, n = -g/|g|,
 *    c' = clamp(c (0.2 + 0.7 |n.L|) + 0.3 |n.L|^32, 0, 1); |g| < 1e-6 keeps c.
 *    Samples with alpha = 0 contribute nothing and are not shaded.
 *  - shading 2, the paper's global shadows ("Foveated Rendering": one shadow
 *    ray per sample towards the light, at a quarter of the main sample
 *    rate): a directional light along the unit vector L (world and voxel
 *    space share directions: the box is scaled uniformly).  From a sample
 *    point p the shadow ray takes samples at s_j = j ds, j = 1, 2, ..., with
 *    ds = rate dt, while s_j < s_exit (where p + s L leaves the box).  Each
 *    stands for rate main steps of its TF opacity, the last one for the part
 *    of its step left inside the box:
 *        T = prod_j (1 - a_j)^(rate min(1, (s_exit - s_j) / ds)),
 *    so T is continuous in s_exit.  The shadow ray stops once T < 2^-14 (the
 *    light it could still carry then moves no output channel by as much).
 *    H = |L - dir|; with |g| >= 1e-6,
 *        c' = clamp(c (0.2 + 0.7 T |n.L|) + 0.3 T |n.H|^32, 0, 1),
 *    otherwise c' = clamp(c (0.2 + 0.7 T), 0, 1); no specular term where
 *    |L - dir| < 1e-12.
 *  - Front-to-back compositing with non-premultiplied colour:
 *    C += (1 - A) a c', A += (1 - A) a; stop after a sample once A >= term.
 *    Output RGB = C + (1 - A) bg, alpha = A, mask channel = 1.  Rays that miss
 *    the box give bg, A = 0, mask = 1.
 *
 * Ambiguity flags (bit 0: the sample count (t_far - t_near)/dt lies within
 * 1e-3 of an integer; bit 1: A came within 1e-6 of the termination threshold;
 * bit 2: a shaded sample had |g| < 1e-5) mark pixels where an FP32
 * implementation of the same definition may legitimately take the other side
 * of a discontinuity.  The windows are a few times the largest FP32 / FP64
 * difference of these quantities met on a foveated 1080p frame (1.6e-4
 * samples for the count, 4.0e-7 for A): FP32 ray geometry at a few hundred
 * voxels from the eye, and FP32 compositing over hundreds of steps, cannot
 * resolve them more finely.  count_shift / term_override let a test compute the
 * alternative result for such pixels.  Shadow rays need no flag: T is
 * continuous in the exit distance, and where FP32 and FP64 disagree on
 * stopping a shadow ray, T differs by less than the 2^-14 cutoff.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_U8 = 0, OR_U16 = 1, OR_F16 = 2, OR_F32 = 3 };

typedef struct {
    const void* data;
    int dtype;
    int n[3];
} or_vol;

/* IEEE-754 binary16 -> double, written from the format definition. */
static double half_to_double(uint16_t h) {
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int m = h & 0x3ff;
    double v;
    if (e == 0) v = ldexp((double)m, -24);                 /* subnormal */
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1.0 + m / 1024.0, e - 15);
    return sign ? -v : v;
}

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

static double voxel(const or_vol* v, int x, int y, int z) {
    if (x < 0) x = 0; if (x > v->n[0] - 1) x = v->n[0] - 1;
    if (y < 0) y = 0; if (y > v->n[1] - 1) y = v->n[1] - 1;
    if (z < 0) z = 0; if (z > v->n[2] - 1) z = v->n[2] - 1;
    size_t i = ((size_t)z * (size_t)v->n[1] + (size_t)y) * (size_t)v->n[0] + (size_t)x;
    switch (v->dtype) {
        case OR_U8: return ((const uint8_t*)v->data)[i] / 255.0;
        case OR_U16: return ((const uint16_t*)v->data)[i] / 65535.0;
        case OR_F16: return clamp01(half_to_double(((const uint16_t*)v->data)[i]));
        default: return clamp01((double)((const float*)v->data)[i]);
    }
}

/* Trilinear interpolation between voxel centres (i + 0.5), clamp to edge. */
static double trilinear(const or_vol* v, double px, double py, double pz) {
    double ux = px - 0.5, uy = py - 0.5, uz = pz - 0.5;
    double fx = floor(ux), fy = floor(uy), fz = floor(uz);
    int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    double tx = ux - fx, ty = uy - fy, tz = uz - fz;
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
                acc += w * voxel(v, ix + dx, iy + dy, iz + dz);
            }
    return acc;
}

/* TF lookup at value val: col[4] = linear interpolation at index val (ntf - 1). */
static void tf_sample(const float* tf, int ntf, double val, double* col) {
    double x = val * (double)(ntf - 1);
    double fi = floor(x);
    int i = (int)fi;
    if (i < 0) i = 0;
    if (i > ntf - 2) i = ntf - 2;
    double fr = x - (double)i;
    for (int ch = 0; ch < 4; ++ch)
        col[ch] = (double)tf[4 * i + ch] * (1.0 - fr) + (double)tf[4 * (i + 1) + ch] * fr;
}

#define SHADOW_CUTOFF (1.0 / 16384.0)

/* Transmittance towards a directional light L (unit) from the voxel-space
 * point p, by the shadow ray defined in the header. */
static double shadow_transmittance(const or_vol* v, const float* tf, int ntf, const double* p, const double* L,
                                   double dt, int rate) {
    double ds = (double)rate * dt;
    double se = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (L[a] == 0.0) continue;
        double s = ((L[a] > 0.0 ? (double)v->n[a] : 0.0) - p[a]) / L[a];
        if (s < se) se = s;
    }
    double T = 1.0;
    for (int64_t j = 1; (double)j * ds < se; ++j) {
        double s = (double)j * ds;
        double col[4];
        tf_sample(tf, ntf, trilinear(v, p[0] + s * L[0], p[1] + s * L[1], p[2] + s * L[2]), col);
        double e = (se - s) / ds;
        if (e > 1.0) e = 1.0;
        if (col[3] > 0.0) T *= pow(1.0 - col[3], (double)rate * e);
        if (T < SHADOW_CUTOFF) break;
    }
    return T;
}

static void normalize3(double* a) {
    double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

typedef struct {
    double o[3];      /* eye in voxel units */
    double f[3], r[3], u[3];
    double tanh_, aspect;
    int W, H;
} or_cam;

static void setup_camera(const double* cam, int W, int H, const or_vol* v, or_cam* c) {
    int nmax = v->n[0];
    if (v->n[1] > nmax) nmax = v->n[1];
    if (v->n[2] > nmax) nmax = v->n[2];
    for (int a = 0; a < 3; ++a) c->o[a] = cam[a] * (double)nmax + 0.5 * v->n[a];
    for (int a = 0; a < 3; ++a) c->f[a] = cam[3 + a] - cam[a];
    normalize3(c->f);
    cross3(c->f, cam + 6, c->r);
    normalize3(c->r);
    cross3(c->r, c->f, c->u);
    c->tanh_ = tan(cam[9] * M_PI / 360.0);
    c->aspect = (double)W / (double)H;
    c->W = W;
    c->H = H;
}

/* One ray; returns the number of classified samples. */
typedef struct {
    double dt, term, bg[3];
    int shading;
    double L[3];      /* shading 2: unit direction towards the light */
    int rate;         /* shading 2: shadow step = rate dt */
} or_mp;

static int64_t march_ray(const or_vol* v, const float* tf, int ntf, const or_cam* c, int px, int py,
                         const or_mp* m, double term, int count_shift, double* rgba, int* amb, double* mg) {
    const double dt = m->dt;
    const double* bg = m->bg;
    const int shading = m->shading;
    double sx = (2.0 * (px + 0.5) / c->W - 1.0) * c->tanh_ * c->aspect;
    double sy = (1.0 - 2.0 * (py + 0.5) / c->H) * c->tanh_;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = c->f[a] + sx * c->r[a] + sy * c->u[a];
    normalize3(d);
    *amb = 0;
    if (mg) mg[0] = mg[1] = INFINITY;
    rgba[0] = bg[0]; rgba[1] = bg[1]; rgba[2] = bg[2]; rgba[3] = 0.0;

    double tn = -INFINITY, tfar = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (c->o[a] < 0.0 || c->o[a] > (double)v->n[a]) return 0;
        } else {
            double t0 = (0.0 - c->o[a]) / d[a];
            double t1 = ((double)v->n[a] - c->o[a]) / d[a];
            if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
            if (t0 > tn) tn = t0;
            if (t1 < tfar) tfar = t1;
        }
    }
    double tnear = tn > 0.0 ? tn : 0.0;
    if (!(tnear < tfar)) return 0;

    double span = (tfar - tnear) / dt;
    if (fabs(span - nearbyint(span)) < 1e-3) *amb |= 1;
    if (mg) mg[0] = fabs(span - nearbyint(span));
    /* number of k >= 0 with tnear + k dt < tfar */
    int64_t nsamp = (int64_t)ceil(span);
    while (nsamp > 0 && tnear + (double)(nsamp - 1) * dt >= tfar) --nsamp;
    while (tnear + (double)nsamp * dt < tfar) ++nsamp;
    nsamp += count_shift;
    if (nsamp < 0) nsamp = 0;

    double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
    int64_t k;
    for (k = 0; k < nsamp; ++k) {
        double t = tnear + (double)k * dt;
        double p[3] = {c->o[0] + t * d[0], c->o[1] + t * d[1], c->o[2] + t * d[2]};
        double col[4];
        tf_sample(tf, ntf, trilinear(v, p[0], p[1], p[2]), col);
        double alpha = col[3];
        if (alpha > 0.0) {
            if (shading) {
                double gx = 0.5 * (trilinear(v, p[0] + 1.0, p[1], p[2]) - trilinear(v, p[0] - 1.0, p[1], p[2]));
                double gy = 0.5 * (trilinear(v, p[0], p[1] + 1.0, p[2]) - trilinear(v, p[0], p[1] - 1.0, p[2]));
                double gz = 0.5 * (trilinear(v, p[0], p[1], p[2] + 1.0) - trilinear(v, p[0], p[1], p[2] - 1.0));
                double gn = sqrt(gx * gx + gy * gy + gz * gz);
                if (gn < 1e-5) *amb |= 4;
                if (shading == 1) {
                    if (gn >= 1e-6) {
                        double ndl = fabs(gx * d[0] + gy * d[1] + gz * d[2]) / gn;
                        double spec = ndl;
                        for (int s = 0; s < 5; ++s) spec = spec * spec; /* ndl^32 */
                        for (int ch = 0; ch < 3; ++ch)
                            col[ch] = clamp01(col[ch] * (0.2 + 0.7 * ndl) + 0.3 * spec);
                    }
                } else {
                    const double* L = m->L;
                    double T = shadow_transmittance(v, tf, ntf, p, L, dt, m->rate);
                    if (gn >= 1e-6) {
                        double ndl = fabs(gx * L[0] + gy * L[1] + gz * L[2]) / gn;
                        double h[3] = {L[0] - d[0], L[1] - d[1], L[2] - d[2]};
                        double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
                        double spec = 0.0;
                        if (hn >= 1e-12) {
                            spec = fabs(gx * h[0] + gy * h[1] + gz * h[2]) / (gn * hn);
                            for (int s = 0; s < 5; ++s) spec = spec * spec; /* ndh^32 */
                        }
                        for (int ch = 0; ch < 3; ++ch)
                            col[ch] = clamp01(col[ch] * (0.2 + 0.7 * T * ndl) + 0.3 * T * spec);
                    } else {
                        for (int ch = 0; ch < 3; ++ch) col[ch] = clamp01(col[ch] * (0.2 + 0.7 * T));
                    }
                }
            }
            double w = (1.0 - A) * alpha;
            C[0] += w * col[0];
            C[1] += w * col[1];
            C[2] += w * col[2];
            A += w;
        }
        if (fabs(A - term) < 1e-6) *amb |= 2;
        if (mg && fabs(A - term) < mg[1]) mg[1] = fabs(A - term);
        if (A >= term) { ++k; break; }
    }
    rgba[0] = C[0] + (1.0 - A) * bg[0];
    rgba[1] = C[1] + (1.0 - A) * bg[1];
    rgba[2] = C[2] + (1.0 - A) * bg[2];
    rgba[3] = A;
    return k;
}

/*
 * mp = {step, term_alpha, bg_r, bg_g, bg_b, shading, light_x, light_y, light_z, shadow_rate}
 * (the light direction is normalised here; the last four only matter for shading 2)
 * cam = {eye[3], target[3], up[3], fov_y_deg}
 * ids == NULL: every pixel (dense).  Otherwise only the listed pixel ids
 * y*W + x are marched and every other pixel of out is 0.
 * out: [5][H][W] float64 (R, G, B, A, M).  amb: [H*W] or NULL.
 * margin: [H*W][2] or NULL; per marched pixel the distances behind its
 * ambiguity flags: |(t_far - t_near) / dt - nearest integer| and the
 * smallest |A - term| over its composited steps (INFINITY where none);
 * a diagnostic of the flags, not part of the rendering.
 * term_override > 0 replaces mp's termination threshold.
 * Returns the total number of classified samples.
 */
int64_t or_march(const void* data, int dtype, int nx, int ny, int nz, const float* tf, int ntf,
                 const double* cam, int W, int H, const double* mp, const int32_t* ids, int64_t nids,
                 int count_shift, double term_override, double* out, uint8_t* amb, double* margin) {
    or_vol v = {data, dtype, {nx, ny, nz}};
    or_cam c;
    setup_camera(cam, W, H, &v, &c);
    const int64_t npix = (int64_t)W * H;
    memset(out, 0, sizeof(double) * 5 * (size_t)npix);
    if (amb) memset(amb, 0, (size_t)npix);
    const int64_t nrays = ids ? nids : npix;
    or_mp m = {mp[0], mp[1], {mp[2], mp[3], mp[4]}, (int)mp[5], {mp[6], mp[7], mp[8]}, (int)mp[9]};
    if (m.shading == 2) normalize3(m.L);
    const double term = term_override > 0.0 ? term_override : mp[1];
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t r = 0; r < nrays; ++r) {
        int64_t pix = ids ? (int64_t)ids[r] : r;
        int px = (int)(pix % W), py = (int)(pix / W);
        double rgba[4];
        int a = 0;
        total += march_ray(&v, tf, ntf, &c, px, py, &m, term, count_shift, rgba, &a,
                           margin ? margin + 2 * pix : NULL);
        out[0 * npix + pix] = rgba[0];
        out[1 * npix + pix] = rgba[1];
        out[2 * npix + pix] = rgba[2];
        out[3 * npix + pix] = rgba[3];
        out[4 * npix + pix] = 1.0;
        if (amb) amb[pix] = (uint8_t)a;
    }
    return total;
}

/* Threads of the OpenMP loops (the CPU baseline also times one core). */
void or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* Normalised trilinear value at voxel-space points p[n][3] (for tests). */
void or_trilinear(const void* data, int dtype, int nx, int ny, int nz, const double* p, int64_t n,
                  double* out) {
    or_vol v = {data, dtype, {nx, ny, nz}};
    for (int64_t i = 0; i < n; ++i) out[i] = trilinear(&v, p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

/* Ray origin (voxel units) and unit direction of pixel (px, py) (for tests). */
void or_ray(const double* cam, int W, int H, int nx, int ny, int nz, int px, int py, double* o,
            double* d) {
    or_vol v = {NULL, OR_F32, {nx, ny, nz}};
    or_cam c;
    setup_camera(cam, W, H, &v, &c);
    double sx = (2.0 * (px + 0.5) / W - 1.0) * c.tanh_ * c.aspect;
    double sy = (1.0 - 2.0 * (py + 0.5) / H) * c.tanh_;
    for (int a = 0; a < 3; ++a) d[a] = c.f[a] + sx * c.r[a] + sy * c.u[a];
    normalize3(d);
    for (int a = 0; a < 3; ++a) o[a] = c.o[a];
}

/* Shadow transmittance (shading 2) at voxel-space points p[n][3] towards the
 * light direction L[3] (normalised here), for tests. */
void or_shadow(const void* data, int dtype, int nx, int ny, int nz, const float* tf, int ntf, const double* p,
               int64_t n, const double* light, double dt, int rate, double* out) {
    or_vol v = {data, dtype, {nx, ny, nz}};
    double L[3] = {light[0], light[1], light[2]};
    normalize3(L);
    for (int64_t i = 0; i < n; ++i) out[i] = shadow_transmittance(&v, tf, ntf, p + 3 * i, L, dt, rate);
}
