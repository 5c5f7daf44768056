// Batched multi-view render: the per-frame path of the paper's pipeline
// (Fig. "pipeline": sample mask -> compaction -> sparse rendering ->
// reconstruction) for up to FVN_MAX_VIEWS views of uneven sizes -- stereo
// pairs, several resolutions, several volumes -- with one launch per stage
// instead of one per view:
//
//   mask + compaction   1 launch over the Z-ordered tiles of every view
//   volume padding      1 launch per distinct volume
//   ray march           1 persistent launch over the rays of every view
//   network             1 launch per layer over the tiles of every view
//
// Per view the arithmetic is that of fvn_render, so each view's output is the
// single-view output bit for bit.  Workspace layout (one device allocation,
// 256-byte aligned pieces): per view its mask (1 B/px), id list (4 B/px),
// sparse frame (20 B/px) and activation buffers (188 B/px at 16/32/64
// channels), then the per-view counts.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace fvn {
namespace {

struct ViewLayout {
    size_t mask, ids, rgbam, plan;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets of every view's pieces; returns the total size.
size_t batch_layout(const fvn_view* views, int n, ViewLayout* lay) {
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t npix = (size_t)views[i].cam.width * views[i].cam.height;
        lay[i].mask = off;
        off += align256(npix);
        lay[i].ids = off;
        off += align256(npix * sizeof(int32_t));
        lay[i].rgbam = off;
        off += align256(5 * npix * sizeof(float));
        lay[i].plan = off;
        off += align256(plan_view(views[i].cam.width, views[i].cam.height, nullptr, nullptr));
    }
    return off + align256(kMaxViews * sizeof(int32_t));
}

fvn_status validate_view(fvn_ctx* ctx, const fvn_view& v, int i) {
    fvn_status st;
    if ((st = validate_volume(ctx, v.vol)) != FVN_OK) return st;
    if ((st = validate_camera(ctx, &v.cam)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, v.tf && v.tf->rgba && v.tf->n >= 2 && v.tf->n <= 4096,
                  "view %d: transfer function needs 2..4096 entries", i);
    FVN_CHECK_ARG(ctx, ((uintptr_t)v.tf->rgba & 15) == 0, "view %d: transfer function must be 16-byte aligned", i);
    const fvn_foveation& f = v.fov;
    FVN_CHECK_ARG(ctx, isfinite(f.focal_px[0]) && isfinite(f.focal_px[1]), "view %d: focal point is not finite", i);
    FVN_CHECK_ARG(ctx, f.fovea_radius >= 0.f && f.falloff_sigma >= 0.f && f.p_base >= 0.f && f.p_base <= 1.f &&
                           isfinite(f.fovea_radius) && isfinite(f.falloff_sigma),
                  "view %d: foveation radius / falloff must be >= 0 and p_base in [0, 1]", i);
    FVN_CHECK_ARG(ctx, v.rgb != nullptr, "view %d: rgb output is NULL", i);
    if (v.prev_rgb && !ctx->recurrent)
        return set_error(ctx, FVN_ERR_STATE, "view %d: a previous frame needs the recurrent network's weights", i);
    return FVN_OK;
}

bool same_volume(const fvn_volume* a, const fvn_volume* b) {
    return a->data == b->data && a->nx == b->nx && a->ny == b->ny && a->nz == b->nz && a->dtype == b->dtype;
}

}  // namespace
}  // namespace fvn

namespace fvn {
namespace {

// The batch; leaves every view's mask and volume copy in
// ctx->batch_ws.view_mask / view_pvol.
fvn_status render_batch_impl(fvn_ctx* ctx, const fvn_view* views, int nviews, const fvn_march_params* mp,
                             int precision, unsigned long long* nsamples, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, views != nullptr, "views is NULL");
    FVN_CHECK_ARG(ctx, nviews >= 1 && nviews <= kMaxViews, "%d views (1..%d)", nviews, kMaxViews);
    fvn_status vs = validate_march_params(ctx, mp);
    if (vs != FVN_OK) return vs;
    FVN_CHECK_ARG(ctx, precision == FVN_PREC_FP16 || precision == FVN_PREC_FP8, "unknown precision %d", precision);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    if (precision == FVN_PREC_FP8 && !ctx->has_fp8)
        return set_error(ctx, FVN_ERR_STATE, "FP8 needs calibrated scales (call fvn_calibrate_fp8 first)");
    // distinct volumes (by pointer, size and type), each padded once
    const fvn_volume* vols[kMaxBatchVolumes];
    int nvol = 0, vol_of[kMaxViews];
    for (int i = 0; i < nviews; ++i) {
        fvn_status st = validate_view(ctx, views[i], i);
        if (st != FVN_OK) return st;
        int k = 0;
        while (k < nvol && !same_volume(vols[k], views[i].vol)) ++k;
        if (k == nvol) {
            FVN_CHECK_ARG(ctx, nvol < kMaxBatchVolumes, "more than %d distinct volumes in one batch",
                          kMaxBatchVolumes);
            vols[nvol++] = views[i].vol;
        }
        vol_of[i] = k;
    }
    int tf_total = 0;   // distinct transfer functions share the march kernel's shared memory
    for (int i = 0; i < nviews; ++i) {
        bool seen = false;
        for (int j = 0; j < i && !seen; ++j)
            seen = views[j].tf->rgba == views[i].tf->rgba && views[j].tf->n == views[i].tf->n;
        if (!seen) tf_total += views[i].tf->n;
    }
    FVN_CHECK_ARG(ctx, tf_total <= 4096, "the batch's transfer functions hold %d entries (at most 4096)", tf_total);

    // ---- workspace (growing it is the one synchronising step) -------------
    ViewLayout lay[kMaxViews];
    const size_t need = batch_layout(views, nviews, lay);
    BatchWorkspace& ws = ctx->batch_ws;
    if (ws.bytes < need) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(ws.base);
        ws.base = nullptr;
        ws.bytes = 0;
        FVN_CUDA(ctx, cudaMalloc(&ws.base, need));
        ws.bytes = need;
    }
    for (int k = 0; k < nvol; ++k) {
        const size_t pb = march_volume_bytes(ctx, vols[k], mp);
        if (ws.pad_bytes[k] < pb) {
            FVN_CUDA(ctx, cudaDeviceSynchronize());
            cudaFree(ws.pad[k]);
            ws.pad[k] = nullptr;
            ws.pad_bytes[k] = 0;
            ws.pad_key[k] = PreparedKey();
            FVN_CUDA(ctx, cudaMalloc(&ws.pad[k], pb));
            ws.pad_bytes[k] = pb;
        }
    }
    char* base = static_cast<char*>(ws.base);
    int32_t* counts = reinterpret_cast<int32_t*>(base + need - align256(kMaxViews * sizeof(int32_t)));
    cudaStream_t st = as_stream(stream);

    // ---- mask + compaction: one launch -------------------------------------
    const fvn_foveation* fov[kMaxViews];
    int w[kMaxViews], h[kMaxViews];
    uint8_t* mask[kMaxViews];
    int32_t* ids[kMaxViews];
    float* rgbam[kMaxViews];
    for (int i = 0; i < nviews; ++i) {
        fov[i] = &views[i].fov;
        w[i] = views[i].cam.width;
        h[i] = views[i].cam.height;
        mask[i] = reinterpret_cast<uint8_t*>(base + lay[i].mask);
        ids[i] = reinterpret_cast<int32_t*>(base + lay[i].ids);
        rgbam[i] = views[i].rgbam ? views[i].rgbam : reinterpret_cast<float*>(base + lay[i].rgbam);
    }
    fvn_status s = make_mask_batch_impl(ctx, fov, w, h, mask, ids, counts, nviews, st);
    if (s != FVN_OK) return s;

    // ---- sparse frames start empty; the march's copy of each volume --------
    for (int i = 0; i < nviews; ++i)
        FVN_CUDA(ctx, cudaMemsetAsync(rgbam[i], 0, 5 * sizeof(float) * (size_t)w[i] * h[i], st));
    for (int k = 0; k < nvol; ++k)
        if ((s = march_volume_prepare_cached(ctx, vols[k], mp, ws.pad[k], ws.pad_key[k], st)) != FVN_OK) return s;

    // ---- one persistent march over every view's rays -----------------------
    BatchMarchView mv[kMaxViews];
    for (int i = 0; i < nviews; ++i)
        mv[i] = BatchMarchView{views[i].vol, ws.pad[vol_of[i]], views[i].tf, &views[i].cam, ids[i], counts + i,
                               rgbam[i]};
    if ((s = march_batch_impl(ctx, mv, nviews, mp, nsamples, st)) != FVN_OK) return s;
    for (int i = 0; i < nviews; ++i) {
        ws.view_mask[i] = mask[i];
        ws.view_pvol[i] = ws.pad[vol_of[i]];
    }

    // ---- network: one launch per layer over every view's tiles ------------
    ReconView rv[kMaxViews];
    for (int i = 0; i < nviews; ++i) {
        plan_view(w[i], h[i], &rv[i].plan, base + lay[i].plan);
        rv[i].rgbam = rgbam[i];
        rv[i].w = w[i];
        rv[i].h = h[i];
        rv[i].rgb = views[i].rgb;
        rv[i].prev = views[i].prev_rgb;
    }
    return reconstruct_tc_views(ctx, rv, nviews, precision, st);
}

}  // namespace
}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_render_batch(fvn_ctx* ctx, const fvn_view* views, int nviews, const fvn_march_params* mp,
                                       int precision, unsigned long long* nsamples, void* stream) {
    return render_batch_impl(ctx, views, nviews, mp, precision, nsamples, stream);
}

extern "C" fvn_status fvn_render_batch_adaptive(fvn_ctx* ctx, const fvn_view* views, int nviews,
                                                const fvn_march_params* mp, int precision, float min_psnr_db,
                                                int max_levels, unsigned long long* nsamples, int* levels_out,
                                                float* psnr_out, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, views != nullptr, "views is NULL");
    FVN_CHECK_ARG(ctx, nviews >= 1 && nviews <= kMaxViews, "%d views (1..%d)", nviews, kMaxViews);
    FVN_CHECK_ARG(ctx, max_levels >= 0 && max_levels <= 8, "max_levels must be in [0, 8]");
    FVN_CHECK_ARG(ctx, isfinite(min_psnr_db), "min_psnr_db is not finite");
    cudaStream_t st = as_stream(stream);
    // probe workspace: per view ids (4 B / px) and samples (20 B / px), then
    // the counts and the error sums
    size_t off[kMaxViews], need = 0;
    for (int i = 0; i < nviews; ++i) {
        FVN_CHECK_ARG(ctx, views[i].cam.width >= 1 && views[i].cam.height >= 1 && views[i].cam.width <= kMaxSide &&
                               views[i].cam.height <= kMaxSide,
                      "view %d: camera size outside [1, %d]", i, kMaxSide);
        off[i] = need;
        need += align256((size_t)views[i].cam.width * views[i].cam.height * 24);
    }
    const size_t cnt_off = need;
    need += align256(kMaxViews * sizeof(int32_t)) + kMaxViews * sizeof(double);
    BatchWorkspace& ws = ctx->batch_ws;
    fvn_view cur[kMaxViews];
    int orig[kMaxViews], level[kMaxViews];
    float est[kMaxViews];
    int n = nviews;
    for (int i = 0; i < nviews; ++i) {
        cur[i] = views[i];
        orig[i] = i;
        level[i] = 0;
        est[i] = 0.f;
    }
    for (;;) {
        fvn_status s = render_batch_impl(ctx, cur, n, mp, precision, nsamples, stream);
        if (s != FVN_OK) return s;
        if (ws.probe_bytes < need) {   // after the first batch: its arguments are validated
            FVN_CUDA(ctx, cudaDeviceSynchronize());
            cudaFree(ws.probe);
            ws.probe = nullptr;
            ws.probe_bytes = 0;
            FVN_CUDA(ctx, cudaMalloc(&ws.probe, need));
            ws.probe_bytes = need;
        }
        char* pb = static_cast<char*>(ws.probe);
        int32_t* counts = reinterpret_cast<int32_t*>(pb + cnt_off);
        double* sums = reinterpret_cast<double*>(pb + cnt_off + align256(kMaxViews * sizeof(int32_t)));
        FVN_CUDA(ctx, cudaMemsetAsync(counts, 0, kMaxViews * sizeof(int32_t), st));
        FVN_CUDA(ctx, cudaMemsetAsync(sums, 0, kMaxViews * sizeof(double), st));
        // probes outside each view's mask, marched in one launch, errors per view
        BatchMarchView mv[kMaxViews];
        for (int a = 0; a < n; ++a) {
            const int i = orig[a];
            const fvn_view& v = cur[a];
            const int w = v.cam.width, h = v.cam.height;
            int32_t* pids = reinterpret_cast<int32_t*>(pb + off[i]);
            float* prgbam = reinterpret_cast<float*>(pb + off[i] + (size_t)w * h * 4);
            if ((s = probe_compact(ctx, w, h, probe_key(&v.fov), ws.view_mask[a], pids, counts + i, st)) != FVN_OK)
                return s;
            mv[a] = BatchMarchView{v.vol, ws.view_pvol[a], v.tf, &v.cam, pids, counts + i, prgbam};
        }
        if ((s = march_batch_impl(ctx, mv, n, mp, nullptr, st)) != FVN_OK) return s;
        for (int a = 0; a < n; ++a) {
            const int i = orig[a];
            const long long plane = (long long)cur[a].cam.width * cur[a].cam.height;
            if ((s = probe_error(ctx, mv[a].ids, mv[a].count, cur[a].rgb, mv[a].rgbam, plane, sums + i, st)) !=
                FVN_OK)
                return s;
        }
        int hc[kMaxViews];
        double hs[kMaxViews];
        FVN_CUDA(ctx, cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, st));
        FVN_CUDA(ctx, cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, st));
        FVN_CUDA(ctx, cudaStreamSynchronize(st));
        // the views below the threshold go again with their periphery density doubled
        int m = 0;
        for (int a = 0; a < n; ++a) {
            const int i = orig[a];
            est[i] = (hc[i] == 0 || hs[i] == 0.0) ? 99.0f : (float)(-10.0 * log10(hs[i] / (3.0 * hc[i])));
            if (est[i] >= min_psnr_db || level[i] >= max_levels || cur[a].fov.p_base >= 1.0f) continue;
            fvn_view nv = cur[a];
            nv.fov.p_base = std::min(1.0f, 2.0f * nv.fov.p_base);
            ++level[i];
            cur[m] = nv;
            orig[m] = i;
            ++m;
        }
        if (m == 0) break;
        n = m;
    }
    for (int i = 0; i < nviews; ++i) {
        if (levels_out) levels_out[i] = level[i];
        if (psnr_out) psnr_out[i] = est[i];
    }
    return FVN_OK;
}
