// Context lifetime, error reporting, argument validation and the one-frame
// driver fvn_render (mask -> compaction -> sparse march -> reconstruction,
// the pipeline of the paper's Fig. "pipeline").
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace {
thread_local std::string g_thread_err;
}

namespace fvn {

fvn_status set_error(fvn_ctx* ctx, fvn_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    g_thread_err = buf;
    return st;
}

fvn_status validate_volume(fvn_ctx* ctx, const fvn_volume* vol) {
    FVN_CHECK_ARG(ctx, vol != nullptr, "volume descriptor is NULL");
    FVN_CHECK_ARG(ctx, vol->data != nullptr, "volume data pointer is NULL");
    FVN_CHECK_ARG(ctx, vol->nx >= 1 && vol->ny >= 1 && vol->nz >= 1 && vol->nx <= kMaxVolSide &&
                           vol->ny <= kMaxVolSide && vol->nz <= kMaxVolSide,
                  "volume dims %d x %d x %d outside [1, %d]", vol->nx, vol->ny, vol->nz, kMaxVolSide);
    FVN_CHECK_ARG(ctx, vol->dtype >= FVN_U8 && vol->dtype <= FVN_F32, "unknown volume dtype %d", vol->dtype);
    return FVN_OK;
}

fvn_status validate_march_params(fvn_ctx* ctx, const fvn_march_params* mp) {
    FVN_CHECK_ARG(ctx, mp != nullptr, "march parameters are NULL");
    FVN_CHECK_ARG(ctx, mp->step_vox > 0.f && isfinite(mp->step_vox), "step_vox must be > 0");
    FVN_CHECK_ARG(ctx, mp->term_alpha > 0.f && mp->term_alpha <= 1.f, "term_alpha must be in (0, 1]");
    FVN_CHECK_ARG(ctx, mp->shading >= 0 && mp->shading <= 2, "shading %d (0 none, 1 headlight, 2 shadows)",
                  mp->shading);
    if (mp->shading == 2) {
        const float* l = mp->light_dir;
        FVN_CHECK_ARG(ctx, isfinite(l[0]) && isfinite(l[1]) && isfinite(l[2]),
                      "light_dir has a non-finite component");
        FVN_CHECK_ARG(ctx, (double)l[0] * l[0] + (double)l[1] * l[1] + (double)l[2] * l[2] > 1e-12,
                      "light_dir is zero");
        FVN_CHECK_ARG(ctx, mp->shadow_rate >= 1 && mp->shadow_rate <= 64, "shadow_rate %d outside [1, 64]",
                      mp->shadow_rate);
    }
    return FVN_OK;
}

fvn_status validate_camera(fvn_ctx* ctx, const fvn_camera* cam) {
    FVN_CHECK_ARG(ctx, cam != nullptr, "camera is NULL");
    FVN_CHECK_ARG(ctx, cam->width >= 1 && cam->height >= 1 && cam->width <= kMaxSide && cam->height <= kMaxSide,
                  "camera size %d x %d outside [1, %d]", cam->width, cam->height, kMaxSide);
    FVN_CHECK_ARG(ctx, cam->fov_y_deg > 0.f && cam->fov_y_deg < 180.f, "fov_y_deg %g outside (0, 180)",
                  (double)cam->fov_y_deg);
    double f[3], up[3];
    for (int a = 0; a < 3; ++a) {
        f[a] = (double)cam->target[a] - cam->eye[a];
        up[a] = cam->up[a];
        FVN_CHECK_ARG(ctx, isfinite(cam->eye[a]) && isfinite(cam->target[a]) && isfinite(cam->up[a]),
                      "camera has a non-finite coordinate");
    }
    double c[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    double cl = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    FVN_CHECK_ARG(ctx, fl > 0.0, "camera eye equals target");
    FVN_CHECK_ARG(ctx, cl > 1e-12 * fl, "camera up is parallel to the view direction");
    return FVN_OK;
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_create(fvn_ctx** out) {
    if (!out) return set_error(nullptr, FVN_ERR_ARG, "out pointer is NULL");
    fvn_ctx* ctx = new (std::nothrow) fvn_ctx();
    if (!ctx) return set_error(nullptr, FVN_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ticket, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_ticket, 0, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_error, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fvn_status st = set_error(nullptr, e == cudaErrorMemoryAllocation ? FVN_ERR_OOM : FVN_ERR_CUDA,
                                  "fvn_create: %s", cudaGetErrorString(e));
        if (ctx->d_ticket) cudaFree(ctx->d_ticket);
        if (ctx->d_error) cudaFree(ctx->d_error);
        delete ctx;
        return st;
    }
    *out = ctx;
    return FVN_OK;
}

extern "C" fvn_status fvn_destroy(fvn_ctx* ctx) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    cudaDeviceSynchronize();
    for (auto& l : ctx->lut) {
        if (l.d_lut) cudaFree(l.d_lut);
        if (l.h_lut) cudaFreeHost(l.h_lut);
    }
    for (auto& L : ctx->layers) {
        cudaFree(L.w16);
        cudaFree(L.w8);
        cudaFree(L.scale8);
        cudaFree(L.bias);
    }
    cudaFree(ctx->head_w16);
    for (cudaEvent_t e : ctx->tm_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(ctx->head_b32);
    cudaFree(ctx->d_error);
    cudaFree(ctx->d_act_scale);
    cudaFree(ctx->d_amax);
    cudaFree(ctx->d_ticket);
    cudaFree(ctx->pad_buf);
    cudaFree(ctx->d_noise);
    cudaFree(ctx->recon_ws.base);
    cudaFree(ctx->render_ws.mask);
    cudaFree(ctx->render_ws.ids);
    cudaFree(ctx->render_ws.count);
    cudaFree(ctx->render_ws.rgbam);
    cudaFree(ctx->probe_ws.ids);
    cudaFree(ctx->probe_ws.count);
    cudaFree(ctx->probe_ws.rgbam);
    cudaFree(ctx->probe_ws.acc);
    cudaFree(ctx->batch_ws.base);
    cudaFree(ctx->wnet.d_w);
    cudaFree(ctx->wnet.ws);
    cudaFree(ctx->wnet.d_wpk);
    cudaFree(ctx->wnet.d_bpk);
    cudaFree(ctx->wnet.tws);
    for (void* p : ctx->batch_ws.pad) cudaFree(p);
    cudaFree(ctx->batch_ws.probe);
    delete ctx;
    return FVN_OK;
}

extern "C" const char* fvn_last_error(const fvn_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_thread_err.c_str();
}

extern "C" fvn_status fvn_set_option(fvn_ctx* ctx, int option, int value) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    switch (option) {
        case FVN_OPT_MARCH_REFILL:
            FVN_CHECK_ARG(ctx, value >= 1 && value <= 32, "refill threshold must be in [1, 32]");
            ctx->march_refill = value;
            return FVN_OK;
        case FVN_OPT_MARCH_BLOCKS_PER_SM:
            FVN_CHECK_ARG(ctx, value >= 0 && value <= 16, "blocks per SM must be in [0, 16]");
            ctx->march_blocks_per_sm = value;
            return FVN_OK;
        case FVN_OPT_MARCH_REFILL_DENSE:
            FVN_CHECK_ARG(ctx, value >= 1 && value <= 32, "refill threshold must be in [1, 32]");
            ctx->march_refill_dense = value;
            return FVN_OK;
        case FVN_OPT_MARCH_BLOCKS_PER_SM_DENSE:
            FVN_CHECK_ARG(ctx, value >= 0 && value <= 16, "blocks per SM must be in [0, 16]");
            ctx->march_blocks_per_sm_dense = value;
            return FVN_OK;
        case FVN_OPT_MARCH_COOP:
            FVN_CHECK_ARG(ctx, value >= 0 && value <= 32, "cooperative-finish threshold must be in [0, 32]");
            ctx->march_coop = value;
            return FVN_OK;
        case FVN_OPT_MARCH_COOP_DENSE:
            FVN_CHECK_ARG(ctx, value >= 0 && value <= 32, "cooperative-finish threshold must be in [0, 32]");
            ctx->march_coop_dense = value;
            return FVN_OK;
        case FVN_OPT_MARCH_GRADIENT_VOLUME:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "gradient-volume option must be 0 or 1");
            ctx->march_grad4 = value;
            return FVN_OK;
        case FVN_OPT_MARCH_COUNT_SHADOW:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "shadow-sample counting option must be 0 or 1");
            ctx->march_count_shadow = value;
            return FVN_OK;
        case FVN_OPT_CONV_ROWS_HALF:
            FVN_CHECK_ARG(ctx, value == 2 || value == 4, "half-resolution tile rows must be 2 or 4");
            ctx->conv_rows_half = value;
            return FVN_OK;
        case FVN_OPT_CONV_ROWS_QUARTER:
            FVN_CHECK_ARG(ctx, value == 1 || value == 2 || value == 4, "quarter-resolution tile rows must be 1, 2 or 4");
            ctx->conv_rows_quarter = value;
            return FVN_OK;
        case FVN_OPT_CONV_ROWS_DEC1:
            FVN_CHECK_ARG(ctx, value == 1 || value == 2, "first decoder layer tile rows must be 1 or 2");
            ctx->conv_rows_dec1 = value;
            return FVN_OK;
        case FVN_OPT_CONV_FUSE_UP_DEC1:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "decoder up-sampling option must be 0 or 1");
            ctx->conv_fuse_up_dec1 = value;
            return FVN_OK;
        case FVN_OPT_WNET_TENSOR_CORES:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "two-stage tensor-core option must be 0 or 1");
            ctx->wnet.tc = value;
            return FVN_OK;
        case FVN_OPT_WNET_FUSED_UPSAMPLING:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "two-stage fused up-sampling option must be 0 or 1");
            ctx->wnet.fuse_up = value;
            return FVN_OK;
        case FVN_OPT_STAGE_TIMING:
            FVN_CHECK_ARG(ctx, value == 0 || value == 1, "stage-timing option must be 0 or 1");
            if (value && !ctx->tm_ev[0])
                for (int k = 0; k < TM_N; ++k) FVN_CUDA(ctx, cudaEventCreate(&ctx->tm_ev[k]));
            ctx->timing = value != 0;
            ctx->timed_frame = false;
            return FVN_OK;
        default:
            return set_error(ctx, FVN_ERR_ARG, "unknown option %d", option);
    }
}

extern "C" fvn_status fvn_device_status(fvn_ctx* ctx) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CUDA(ctx, cudaDeviceSynchronize());
    int flag = 0;
    FVN_CUDA(ctx, cudaMemcpy(&flag, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        FVN_CUDA(ctx, cudaMemset(ctx->d_error, 0, sizeof(int)));
        return set_error(ctx, FVN_ERR_TIMEOUT, "a kernel gave up waiting for the tensor cores (flag %d)", flag);
    }
    return FVN_OK;
}

static fvn_status render_entry(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                               const fvn_foveation* fov, const fvn_march_params* mp, int precision, const float* prev,
                               float* rgb, float* rgbam_out, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    fvn_status st;
    if ((st = validate_volume(ctx, vol)) != FVN_OK) return st;
    if ((st = validate_camera(ctx, cam)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, tf && tf->rgba && tf->n >= 2 && tf->n <= 4096, "bad transfer function");
    FVN_CHECK_ARG(ctx, fov != nullptr, "foveation is NULL");
    if ((st = validate_march_params(ctx, mp)) != FVN_OK) return st;
    FVN_CHECK_ARG(ctx, rgb != nullptr, "rgb output is NULL");
    FVN_CHECK_ARG(ctx, precision == FVN_PREC_FP16 || precision == FVN_PREC_FP8, "unknown precision %d", precision);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    if (prev && !ctx->recurrent)
        return set_error(ctx, FVN_ERR_STATE, "a previous frame needs the recurrent network's weights");
    const int w = cam->width, h = cam->height;
    RenderWorkspace& ws = ctx->render_ws;
    if (ws.w != w || ws.h != h) {
        // Growing the workspace is the one synchronising step of this call.
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(ws.mask);
        cudaFree(ws.ids);
        cudaFree(ws.count);
        cudaFree(ws.rgbam);
        ws = RenderWorkspace();
        size_t npix = (size_t)w * h;
        FVN_CUDA(ctx, cudaMalloc(&ws.mask, npix));
        FVN_CUDA(ctx, cudaMalloc(&ws.ids, npix * sizeof(int32_t)));
        FVN_CUDA(ctx, cudaMalloc(&ws.count, sizeof(int32_t)));
        FVN_CUDA(ctx, cudaMalloc(&ws.rgbam, 5 * npix * sizeof(float)));
        ws.w = w;
        ws.h = h;
    }
    cudaStream_t s = as_stream(stream);
    float* rgbam = rgbam_out ? rgbam_out : ws.rgbam;
    struct InRender {   // the stages of this call are the ones recorded
        fvn_ctx* c;
        explicit InRender(fvn_ctx* x) : c(x) { c->in_render = true; c->timed_frame = false; }
        ~InRender() { c->in_render = false; }
    } guard(ctx);
    stage_mark(ctx, TM_START, s);
    if ((st = make_mask_impl(ctx, fov, w, h, ws.mask, ws.ids, ws.count, s)) != FVN_OK) return st;
    stage_mark(ctx, TM_MASK, s);
    if ((st = march_impl(ctx, vol, tf, cam, mp, ws.ids, ws.count, rgbam, nullptr, s)) != FVN_OK) return st;
    if ((st = reconstruct_impl(ctx, rgbam, prev, w, h, precision, rgb, s)) != FVN_OK) return st;
    stage_mark(ctx, TM_NET, s);
    ctx->timed_frame = ctx->timing;
    return FVN_OK;
}

extern "C" fvn_status fvn_stage_times(fvn_ctx* ctx, float* ms) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, ms != nullptr, "ms is NULL");
    if (!ctx->timing || !ctx->timed_frame)
        return set_error(ctx, FVN_ERR_STATE, "no frame rendered with stage timing on (FVN_OPT_STAGE_TIMING)");
    FVN_CUDA(ctx, cudaEventSynchronize(ctx->tm_ev[TM_NET]));
    float t[TM_N - 1];
    for (int k = 0; k + 1 < TM_N; ++k) FVN_CUDA(ctx, cudaEventElapsedTime(&t[k], ctx->tm_ev[k], ctx->tm_ev[k + 1]));
    for (int k = 0; k + 1 < TM_N; ++k) ms[k] = t[k];
    return FVN_OK;
}

extern "C" fvn_status fvn_render(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                                 const fvn_foveation* fov, const fvn_march_params* mp, int precision, float* rgb,
                                 float* rgbam_out, void* stream) {
    return render_entry(ctx, vol, tf, cam, fov, mp, precision, nullptr, rgb, rgbam_out, stream);
}

extern "C" fvn_status fvn_render_recurrent(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf,
                                           const fvn_camera* cam, const fvn_foveation* fov,
                                           const fvn_march_params* mp, int precision, const float* prev_rgb,
                                           float* rgb, float* rgbam_out, void* stream) {
    return render_entry(ctx, vol, tf, cam, fov, mp, precision, prev_rgb, rgb, rgbam_out, stream);
}
