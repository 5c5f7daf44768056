// Reconstruction network inference (paper: "Reconstruction Network", Fig.
// "network architecture"; "Model Precision & Optimization": weights truncated
// to 16 bit).  Slim U-Net of 16/32/64 channels, then the 1x1 head, the 5x5
// kernel prediction on the sparse samples and the blend.
//
// This file holds the network's host side: the layer table and the flat
// weight order, the activation workspace plan (FP16 / FP8 chunk-planar
// tensors per resolution level of the frame padded to a multiple of 4), the
// weight conversion to the tensor-core operand layouts (FP16, and E4M3 with
// per-output-channel scales after calibration) and the entry points.  The
// kernels are the tcgen05 convolutions of conv_tc.cu / conv_ws.cuh.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_fp8.h>

#include "common.cuh"

namespace fvn {

// ---------------------------------------------------------------------------
// layer table (flat weight order of fvn_load_weights)
// ---------------------------------------------------------------------------
struct LayerSpec {
    int cin, cout, k;
};
static const LayerSpec kLayers[kNumLayers] = {
    {5, 16, 3},  {16, 16, 3}, {16, 32, 3}, {32, 32, 3}, {32, 64, 3}, {64, 64, 3},
    {96, 32, 3}, {32, 32, 3}, {48, 16, 3}, {16, 16, 3}, {16, 29, 1},
};
constexpr int kHeadC = 29;

// Layer li of the plain network, or of the recurrent one (paper:
// "Recurrence": the previous output enters the first layer as three more
// input channels).
static LayerSpec layer_spec(bool recurrent, int li) {
    LayerSpec s = kLayers[li];
    if (li == 0 && recurrent) s.cin = 8;
    return s;
}

static size_t weight_count(bool recurrent = false) {
    size_t n = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec l = layer_spec(recurrent, li);
        n += (size_t)l.cout * l.cin * l.k * l.k + l.cout;
    }
    return n;
}


// separate_up: give the up-sampled decoder inputs buffers of their own
// (FP8 calibration reads every activation after the pass).
static size_t plan_buffers(int W4, int H4, ReconPlan* b, char* base, bool separate_up = false) {
    const size_t n0 = (size_t)W4 * H4, n1 = n0 / 4, n2 = n0 / 16;
    const size_t sizes[12] = {n0 * 16, n0 * 16, n1 * 16, n1 * 32, n1 * 32, n2 * 32,
                              n2 * 64, n2 * 64, n1 * 32, n1 * 32, n0 * 16, n0 * 16};
    __half** ptrs[12] = {&b->e0a, &b->e0, &b->p0, &b->e1a, &b->e1, &b->p1,
                         &b->ba,  &b->bt, &b->d1a, &b->d1, &b->d0a, &b->d0};
    size_t off = 0;
    for (int i = 0; i < 12; ++i) {
        if (base) *ptrs[i] = reinterpret_cast<__half*>(base + off);
        off += (sizes[i] * sizeof(__half) + 255) & ~(size_t)255;
    }
    // up-sampled decoder inputs on dead buffers: u1 (n1 x 64) on e0a (n0 x 16,
    // dead after the second layer); u0 (n0 x 32) from p0 on, over p0, e1a,
    // e1, p1, ba, bt, d1a (n0 x 38 in total, all dead once d1 is written)
    if (separate_up) {
        if (base) {
            b->u1 = reinterpret_cast<__half*>(base + off);
            b->u0 = reinterpret_cast<__half*>(base + off + ((n1 * 64 * sizeof(__half) + 255) & ~(size_t)255));
        }
        return off + ((n1 * 64 * sizeof(__half) + 255) & ~(size_t)255) + ((n0 * 32 * sizeof(__half) + 255) & ~(size_t)255);
    }
    if (base) {
        b->u1 = b->e0a;
        b->u0 = b->p0;
    }
    return off;
}

size_t recon_workspace_bytes(int w, int h) {
    return plan_buffers((w + 3) & ~3, (h + 3) & ~3, nullptr, nullptr);
}

size_t plan_view(int w, int h, ReconPlan* plan, char* base) {
    ReconPlan tmp;
    return plan_buffers((w + 3) & ~3, (h + 3) & ~3, plan ? plan : &tmp, base);
}

fvn_status reconstruct_impl(fvn_ctx* ctx, const float* rgbam, const float* prev, int w, int h, int precision,
                            float* rgb, cudaStream_t st) {
    if (precision == FVN_PREC_FP8 && !ctx->has_fp8)
        return set_error(ctx, FVN_ERR_STATE, "FP8 needs calibrated scales (call fvn_calibrate_fp8 first)");
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    ReconWorkspace& ws = ctx->recon_ws;
    if (ws.w != W4 || ws.h != H4) {
        FVN_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(ws.base);
        ws = ReconWorkspace();
        size_t bytes = plan_buffers(W4, H4, nullptr, nullptr);
        FVN_CUDA(ctx, cudaMalloc(&ws.base, bytes));
        ws.bytes = bytes;
        ws.w = W4;
        ws.h = H4;
    }
    return reconstruct_on(ctx, ws.base, rgbam, prev, w, h, precision, rgb, st);
}

fvn_status reconstruct_on(fvn_ctx* ctx, void* workspace, const float* rgbam, const float* prev, int w, int h,
                          int precision, float* rgb, cudaStream_t st) {
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    ReconPlan B;
    plan_buffers(W4, H4, &B, static_cast<char*>(workspace));
    if (precision == FVN_PREC_FP8) {
        if (!ctx->has_fp8)
            return set_error(ctx, FVN_ERR_STATE, "FP8 needs calibrated scales (call fvn_calibrate_fp8 first)");
        return reconstruct_tc_fp8(ctx, B, rgbam, prev, w, h, rgb, st);
    }
    return reconstruct_tc(ctx, B, rgbam, prev, w, h, rgb, st);
}

}  // namespace fvn

using namespace fvn;

extern "C" size_t fvn_weight_count(void) { return weight_count(false); }

extern "C" size_t fvn_weight_count_recurrent(void) { return weight_count(true); }

extern "C" fvn_status fvn_load_weights(fvn_ctx* ctx, const float* host_w, size_t n) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, host_w != nullptr, "weights pointer is NULL");
    FVN_CHECK_ARG(ctx, n == weight_count(false) || n == weight_count(true),
                  "weight vector has %zu entries, expected %zu (or %zu for the recurrent network)", n,
                  weight_count(false), weight_count(true));
    const bool recurrent = n == weight_count(true);
    for (size_t i = 0; i < n; ++i)
        FVN_CHECK_ARG(ctx, isfinite(host_w[i]), "weight %zu is not finite", i);
    FVN_CUDA(ctx, cudaDeviceSynchronize());
    ctx->host_weights.assign(host_w, host_w + n);
    ctx->has_fp8 = false;   // FP8 weights follow the FP32 weights: calibrate again
    ctx->has_weights = false;
    size_t off = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec sp = layer_spec(recurrent, li);
        const float* W = host_w + off;
        const float* b = W + (size_t)sp.cout * sp.cin * sp.k * sp.k;
        off += (size_t)sp.cout * sp.cin * sp.k * sp.k + sp.cout;
        ConvW& L = ctx->layers[li];
        L.cin = sp.cin;
        L.cout = sp.cout;
        L.k = sp.k;
        if (sp.k == 1) {   // head (16 -> 29, 1x1) as a tensor-core operand: [k chunk 2][n 32][8], output rows 29..31 zero
            std::vector<__half> h16(2 * 32 * 8, __float2half(0.f));
            std::vector<float> hb(32, 0.f);
            for (int o = 0; o < kHeadC; ++o) {
                for (int c = 0; c < 16; ++c) h16[((c / 8) * 32 + o) * 8 + (c % 8)] = __float2half(W[o * sp.cin + c]);
                hb[o] = b[o];
            }
            if (!ctx->head_w16) FVN_CUDA(ctx, cudaMalloc(&ctx->head_w16, h16.size() * sizeof(__half)));
            if (!ctx->head_b32) FVN_CUDA(ctx, cudaMalloc(&ctx->head_b32, hb.size() * sizeof(float)));
            FVN_CUDA(ctx, cudaMemcpy(ctx->head_w16, h16.data(), h16.size() * sizeof(__half), cudaMemcpyHostToDevice));
            FVN_CUDA(ctx, cudaMemcpy(ctx->head_b32, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice));
            continue;
        }
        const int cp = (sp.cin + 15) & ~15;
        L.cin_pad = cp;
        const int chunks = cp / 8;
        std::vector<__half> w16((size_t)9 * cp * sp.cout, __float2half(0.f));
        for (int o = 0; o < sp.cout; ++o)
            for (int c = 0; c < sp.cin; ++c)
                for (int tap = 0; tap < 9; ++tap) {
                    const float v = W[((size_t)o * sp.cin + c) * 9 + tap];
                    w16[(((size_t)tap * chunks + c / 8) * sp.cout + o) * 8 + (c % 8)] = __float2half(v);
                }
        if (!L.w16) FVN_CUDA(ctx, cudaMalloc(&L.w16, w16.size() * sizeof(__half)));
        if (!L.bias) FVN_CUDA(ctx, cudaMalloc(&L.bias, sp.cout * sizeof(float)));
        FVN_CUDA(ctx, cudaMemcpy(L.w16, w16.data(), w16.size() * sizeof(__half), cudaMemcpyHostToDevice));
        FVN_CUDA(ctx, cudaMemcpy(L.bias, b, sp.cout * sizeof(float), cudaMemcpyHostToDevice));
    }
    ctx->recurrent = recurrent;
    ctx->has_weights = true;
    return FVN_OK;
}

static fvn_status reconstruct_entry(fvn_ctx* ctx, const float* rgbam, const float* prev, int w, int h,
                                    int precision, float* rgb, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam && rgb, "rgbam and rgb must be device pointers");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    FVN_CHECK_ARG(ctx, precision == FVN_PREC_FP16 || precision == FVN_PREC_FP8, "unknown precision %d", precision);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    if (prev && !ctx->recurrent)
        return set_error(ctx, FVN_ERR_STATE, "a previous frame needs the recurrent network's weights");
    return reconstruct_impl(ctx, rgbam, prev, w, h, precision, rgb, as_stream(stream));
}

extern "C" fvn_status fvn_reconstruct(fvn_ctx* ctx, const float* rgbam, int w, int h, int precision, float* rgb,
                                      void* stream) {
    return reconstruct_entry(ctx, rgbam, nullptr, w, h, precision, rgb, stream);
}

extern "C" fvn_status fvn_reconstruct_recurrent(fvn_ctx* ctx, const float* rgbam, const float* prev_rgb, int w,
                                                int h, int precision, float* rgb, void* stream) {
    return reconstruct_entry(ctx, rgbam, prev_rgb, w, h, precision, rgb, stream);
}

namespace fvn {

// Input tensor of every input channel of a layer, and the layer's output /
// pooled tensor (FP8 scales; see conv_tc.cu).
static void fp8_tensors(int layer, int c, int* in_t) {
    static const int single[kNumLayers] = {FP8_RGBAM, FP8_E0A, FP8_P0, FP8_E1A, FP8_P1, FP8_BA,
                                           -1,        FP8_D1A, -1,     FP8_D0A, -1};
    if (layer == 6) *in_t = c < 64 ? FP8_BT : FP8_E1;          // [up(bt), e1]
    else if (layer == 8) *in_t = c < 32 ? FP8_D1 : FP8_E0;     // [up(d1), e0]
    else *in_t = single[layer];
}

// Quantise every 3x3 layer to E4M3 with the activation scales folded in:
// w' = w s_in(c); s_w[o] = max |w'| / 448; q = e4m3(w' / s_w[o]).  Layout
// [tap][cin_pad / 16][cout][16 bytes] (cin padded to a multiple of 32).
static fvn_status build_fp8_weights(fvn_ctx* ctx) {
    const float* hw = ctx->host_weights.data();
    float s[FP8_NT];
    for (int t = 0; t < FP8_NT; ++t) {
        const float amax = t == FP8_RGBAM ? 1.0f : ctx->fp8_amax[t];
        s[t] = amax > 0.f ? amax / 448.0f : 1.0f;
        ctx->fp8_inv_scale[t] = 1.0f / s[t];
    }
    size_t off = 0;
    for (int li = 0; li < kNumLayers; ++li) {
        const LayerSpec sp = layer_spec(ctx->recurrent, li);
        const float* W = hw + off;
        off += (size_t)sp.cout * sp.cin * sp.k * sp.k + sp.cout;
        if (sp.k != 3) continue;
        const int cp = (sp.cin + 31) & ~31;
        std::vector<float> wf((size_t)sp.cout * sp.cin * 9);
        std::vector<float> sw(sp.cout, 1.0f);
        for (int o = 0; o < sp.cout; ++o) {
            float m = 0.f;
            for (int c = 0; c < sp.cin; ++c) {
                int t;
                fp8_tensors(li, c, &t);
                for (int tap = 0; tap < 9; ++tap) {
                    const size_t i = ((size_t)o * sp.cin + c) * 9 + tap;
                    wf[i] = W[i] * s[t];
                    m = std::max(m, std::fabs(wf[i]));
                }
            }
            sw[o] = m > 0.f ? m / 448.0f : 1.0f;
        }
        std::vector<uint8_t> q((size_t)9 * cp * sp.cout, 0);
        for (int o = 0; o < sp.cout; ++o)
            for (int c = 0; c < sp.cin; ++c)
                for (int tap = 0; tap < 9; ++tap) {
                    const float v = wf[((size_t)o * sp.cin + c) * 9 + tap] / sw[o];
                    q[(((size_t)tap * (cp / 16) + c / 16) * sp.cout + o) * 16 + (c % 16)] =
                        (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
                }
        ConvW& L = ctx->layers[li];
        if (!L.w8) FVN_CUDA(ctx, cudaMalloc(&L.w8, q.size()));
        if (!L.scale8) FVN_CUDA(ctx, cudaMalloc(&L.scale8, sp.cout * sizeof(float)));
        FVN_CUDA(ctx, cudaMemcpy(L.w8, q.data(), q.size(), cudaMemcpyHostToDevice));
        FVN_CUDA(ctx, cudaMemcpy(L.scale8, sw.data(), sp.cout * sizeof(float), cudaMemcpyHostToDevice));
    }
    ctx->has_fp8 = true;
    return FVN_OK;
}

}  // namespace fvn

extern "C" fvn_status fvn_calibrate_fp8(fvn_ctx* ctx, const float* rgbam, int w, int h, int reset, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam != nullptr, "rgbam must be a device pointer");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    cudaStream_t st = as_stream(stream);
    // run the FP16 tensor-core network on this frame into a workspace where
    // no activation is overwritten, then reduce every activation's amax
    const int W4 = (w + 3) & ~3, H4 = (h + 3) & ~3;
    float* out = nullptr;
    char* wsp = nullptr;
    FVN_CUDA(ctx, cudaMalloc(&out, sizeof(float) * 3 * (size_t)w * h));
    if (cudaMalloc(&wsp, plan_buffers(W4, H4, nullptr, nullptr, true)) != cudaSuccess) {
        cudaFree(out);
        return set_error(ctx, FVN_ERR_OOM, "no memory for the calibration workspace");
    }
    ReconView v;
    plan_buffers(W4, H4, &v.plan, wsp, true);
    v.rgbam = rgbam;
    v.w = w;
    v.h = h;
    v.rgb = out;
    fvn_status s = reconstruct_tc_views(ctx, &v, 1, FVN_PREC_FP16, st);
    if (s == FVN_OK && !ctx->d_amax && cudaMalloc(&ctx->d_amax, FP8_NT * sizeof(float)) != cudaSuccess)
        s = set_error(ctx, FVN_ERR_OOM, "no memory for the amax accumulators");
    if (s == FVN_OK && cudaMemsetAsync(ctx->d_amax, 0, FP8_NT * sizeof(float), st) != cudaSuccess)
        s = set_error(ctx, FVN_ERR_CUDA, "cudaMemsetAsync failed");
    if (s == FVN_OK) s = calibrate_amax(ctx, v.plan, w, h, ctx->d_amax, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaFree(out);
    cudaFree(wsp);
    if (s != FVN_OK) return s;
    if (se != cudaSuccess) return set_error(ctx, FVN_ERR_CUDA, "calibration pass failed: %s", cudaGetErrorString(se));
    float amax[FP8_NT];
    FVN_CUDA(ctx, cudaMemcpy(amax, ctx->d_amax, sizeof amax, cudaMemcpyDeviceToHost));
    for (int t = 0; t < FP8_NT; ++t) ctx->fp8_amax[t] = reset ? amax[t] : std::max(ctx->fp8_amax[t], amax[t]);
    return build_fp8_weights(ctx);
}
