// Shared host-side definitions of libfvn: the context, error reporting and
// launch helpers.  Device kernels live in the per-stage .cu files.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/fvn.h"

namespace fvn {

constexpr int kLutBins = 16384;       // threshold-table entries
constexpr int kLutCache = 16;         // distinct foveation profiles kept per context
constexpr int kMaxSide = 16384;       // largest frame side accepted
constexpr int kMaxVolSide = 4096;     // largest volume side accepted
constexpr int kMaxViews = FVN_MAX_VIEWS;   // views of one batched render
constexpr int kMaxBatchVolumes = 4;   // distinct volumes of one batched render
// a batch's views never evict one another's threshold tables (least recently
// used eviction only reaches profiles older than the batch)
static_assert(kLutCache >= kMaxViews, "threshold-table cache smaller than a batch");

struct LutEntry {
    bool valid = false;
    int w = 0, h = 0;
    float r0 = 0.f, s = 0.f, pb = 0.f;
    int shift = 0;
    uint64_t last_use = 0;
    uint32_t* d_lut = nullptr;        // device copy, kLutBins entries
    uint32_t* h_lut = nullptr;        // pinned host copy, never modified after upload
};

// Per-layer inference weights: FP16 in the shared-memory layout of the conv
// kernels ([tap][cin/8][cout][8]) plus FP32 bias; FP8 copies with per-output
// channel scales.
struct ConvW {
    int cin = 0, cin_pad = 0, cout = 0, k = 0;
    __half* w16 = nullptr;
    uint8_t* w8 = nullptr;            // e4m3, same layout as w16
    float* scale8 = nullptr;          // per output channel dequantisation scale
    float* bias = nullptr;
};

constexpr int kNumLayers = 11;

struct ReconWorkspace {
    int w = 0, h = 0;                 // frame the buffers were sized for
    size_t bytes = 0;
    void* base = nullptr;
};

// Activation buffers of one reconstruction (FP16 NHWC, per level).  u1 and
// u0 hold the up-sampled inputs of the two decoder convolutions; they alias
// buffers that are dead by then (u1 = e0a, u0 spans p0 .. d1a).
struct ReconPlan {
    __half *e0a, *e0, *p0, *e1a, *e1, *p1, *ba, *bt, *d1a, *d1, *d0a, *d0;
    __half *u1, *u0;
};

// One view of a batched reconstruction: its activation buffers, sparse
// frame and output.
struct ReconView {
    ReconPlan plan;
    const float* rgbam;
    int w, h;
    float* rgb;
    const float* prev = nullptr;      // recurrent model: previous output [3][h][w] (NULL: zeros)
};

// The source of a prepared volume copy (padded copy, gradient volume or
// shadow cells): the copy is reused while a volume with a non-zero
// generation names the same data, sizes, voxel type, generation and kind.
struct PreparedKey {
    const void* data = nullptr;
    int nx = 0, ny = 0, nz = 0, dtype = -1, kind = -1;
    uint32_t generation = 0;          // 0: nothing reusable
    bool matches(const fvn_volume* v, int k) const {
        return generation != 0 && v->generation == generation && v->data == data && v->nx == nx &&
               v->ny == ny && v->nz == nz && v->dtype == dtype && k == kind;
    }
};

// Workspace of fvn_render_batch, one allocation carved per view.
struct BatchWorkspace {
    size_t bytes = 0;
    void* base = nullptr;
    int32_t* counts = nullptr;        // per-view sampled-pixel counts
    void* pad[kMaxBatchVolumes] = {}; // padded volume copies
    size_t pad_bytes[kMaxBatchVolumes] = {};
    PreparedKey pad_key[kMaxBatchVolumes];
    uint8_t* view_mask[kMaxViews] = {};      // the last batch's masks and volume copies, per view
    const void* view_pvol[kMaxViews] = {};
    // probes of fvn_render_batch_adaptive: per view ids and samples (24 B per
    // pixel), then counts and error sums
    void* probe = nullptr;
    size_t probe_bytes = 0;
};

// Two-stage network: configuration, FP32 weights on the device (the flat
// layout of fvn_wnet_weight_count) and an activation workspace for one frame
// size.
constexpr int kWnetMaxLayers = 64;
struct WnetState {
    fvn_wnet_config cfg{};
    float* d_w = nullptr;
    size_t n = 0, cap = 0;            // weights in use / floats allocated
    bool loaded = false;              // a complete set of weights is in place
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int ws_w = 0, ws_h = 0;           // padded frame the workspace was carved for
    // tensor-core path (FVN_OPT_WNET_TENSOR_CORES): the layers' weights packed
    // for the K-streamed convolution (FP16) and their zero-padded biases
    int tc = 0;                       // the option
    int fuse_up = 1;                  // decoder up-sampling inside the convolutions (tensor-core path)
    bool tc_ok = false;               // the widths allow the tensor-core path
    void* d_wpk = nullptr;            // packed FP16 weights of every layer
    float* d_bpk = nullptr;           // padded biases of every layer
    size_t wpk_off[kWnetMaxLayers] = {}, bpk_off[kWnetMaxLayers] = {};   // per layer, in halves / floats
    // each K decoder level's tap and blend heads packed as one 10-output layer
    size_t wpk_tb_off[FVN_WNET_MAX_LEVELS] = {}, bpk_tb_off[FVN_WNET_MAX_LEVELS] = {};
    void* tws = nullptr;              // tensor-core workspace
    size_t tws_bytes = 0;
    int tws_w = 0, tws_h = 0;
};

// Activation tensors with an FP8 scale (per tensor, from calibration).
enum Fp8Tensor {
    FP8_RGBAM = 0, FP8_E0A, FP8_E0, FP8_P0, FP8_E1A, FP8_E1, FP8_P1, FP8_BA, FP8_BT, FP8_D1A, FP8_D1, FP8_D0A,
    FP8_NT
};

// Stage timing of fvn_render (FVN_OPT_STAGE_TIMING): events recorded on the
// frame's stream at the stage boundaries.
enum StageMark { TM_START = 0, TM_MASK, TM_SETUP, TM_PREP, TM_MARCH, TM_NET, TM_N };

struct ProbeWorkspace {
    int w = 0, h = 0;
    int32_t* ids = nullptr;
    int32_t* count = nullptr;
    float* rgbam = nullptr;
    double* acc = nullptr;
};

struct RenderWorkspace {
    int w = 0, h = 0;
    uint8_t* mask = nullptr;
    int32_t* ids = nullptr;
    int32_t* count = nullptr;
    float* rgbam = nullptr;
};

}  // namespace fvn

struct fvn_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    fvn::LutEntry lut[fvn::kLutCache];
    uint64_t lut_clock = 0;
    int* d_ticket = nullptr;          // 64 march work-queue counters (stream-ordered reset)
    unsigned ticket_ring = 0;         // next counter to use, so queued launches do not share one
    bool has_weights = false;
    bool recurrent = false;           // the loaded weights take the previous output as input
    fvn::ConvW layers[fvn::kNumLayers];
    __half* head_w16 = nullptr;       // head weights as a tensor-core operand: [2][32][8] FP16 (rows 29-31 zero)
    float* head_b32 = nullptr;        // head bias padded to 32
    int* d_error = nullptr;           // device-side error flag (a bounded wait gave up)
    std::vector<float> host_weights;  // FP32 weights as loaded (re-quantised at FP8 calibration)
    bool has_fp8 = false;
    float fp8_amax[fvn::FP8_NT] = {};
    float fp8_inv_scale[fvn::FP8_NT] = {};
    float* d_amax = nullptr;          // device amax accumulators [FP8_NT]
    int march_refill = 1;             // sparse march: refill idle lanes once fewer than this many are busy
    int march_blocks_per_sm = 0;      // sparse march CTAs per SM, 0 = occupancy limit
    int march_refill_dense = 1;       // dense march: 1 = whole 32-ray packets only
    int march_blocks_per_sm_dense = 0;
    int march_coop = 0;               // sparse march: finish a warp's rays with the whole warp once at most this many are left
    int march_coop_dense = 0;
    int march_grad4 = 1;              // shaded marches read a gradient volume when it fits
    int march_count_shadow = 0;       // shadowed marches also count the shadow rays' samples
    int conv_rows_half = 4;           // output rows per tile of the half-resolution 32-channel layers
    int conv_rows_quarter = 2;        // ... of the quarter-resolution bottleneck layers
    int conv_rows_dec1 = 1;           // ... of the first decoder layer (96 input channels)
    int conv_fuse_up_dec1 = 0;        // first decoder layer computes its up-sampled input itself
    uint32_t* d_noise = nullptr;      // sample-map noise tiles (NULL: the hash), [frames][T][T]
    int noise_log2 = 0, noise_frames = 0;
    void* pad_buf = nullptr;          // padded copy of the volume read by the march
    size_t pad_bytes = 0;
    fvn::PreparedKey pad_key;         // what pad_buf holds
    float* d_act_scale = nullptr;     // FP8 per-layer activation scales
    fvn::ReconWorkspace recon_ws;
    fvn::RenderWorkspace render_ws;
    fvn::ProbeWorkspace probe_ws;
    fvn::BatchWorkspace batch_ws;
    fvn::WnetState wnet;
    bool timing = false;              // record stage events (FVN_OPT_STAGE_TIMING)
    bool in_render = false;           // inside fvn_render: its stages are the ones recorded
    bool timed_frame = false;         // a whole fvn_render was recorded since timing was enabled
    cudaEvent_t tm_ev[fvn::TM_N] = {};
};

namespace fvn {

// A kernel that uses more than 48 KB of dynamic shared memory must opt in,
// once per device (the attribute belongs to the device's copy of the
// kernel).  `done` is the kernel's own record of the devices already set up
// (bit d for device d < 64; higher device indices set it on every call).
template <typename K>
inline cudaError_t opt_in_smem(int device, K kern, int bytes, std::atomic<unsigned long long>& done) {
    const unsigned long long bit = device >= 0 && device < 64 ? 1ull << device : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}
template <typename K>
inline cudaError_t opt_in_smem(const fvn_ctx* ctx, K kern, int bytes, std::atomic<unsigned long long>& done) {
    return opt_in_smem(ctx->device, kern, bytes, done);
}

// K-streamed tensor-core convolution of FP16 chunk-planar tensors
// ([chunks][H][W][8 halves]; conv_tc.cu): the input is source 0's ch0
// chunks followed by source 1's ch1; wpk holds the weights packed as
// [ceil((ch0 + ch1) / 2)][k * k][2][ks_coutp(cout)][8] FP16 and bias
// ks_coutp(cout) floats (zero padded).  Writes ceil(cout / 8) chunks of out
// and / or cout FP32 planes of out32.  up = 1: source 0 is a coarse tensor of
// H / 2 x W / 2 pixels whose bilinear x2 up-sampling the kernel computes
// (H, W and ch0 even).
struct KsConv {
    const void* in0;
    int ch0;
    const void* in1;
    int ch1;
    int H, W;
    const void* wpk;
    const float* bias;
    int cout, k, relu;
    void* out;
    float* out32;
    int up;
};
int ks_coutp(int cout);
fvn_status ks_conv(fvn_ctx* ctx, const KsConv& c, cudaStream_t st);

fvn_status set_error(fvn_ctx* ctx, fvn_status st, const char* fmt, ...);

#define FVN_CHECK_ARG(ctx, cond, ...)                                   \
    do {                                                                \
        if (!(cond)) return ::fvn::set_error((ctx), FVN_ERR_ARG, __VA_ARGS__); \
    } while (0)

#define FVN_CUDA(ctx, call)                                                           \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::fvn::set_error((ctx), e_ == cudaErrorMemoryAllocation ? FVN_ERR_OOM : FVN_ERR_CUDA, \
                                    "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Record stage boundary k of the fvn_render in progress when stage timing
// is on (the stages of other calls are not recorded).
inline void stage_mark(fvn_ctx* ctx, int k, cudaStream_t st) {
    if (ctx->timing && ctx->in_render) cudaEventRecord(ctx->tm_ev[k], st);
}

// Launch-error check after a kernel launch.
#define FVN_LAUNCH_CHECK(ctx) FVN_CUDA((ctx), cudaGetLastError())

fvn_status validate_volume(fvn_ctx* ctx, const fvn_volume* vol);
fvn_status validate_camera(fvn_ctx* ctx, const fvn_camera* cam);
fvn_status validate_march_params(fvn_ctx* ctx, const fvn_march_params* mp);

// Stage entry points used by fvn_render (no argument validation).
fvn_status make_mask_impl(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, uint8_t* mask, int32_t* ids,
                          int32_t* count, cudaStream_t st);
fvn_status march_impl(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                      const fvn_march_params* mp, const int32_t* ids, const int32_t* count, float* rgbam,
                      unsigned long long* nsamples, cudaStream_t st, const uint8_t* reject = nullptr);
fvn_status reconstruct_impl(fvn_ctx* ctx, const float* rgbam, const float* prev, int w, int h, int precision,
                            float* rgb, cudaStream_t st);
// One view of the batched march: its volume and padded copy, transfer
// function, camera, compacted ids / count (device) and sparse frame.
struct BatchMarchView {
    const fvn_volume* vol;
    const void* pvol;
    const fvn_tf* tf;
    const fvn_camera* cam;
    const int32_t* ids;
    const int32_t* count;
    float* rgbam;
};
// Every view's rays in one persistent launch (rgbam must already be zero
// outside the sampled pixels).
fvn_status march_batch_impl(fvn_ctx* ctx, const BatchMarchView* views, int n, const fvn_march_params* mp,
                            unsigned long long* nsamples, cudaStream_t st);
// The march's copy of a volume: a gradient volume for shaded marches that
// fit (march_uses_grad4), else a padded scalar copy; its size and one pass
// that writes it.
bool march_uses_grad4(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp);
size_t march_volume_bytes(const fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp);
fvn_status march_volume_prepare(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, void* buf,
                                cudaStream_t st);
// march_volume_prepare unless `key` says buf already holds that copy (the
// volume's generation is non-zero and unchanged); records the new source.
fvn_status march_volume_prepare_cached(fvn_ctx* ctx, const fvn_volume* vol, const fvn_march_params* mp, void* buf,
                                       PreparedKey& key, cudaStream_t st);
// Masks and id lists of n views in one launch: view i writes mask[i] and its
// ids at ids[i], its count at counts[i] (counts zeroed here).
fvn_status make_mask_batch_impl(fvn_ctx* ctx, const fvn_foveation* const* fov, const int* w, const int* h,
                                uint8_t* const* mask, int32_t* const* ids, int32_t* counts, int n,
                                cudaStream_t st);
// Error-estimate probes of the denser-mask fallback: the key of a frame's
// second hash, the compaction of the probe pixels (second hash below 1/256,
// outside the mask) and the sum of squared errors of the clamped RGB at them.
uint32_t probe_key(const fvn_foveation* f);
fvn_status probe_compact(fvn_ctx* ctx, int w, int h, uint32_t key2, const uint8_t* mask, int32_t* ids,
                         int32_t* count, cudaStream_t st);
fvn_status probe_error(fvn_ctx* ctx, const int32_t* ids, const int32_t* count, const float* rgb, const float* probe,
                       long long plane, double* acc, cudaStream_t st);
// The network launch sequence on a caller-provided workspace of at least
// recon_workspace_bytes(w, h) bytes (256-byte aligned).
fvn_status reconstruct_on(fvn_ctx* ctx, void* workspace, const float* rgbam, const float* prev, int w, int h,
                          int precision, float* rgb, cudaStream_t st);
size_t recon_workspace_bytes(int w, int h);
fvn_status reconstruct_tc(fvn_ctx* ctx, const ReconPlan& B, const float* rgbam, const float* prev, int w, int h,
                          float* rgb, cudaStream_t st);
fvn_status reconstruct_tc_fp8(fvn_ctx* ctx, const ReconPlan& B, const float* rgbam, const float* prev, int w,
                              int h, float* rgb, cudaStream_t st);
fvn_status calibrate_amax(fvn_ctx* ctx, const ReconPlan& B, int w, int h, float* d_amax, cudaStream_t st);
// The network over n views, one launch per layer for all of them (tcgen05).
fvn_status reconstruct_tc_views(fvn_ctx* ctx, const ReconView* views, int n, int precision, cudaStream_t st);
// Activation buffers of one view carved from `base` (nullptr: size only).
size_t plan_view(int w, int h, ReconPlan* plan, char* base);

}  // namespace fvn
