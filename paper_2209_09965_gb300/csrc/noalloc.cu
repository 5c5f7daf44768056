// fvn_reconstruct_noalloc: the reconstruction network of fvn_reconstruct on
// a workspace that is never allocated at run time.
//
// Some callers cannot allocate device memory at the moment they reconstruct
// a frame: code that runs while a stream is being captured into a CUDA graph
// (cudaMalloc is not a stream operation and breaks the capture), engines that
// hand the library a fixed memory budget up front and forbid allocation
// afterwards, or real-time loops where an allocation's implicit device
// synchronisation would stall the frame.  fvn_reconstruct grows a per-context
// workspace with cudaMalloc whenever the frame size changes; this entry point
// instead runs the same kernels on a file-scope device array of fixed size.
//
// The array is 64 MiB of device global memory, reserved on every GPU that
// loads this library until the process exits.  It holds the activations of
// frames up to 512 x 512 pixels (any frame whose padded activation planes
// fit; larger frames are rejected before anything is enqueued).
#include <mutex>

#include "common.cuh"

namespace fvn {

constexpr size_t kNoAllocBytes = 64ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_workspace[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[kMaxDevices];   // device address of the array, per device

// In host code g_noalloc_workspace names a host-side stand-in, not device
// memory: the device address is looked up once per device, with that device
// current, and cached.
static fvn_status noalloc_workspace(fvn_ctx* ctx, void** out) {
    int dev = -1;
    FVN_CUDA(ctx, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(ctx, FVN_ERR_UNSUPPORTED, "device index %d not supported by the no-alloc path", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        FVN_CUDA(ctx, cudaGetSymbolAddress(&p, g_noalloc_workspace));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FVN_OK;
}

}  // namespace fvn

using namespace fvn;

extern "C" fvn_status fvn_reconstruct_noalloc(fvn_ctx* ctx, const float* rgbam, int w, int h, int precision,
                                              float* rgb, void* stream) {
    if (!ctx) return set_error(nullptr, FVN_ERR_ARG, "ctx is NULL");
    FVN_CHECK_ARG(ctx, rgbam && rgb, "rgbam and rgb must be device pointers");
    FVN_CHECK_ARG(ctx, w >= 1 && h >= 1 && w <= kMaxSide && h <= kMaxSide, "frame %d x %d outside [1, %d]", w, h,
                  kMaxSide);
    FVN_CHECK_ARG(ctx, precision == FVN_PREC_FP16 || precision == FVN_PREC_FP8, "unknown precision %d", precision);
    const size_t need = recon_workspace_bytes(w, h);
    FVN_CHECK_ARG(ctx, need <= kNoAllocBytes,
                  "frame %d x %d needs %zu bytes of workspace; fvn_reconstruct_noalloc has a fixed %zu "
                  "(frames up to 512 x 512 pixels)",
                  w, h, need, kNoAllocBytes);
    if (!ctx->has_weights) return set_error(ctx, FVN_ERR_STATE, "no weights loaded (call fvn_load_weights)");
    int dev = -1;
    FVN_CUDA(ctx, cudaGetDevice(&dev));
    if (dev != ctx->device)
        return set_error(ctx, FVN_ERR_ARG, "current device %d is not the context's device %d", dev, ctx->device);
    void* ws = nullptr;
    fvn_status st = noalloc_workspace(ctx, &ws);
    if (st != FVN_OK) return st;
    return reconstruct_on(ctx, ws, rgbam, nullptr, w, h, precision, rgb, as_stream(stream));
}
