/*
 * fvn.h -- C ABI of the GB300 foveated volume renderer (libfvn.so).
 *
 * The hot path of FoVolNet (Bauer, Wu, Ma, arXiv 2209.09965): a seeded
 * foveated sample mask and its compaction, a sparse ray march of a scalar
 * volume through the compacted pixel list, and neural reconstruction of the
 * full frame from the sparse samples.
 *
 * Conventions for every call:
 *  - Buffers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them.  Buffers named "host" are ordinary host memory
 *    read before the call returns.
 *  - Calls that take a `stream` (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream) only enqueue work on it and return without
 *    synchronising the host, unless stated otherwise.
 *  - Every argument is validated before anything is enqueued.  On error the
 *    call returns a negative fvn_status, leaves every output untouched and
 *    records a message for fvn_last_error().  Nothing throws across the ABI.
 *  - Images are planar float32: [C][H][W], x fastest, y = 0 at the top.
 *    Volumes are [nz][ny][nx], x fastest.
 *  - A context is used by one host thread at a time.
 */
#ifndef FVN_H
#define FVN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FVN_OK = 0,
    FVN_ERR_ARG = -1,          /* invalid argument (null pointer, size, range) */
    FVN_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    FVN_ERR_OOM = -3,          /* device or pinned allocation failed */
    FVN_ERR_UNSUPPORTED = -4,  /* valid request this build does not support */
    FVN_ERR_STATE = -5,        /* call out of order (e.g. no weights loaded) */
    FVN_ERR_TIMEOUT = -6       /* a kernel gave up a bounded wait (see fvn_device_status) */
} fvn_status;

/* Voxel types; integer types are normalised by their maximum (u8 / 255,
 * u16 / 65535), floating types are clamped to [0, 1]. */
typedef enum { FVN_U8 = 0, FVN_U16 = 1, FVN_F16 = 2, FVN_F32 = 3 } fvn_dtype;

/* Arithmetic of the reconstruction convolutions (FP32 accumulation). */
typedef enum { FVN_PREC_FP16 = 0, FVN_PREC_FP8 = 1 } fvn_precision;

typedef struct fvn_ctx fvn_ctx;

/* Scalar volume; data is a device pointer, 1 <= nx, ny, nz <= 4096.
 * generation: 0 = the library makes its working copy of the volume (padded
 * copy, gradient volume or shadow cells, one pass over the volume) on every
 * march; any other value lets a context reuse the copy it made last for the
 * same data pointer, sizes, voxel type, generation and kind of copy, so a
 * static volume is prepared once.  The caller must then change generation
 * whenever it changes the voxels, and order its calls on the device (one
 * stream, or events) so that a reuse follows the pass that made the copy. */
typedef struct {
    const void* data;
    int nx, ny, nz;
    int dtype;                 /* fvn_dtype */
    uint32_t generation;
} fvn_volume;

/* 1-D RGBA transfer function: device pointer to n entries of float RGBA
 * (n in [2, 4096]); looked up at continuous index v (n - 1), linear between
 * entries, alpha is the per-sample opacity. */
typedef struct {
    const float* rgba;
    int n;
} fvn_tf;

/* Pinhole camera in world space; the volume box is centred at the origin and
 * scaled so that its longest axis has length 1.  fov_y_deg in (0, 180);
 * 1 <= width, height <= 16384. */
typedef struct {
    float eye[3], target[3], up[3];
    float fov_y_deg;
    int width, height;
} fvn_camera;

/* Foveation (Eq. 1-2 of the paper).  focal_px: focal point in pixels
 * (pixel centres at x + 0.5).  fovea_radius r0 and falloff_sigma s are
 * fractions of the half diagonal R = sqrt(W^2 + H^2) / 2; p_base is the
 * periphery density P_b.  tau(d) = 1 for d <= r0, else
 * P_b + (1 - P_b) exp(-((d - r0) / s)^2 / 2).  seed and frame select the
 * per-pixel hashed noise. */
typedef struct {
    float focal_px[2];
    float fovea_radius, falloff_sigma, p_base;
    uint32_t seed, frame;
} fvn_foveation;

/* Ray-march parameters: step in voxels (> 0), early-termination opacity
 * (0, 1], background colour, and the shading:
 *   0  none (the TF colour);
 *   1  Phong with a headlight (light and view along the ray);
 *   2  Phong lit by a directional light, with global shadows as in the
 *      paper's renderer ("Foveated Rendering": one shadow ray per sample
 *      towards the light at a quarter of the main sample rate).  From every
 *      sample with opacity > 0 a shadow ray takes samples at j * ds,
 *      j = 1, 2, ..., ds = shadow_rate * step_vox, until it leaves the box;
 *      each multiplies the light's transmittance T by (1 - a)^shadow_rate
 *      (a = TF opacity there; the last sample by the power for the part of
 *      its step inside the box), and the ray stops once T < 2^-14.  The
 *      shaded colour is clamp(c (0.2 + 0.7 T |n.L|) + 0.3 T |n.H|^32) with
 *      H = |L - dir|, or clamp(c (0.2 + 0.7 T)) where the gradient is < 1e-6.
 * light_dir (world space, towards the light; normalised by the library) and
 * shadow_rate (1..64; the paper uses 4) matter for shading 2 only. */
typedef struct {
    float step_vox;
    float term_alpha;
    float bg[3];
    int shading;
    float light_dir[3];
    int shadow_rate;
} fvn_march_params;

/* Create a context on the current CUDA device.  Synchronises the host. */
fvn_status fvn_create(fvn_ctx** out);

/* Free a context and everything it owns.  Synchronises the device. */
fvn_status fvn_destroy(fvn_ctx* ctx);

/* Tuning options (fvn_set_option).  Defaults: whole 32-ray packets, no
 * cooperative finish, as many march CTAs as fit; with these the march is
 * deterministic (each ray's arithmetic is independent of which rays share
 * its warp).  Every setting computes the same result (the cooperative finish
 * up to FP32 rounding order); the autotuner times them.
 *  FVN_OPT_MARCH_REFILL: a sparse-march warp refills idle lanes with new
 *      rays once fewer than this many lanes (1..32) are busy (1 = only whole
 *      32-ray packets).
 *  FVN_OPT_MARCH_BLOCKS_PER_SM: persistent sparse-march CTAs per SM (0 = as
 *      many as fit).
 *  FVN_OPT_MARCH_COOP: once at most this many lanes (0..32) of a sparse-march
 *      warp still hold rays, the warp marches each of them with all 32 lanes
 *      (32 samples per step, composited by a product scan of the
 *      transmittances; the same result up to FP32 rounding order); 0 = never;
 *      32 = every ray, a warp taking one ray at a time from the queue.
 *  FVN_OPT_MARCH_REFILL_DENSE, FVN_OPT_MARCH_BLOCKS_PER_SM_DENSE,
 *  FVN_OPT_MARCH_COOP_DENSE: the same for the dense march (ids == NULL).
 *  FVN_OPT_MARCH_GRADIENT_VOLUME: 1 (default) = a shaded march first writes a
 *      gradient volume, (v, dv/dx, dv/dy, dv/dz) as central differences per
 *      padded voxel (16 bytes each, used when that takes at most 4 GiB), and
 *      reads 8 of those per sample instead of 32 voxels; 0 = always the
 *      32-voxel stencil.  Same result up to FP32 rounding order.
 *  FVN_OPT_MARCH_COUNT_SHADOW: 1 = with shading 2, the nsamples counter of a
 *      march also counts the samples of the shadow rays (default 0: primary
 *      samples only).
 *  FVN_OPT_STAGE_TIMING: 1 = fvn_render records CUDA events at its stage
 *      boundaries (read with fvn_stage_times); 0 (default) = none.
 *  FVN_OPT_CONV_ROWS_HALF (2 or 4, default 4), FVN_OPT_CONV_ROWS_QUARTER
 *      (1, 2 or 4, default 2), FVN_OPT_CONV_ROWS_DEC1 (1 or 2, default 1):
 *      output rows per tile of the network's half-resolution 32-channel
 *      convolutions, of its quarter-resolution bottleneck convolutions and of
 *      its first decoder convolution (96 input channels).  Every setting
 *      computes the same result bit for bit (each output pixel's sums are
 *      formed in the same order).
 *  FVN_OPT_CONV_FUSE_UP_DEC1: 1 = the first decoder convolution up-samples
 *      the bottleneck output itself instead of reading a pass's up-sampled
 *      copy (0, default); the in-kernel up-sampling interpolates in half
 *      precision, so the two differ by FP16 rounding.
 *  FVN_OPT_WNET_TENSOR_CORES: 1 = fvn_reconstruct_wnet runs its convolutions
 *      on the tensor cores (FP16 operands and activations, FP32
 *      accumulation; needs every width a multiple of 8 and at most 128,
 *      else FVN_ERR_UNSUPPORTED); 0 (default) = FP32 kernels throughout.
 *  FVN_OPT_WNET_FUSED_UPSAMPLING: 1 (default) = on the tensor cores, the
 *      first convolution of each decoder level computes the bilinear x2
 *      up-sampling of its coarse input itself (when that input's channels
 *      fill whole 16-channel groups); 0 = a separate up-sampling pass writes
 *      the fine copy it reads.  The same bits either way.
 * A shadowed march (shading 2) first writes, besides the padded copy, a cell
 * volume -- per padded voxel the 2 x 2 block of voxels (x..x+1, y..y+1) in
 * the voxel type -- so that a shadow sample reads two cells instead of
 * eight voxels; the gradient-volume option does not apply to it. */
enum {
    FVN_OPT_MARCH_REFILL = 2,
    FVN_OPT_MARCH_BLOCKS_PER_SM = 3,
    FVN_OPT_MARCH_REFILL_DENSE = 4,
    FVN_OPT_MARCH_BLOCKS_PER_SM_DENSE = 5,
    FVN_OPT_MARCH_COOP = 6,
    FVN_OPT_MARCH_COOP_DENSE = 7,
    FVN_OPT_MARCH_GRADIENT_VOLUME = 8,
    FVN_OPT_MARCH_COUNT_SHADOW = 9,
    FVN_OPT_STAGE_TIMING = 10,
    FVN_OPT_CONV_ROWS_HALF = 11,
    FVN_OPT_CONV_ROWS_QUARTER = 12,
    FVN_OPT_CONV_ROWS_DEC1 = 13,
    FVN_OPT_CONV_FUSE_UP_DEC1 = 14,
    FVN_OPT_WNET_TENSOR_CORES = 15,
    FVN_OPT_WNET_FUSED_UPSAMPLING = 16
};
fvn_status fvn_set_option(fvn_ctx* ctx, int option, int value);

/* Stage times of the last fvn_render / fvn_render_recurrent of this context,
 * with FVN_OPT_STAGE_TIMING set to 1 before it (the option makes fvn_render
 * record CUDA events on its stream at the stage boundaries; paper: the
 * per-stage frame times of its evaluation, section "Performance").  Waits
 * for that frame, then writes five host floats, in milliseconds: mask and
 * compaction; the march's setup (clearing the sparse frame); the volume
 * preparation (0 when a reusable copy was current); the march kernel; the
 * reconstruction network.  FVN_ERR_STATE when no frame was recorded. */
fvn_status fvn_stage_times(fvn_ctx* ctx, float* ms);

/* Synchronise the device and report a device-side failure recorded by this
 * context's kernels since the last call: FVN_ERR_TIMEOUT when a tensor-core
 * wait gave up after its iteration limit (the kernel then skipped its
 * remaining work and left its outputs incomplete).  Clears the flag. */
fvn_status fvn_device_status(fvn_ctx* ctx);

/* Diagnostic of that failure path: launches one kernel that waits, with the
 * same bounded mbarrier wait the tensor-core kernels use, on a barrier that
 * nothing completes; after `limit` polls (1..2^20) it gives up and records
 * the give-up in the context's error flag, so the next fvn_device_status
 * returns FVN_ERR_TIMEOUT and clears it -- the context stays usable.  No
 * other work is touched. */
fvn_status fvn_selftest_wait_timeout(fvn_ctx* ctx, unsigned limit, void* stream);

/* Last error message of this context (or of the calling thread when ctx is
 * NULL); never NULL, "" when there was none. */
const char* fvn_last_error(const fvn_ctx* ctx);

/*
 * fvn_make_mask -- binary sample mask and its stream compaction.
 * Paper: "Sample Maps" (M(u, v) = 1 iff N(u, v) < tau(u, v); Eq. 1-2) and
 * "Stream Compaction" (pack the valid pixels into a small buffer).
 *
 * N(u, v) is the top 24 bits of a 32-bit integer hash of (seed, frame, x, y),
 * or, after fvn_set_noise_tiles, the context's noise tile for the frame;
 * tau is taken from a 16384-entry table of floor(tau 2^24) indexed by the
 * squared half-pixel distance to the focal point (built on the host in
 * float64 and cached in the context).  The decision is integer-only and
 * bit-exact.
 *
 * mask  : device uint8 [h][w], written 0 / 1 for every pixel.
 * ids   : device int32 [>= w*h], receives the ids y*w + x of the sampled
 *         pixels in an unspecified order (tile by tile).
 * count : device int32, receives the number of sampled pixels.
 * The first call with a new (w, h, r0, s, P_b) builds and uploads the table
 * and is the only one that does host work beyond argument checks.
 */
fvn_status fvn_make_mask(fvn_ctx* ctx, const fvn_foveation* fov, int w, int h, uint8_t* mask,
                         int32_t* ids, int32_t* count, void* stream);

/*
 * fvn_set_noise_tiles -- the noise of the sample maps from a looping series
 * of tiles instead of the hash.  Paper: "Noise Patterns" (masks from a
 * pre-computed series of 64 spatio-temporal blue-noise tiles of 16^2 to
 * 256^2 pixels, tiled over the frame and looped over the frames).
 *
 * tiles : HOST uint32 [frames][tile][tile], every value below 2^24; the
 *         context keeps its own device copy (the caller's array may be freed).
 *         NULL reverts to the hash.
 * tile  : side of a tile, a power of two in [16, 256].
 * frames: number of tiles, 1..256; frame f of a foveation uses tile f mod frames.
 * From then on every mask of the context (fvn_make_mask, fvn_render,
 * fvn_render_batch, fvn_render_adaptive) takes
 * N(x, y) = tiles[frame mod frames][y mod tile][x mod tile].  Synchronises the
 * device (masks already queued may read the previous tiles); nothing changes
 * on error.
 */
fvn_status fvn_set_noise_tiles(fvn_ctx* ctx, const uint32_t* tiles, int tile, int frames);

/*
 * fvn_march -- emission-absorption ray march of the volume.
 * Paper: "Foveated Rendering" / "Rendering" (a CUDA ray-marching DVR renderer
 * casting one ray per valid pixel of the compacted buffer, with the results
 * projected back to their full-frame positions).
 *
 * Per ray: slab test against the volume box, samples at
 * t_k = max(t_enter, 0) + k step for every t_k < t_exit, trilinear fetch
 * (clamp to edge), transfer-function lookup, optional Phong shading from
 * central differences, front-to-back compositing, termination once
 * A >= term_alpha.
 *
 * ids == NULL: dense march, every pixel of the camera frame.
 * ids != NULL: sparse march of the *count pixel ids in ids (count is a
 *              device int32, read by the kernel, so the call needs no host
 *              synchronisation after fvn_make_mask); every other pixel of
 *              rgbam is written 0.
 * rgbam    : device float [5][h][w]: R, G, B (composited over bg), A, and the
 *            mask channel M (1 where a ray was cast).
 * nsamples : optional device uint64 accumulator; the number of classified
 *            samples is ADDED to it (NULL to skip).
 */
fvn_status fvn_march(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                     const fvn_march_params* mp, const int32_t* ids, const int32_t* count, float* rgbam,
                     unsigned long long* nsamples, void* stream);

/*
 * fvn_march_masked -- the naive alternative to compaction.
 * Paper: "Rendering" (a kernel over the full frame whose invalid pixels are
 * simply discarded at kernel level, so a warp still waits for its slowest
 * lane).  Dense ray numbering over the whole frame; pixels whose byte in
 * mask (device uint8 [h][w]) is 0 are skipped in place and written 0, the
 * others are marched exactly as fvn_march does.  Kept as the baseline of the
 * compaction-efficiency measurement.
 */
fvn_status fvn_march_masked(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                            const fvn_march_params* mp, const uint8_t* mask, float* rgbam,
                            unsigned long long* nsamples, void* stream);

/*
 * fvn_load_weights -- install reconstruction-network weights.
 * Paper: "Model Precision & Optimization" (train in FP32, run with weights
 * truncated to 16-bit).  host_w: host float32, the flat layer order
 * enc0a(5->16) enc0b(16->16) enc1a(16->32) enc1b(32->32) bota(32->64)
 * botb(64->64) dec1a(96->32) dec1b(32->32) dec0a(48->16) dec0b(16->16)
 * head(16->29, 1x1); each layer W[cout][cin][k][k] then b[cout].  n must
 * equal fvn_weight_count(), or fvn_weight_count_recurrent() for the
 * recurrent network, whose enc0a takes 8 channels: the 5 of the sparse frame
 * and the previous frame's output RGB (paper: "Recurrence": the output of D
 * is passed back to its input in the next run, concatenated along the
 * channels).  Converts to the FP16 and FP8 layouts of the kernels.
 * Synchronises the host.
 */
fvn_status fvn_load_weights(fvn_ctx* ctx, const float* host_w, size_t n);
size_t fvn_weight_count(void);
size_t fvn_weight_count_recurrent(void);

/*
 * fvn_reconstruct -- full frame from the sparse samples.
 * Paper: "Reconstruction Network" (a U-Net direct prediction "D" whose
 * decoder state drives per-pixel kernel prediction "K"; Fig. "network
 * architecture"), slim variant: 3 levels of 16/32/64 channels, two 3x3
 * conv + ReLU per level, 2x2 average pooling, bilinear x2 up-sampling with
 * skip concatenation, a 1x1 head giving the direct RGB, 25 kernel logits and
 * a blend logit; softmax 5x5 kernel applied to the sparse samples normalised
 * by the sampled weights, blended with the direct RGB by sigmoid(blend).
 *
 * rgbam : device float [5][h][w] from fvn_march (M = 0 where not sampled).
 * rgb   : device float [3][h][w] output.
 * precision : FVN_PREC_FP16 or FVN_PREC_FP8 operands, FP32 accumulation.
 * Needs fvn_load_weights first (FVN_ERR_STATE otherwise).  Uses context
 * workspace sized on first use for (w, h).
 */
fvn_status fvn_reconstruct(fvn_ctx* ctx, const float* rgbam, int w, int h, int precision, float* rgb,
                           void* stream);

/*
 * fvn_reconstruct_recurrent -- fvn_reconstruct with the recurrent network:
 * prev_rgb (device float [3][h][w], the previous frame's output, clamped to
 * [0, 1] as input; NULL reads zeros, for the first frame of a sequence)
 * enters the first layer beside the sparse frame.  rgb must not alias
 * prev_rgb.  FVN_ERR_STATE when prev_rgb is set and the loaded weights are
 * not the recurrent network's.  (fvn_reconstruct with recurrent weights is
 * this call with prev_rgb = NULL.)
 */
fvn_status fvn_reconstruct_recurrent(fvn_ctx* ctx, const float* rgbam, const float* prev_rgb, int w, int h,
                                     int precision, float* rgb, void* stream);

/*
 * fvn_calibrate_fp8 -- activation scales and E4M3 weights for
 * FVN_PREC_FP8.  Paper: "Model Precision & Optimization" (post-training
 * reduction of precision; the paper's INT8 path used a calibrating engine
 * builder).  Runs the FP16 network on the sparse frame rgbam ([5][h][w],
 * device), takes the largest value of every activation tensor (a running
 * maximum over calls unless reset != 0), sets each tensor's scale to
 * amax / 448 and re-quantises the weights to E4M3 with those input scales
 * folded in and one scale per output channel.  Synchronises the host.
 * fvn_load_weights discards the FP8 state.
 */
fvn_status fvn_calibrate_fp8(fvn_ctx* ctx, const float* rgbam, int w, int h, int reset, void* stream);

/*
 * fvn_reconstruct_noalloc -- fvn_reconstruct without any allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they reconstruct a frame, such as code
 * running while a stream is captured into a CUDA graph, engines that fix
 * their memory budget up front, or real-time loops that cannot afford the
 * device synchronisation an allocation implies.  Same arguments, kernels and
 * results as fvn_reconstruct, but the activation workspace is a fixed 64 MiB
 * device array inside the library (reserved on every GPU that loads the
 * library, until the process exits) instead of context memory grown with
 * cudaMalloc.  It never calls cudaMalloc, cudaFree or an allocating routine.
 *  - Frames whose workspace exceeds 64 MiB (larger than about 512 x 512
 *    pixels) are rejected with FVN_ERR_ARG before anything is enqueued.
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    stream capture.
 *  - Every call, from every context and stream, shares the one array and
 *    leaves its activations there; calls that overlap on the GPU race on
 *    it, so serialise them (one stream, or events).  Nothing in the array
 *    needs to start at zero: every activation is written before it is read.
 * Needs fvn_load_weights on ctx first (FVN_ERR_STATE otherwise).
 */
fvn_status fvn_reconstruct_noalloc(fvn_ctx* ctx, const float* rgbam, int w, int h, int precision, float* rgb,
                                   void* stream);

/*
 * fvn_render -- one foveated frame: fvn_make_mask, sparse fvn_march and
 * fvn_reconstruct on context workspace, no host synchronisation.
 * Paper: Fig. "pipeline" (sample mask -> compaction -> sparse rendering ->
 * reconstruction).  rgb: device float [3][h][w] with (w, h) from the camera.
 * rgbam_out: optional device float [5][h][w] copy target for the sparse frame
 * (NULL to skip).
 */
fvn_status fvn_render(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                      const fvn_foveation* fov, const fvn_march_params* mp, int precision, float* rgb,
                      float* rgbam_out, void* stream);

/* fvn_render with the recurrent network and the previous frame's output
 * prev_rgb (as fvn_reconstruct_recurrent; rgb must not alias it). */
fvn_status fvn_render_recurrent(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                                const fvn_foveation* fov, const fvn_march_params* mp, int precision,
                                const float* prev_rgb, float* rgb, float* rgbam_out, void* stream);

/*
 * fvn_render_adaptive -- fvn_render with a denser-mask fallback (the paper
 * has no counterpart; this is the frame-quality guard of this library).
 * After each frame a probe set -- the pixels whose second hash of
 * (seed ^ 0x9E3779B9, frame, y, x) has its top 24 bits below 2^16 (1/256 of
 * the frame) and that the mask left out -- is ray-marched too, and the PSNR
 * of the reconstruction against those probes (RGB clamped to [0, 1]) is the
 * frame's error estimate.  While the estimate is below min_psnr_db and fewer
 * than max_levels re-renders were made, the frame is rendered again with
 * P_b doubled (capped at 1).  level_out / psnr_out (host, optional) receive
 * the number of re-renders and the last estimate.  Synchronises the host
 * once per level (it reads the 12-byte error sum).
 */
fvn_status fvn_render_adaptive(fvn_ctx* ctx, const fvn_volume* vol, const fvn_tf* tf, const fvn_camera* cam,
                               const fvn_foveation* fov, const fvn_march_params* mp, int precision,
                               float min_psnr_db, int max_levels, float* rgb, int* level_out, float* psnr_out,
                               void* stream);

/* Most views one fvn_render_batch call takes. */
#define FVN_MAX_VIEWS 16

/* One view of a batch.  vol, tf: as for fvn_render (read before the call
 * returns; views may share them).  cam, fov: the view's camera (its width x
 * height is the view's size) and foveation.  rgb: device float [3][h][w]
 * output.  rgbam: optional device float [5][h][w] that receives the view's
 * sparse frame (NULL: kept in the context's workspace).  prev_rgb: the
 * view's previous output for the recurrent network (as
 * fvn_reconstruct_recurrent), or NULL. */
typedef struct {
    const fvn_volume* vol;
    const fvn_tf* tf;
    fvn_camera cam;
    fvn_foveation fov;
    float* rgb;
    float* rgbam;
    const float* prev_rgb;
} fvn_view;

/*
 * fvn_render_batch -- fvn_render for 1..FVN_MAX_VIEWS views of any sizes
 * (stereo pairs, several resolutions) over up to 4 distinct volumes (of any
 * voxel types) in one pass: one mask + compaction launch for all views, one
 * padding launch per distinct volume, ONE persistent march launch over the
 * rays of every view, and one launch per network layer over the tiles of
 * every view.  The paper renders one view per frame (Fig. "pipeline"); the
 * batch is this library's multi-view form of that frame, and each view's rgb
 * (and rgbam) equals what fvn_render gives for that view alone, bit for bit.
 * The distinct transfer functions together hold at most 4096 entries.
 * nsamples: optional device counter, incremented by the samples of all
 * views.  The context keeps a batch workspace (about 215 B per pixel);
 * growing it synchronises the device, so capture the call in a CUDA graph
 * only after one call with the same view sizes.
 */
fvn_status fvn_render_batch(fvn_ctx* ctx, const fvn_view* views, int nviews, const fvn_march_params* mp,
                            int precision, unsigned long long* nsamples, void* stream);

/*
 * fvn_render_batch_adaptive -- fvn_render_batch with the denser-mask
 * fallback of fvn_render_adaptive applied to every view (the paper has no
 * counterpart; this is the library's frame-quality guard).  After each
 * batch, every view's probes (its second hash below 1/256, outside its mask)
 * are ray-marched in one launch and the PSNR of its reconstruction there
 * estimates the view's PSNR; the views below min_psnr_db that have made
 * fewer than max_levels (0..8) re-renders and whose P_b is below 1 are
 * rendered again, together, with P_b doubled (capped at 1).  Each view ends
 * with the output fvn_render_adaptive gives for it alone.  levels_out /
 * psnr_out: optional host arrays of nviews entries (re-renders, last
 * estimate).  nsamples counts the samples of every batch pass.  Synchronises
 * the host once per pass; keeps a probe workspace of 24 bytes per pixel.
 */
fvn_status fvn_render_batch_adaptive(fvn_ctx* ctx, const fvn_view* views, int nviews, const fvn_march_params* mp,
                                     int precision, float min_psnr_db, int max_levels, unsigned long long* nsamples,
                                     int* levels_out, float* psnr_out, void* stream);

/* ------------------------------------------------------------------------
 * Training kernels (FP32, NCHW with batch N).  Paper: "Training" and "Loss"
 * sections (the network is trained in FP32).  These are the forward and
 * backward pieces behind the Python autograd functions; all pointers are
 * device float32, all calls asynchronous on `stream`.
 * ------------------------------------------------------------------------ */

/* y = conv_k(x) + b, optional ReLU; x is the channel concatenation of xa
 * [N][ca][H][W] and xb [N][cb][H][W] (xb may be NULL with cb = 0);
 * w [cout][ca+cb][k][k]; k in {1, 3}, zero padding k/2. */
fvn_status fvn_conv_fwd(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                        const float* w, const float* b, int cout, int k, int relu, float* y, void* stream);

/* Gradients of the layer above.  gy is dL/dy; y_relu (the saved ReLU output,
 * or NULL for a layer without ReLU) masks it to dL/dz.  gxa / gxb receive
 * dL/dx (overwritten; either may be NULL to skip), gw / gb receive dL/dw,
 * dL/db (overwritten). */
fvn_status fvn_conv_bwd(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                        const float* w, int cout, int k, const float* gy, const float* y_relu,
                        float* gxa, float* gxb, float* gw, float* gb, void* stream);

/* The 3x3 layers on the tensor cores (tcgen05, BF16 operands rounded from
 * the FP32 tensors while staged, FP32 accumulation; paper: "Model Precision &
 * Optimization" -- FP32 master weights, 16-bit arithmetic).
 * fvn_conv3x3_fwd_bf16: as fvn_conv_fwd with k = 3.  fvn_conv3x3_dgrad_bf16:
 * dL/dx of the layer (ca + cb input channels, cout outputs, weights w
 * [cout][ca+cb][3][3]) from gy [N][cout][H][W], masked by y_relu > 0 when
 * y_relu is set, into gxa [N][ca][H][W] and gxb [N][cb][H][W] (either may be
 * NULL to skip).  Channel pairs (in -> out, padded to multiples of 16) of
 * 16/32/48/64/96 channels as the slim network's layers need;
 * FVN_ERR_UNSUPPORTED for others.  fvn_train_device_status synchronises and
 * returns FVN_ERR_TIMEOUT (clearing the flag) when one of these kernels gave
 * up a bounded wait. */
fvn_status fvn_conv3x3_fwd_bf16(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                const float* w, const float* b, int cout, int relu, float* y, void* stream);
fvn_status fvn_conv3x3_dgrad_bf16(const float* gy, const float* y_relu, int cout, int n, int h, int w_,
                                  const float* w, int ca, int cb, float* gxa, float* gxb, void* stream);
fvn_status fvn_train_device_status(void);
/* dL/dw [cout][ca+cb][3][3] and dL/db [cout] (overwritten) of a 3x3 layer on
 * the tensor cores: the sum over images and pixels of gy (masked by
 * y_relu > 0 when set) times the shifted inputs xa / xb, as a GEMM over the
 * pixels with BF16 operands and FP32 accumulation (cout up to 96). */
fvn_status fvn_conv3x3_wgrad_bf16(const float* xa, int ca, const float* xb, int cb, int n, int h, int w_,
                                  const float* gy, const float* y_relu, int cout, float* gw, float* gb, void* stream);

/* 2x2 average pooling and its adjoint ([N][C][H][W] -> [N][C][H/2][W/2]). */
fvn_status fvn_avgpool2_fwd(const float* x, int nc, int h, int w_, float* y, void* stream);
fvn_status fvn_avgpool2_bwd(const float* gy, int nc, int h, int w_, float* gx, void* stream);

/* Bilinear x2 up-sampling (half-pixel centres, edge clamp) and its adjoint;
 * h, w are the input (coarse) sizes. */
fvn_status fvn_upsample2_fwd(const float* x, int nc, int h, int w_, float* y, void* stream);
fvn_status fvn_upsample2_bwd(const float* gy, int nc, int h, int w_, float* gx, void* stream);

/* Kernel prediction + blend: head [N][29][H][W], sparse [N][5][H][W] ->
 * out [N][3][H][W]; and dL/dhead from dL/dout. */
fvn_status fvn_kp_blend_fwd(const float* head, const float* sparse, int n, int h, int w_, float* out,
                            void* stream);
fvn_status fvn_kp_blend_bwd(const float* head, const float* sparse, const float* gout, int n, int h,
                            int w_, float* ghead, void* stream);

/* The 1x1 head and the kernel-prediction blend fused (the paper's "Kernel
 * Prediction" subsection).  Forward: head = w x + b ([N][16][H][W] ->
 * [N][29][H][W], written for the backward pass; w [29][16], b [29]) and
 * out [N][3][H][W] as fvn_kp_blend_fwd computes it from head.  Backward:
 * from dL/dout, dL/dx (overwritten) and the head's dL/dw, dL/db
 * (overwritten); dL/dhead is not stored.  FP32 throughout; the weight
 * gradients are summed with atomics (order not fixed). */
fvn_status fvn_head_kp_fwd(const float* x, int n, int h, int w_, const float* w, const float* b,
                           const float* sparse, float* head, float* out, void* stream);
fvn_status fvn_head_kp_bwd(const float* x, const float* head, const float* sparse, const float* w,
                           const float* gout, int n, int h, int w_, float* gx, float* gw, float* gb, void* stream);

/* L1 + lam * (L1 of x / y forward differences), each a mean over its own
 * elements, over pred / target [N][C][H][W].  loss: device float scalar
 * (overwritten); gpred: dL/dpred (overwritten). */
fvn_status fvn_loss_l1grad(const float* pred, const float* target, int nc, int h, int w_, float lam,
                           float* loss, float* gpred, void* stream);

/* One bias-corrected Adam step on n parameters (step >= 1). */
fvn_status fvn_adam_step(float* p, const float* g, float* m, float* v, size_t n, int step, float lr,
                         float beta1, float beta2, float eps, void* stream);
/* The same with the step count (int, >= 1) read from device memory when the
 * kernel runs, so that a step captured in a CUDA graph can be replayed. */
fvn_status fvn_adam_step_dev(float* p, const float* g, float* m, float* v, size_t n, const int* step, float lr,
                             float beta1, float beta2, float eps, void* stream);

/* ------------------------------------------------------------------------
 * Two-stage network (paper: "Reconstruction Network" -- a first U-Net D
 * predicts a coarse image O_d directly and keeps its decoder's hidden states
 * H_d; a second U-Net K predicts per-pixel filter kernels from H_d at several
 * scales, in its encoder and its decoder blocks, and passes O_d through them
 * in sequence; "Model Configuration": both follow the block plan
 * e64-e64-e80-d96-d80-d64-d64, D's blocks hold two 3x3 convolutions with
 * ReLU, K's blocks one 1x1 convolution).  Readings where the paper is
 * silent: K's blocks take D's decoder state of their own scale (the
 * encoder blocks also the pooled output of the block above, the decoder
 * blocks the up-sampled output of the block below); each block's 1x1 heads
 * give 9 logits of a 3x3 kernel (softmax over the taps inside the frame) and,
 * in the decoder blocks, one blend logit z; the image is filtered by the
 * encoder blocks (pooled between scales), by the coarsest block, then, going
 * up, joined to the encoder image of each scale by
 * X = J + sigmoid(z) up(Y - pool J) and filtered by that decoder block.
 * FP32 throughout (CUDA cores), NCHW.
 * ------------------------------------------------------------------------ */

#define FVN_WNET_MAX_LEVELS 4

/* Block widths: enc[s] / dec[s] of the encoder / decoder block at scale s
 * (resolution 2^-s), 0 <= s < levels; bot of the block at scale `levels`.
 * levels 1..4, widths 1..256.  The paper's plan: levels 3, enc {64, 64, 80},
 * bot 96, dec {64, 64, 80}. */
typedef struct {
    int levels;
    int enc[FVN_WNET_MAX_LEVELS];
    int bot;
    int dec[FVN_WNET_MAX_LEVELS];
} fvn_wnet_config;

/* Number of float weights of a configuration; 0 when it is invalid.  Order
 * (each layer W[cout][cin][k][k] then b[cout]):
 *   D: per scale s = 0..L-1 enc_s a (cin -> enc[s], 3x3; cin = 5 at s = 0,
 *      else enc[s-1]), enc_s b (enc[s] -> enc[s]); bot a (enc[L-1] -> bot),
 *      bot b; per s = L-1..0 dec_s a ((bot or dec[s+1]) + enc[s] -> dec[s],
 *      input order [up-sampled, skip]), dec_s b; out (dec[0] -> 3, 1x1).
 *   K (all 1x1): per s = 0..L-1 enc_s ([pooled K enc_(s-1) (s > 0), D dec_s]
 *      -> enc[s]), enc_s taps (enc[s] -> 9); bot ([pooled K enc_(L-1), D bot]
 *      -> bot), bot taps (bot -> 9); per s = L-1..0 dec_s ([up-sampled K
 *      (bot or dec_(s+1)), D dec_s] -> dec[s]), dec_s taps (dec[s] -> 9),
 *      dec_s blend (dec[s] -> 1). */
size_t fvn_wnet_weight_count(const fvn_wnet_config* cfg);

/* Install two-stage weights (host float array of fvn_wnet_weight_count(cfg)
 * entries, all finite; copied, synchronises).  Independent of
 * fvn_load_weights.  An argument error (FVN_ERR_ARG) keeps the weights
 * installed before; a CUDA error during the copy leaves none installed. */
fvn_status fvn_load_wnet_weights(fvn_ctx* ctx, const fvn_wnet_config* cfg, const float* host_w, size_t n);

/* The two-stage network on one sparse frame: rgbam device float [5][h][w]
 * (as fvn_reconstruct) -> rgb device float [3][h][w].  The frame is padded
 * with zeros at the bottom / right to a multiple of 2^levels and cropped
 * back.  Uses a context workspace (reallocated, with a device
 * synchronisation, when the frame size changes).  FVN_ERR_STATE without
 * fvn_load_wnet_weights. */
fvn_status fvn_reconstruct_wnet(fvn_ctx* ctx, const float* rgbam, int w, int h, float* rgb, void* stream);

/* Training pieces of the two-stage network (FP32, NCHW, device pointers).
 * fvn_filter3_fwd: out[n][c] (p) = sum_q w_q(p) img[n][c](p + q), c < 3,
 * w = softmax of logits[n][0..8](p) over the taps q = (q/3 - 1, q%3 - 1)
 * with p + q inside the h x w frame (h and n at most 65535, else
 * FVN_ERR_ARG).  fvn_filter3_bwd: dL/dimg and dL/dlogits (overwritten)
 * from dL/dout. */
fvn_status fvn_filter3_fwd(const float* img, const float* logits, int n, int h, int w_, float* out, void* stream);
fvn_status fvn_filter3_bwd(const float* img, const float* logits, int n, int h, int w_, const float* gout,
                           float* gimg, float* glogits, void* stream);

/* fvn_wnet_join_fwd: x = j + sigmoid(z) up(y - pool j), j / x [N][3][h][w],
 * y [N][3][h/2][w/2], z [N][1][h][w]; h, w even; the forward pass takes h
 * and N up to 65535.  fvn_wnet_join_bwd: dL/dj,
 * dL/dy and dL/dz (overwritten) from dL/dx. */
fvn_status fvn_wnet_join_fwd(const float* j, const float* y, const float* z, int n, int h, int w_, float* x,
                             void* stream);
fvn_status fvn_wnet_join_bwd(const float* j, const float* y, const float* z, int n, int h, int w_,
                             const float* gx, float* gj, float* gy, float* gz, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FVN_H */
