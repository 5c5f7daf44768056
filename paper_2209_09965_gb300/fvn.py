"""Python binding of libfvn (ctypes): argument marshalling only.

Every function forwards torch CUDA tensors (as device pointers) and the
current CUDA stream to the C ABI declared in ``include/fvn.h``; every step of
the computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing or was not built, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfvn.so")

FVN_OK = 0
U8, U16, F16, F32 = 0, 1, 2, 3
PREC_FP16, PREC_FP8 = 0, 1

_STATUS = {0: "FVN_OK", -1: "FVN_ERR_ARG", -2: "FVN_ERR_CUDA", -3: "FVN_ERR_OOM", -4: "FVN_ERR_UNSUPPORTED",
           -5: "FVN_ERR_STATE", -6: "FVN_ERR_TIMEOUT"}

# every symbol include/fvn.h declares
EXPORTS = (
    "fvn_create", "fvn_destroy", "fvn_last_error", "fvn_make_mask", "fvn_march", "fvn_load_weights",
    "fvn_weight_count", "fvn_reconstruct", "fvn_render", "fvn_conv_fwd", "fvn_conv_bwd", "fvn_avgpool2_fwd",
    "fvn_avgpool2_bwd", "fvn_upsample2_fwd", "fvn_upsample2_bwd", "fvn_kp_blend_fwd", "fvn_kp_blend_bwd",
    "fvn_loss_l1grad", "fvn_adam_step", "fvn_reconstruct_noalloc", "fvn_set_option", "fvn_device_status",
    "fvn_calibrate_fp8", "fvn_render_adaptive", "fvn_march_masked", "fvn_render_batch", "fvn_set_noise_tiles",
    "fvn_weight_count_recurrent", "fvn_reconstruct_recurrent", "fvn_render_recurrent", "fvn_selftest_wait_timeout",
    "fvn_wnet_weight_count", "fvn_load_wnet_weights", "fvn_reconstruct_wnet", "fvn_filter3_fwd", "fvn_filter3_bwd",
    "fvn_wnet_join_fwd", "fvn_wnet_join_bwd", "fvn_stage_times", "fvn_render_batch_adaptive",
    "fvn_conv3x3_fwd_bf16", "fvn_conv3x3_dgrad_bf16", "fvn_train_device_status", "fvn_conv3x3_wgrad_bf16",
    "fvn_head_kp_fwd", "fvn_head_kp_bwd", "fvn_adam_step_dev",
)
WNET_MAX_LEVELS = 4
MAX_VIEWS = 16
OPT_MARCH_REFILL, OPT_MARCH_BLOCKS_PER_SM = 2, 3
OPT_MARCH_REFILL_DENSE, OPT_MARCH_BLOCKS_PER_SM_DENSE = 4, 5
OPT_MARCH_COOP, OPT_MARCH_COOP_DENSE = 6, 7
OPT_MARCH_GRADIENT_VOLUME = 8
OPT_MARCH_COUNT_SHADOW = 9
OPT_STAGE_TIMING = 10
OPT_CONV_ROWS_HALF, OPT_CONV_ROWS_QUARTER, OPT_CONV_ROWS_DEC1 = 11, 12, 13
OPT_CONV_FUSE_UP_DEC1 = 14
OPT_WNET_TENSOR_CORES = 15
OPT_WNET_FUSED_UPSAMPLING = 16
STAGES = ("mask", "march_setup", "volume_prep", "march", "network")


class FvnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Volume(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dtype", ctypes.c_int), ("generation", ctypes.c_uint32)]


class TF(ctypes.Structure):
    _fields_ = [("rgba", ctypes.c_void_p), ("n", ctypes.c_int)]


class CameraC(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fov_y_deg", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class FoveationC(ctypes.Structure):
    _fields_ = [("focal_px", ctypes.c_float * 2), ("fovea_radius", ctypes.c_float),
                ("falloff_sigma", ctypes.c_float), ("p_base", ctypes.c_float), ("seed", ctypes.c_uint32),
                ("frame", ctypes.c_uint32)]


class MarchParamsC(ctypes.Structure):
    _fields_ = [("step_vox", ctypes.c_float), ("term_alpha", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("shading", ctypes.c_int), ("light_dir", ctypes.c_float * 3), ("shadow_rate", ctypes.c_int)]


class WnetConfigC(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("enc", ctypes.c_int * WNET_MAX_LEVELS), ("bot", ctypes.c_int),
                ("dec", ctypes.c_int * WNET_MAX_LEVELS)]


def wnet_config(cfg) -> WnetConfigC:
    """(enc widths, bottom width, dec widths), dec indexed by scale like enc."""
    enc, bot, dec = cfg
    c = WnetConfigC()
    c.levels = len(enc)     # more than WNET_MAX_LEVELS: the library rejects it
    for s in range(min(len(enc), WNET_MAX_LEVELS)):
        c.enc[s] = int(enc[s])
        c.dec[s] = int(dec[s])
    c.bot = int(bot)
    return c


class ViewC(ctypes.Structure):
    _fields_ = [("vol", ctypes.POINTER(Volume)), ("tf", ctypes.POINTER(TF)), ("cam", CameraC),
                ("fov", FoveationC), ("rgb", ctypes.c_void_p), ("rgbam", ctypes.c_void_p),
                ("prev_rgb", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfvn is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    sig = {
        "fvn_create": [P],
        "fvn_destroy": [P],
        "fvn_make_mask": [P, P, I, I, P, P, P, P],
        "fvn_march": [P, P, P, P, P, P, P, P, P, P],
        "fvn_load_weights": [P, P, ctypes.c_size_t],
        "fvn_reconstruct": [P, P, I, I, I, P, P],
        "fvn_reconstruct_recurrent": [P, P, P, I, I, I, P, P],
        "fvn_render_recurrent": [P, P, P, P, P, P, I, P, P, P, P],
        "fvn_reconstruct_noalloc": [P, P, I, I, I, P, P],
        "fvn_set_option": [P, I, I],
        "fvn_calibrate_fp8": [P, P, I, I, I, P],
        "fvn_march_masked": [P, P, P, P, P, P, P, P, P],
        "fvn_render_adaptive": [P, P, P, P, P, P, I, F, I, P, P, P, P],
        "fvn_device_status": [P],
        "fvn_render": [P, P, P, P, P, P, I, P, P, P],
        "fvn_render_batch": [P, P, I, P, I, P, P],
        "fvn_set_noise_tiles": [P, P, I, I],
        "fvn_selftest_wait_timeout": [P, ctypes.c_uint, P],
        "fvn_conv_fwd": [P, I, P, I, I, I, I, P, P, I, I, I, P, P],
        "fvn_conv_bwd": [P, I, P, I, I, I, I, P, I, I, P, P, P, P, P, P, P],
        "fvn_avgpool2_fwd": [P, I, I, I, P, P],
        "fvn_avgpool2_bwd": [P, I, I, I, P, P],
        "fvn_upsample2_fwd": [P, I, I, I, P, P],
        "fvn_upsample2_bwd": [P, I, I, I, P, P],
        "fvn_kp_blend_fwd": [P, P, I, I, I, P, P],
        "fvn_kp_blend_bwd": [P, P, P, I, I, I, P, P],
        "fvn_loss_l1grad": [P, P, I, I, I, F, P, P, P],
        "fvn_adam_step": [P, P, P, P, ctypes.c_size_t, I, F, F, F, F, P],
        "fvn_load_wnet_weights": [P, P, P, ctypes.c_size_t],
        "fvn_reconstruct_wnet": [P, P, I, I, P, P],
        "fvn_filter3_fwd": [P, P, I, I, I, P, P],
        "fvn_filter3_bwd": [P, P, I, I, I, P, P, P, P],
        "fvn_wnet_join_fwd": [P, P, P, I, I, I, P, P],
        "fvn_wnet_join_bwd": [P, P, P, I, I, I, P, P, P, P, P],
        "fvn_stage_times": [P, P],
        "fvn_render_batch_adaptive": [P, P, I, P, I, F, I, P, P, P, P],
        "fvn_conv3x3_fwd_bf16": [P, I, P, I, I, I, I, P, P, I, I, P, P],
        "fvn_conv3x3_dgrad_bf16": [P, P, I, I, I, I, P, I, I, P, P, P],
        "fvn_train_device_status": [],
        "fvn_conv3x3_wgrad_bf16": [P, I, P, I, I, I, I, P, P, I, P, P, P],
        "fvn_head_kp_fwd": [P, I, I, I, P, P, P, P, P, P],
        "fvn_head_kp_bwd": [P, P, P, P, P, I, I, I, P, P, P, P],
        "fvn_adam_step_dev": [P, P, P, P, ctypes.c_size_t, P, F, F, F, F, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.fvn_last_error.argtypes = [P]
    lib.fvn_last_error.restype = ctypes.c_char_p
    lib.fvn_weight_count.argtypes = []
    lib.fvn_weight_count.restype = ctypes.c_size_t
    lib.fvn_weight_count_recurrent.argtypes = []
    lib.fvn_weight_count_recurrent.restype = ctypes.c_size_t
    lib.fvn_wnet_weight_count.argtypes = [P]
    lib.fvn_wnet_weight_count.restype = ctypes.c_size_t
    return lib


lib = _load()


def _check(status, ctx=None):
    if status != FVN_OK:
        msg = lib.fvn_last_error(ctx).decode(errors="replace")
        raise FvnError(status, msg)


def _ptr(t, dtype=torch.float32):
    """Device pointer of a contiguous CUDA tensor of the expected dtype."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_DTYPE = {torch.uint8: U8, torch.int16: U16, torch.float16: F16, torch.float32: F32}
if hasattr(torch, "uint16"):
    _DTYPE[torch.uint16] = U16


def volume(t: torch.Tensor, generation: int = 0) -> Volume:
    """Descriptor of a [nz, ny, nx] CUDA volume (uint16 may be carried as
    int16).  generation != 0 lets the library reuse its prepared copy of an
    unchanged volume (change it whenever the voxels change)."""
    if t.dim() != 3 or t.dtype not in _DTYPE:
        raise ValueError("volume must be a 3-D uint8 / uint16 / float16 / float32 CUDA tensor")
    nz, ny, nx = t.shape
    return Volume(_ptr(t, None), nx, ny, nz, _DTYPE[t.dtype], int(generation) & 0xFFFFFFFF)


def transfer_function(t: torch.Tensor) -> TF:
    if t.dim() != 2 or t.shape[1] != 4 or t.dtype != torch.float32:
        raise ValueError("transfer function must be a [n, 4] float32 CUDA tensor")
    return TF(_ptr(t), t.shape[0])


def camera(cam) -> CameraC:
    c = CameraC()
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_y_deg = float(cam.fov_y_deg)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def foveation(f) -> FoveationC:
    c = FoveationC()
    c.focal_px[:] = [float(f.focal_px[0]), float(f.focal_px[1])]
    c.fovea_radius, c.falloff_sigma, c.p_base = float(f.fovea_radius), float(f.falloff_sigma), float(f.p_base)
    c.seed, c.frame = int(f.seed) & 0xFFFFFFFF, int(f.frame) & 0xFFFFFFFF
    return c


def march_params(mp) -> MarchParamsC:
    c = MarchParamsC()
    c.step_vox, c.term_alpha = float(mp.step_vox), float(mp.term_alpha)
    c.bg[:] = [float(v) for v in mp.bg]
    c.shading = int(mp.shading)
    c.light_dir[:] = [float(v) for v in getattr(mp, "light_dir", (0.0, 1.0, 0.0))]
    c.shadow_rate = int(getattr(mp, "shadow_rate", 4))
    return c


def weight_count() -> int:
    return int(lib.fvn_weight_count())


def weight_count_recurrent() -> int:
    return int(lib.fvn_weight_count_recurrent())


class Context:
    """Owns an fvn_ctx (threshold tables, work-queue counters, weights and
    reconstruction workspace) on the current CUDA device."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib.fvn_create(ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            lib.fvn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        self._chk(lib.fvn_set_option(self.h, int(option), int(value)))

    def selftest_wait_timeout(self, limit=1000, stream=None):
        """Run the bounded-wait failure path once (fvn_selftest_wait_timeout)."""
        self._chk(lib.fvn_selftest_wait_timeout(self.h, int(limit), _stream(stream)))

    def stage_times(self):
        """Per-stage ms of the last render with OPT_STAGE_TIMING on (waits for it)."""
        ms = (ctypes.c_float * len(STAGES))()
        self._chk(lib.fvn_stage_times(self.h, ms))
        return dict(zip(STAGES, (float(x) for x in ms)))

    def device_status(self):
        """Synchronise; raise FvnError(FVN_ERR_TIMEOUT) if a kernel gave up a bounded wait."""
        self._chk(lib.fvn_device_status(self.h))

    def last_error(self) -> str:
        return lib.fvn_last_error(self.h).decode(errors="replace")

    def _chk(self, st):
        _check(st, self.h)

    # --- hot path -----------------------------------------------------------
    def set_noise_tiles(self, tiles):
        """Install a looping series of sample-map noise tiles (numpy uint32
        [frames, tile, tile], values < 2^24), or None to go back to the hash."""
        if tiles is None:
            self._chk(lib.fvn_set_noise_tiles(self.h, None, 0, 0))
            return
        import numpy as np
        t = np.ascontiguousarray(tiles, dtype=np.uint32)
        if t.ndim != 3 or t.shape[1] != t.shape[2]:
            raise ValueError("noise tiles must be [frames, tile, tile]")
        self._chk(lib.fvn_set_noise_tiles(self.h, t.ctypes.data_as(ctypes.c_void_p), t.shape[1], t.shape[0]))

    def make_mask(self, fov, w, h, mask, ids, count, stream=None):
        self._chk(lib.fvn_make_mask(self.h, ctypes.byref(foveation(fov)), int(w), int(h), _ptr(mask, torch.uint8),
                                    _ptr(ids, torch.int32), _ptr(count, torch.int32), _stream(stream)))

    def march(self, vol, tf, cam, mp, rgbam, ids=None, count=None, nsamples=None, stream=None, generation=0):
        v, t, c, m = volume(vol, generation), transfer_function(tf), camera(cam), march_params(mp)
        self._chk(lib.fvn_march(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(c), ctypes.byref(m),
                                _ptr(ids, torch.int32), _ptr(count, torch.int32), _ptr(rgbam),
                                _ptr(nsamples, torch.int64), _stream(stream)))

    def march_masked(self, vol, tf, cam, mp, mask, rgbam, nsamples=None, stream=None, generation=0):
        """Naive rejection: dense ray numbering, pixels with mask 0 skipped in place."""
        v, t, c, m = volume(vol, generation), transfer_function(tf), camera(cam), march_params(mp)
        self._chk(lib.fvn_march_masked(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(c), ctypes.byref(m),
                                       _ptr(mask, torch.uint8), _ptr(rgbam), _ptr(nsamples, torch.int64),
                                       _stream(stream)))

    def load_weights(self, flat):
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        self._chk(lib.fvn_load_weights(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size))

    def load_wnet_weights(self, cfg, flat):
        """Two-stage network weights for widths cfg = (enc, bot, dec)."""
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        c = wnet_config(cfg)
        self._chk(lib.fvn_load_wnet_weights(self.h, ctypes.byref(c), a.ctypes.data_as(ctypes.c_void_p), a.size))

    def reconstruct_wnet(self, rgbam, w, h, rgb, stream=None):
        self._chk(lib.fvn_reconstruct_wnet(self.h, _ptr(rgbam), int(w), int(h), _ptr(rgb), _stream(stream)))

    def reconstruct(self, rgbam, w, h, rgb, precision=PREC_FP16, stream=None, prev=None):
        """prev: the previous output [3, h, w] for the recurrent network (fvn_reconstruct_recurrent)."""
        if prev is None:
            self._chk(lib.fvn_reconstruct(self.h, _ptr(rgbam), int(w), int(h), int(precision), _ptr(rgb),
                                          _stream(stream)))
        else:
            self._chk(lib.fvn_reconstruct_recurrent(self.h, _ptr(rgbam), _ptr(prev), int(w), int(h), int(precision),
                                                    _ptr(rgb), _stream(stream)))

    def render_adaptive(self, vol, tf, cam, fov, mp, rgb, min_psnr_db=35.0, max_levels=3, precision=PREC_FP16,
                        stream=None, generation=0):
        """fvn_render with the denser-mask fallback; returns (levels, PSNR estimate)."""
        v, t, c, m = volume(vol, generation), transfer_function(tf), camera(cam), march_params(mp)
        f = foveation(fov)
        lvl = ctypes.c_int(0)
        est = ctypes.c_float(0.0)
        self._chk(lib.fvn_render_adaptive(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(c), ctypes.byref(f),
                                          ctypes.byref(m), int(precision), float(min_psnr_db), int(max_levels),
                                          _ptr(rgb), ctypes.byref(lvl), ctypes.byref(est), _stream(stream)))
        return lvl.value, est.value

    def calibrate_fp8(self, rgbam, w, h, reset=True, stream=None):
        """Set the FP8 activation scales from this sparse frame (synchronises)."""
        self._chk(lib.fvn_calibrate_fp8(self.h, _ptr(rgbam), int(w), int(h), int(bool(reset)), _stream(stream)))

    def reconstruct_noalloc(self, rgbam, w, h, rgb, precision=PREC_FP16, stream=None):
        """fvn_reconstruct on the library's fixed workspace: never allocates
        (frames up to 512 x 512; calls sharing the workspace must not overlap)."""
        self._chk(lib.fvn_reconstruct_noalloc(self.h, _ptr(rgbam), int(w), int(h), int(precision), _ptr(rgb),
                                              _stream(stream)))

    def render(self, vol, tf, cam, fov, mp, rgb, precision=PREC_FP16, rgbam_out=None, stream=None, prev=None,
               generation=0):
        """prev: the previous output [3, h, w] for the recurrent network (fvn_render_recurrent).
        generation != 0: reuse the prepared copy of an unchanged volume (fvn_volume.generation)."""
        v, t, c, m = volume(vol, generation), transfer_function(tf), camera(cam), march_params(mp)
        f = foveation(fov)
        if prev is None:
            self._chk(lib.fvn_render(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(c), ctypes.byref(f),
                                     ctypes.byref(m), int(precision), _ptr(rgb), _ptr(rgbam_out), _stream(stream)))
        else:
            self._chk(lib.fvn_render_recurrent(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(c),
                                               ctypes.byref(f), ctypes.byref(m), int(precision), _ptr(prev),
                                               _ptr(rgb), _ptr(rgbam_out), _stream(stream)))

    def _batch_views(self, views):
        n = len(views)
        arr = (ViewC * max(n, 1))()
        keep = []   # descriptors referenced by pointer must outlive the call
        vol_desc, tf_desc = {}, {}
        for i, v in enumerate(views):
            vt, tt = v["vol"], v["tf"]
            kv = (vt.data_ptr(), tuple(vt.shape), vt.dtype)
            if kv not in vol_desc:
                vol_desc[kv] = volume(vt, v.get("generation", 0))
            kt = (tt.data_ptr(), tuple(tt.shape))
            if kt not in tf_desc:
                tf_desc[kt] = transfer_function(tt)
            vd, td = vol_desc[kv], tf_desc[kt]
            keep += [vd, td]
            arr[i].vol = ctypes.pointer(vd)
            arr[i].tf = ctypes.pointer(td)
            arr[i].cam = camera(v["cam"])
            arr[i].fov = foveation(v["fov"])
            arr[i].rgb = _ptr(v["rgb"])
            arr[i].rgbam = _ptr(v.get("rgbam"))
            arr[i].prev_rgb = _ptr(v.get("prev"))
        return arr, keep

    def render_batch(self, views, mp, precision=PREC_FP16, nsamples=None, stream=None):
        """fvn_render for several views in one pass.  ``views`` is a list of
        dicts with keys vol, tf (CUDA tensors), cam, fov and rgb (CUDA
        [3, h, w] float32), optionally rgbam (CUDA [5, h, w] float32),
        prev (the view's previous output, recurrent network) and generation
        (of the view's volume, see fvn_volume)."""
        arr, keep = self._batch_views(views)
        m = march_params(mp)
        ns = None if nsamples is None else _ptr(nsamples, torch.int64)
        self._chk(lib.fvn_render_batch(self.h, arr, len(views), ctypes.byref(m), int(precision), ns,
                                       _stream(stream)))

    def render_batch_adaptive(self, views, mp, min_psnr_db=35.0, max_levels=3, precision=PREC_FP16, nsamples=None,
                              stream=None):
        """render_batch with the per-view denser-mask fallback; returns
        (levels, PSNR estimates), one entry per view."""
        arr, keep = self._batch_views(views)
        m = march_params(mp)
        n = len(views)
        lv = (ctypes.c_int * n)()
        est = (ctypes.c_float * n)()
        ns = None if nsamples is None else _ptr(nsamples, torch.int64)
        self._chk(lib.fvn_render_batch_adaptive(self.h, arr, n, ctypes.byref(m), int(precision), float(min_psnr_db),
                                                int(max_levels), ns, lv, est, _stream(stream)))
        return list(lv), [float(x) for x in est]



# --- training kernels (context-free) -----------------------------------------
def conv_fwd(xa, xb, w, b, relu, y, stream=None):
    n, ca, h, wd = xa.shape
    cb = 0 if xb is None else xb.shape[1]
    cout, _, k, _ = w.shape
    _check(lib.fvn_conv_fwd(_ptr(xa), ca, _ptr(xb), cb, n, h, wd, _ptr(w), _ptr(b), cout, k, int(bool(relu)),
                            _ptr(y), _stream(stream)))


def conv_bwd(xa, xb, w, gy, y_relu, gxa, gxb, gw, gb, stream=None):
    n, ca, h, wd = xa.shape
    cb = 0 if xb is None else xb.shape[1]
    cout, _, k, _ = w.shape
    _check(lib.fvn_conv_bwd(_ptr(xa), ca, _ptr(xb), cb, n, h, wd, _ptr(w), cout, k, _ptr(gy), _ptr(y_relu),
                            _ptr(gxa), _ptr(gxb), _ptr(gw), _ptr(gb), _stream(stream)))


def conv3x3_fwd_bf16(xa, xb, w, b, relu, y, stream=None):
    """3x3 convolution forward on the tensor cores (BF16 operands, FP32 accumulation)."""
    n, ca, h, wd = xa.shape
    cb = 0 if xb is None else xb.shape[1]
    _check(lib.fvn_conv3x3_fwd_bf16(_ptr(xa), ca, _ptr(xb), cb, n, h, wd, _ptr(w), _ptr(b), w.shape[0],
                                    int(bool(relu)), _ptr(y), _stream(stream)))


def conv3x3_dgrad_bf16(gy, y_relu, w, ca, cb, gxa, gxb, stream=None):
    """Data gradient of a 3x3 convolution on the tensor cores: gy [N, cout, H, W]
    masked by y_relu > 0 (None: no mask) into gxa [N, ca, H, W], gxb [N, cb, H, W]."""
    n, cout, h, wd = gy.shape
    _check(lib.fvn_conv3x3_dgrad_bf16(_ptr(gy), _ptr(y_relu), cout, n, h, wd, _ptr(w), int(ca), int(cb), _ptr(gxa),
                                      _ptr(gxb), _stream(stream)))


def conv3x3_wgrad_bf16(xa, xb, gy, y_relu, gw, gb, stream=None):
    """Weight and bias gradients of a 3x3 layer on the tensor cores (overwritten)."""
    n, ca, h, wd = xa.shape
    cb = 0 if xb is None else xb.shape[1]
    _check(lib.fvn_conv3x3_wgrad_bf16(_ptr(xa), ca, _ptr(xb), cb, n, h, wd, _ptr(gy), _ptr(y_relu), gy.shape[1],
                                      _ptr(gw), _ptr(gb), _stream(stream)))


def head_kp_fwd(x, w, b, sparse, head, out, stream=None):
    """The 1x1 head (x [N][16][H][W] -> head [N][29][H][W]) and the kernel-prediction blend -> out [N][3][H][W]."""
    n, _, h, wd = x.shape
    _check(lib.fvn_head_kp_fwd(_ptr(x), n, h, wd, _ptr(w), _ptr(b), _ptr(sparse), _ptr(head), _ptr(out),
                               _stream(stream)))


def head_kp_bwd(x, head, sparse, w, gout, gx, gw, gb, stream=None):
    """dL/dx, and the head's dL/dw, dL/db (overwritten), from dL/dout of the blend."""
    n, _, h, wd = x.shape
    _check(lib.fvn_head_kp_bwd(_ptr(x), _ptr(head), _ptr(sparse), _ptr(w), _ptr(gout), n, h, wd, _ptr(gx),
                               _ptr(gw), _ptr(gb), _stream(stream)))


def train_device_status():
    """Synchronise; FvnError(TIMEOUT) if a training tensor-core wait gave up."""
    _check(lib.fvn_train_device_status())


def avgpool2_fwd(x, y, stream=None):
    n, c, h, w = x.shape
    _check(lib.fvn_avgpool2_fwd(_ptr(x), n * c, h, w, _ptr(y), _stream(stream)))


def avgpool2_bwd(gy, gx, stream=None):
    n, c, h, w = gx.shape
    _check(lib.fvn_avgpool2_bwd(_ptr(gy), n * c, h, w, _ptr(gx), _stream(stream)))


def upsample2_fwd(x, y, stream=None):
    n, c, h, w = x.shape
    _check(lib.fvn_upsample2_fwd(_ptr(x), n * c, h, w, _ptr(y), _stream(stream)))


def upsample2_bwd(gy, gx, stream=None):
    n, c, h, w = gx.shape
    _check(lib.fvn_upsample2_bwd(_ptr(gy), n * c, h, w, _ptr(gx), _stream(stream)))


def kp_blend_fwd(head, sparse, out, stream=None):
    n, _, h, w = head.shape
    _check(lib.fvn_kp_blend_fwd(_ptr(head), _ptr(sparse), n, h, w, _ptr(out), _stream(stream)))


def kp_blend_bwd(head, sparse, gout, ghead, stream=None):
    n, _, h, w = head.shape
    _check(lib.fvn_kp_blend_bwd(_ptr(head), _ptr(sparse), _ptr(gout), n, h, w, _ptr(ghead), _stream(stream)))


def loss_l1grad(pred, target, lam, loss, gpred, stream=None):
    n, c, h, w = pred.shape
    _check(lib.fvn_loss_l1grad(_ptr(pred), _ptr(target), n * c, h, w, float(lam), _ptr(loss), _ptr(gpred),
                               _stream(stream)))


def wnet_weight_count(cfg) -> int:
    c = wnet_config(cfg)
    return int(lib.fvn_wnet_weight_count(ctypes.byref(c)))


def filter3_fwd(img, logits, out, stream=None):
    n, _, h, w = img.shape
    _check(lib.fvn_filter3_fwd(_ptr(img), _ptr(logits), n, h, w, _ptr(out), _stream(stream)))


def filter3_bwd(img, logits, gout, gimg, glogits, stream=None):
    n, _, h, w = img.shape
    _check(lib.fvn_filter3_bwd(_ptr(img), _ptr(logits), n, h, w, _ptr(gout), _ptr(gimg), _ptr(glogits),
                               _stream(stream)))


def wnet_join_fwd(j, y, z, x, stream=None):
    n, _, h, w = j.shape
    _check(lib.fvn_wnet_join_fwd(_ptr(j), _ptr(y), _ptr(z), n, h, w, _ptr(x), _stream(stream)))


def wnet_join_bwd(j, y, z, gx, gj, gy, gz, stream=None):
    n, _, h, w = j.shape
    _check(lib.fvn_wnet_join_bwd(_ptr(j), _ptr(y), _ptr(z), n, h, w, _ptr(gx), _ptr(gj), _ptr(gy), _ptr(gz),
                                 _stream(stream)))


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib.fvn_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), int(step), float(lr), float(beta1),
                             float(beta2), float(eps), _stream(stream)))


def adam_step_dev(p, g, m, v, step_t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Adam with the step count in a device int32 tensor (read when the kernel runs)."""
    _check(lib.fvn_adam_step_dev(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), _ptr(step_t, torch.int32), float(lr),
                                 float(beta1), float(beta2), float(eps), _stream(stream)))
