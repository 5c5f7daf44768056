"""Oracle: Python loader for the FP64 C ray marcher (``march.c``).

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  See ``march.c`` for the definition of
what is computed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "march.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_march.so")

DTYPES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float16): 2, np.dtype(np.float32): 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile march.c with gcc (-O2 -fopenmp, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.or_march.restype = ctypes.c_int64
        lib.or_march.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                 P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_double, P, P, P]
        lib.or_trilinear.restype = None
        lib.or_trilinear.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                     ctypes.c_int64, P]
        lib.or_shadow.restype = None
        lib.or_shadow.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                                  ctypes.c_int64, P, ctypes.c_double, ctypes.c_int, P]
        lib.or_set_threads.restype = None
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_ray.restype = None
        lib.or_ray.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cam_array(cam):
    return np.array(list(cam.eye) + list(cam.target) + list(cam.up) + [cam.fov_y_deg], dtype=np.float64)


def _mp_array(mp):
    light = getattr(mp, "light_dir", (0.0, 1.0, 0.0))
    rate = getattr(mp, "shadow_rate", 4)
    return np.array([mp.step_vox, mp.term_alpha, *mp.bg, float(mp.shading), *light, float(rate)],
                    dtype=np.float64)


def _vol_args(vol):
    vol = np.ascontiguousarray(vol)
    if vol.dtype == np.int16:          # uint16 bit pattern carried in int16
        vol = vol.view(np.uint16)
    if vol.dtype not in DTYPES:
        raise TypeError(f"unsupported volume dtype {vol.dtype}")
    nz, ny, nx = vol.shape
    return vol, DTYPES[vol.dtype], nx, ny, nz


def march(vol, tf, cam, mp, ids=None, count_shift=0, term_override=0.0, margins=False):
    """Return (out [5, H, W] float64, amb [H, W] uint8, nsamples), and with
    margins=True also margin [2, H, W]: per marched pixel the distance of the
    sample count (t_far - t_near) / dt to the nearest integer and the smallest
    |A - term| over its steps -- the quantities the ambiguity flags test."""
    vol, dt, nx, ny, nz = _vol_args(vol)
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    camv = _cam_array(cam)
    mpv = _mp_array(mp)
    W, H = cam.width, cam.height
    out = np.empty((5, H, W), dtype=np.float64)
    amb = np.empty((H, W), dtype=np.uint8)
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        idp, nids = _ptr(ids), ids.size
    else:
        idp, nids = None, 0
    mg = np.full((H * W, 2), np.inf, dtype=np.float64) if margins else None
    ns = _load().or_march(_ptr(vol), dt, nx, ny, nz, _ptr(tf), tf.shape[0], _ptr(camv), W, H, _ptr(mpv),
                          idp, nids, int(count_shift), float(term_override), _ptr(out), _ptr(amb),
                          _ptr(mg) if margins else None)
    if margins:
        return out, amb, int(ns), mg.T.reshape(2, H, W).copy()
    return out, amb, int(ns)


def trilinear(vol, points):
    vol, dt, nx, ny, nz = _vol_args(vol)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty(p.shape[0], dtype=np.float64)
    _load().or_trilinear(_ptr(vol), dt, nx, ny, nz, _ptr(p), p.shape[0], _ptr(out))
    return out


def ray(cam, dims, px, py):
    camv = _cam_array(cam)
    o = np.empty(3)
    d = np.empty(3)
    nx, ny, nz = dims
    _load().or_ray(_ptr(camv), cam.width, cam.height, nx, ny, nz, px, py, _ptr(o), _ptr(d))
    return o, d


def shadow(vol, tf, points, light_dir, step_vox=0.5, rate=4):
    """Shadow transmittance (shading 2) at voxel-space points towards the light."""
    vol, dt, nx, ny, nz = _vol_args(vol)
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    L = np.ascontiguousarray(light_dir, dtype=np.float64)
    out = np.empty(p.shape[0], dtype=np.float64)
    _load().or_shadow(_ptr(vol), dt, nx, ny, nz, _ptr(tf), tf.shape[0], _ptr(p), p.shape[0], _ptr(L),
                      float(step_vox), int(rate), _ptr(out))
    return out


def set_threads(n: int):
    """Number of OpenMP threads of the marcher."""
    _load().or_set_threads(int(n))
