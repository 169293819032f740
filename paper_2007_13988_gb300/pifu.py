"""Thin Python binding of libpifu (include/pifu.h): the same entry points,
argument marshalling only.  Every step of the path runs in the library's
CUDA kernels; PyTorch supplies device memory and streams.

Loading fails loudly when the library is missing or cannot be opened: there
is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

from . import build as _build

PIFU_OK = 0
PIFU_ERR_ARG = -1
PIFU_ERR_FORMAT = -2
PIFU_ERR_CUDA = -3
PIFU_ERR_OOM = -4
PIFU_ERR_NOT_CONVERGED = -5
PIFU_ERR_TIMEOUT = -6
PIFU_ERR_STATE = -7
PIFU_ERR_UNSUPPORTED = -8
PIFU_ERR_CAPACITY = -9

PIFU_F32 = 0
PIFU_BF16 = 1
PIFU_PREC_FP32 = 0
PIFU_PREC_BF16 = 1
PIFU_PREC_MIXED = 2
PIFU_PREC_FP8_MIXED = 3
PIFU_PREC_FP8 = 4
PIFU_SUBDIV_METHOD = 0
PIFU_SUBDIV_BINARIZED = 1
PIFU_SUBDIV_THRESHOLD = 2

# Every symbol include/pifu.h declares.
EXPORTS = ("pifu_create", "pifu_destroy", "pifu_query", "pifu_query_colour", "pifu_localize",
           "pifu_render", "pifu_sync_stats", "pifu_status_string", "pifu_last_error",
           "pifu_profile", "pifu_profile_read", "pifu_query_noalloc", "pifu_query_ex",
           "pifu_frame", "pifu_surrogate_init", "pifu_surrogate_samples", "pifu_surrogate_grad",
           "pifu_surrogate_train", "pifu_surrogate_params", "pifu_surrogate_query",
           "pifu_calibrate_fp8", "pifu_frames", "pifu_autotune", "pifu_surrogate_ohem_init",
           "pifu_surrogate_ohem_weights", "pifu_surrogate_ohem_sample",
           "pifu_surrogate_train_ohem", "pifu_set_tiles", "pifu_set_schedule", "pifu_stream",
           "pifu_set_recheck", "pifu_test_starve_wait", "pifu_frame_async", "pifu_frame_wait")

KERNEL_CLASSES = ("gather", "mlp_hidden", "mlp_last", "level", "select", "render", "mlp_f32",
                  "cbn_tc")


class pifu_fmap(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("C", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class pifu_levels(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("margin", ctypes.c_float), ("use_surrogate", ctypes.c_int32),
                ("surrogate_margin", ctypes.c_float), ("subdivision", ctypes.c_int32),
                ("threshold", ctypes.c_float)]


class pifu_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("background", ctypes.c_float * 3), ("precision", ctypes.c_int32),
                ("final_level", ctypes.c_int32)]


class pifu_volume(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("row_words", ctypes.c_int32),
                ("occ_bits_dev", ctypes.c_void_p), ("eval_bits_dev", ctypes.c_void_p),
                ("values_dev", ctypes.c_void_p), ("n_eval", ctypes.c_int64),
                ("evals_per_level", ctypes.c_int64 * 8),
                ("candidates_per_level", ctypes.c_int64 * 8),
                ("rechecked_per_level", ctypes.c_int64 * 8),
                ("fallback_per_level", ctypes.c_int64 * 8),
                ("conflict_rounds", ctypes.c_int32 * 8)]


class pifu_frame_time(ctypes.Structure):
    _fields_ = [("admit_ms", ctypes.c_float), ("done_ms", ctypes.c_float),
                ("slot", ctypes.c_int32), ("stream_rounds", ctypes.c_int32)]


class pifu_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class PifuError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        msg = f"{what}: {_lib().pifu_status_string(status).decode()} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_LIB = None


def library_path() -> str:
    return _build.LIB


def _lib():
    """Open libpifu.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libpifu not found at {path}")
    lib = ctypes.CDLL(path)
    P, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    lib.pifu_create.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(P)]
    lib.pifu_create.restype = I
    lib.pifu_destroy.argtypes = [P]
    lib.pifu_destroy.restype = None
    lib.pifu_query.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), P, I64, P, P]
    lib.pifu_query.restype = I
    lib.pifu_query_ex.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), P, I64, P, I, F,
                                  P]
    lib.pifu_query_ex.restype = I
    lib.pifu_query_colour.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(pifu_fmap),
                                      ctypes.POINTER(F), P, I64, P, P]
    lib.pifu_query_colour.restype = I
    lib.pifu_localize.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F),
                                  ctypes.POINTER(pifu_levels), P, ctypes.POINTER(pifu_volume)]
    lib.pifu_localize.restype = I
    lib.pifu_render.argtypes = [P, ctypes.POINTER(pifu_camera), ctypes.POINTER(pifu_fmap),
                                ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), P, P, P, P]
    lib.pifu_render.restype = I
    lib.pifu_frame.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(pifu_fmap),
                               ctypes.POINTER(F), ctypes.POINTER(pifu_levels),
                               ctypes.POINTER(pifu_camera), P, P, P, P, ctypes.POINTER(pifu_volume)]
    lib.pifu_frame.restype = I
    lib.pifu_frame_async.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(pifu_fmap),
                                     ctypes.POINTER(F), ctypes.POINTER(pifu_levels),
                                     ctypes.POINTER(pifu_camera), P, P, P, P]
    lib.pifu_frame_async.restype = I
    lib.pifu_frame_wait.argtypes = [P, P, ctypes.POINTER(pifu_volume)]
    lib.pifu_frame_wait.restype = I
    U64, D = ctypes.c_uint64, ctypes.c_double
    lib.pifu_frames.argtypes = [P, I, ctypes.POINTER(pifu_fmap), ctypes.POINTER(pifu_fmap),
                                ctypes.POINTER(F), ctypes.POINTER(pifu_levels),
                                ctypes.POINTER(pifu_camera), P, P, P, P, ctypes.POINTER(pifu_volume)]
    lib.pifu_frames.restype = I
    lib.pifu_stream.argtypes = [P, I, ctypes.POINTER(pifu_fmap), ctypes.POINTER(pifu_fmap),
                                ctypes.POINTER(F), I, ctypes.POINTER(pifu_levels),
                                ctypes.POINTER(pifu_camera), P, P, P, P, P,
                                ctypes.POINTER(pifu_volume), ctypes.POINTER(pifu_frame_time)]
    lib.pifu_stream.restype = I
    lib.pifu_autotune.argtypes = [P, I64, P, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double), I, ctypes.POINTER(I)]
    lib.pifu_autotune.restype = I
    lib.pifu_set_tiles.argtypes = [P, ctypes.POINTER(ctypes.c_int32), I]
    lib.pifu_set_tiles.restype = I
    lib.pifu_set_schedule.argtypes = [P, I]
    lib.pifu_set_schedule.restype = I
    lib.pifu_set_recheck.argtypes = [P, I]
    lib.pifu_set_recheck.restype = I
    lib.pifu_test_starve_wait.argtypes = [P, I]
    lib.pifu_test_starve_wait.restype = I
    lib.pifu_calibrate_fp8.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), I, P]
    lib.pifu_calibrate_fp8.restype = I
    lib.pifu_surrogate_init.argtypes = [P, I, I, U64]
    lib.pifu_surrogate_init.restype = I
    lib.pifu_surrogate_samples.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), P, I64,
                                           P, P, P]
    lib.pifu_surrogate_samples.restype = I
    lib.pifu_surrogate_query.argtypes = [P, ctypes.POINTER(pifu_fmap), ctypes.POINTER(F), P, I64,
                                         P, I, P]
    lib.pifu_surrogate_query.restype = I
    lib.pifu_surrogate_grad.argtypes = [P, P, P, I64, ctypes.POINTER(F), ctypes.POINTER(D), P]
    lib.pifu_surrogate_grad.restype = I
    lib.pifu_surrogate_train.argtypes = [P, P, P, I64, I, I, F, ctypes.POINTER(D), P]
    lib.pifu_surrogate_train.restype = I
    lib.pifu_surrogate_ohem_init.argtypes = [P, I64]
    lib.pifu_surrogate_ohem_init.restype = I
    lib.pifu_surrogate_ohem_weights.argtypes = [P, ctypes.POINTER(F), I64, I]
    lib.pifu_surrogate_ohem_weights.restype = I
    lib.pifu_surrogate_ohem_sample.argtypes = [P, U64, I, I, P, P]
    lib.pifu_surrogate_ohem_sample.restype = I
    lib.pifu_surrogate_train_ohem.argtypes = [P, P, P, I64, I, I, F, F, F, U64,
                                              ctypes.POINTER(D), P]
    lib.pifu_surrogate_train_ohem.restype = I
    lib.pifu_surrogate_params.argtypes = [P, ctypes.POINTER(F), I64, I]
    lib.pifu_surrogate_params.restype = I
    lib.pifu_sync_stats.argtypes = [P, ctypes.POINTER(pifu_volume)]
    lib.pifu_sync_stats.restype = I
    lib.pifu_status_string.argtypes = [I]
    lib.pifu_status_string.restype = ctypes.c_char_p
    lib.pifu_last_error.argtypes = [P]
    lib.pifu_last_error.restype = ctypes.c_char_p
    lib.pifu_profile.argtypes = [P, I]
    lib.pifu_profile.restype = I
    lib.pifu_profile_read.argtypes = [P, ctypes.POINTER(pifu_kernel_stats)]
    lib.pifu_profile_read.restype = I
    lib.pifu_query_noalloc.argtypes = [P, ctypes.c_size_t, P, ctypes.POINTER(pifu_fmap),
                                       ctypes.POINTER(F), P, I64, P, P]
    lib.pifu_query_noalloc.restype = I
    _LIB = lib
    return lib


def load():
    """The opened ctypes library."""
    return _lib()


# --------------------------------------------------------------------------
# Weight blob (format in include/pifu.h)
# --------------------------------------------------------------------------

def blob_from_nets(occ_net, col_net) -> bytes:
    """Serialise the occupancy and colour MLPs into the library's blob."""
    parts = [b"PIFU", struct.pack("<II", 1, 2)]
    f4 = lambda a: np.ascontiguousarray(a, dtype="<f4").tobytes()
    for kind, net in ((0, occ_net), (1, col_net)):
        if getattr(net, "kind", "mlp") == "cbn":
            # kind 2: the CBN + SoftZ occupancy network
            parts.append(struct.pack("<IIIIIf", 2, net.C, net.n_z, net.width, net.n_blocks,
                                     net.eps))
            parts += [f4(net.Wz), f4(net.bz)]
            for i in range(net.n_blocks):
                parts += [f4(net.Gg[i]), f4(net.gg[i]), f4(net.Gb[i]), f4(net.gb[i]),
                          f4(net.mu[i]), f4(net.var[i]), f4(net.W[i]), f4(net.b[i])]
            continue
        L = len(net.W)
        skip_mask = 0
        for l in net.skip:
            skip_mask |= 1 << l
        parts.append(struct.pack("<IIIf", kind, net.d_in, L, net.slope))
        parts.append(struct.pack(f"<{L}I", *[w.shape[0] for w in net.W]))
        parts.append(struct.pack("<I", skip_mask))
        for W, b in zip(net.W, net.b):
            parts.append(np.ascontiguousarray(W, dtype="<f4").tobytes())
            parts.append(np.ascontiguousarray(b, dtype="<f4").tobytes())
    return b"".join(parts)


# --------------------------------------------------------------------------
# Marshalling helpers
# --------------------------------------------------------------------------

def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def fmap(t):
    """pifu_fmap describing a contiguous [H][W][C] CUDA tensor (float32/bf16)."""
    import torch
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or t.dim() != 3:
        raise ValueError("feature map must be a contiguous [H][W][C] CUDA tensor")
    dt = {torch.float32: PIFU_F32, torch.bfloat16: PIFU_BF16}[t.dtype]
    return pifu_fmap(t.data_ptr(), t.shape[0], t.shape[1], t.shape[2], dt)


def _calib(c):
    a = np.ascontiguousarray(np.asarray(c, dtype=np.float32).reshape(12))
    return (ctypes.c_float * 12)(*a.tolist())


def _check(status, what, ctx=None):
    if status != PIFU_OK:
        detail = ""
        if ctx is not None and status in (PIFU_ERR_CUDA, PIFU_ERR_OOM):
            detail = _lib().pifu_last_error(ctx).decode()
        raise PifuError(status, what, detail)


# --------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def pifu_create(blob: bytes):
    lib = _lib()
    ctx = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib.pifu_create(buf, len(blob), ctypes.byref(ctx)), "pifu_create")
    return ctx


def pifu_destroy(ctx):
    _lib().pifu_destroy(ctx)


def pifu_query(ctx, occ_map, calib, pts, out, stream=None):
    """out[p] = O(pts[p]) (Eq. 1); pts [m][3] and out [m] float32 CUDA tensors."""
    m = pts.shape[0]
    fm = fmap(occ_map)
    st = _lib().pifu_query(ctx, ctypes.byref(fm), _calib(calib), _ptr(pts), m, _ptr(out),
                           _stream(stream))
    _check(st, "pifu_query", ctx)
    return out


def pifu_query_ex(ctx, occ_map, calib, pts, out, precision=PIFU_PREC_FP32, margin=0.02,
                  stream=None):
    """pifu_query with a choice of MLP arithmetic (PIFU_PREC_FP32 / _BF16 / _MIXED)."""
    m = pts.shape[0]
    fm = fmap(occ_map)
    st = _lib().pifu_query_ex(ctx, ctypes.byref(fm), _calib(calib), _ptr(pts), m, _ptr(out),
                              precision, margin, _stream(stream))
    _check(st, "pifu_query_ex", ctx)
    return out


def pifu_query_colour(ctx, occ_map, col_map, calib, pts, out, stream=None):
    """out[p] = T(pts[p]) in [0, 1]^3 (Eq. 2); out [m][3]."""
    m = pts.shape[0]
    fo = fmap(occ_map)
    fc = fmap(col_map)
    st = _lib().pifu_query_colour(ctx, ctypes.byref(fo), ctypes.byref(fc) if fc else None,
                                  _calib(calib), _ptr(pts), m, _ptr(out), _stream(stream))
    _check(st, "pifu_query_colour", ctx)
    return out


def pifu_localize(ctx, occ_map, calib, n0, num_levels, precision=PIFU_PREC_FP32,
                  max_rounds=0, margin=0.02, use_surrogate=False, surrogate_margin=0.1,
                  stream=None, subdivision=PIFU_SUBDIV_METHOD, threshold=0.0) -> pifu_volume:
    """subdivision: PIFU_SUBDIV_METHOD (Sec. 3.2), or one of the octree
    baselines of Fig. 3 (BINARIZED; THRESHOLD with `threshold`)."""
    fm = fmap(occ_map)
    lv = pifu_levels(n0, num_levels, precision, max_rounds, margin, 1 if use_surrogate else 0,
                     surrogate_margin, subdivision, threshold)
    vol = pifu_volume()
    st = _lib().pifu_localize(ctx, ctypes.byref(fm), _calib(calib), ctypes.byref(lv),
                              _stream(stream), ctypes.byref(vol))
    _check(st, "pifu_localize", ctx)
    return vol


def pifu_render(ctx, width, height, occ_map, col_map, calib, depth=None, rgb=None, mask=None,
                background=(0.0, 0.0, 0.0), precision=PIFU_PREC_FP32, stream=None,
                final_level=0):
    cam = pifu_camera(width, height, (ctypes.c_float * 3)(*background), precision, final_level)
    fo = fmap(occ_map)
    fc = fmap(col_map)
    st = _lib().pifu_render(ctx, ctypes.byref(cam), ctypes.byref(fo) if fo else None,
                            ctypes.byref(fc) if fc else None, _calib(calib), _stream(stream),
                            _ptr(depth), _ptr(rgb), _ptr(mask))
    _check(st, "pifu_render", ctx)


def pifu_frame(ctx, occ_map, col_map, calib, n0, num_levels, width, height, depth=None, rgb=None,
               mask=None, precision=PIFU_PREC_MIXED, margin=0.02, max_rounds=0,
               background=(0.0, 0.0, 0.0), stream=None, use_surrogate=False,
               surrogate_margin=0.0, final_level=0) -> pifu_volume:
    """Localization + render of one frame as a (cached) CUDA graph."""
    fo = fmap(occ_map)
    fc = fmap(col_map)
    lv = pifu_levels(n0, num_levels, precision, max_rounds, margin, int(bool(use_surrogate)),
                     surrogate_margin)
    cam = pifu_camera(width, height, (ctypes.c_float * 3)(*background), PIFU_PREC_BF16,
                      final_level)
    vol = pifu_volume()
    st = _lib().pifu_frame(ctx, ctypes.byref(fo), ctypes.byref(fc) if fc else None, _calib(calib),
                           ctypes.byref(lv), ctypes.byref(cam), _stream(stream), _ptr(depth),
                           _ptr(rgb), _ptr(mask), ctypes.byref(vol))
    _check(st, "pifu_frame", ctx)
    return vol


def pifu_frame_async(ctx, occ_map, col_map, calib, n0, num_levels, width, height, depth=None,
                     rgb=None, mask=None, precision=PIFU_PREC_MIXED, margin=0.02, max_rounds=0,
                     background=(0.0, 0.0, 0.0), stream=None, use_surrogate=False,
                     surrogate_margin=0.0, final_level=0) -> None:
    """pifu_frame enqueued on `stream` without waiting for it; errors and the
    volume come from pifu_frame_wait."""
    fo = fmap(occ_map)
    fc = fmap(col_map)
    lv = pifu_levels(n0, num_levels, precision, max_rounds, margin, int(bool(use_surrogate)),
                     surrogate_margin)
    cam = pifu_camera(width, height, (ctypes.c_float * 3)(*background), PIFU_PREC_BF16,
                      final_level)
    st = _lib().pifu_frame_async(ctx, ctypes.byref(fo), ctypes.byref(fc) if fc else None,
                                 _calib(calib), ctypes.byref(lv), ctypes.byref(cam),
                                 _stream(stream), _ptr(depth), _ptr(rgb), _ptr(mask))
    _check(st, "pifu_frame_async", ctx)


def pifu_frame_wait(ctx, stream=None) -> pifu_volume:
    """Waits for the frames pifu_frame_async enqueued; raises the error any of
    them latched; returns the last frame's volume."""
    vol = pifu_volume()
    st = _lib().pifu_frame_wait(ctx, _stream(stream), ctypes.byref(vol))
    _check(st, "pifu_frame_wait", ctx)
    return vol


def pifu_frames(ctx, occ_maps, col_maps, calibs, n0, num_levels, width, height, depth=None,
                rgb=None, mask=None, precision=PIFU_PREC_MIXED, margin=0.02, max_rounds=0,
                background=(0.0, 0.0, 0.0), stream=None, use_surrogate=False,
                surrogate_margin=0.0):
    """B frames in lockstep as one (cached) CUDA graph; returns B volumes.
    occ_maps / col_maps: sequences of device tensors (col_maps may be None),
    calibs: B calibrations; depth/rgb/mask: [B][H][W](x3) device tensors."""
    B = len(occ_maps)
    fo = (pifu_fmap * B)(*[fmap(m) for m in occ_maps])
    fc = (pifu_fmap * B)(*[fmap(m) for m in col_maps]) if col_maps is not None else None
    cal = np.ascontiguousarray(np.asarray(calibs, np.float32).reshape(B, 12))
    cal_p = cal.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    lv = pifu_levels(n0, num_levels, precision, max_rounds, margin, int(bool(use_surrogate)),
                     surrogate_margin)
    cam = pifu_camera(width, height, (ctypes.c_float * 3)(*background), PIFU_PREC_BF16)
    vols = (pifu_volume * B)()
    st = _lib().pifu_frames(ctx, B, fo, fc, cal_p, ctypes.byref(lv), ctypes.byref(cam),
                            _stream(stream), _ptr(depth), _ptr(rgb), _ptr(mask), vols)
    _check(st, "pifu_frames", ctx)
    return list(vols)


def pifu_stream(ctx, occ_maps, col_maps, calibs, slots, n0, num_levels, width, height, depth=None,
                rgb=None, mask=None, occ_bits=None, precision=PIFU_PREC_MIXED, margin=0.02,
                max_rounds=0, background=(0.0, 0.0, 0.0), stream=None, use_surrogate=False,
                surrogate_margin=0.0):
    """F frames through `slots` frame slots fed by a device work queue, as one
    (cached) CUDA graph; returns (F volumes, F pifu_frame_time).
    occ_maps / col_maps: sequences of device tensors (col_maps may be None),
    calibs: F calibrations; depth/rgb/mask: [F][H][W](x3) device tensors;
    occ_bits: optional [F][words] int32 device tensor for each frame's
    binarized finest level."""
    F = len(occ_maps)
    fo = (pifu_fmap * F)(*[fmap(m) for m in occ_maps])
    fc = (pifu_fmap * F)(*[fmap(m) for m in col_maps]) if col_maps is not None else None
    cal = np.ascontiguousarray(np.asarray(calibs, np.float32).reshape(F, 12))
    cal_p = cal.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    lv = pifu_levels(n0, num_levels, precision, max_rounds, margin, int(bool(use_surrogate)),
                     surrogate_margin)
    cam = pifu_camera(width, height, (ctypes.c_float * 3)(*background), PIFU_PREC_BF16)
    vols = (pifu_volume * F)()
    times = (pifu_frame_time * F)()
    st = _lib().pifu_stream(ctx, F, fo, fc, cal_p, int(slots), ctypes.byref(lv),
                            ctypes.byref(cam), _stream(stream), _ptr(depth), _ptr(rgb), _ptr(mask),
                            _ptr(occ_bits), vols, times)
    _check(st, "pifu_stream", ctx)
    return list(vols), list(times)


# Tile code of the CTA-pair form (two CTAs on a 256 x 256 tile).
PIFU_TILE_PAIR = 512


def pifu_autotune(ctx, rows, stream=None, n_max=32):
    """Tile codes chosen per tensor-core layer: list of (code, ms per launch);
    code = BN of a single-CTA 128 x BN tile, or PIFU_TILE_PAIR."""
    bn = (ctypes.c_int32 * n_max)()
    ms = (ctypes.c_double * n_max)()
    n = ctypes.c_int(0)
    _check(_lib().pifu_autotune(ctx, int(rows), _stream(stream), bn, ms, n_max, ctypes.byref(n)),
           "pifu_autotune", ctx)
    return [(int(bn[i]), float(ms[i])) for i in range(min(n.value, n_max))]


PIFU_SCHED_PER_LAYER = 0
PIFU_SCHED_CHAINED = 1


def pifu_set_schedule(ctx, schedule):
    """Per-layer launches (default) or chained (all hidden layers in one launch)."""
    _check(_lib().pifu_set_schedule(ctx, int(schedule)), "pifu_set_schedule", ctx)


PIFU_RECHECK_TENSOR = 0
PIFU_RECHECK_SIMT = 1
PIFU_RECHECK_TENSOR_ALL = 2


def pifu_set_recheck(ctx, form):
    """Arithmetic of the MIXED forms' FP32 passes: split TF32 on the tensor
    cores above 192 points (default), the FP32 SIMT network, or split TF32
    for every pass."""
    _check(_lib().pifu_set_recheck(ctx, int(form)), "pifu_set_recheck", ctx)


def pifu_test_starve_wait(ctx, starve):
    """Test hook: the split-TF32 kernels' cross-CTA wait runs out (1) or not (0)."""
    _check(_lib().pifu_test_starve_wait(ctx, int(starve)), "pifu_test_starve_wait", ctx)


def pifu_set_tiles(ctx, codes):
    """Set every tuned layer's tile code (pifu_autotune's order and codes)."""
    arr = (ctypes.c_int32 * max(len(codes), 1))(*[int(c) for c in codes])
    _check(_lib().pifu_set_tiles(ctx, arr, len(codes)), "pifu_set_tiles", ctx)


def pifu_surrogate_ohem_init(ctx, m):
    _check(_lib().pifu_surrogate_ohem_init(ctx, int(m)), "pifu_surrogate_ohem_init", ctx)


def pifu_surrogate_ohem_weights(ctx, n, values=None):
    """Read the n OHEM weights (values None) or upload them."""
    buf = np.ascontiguousarray(np.zeros(n, np.float32) if values is None else
                               np.asarray(values, np.float32))
    ptr = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    _check(_lib().pifu_surrogate_ohem_weights(ctx, ptr, n, 0 if values is None else 1),
           "pifu_surrogate_ohem_weights", ctx)
    return buf


def pifu_surrogate_ohem_sample(ctx, seed, step, idx, stream=None):
    """Draw idx.shape[0] indices (int32 CUDA tensor) by the current weights."""
    _check(_lib().pifu_surrogate_ohem_sample(ctx, seed, step, idx.shape[0], _ptr(idx),
                                             _stream(stream)), "pifu_surrogate_ohem_sample", ctx)


def pifu_surrogate_train_ohem(ctx, x, y, batch=4096, steps=100, lr=1e-3, alpha=0.7, beta=0.0,
                              seed=0, stream=None):
    loss = (ctypes.c_double * 2)()
    _check(_lib().pifu_surrogate_train_ohem(ctx, _ptr(x), _ptr(y), x.shape[0], batch, steps, lr,
                                            alpha, beta, seed, loss, _stream(stream)),
           "pifu_surrogate_train_ohem", ctx)
    return float(loss[0]), float(loss[1])


def pifu_calibrate_fp8(ctx, occ_map, calib, n0=32, stream=None):
    """Scales and E4M3 weights of f_O's FP8 form from the dense n0^3 grid."""
    fm = fmap(occ_map)
    _check(_lib().pifu_calibrate_fp8(ctx, ctypes.byref(fm), _calib(calib), n0, _stream(stream)),
           "pifu_calibrate_fp8", ctx)


def pifu_surrogate_init(ctx, h1=128, h2=64, seed=0):
    _check(_lib().pifu_surrogate_init(ctx, h1, h2, seed), "pifu_surrogate_init", ctx)


def pifu_surrogate_samples(ctx, occ_map, calib, pts, x_out, o_out, stream=None):
    """Distillation tuples: x_out [m][row width of f_O] gathered rows, o_out [m]
    f_O's FP32 occupancy at the points."""
    fm = fmap(occ_map)
    st = _lib().pifu_surrogate_samples(ctx, ctypes.byref(fm), _calib(calib), _ptr(pts),
                                       pts.shape[0], _ptr(x_out), _ptr(o_out), _stream(stream))
    _check(st, "pifu_surrogate_samples", ctx)


def pifu_surrogate_query(ctx, occ_map, calib, pts, out, precision=PIFU_PREC_FP32, stream=None):
    fm = fmap(occ_map)
    st = _lib().pifu_surrogate_query(ctx, ctypes.byref(fm), _calib(calib), _ptr(pts),
                                     pts.shape[0], _ptr(out), precision, _stream(stream))
    _check(st, "pifu_surrogate_query", ctx)
    return out


def surrogate_param_count(h1, h2, d_in):
    return h1 * d_in + h1 + h2 * h1 + h2 + h2 + 1


def pifu_surrogate_grad(ctx, x, y, n_params, stream=None):
    """(loss, gradient in the unpadded parameter layout) of one batch."""
    g = (ctypes.c_float * n_params)()
    loss = ctypes.c_double()
    st = _lib().pifu_surrogate_grad(ctx, _ptr(x), _ptr(y), x.shape[0], g, ctypes.byref(loss),
                                    _stream(stream))
    _check(st, "pifu_surrogate_grad", ctx)
    return loss.value, np.frombuffer(g, dtype=np.float32).copy()


def pifu_surrogate_train(ctx, x, y, batch=4096, steps=1000, lr=1e-3, stream=None):
    """Adam steps over consecutive batches; returns (first, last) batch loss."""
    loss = (ctypes.c_double * 2)()
    st = _lib().pifu_surrogate_train(ctx, _ptr(x), _ptr(y), x.shape[0], batch, steps, lr, loss,
                                     _stream(stream))
    _check(st, "pifu_surrogate_train", ctx)
    return loss[0], loss[1]


def pifu_surrogate_params(ctx, n_params, values=None):
    """Get (values None) or set the surrogate's parameters (unpadded layout)."""
    buf = (ctypes.c_float * n_params)()
    if values is not None:
        buf[:] = np.asarray(values, np.float32).tolist()
    st = _lib().pifu_surrogate_params(ctx, buf, n_params, 0 if values is None else 1)
    _check(st, "pifu_surrogate_params", ctx)
    return None if values is not None else np.frombuffer(buf, dtype=np.float32).copy()


def pifu_sync_stats(ctx) -> pifu_volume:
    vol = pifu_volume()
    _check(_lib().pifu_sync_stats(ctx, ctypes.byref(vol)), "pifu_sync_stats")
    return vol


def pifu_query_noalloc(blob: bytes, blob_dev, occ_map, calib, pts, out, stream=None):
    """pifu_query without a context and without any allocation by the
    library: blob is the host weight blob, blob_dev a device copy of its
    bytes owned by the caller (e.g. a uint8 CUDA tensor)."""
    buf = ctypes.create_string_buffer(blob, len(blob))
    fm = fmap(occ_map)
    st = _lib().pifu_query_noalloc(buf, len(blob), _ptr(blob_dev), ctypes.byref(fm),
                                   _calib(calib), _ptr(pts), pts.shape[0], _ptr(out),
                                   _stream(stream))
    _check(st, "pifu_query_noalloc")
    return out


def pifu_profile(ctx, enable: bool):
    _check(_lib().pifu_profile(ctx, 1 if enable else 0), "pifu_profile", ctx)


def pifu_profile_read(ctx) -> dict:
    """{class name: {launches, ms, flops, bytes}} since the last pifu_profile."""
    arr = (pifu_kernel_stats * len(KERNEL_CLASSES))()
    _check(_lib().pifu_profile_read(ctx, arr), "pifu_profile_read", ctx)
    return {n: {"launches": int(a.launches), "ms": float(a.ms), "flops": float(a.flops),
                "bytes": float(a.bytes)} for n, a in zip(KERNEL_CLASSES, arr)}


def pifu_status_string(status: int) -> str:
    return _lib().pifu_status_string(status).decode()


# --------------------------------------------------------------------------
# Views of a localized volume (device tensors over context memory)
# --------------------------------------------------------------------------

def volume_tensors(vol: pifu_volume):
    """(occ_bits, eval_bits, values) as CUDA tensors aliasing context memory
    (valid until the next pifu_localize on the context)."""
    import torch
    n1 = vol.n + 1
    words = n1 * n1 * vol.row_words

    def view(ptr, count, dtype):
        # wrap raw device memory through the CUDA array interface
        class _A:
            __cuda_array_interface__ = {"shape": (count,), "typestr": dtype, "data": (ptr, False),
                                        "version": 3}
        return torch.as_tensor(_A(), device="cuda")

    occ = view(vol.occ_bits_dev, words, "<i4")
    ev = view(vol.eval_bits_dev, words, "<i4")
    val = view(vol.values_dev, n1 ** 3, "<f4")
    return occ, ev, val


def unpack_bits(words, n, row_words):
    """Host bool array [n+1]^3 ([z][y][x]) from a bitset in the row layout."""
    w = np.asarray(words, dtype=np.int32).view(np.uint32).reshape(n + 1, n + 1, row_words)
    bits = np.unpackbits(w.view(np.uint8).reshape(n + 1, n + 1, row_words * 4), axis=2,
                         bitorder="little")
    return bits[:, :, :n + 1].astype(bool)
