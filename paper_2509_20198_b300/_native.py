"""ctypes view of liblidarscout.so (the C ABI declared in include/lidarscout.h).

Argument marshalling only: every step of the heightmap build runs in the CUDA
library.  Loading fails loudly when the library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblidarscout.so")

I32, I64, U64, DBL, FLT = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_float
VP = ctypes.c_void_p


class LsPoints(ctypes.Structure):
    _fields_ = [("x", VP), ("y", VP), ("z", VP), ("r", VP), ("g", VP), ("b", VP),
                ("n", I64), ("tile_offsets", VP)]


class LsRegion(ctypes.Structure):
    _fields_ = [("x0_cm", I64), ("y0_cm", I64), ("tile_cm", I32), ("tiles_x", I32),
                ("tiles_y", I32), ("z_scale", DBL), ("z_offset", DBL)]


class LsBins(ctypes.Structure):
    _fields_ = [("cells", I32), ("count", VP), ("zsum", VP), ("zmin", VP), ("zmax", VP),
                ("rsum", VP), ("gsum", VP), ("bsum", VP)]


class LsFillParams(ctypes.Structure):
    _fields_ = [("res", I32), ("radius_cm", I32), ("sigma_cm", FLT)]


class LsInterpParams(ctypes.Structure):
    _fields_ = [("res", I32), ("pad_cm", I32)]


class LsInterpOutputs(ctypes.Structure):
    _fields_ = [("nn_height", VP), ("nn_rgb", VP), ("lin_height", VP), ("lin_rgb", VP), ("inside", VP),
                ("triangles", VP), ("tri_count", VP), ("tri_cap", I32)]


class LsCamera(ctypes.Structure):
    _fields_ = [("origin_cm", I64 * 3), ("view_proj", FLT * 16), ("width", I32), ("height", I32)]


class LsConvShape(ctypes.Structure):
    _fields_ = [("n", I32), ("h", I32), ("w", I32), ("cin", I32), ("cout", I32)]


class LsBinShape(ctypes.Structure):
    _fields_ = [("spans_per_cta", I32), ("prefetch_batches", I32)]


class LsFillShape(ctypes.Structure):
    _fields_ = [("split", I32), ("ctas_per_sm", I32)]


class LsSampleBuffers(ctypes.Structure):
    _fields_ = [("x", VP), ("y", VP), ("z", VP), ("r", VP), ("g", VP), ("b", VP)]


P = ctypes.POINTER
SIGNATURES = {
    "ls_bin_points": ([P(LsPoints), P(LsRegion), P(LsBins), I32, VP, VP], I32),
    "ls_bin_points_fixed_scratch": ([P(LsPoints), P(LsRegion), P(LsBins), I32, VP, VP], I32),
    "ls_bin_points_accumulate": ([P(LsPoints), P(LsRegion), P(LsBins), I32, VP, VP], I32),
    "ls_bin_stats": ([VP, I32], I32),
    "ls_bin_shape_get": ([P(LsPoints), P(LsBins), I32, P(LsBinShape)], I32),
    "ls_bin_shape_set": ([P(LsPoints), P(LsBins), I32, P(LsBinShape)], I32),
    "ls_fill_shape_get": ([P(LsPoints), P(LsFillParams), I64, P(LsFillShape)], I32),
    "ls_fill_shape_set": ([P(LsPoints), P(LsFillParams), I64, P(LsFillShape)], I32),
    "ls_tune_clear": ([], I32),
    "ls_tune_bin_points": ([P(LsPoints), P(LsRegion), P(LsBins), I32, VP, I32, VP, P(LsBinShape), P(FLT)], I32),
    "ls_tune_fill_sparse": ([P(LsPoints), P(LsRegion), P(LsFillParams), VP, I64, VP, VP, I32, VP, P(LsFillShape),
                             P(FLT)], I32),
    "ls_extract_samples": ([P(LsPoints), I64, I32, VP, P(LsSampleBuffers), I64, VP], I32),
    "ls_fill_sparse": ([P(LsPoints), P(LsRegion), P(LsFillParams), VP, I64, VP, VP, VP], I32),
    "ls_update_tile": ([P(LsBins), P(LsRegion), VP, I64, VP, VP, VP], I32),
    "ls_fill_interp": ([P(LsPoints), P(LsRegion), P(LsInterpParams), VP, I64, P(LsInterpOutputs), VP], I32),
    "ls_cnn_create": ([I32, I32, I32, P(VP)], I32),
    "ls_cnn_destroy": ([VP], None),
    "ls_cnn_param_count": ([VP], I64),
    "ls_cnn_layer_count": ([VP], I32),
    "ls_cnn_layer_info": ([VP, I32, P(I32), P(I32), P(I32), P(I64), P(I64)], I32),
    "ls_cnn_load": ([VP, VP, VP], I32),
    "ls_cnn_forward": ([VP, VP, VP, I32, VP, VP], I32),
    "ls_cnn_backward": ([VP, VP, VP, I32, VP, VP], I32),
    "ls_cnn_inputs": ([VP, VP, VP, VP, I64, I32, FLT, VP, VP, VP], I32),
    "ls_render_clear": ([VP, I32, I32, VP], I32),
    "ls_render_points": ([P(LsPoints), P(LsCamera), VP, VP], I32),
    "ls_render_heightmaps": ([VP, VP, VP, I64, I32, P(LsRegion), P(LsCamera), VP, VP], I32),
    "ls_render_resolve": ([VP, I32, I32, ctypes.c_uint32, VP, VP], I32),
    "ls_conv3x3_packed_elems": ([I32, I32], I64),
    "ls_conv3x3_pack": ([VP, I32, I32, I32, VP, VP], I32),
    "ls_conv3x3_forward": ([VP, VP, VP, VP, I32, P(LsConvShape), VP, VP], I32),
    "ls_conv3x3_wgrad": ([VP, VP, P(LsConvShape), VP, VP, VP], I32),
    "ls_model_create": ([I32, VP, I32, I32, P(VP)], I32),
    "ls_model_create_opts": ([I32, VP, I32, I32, I32, P(VP)], I32),
    "ls_model_device_bytes": ([VP], ctypes.c_size_t),
    "ls_model_destroy": ([VP], None),
    "ls_model_param_count": ([VP], I64),
    "ls_model_layer_count": ([VP], I32),
    "ls_model_layer_info": ([VP, I32, P(I32), P(I32), P(I32), P(I64), P(I64)], I32),
    "ls_model_load": ([VP, VP, VP], I32),
    "ls_filler_forward": ([VP, VP, VP, I32, VP, VP], I32),
    "ls_filler_backward": ([VP, VP, VP, I32, VP, VP], I32),
    "ls_filler_loss": ([VP, VP, VP, VP, I64, FLT, I32, VP, VP, VP, VP], I32),
    "ls_adamw_step": ([VP, VP, VP, VP, I64, FLT, FLT, FLT, FLT, FLT, I32, VP], I32),
    "ls_learned_inputs": ([P(LsPoints), P(LsRegion), P(LsFillParams), VP, I64, VP, VP, VP, VP, VP, VP, VP], I32),
    "ls_learned_targets": ([P(LsBins), P(LsRegion), VP, I64, VP, VP, VP, VP], I32),
    "ls_learned_finish": ([VP, VP, VP, I64, I32, P(LsRegion), FLT, VP, VP, VP, VP, VP, VP, VP], I32),
    "ls_fill_learned_scratch_bytes": ([VP], ctypes.c_size_t),
    "ls_fill_learned": ([VP, VP, P(LsPoints), P(LsRegion), P(LsFillParams), VP, I64, FLT, VP, VP, VP, VP, VP,
                         ctypes.c_size_t, VP], I32),
    "ls_status_string": ([I32], ctypes.c_char_p),
    "ls_last_error": ([], I32),
    "ls_set_spin_limit": ([I32], I32),
    "ls_probe_wait": ([VP, VP], I32),
    "ls_release_workspace": ([], I32),
    "ls_version": ([], I32),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblidarscout.so not found at {LIB_PATH}: run "
                               "`python -m paper_2509_20198_b300.build` (nvcc, sm_103a) first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class LsError(RuntimeError):
    def __init__(self, fn, status):
        msg = lib().ls_status_string(status).decode()
        super().__init__(f"{fn} failed: {msg} ({status})")
        self.status = status


def check(fn, status):
    if status != 0:
        raise LsError(fn, status)
