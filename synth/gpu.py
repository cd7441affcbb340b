"""GPU twin of the seeded generator (libsynth.so): same integer definition as the
numpy generator in synth/__init__.py, used to build the large workloads on the device.
Input generation only; no arithmetic of the heightmap method."""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_SO = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
_lib = None
I64, U64, VP = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError("synth/libsynth.so not built (paper_2509_20198_b300.build.build_synth)")
        L = ctypes.CDLL(_SO)
        L.synth_region_points.argtypes = [U64, I64, I64, I64, I64, VP, I64, I64] + [VP] * 7
        L.synth_region_points.restype = ctypes.c_int
        L.synth_region_samples.argtypes = [U64, I64, I64, I64, I64, VP, VP, I64, I64, I64] + [VP] * 7
        L.synth_region_samples.restype = ctypes.c_int
        _lib = L
    return _lib


def _alloc(n, device):
    return {"x": torch.empty(n, dtype=torch.int32, device=device),
            "y": torch.empty(n, dtype=torch.int32, device=device),
            "z": torch.empty(n, dtype=torch.int32, device=device),
            "r": torch.empty(n, dtype=torch.uint16, device=device),
            "g": torch.empty(n, dtype=torch.uint16, device=device),
            "b": torch.empty(n, dtype=torch.uint16, device=device)}


def region_points(seed, region, counts, device="cuda", stream=None):
    counts = np.asarray(counts, dtype=np.int64)
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    total = int(offs[-1])
    out = _alloc(max(total, 1), device)
    out = {k: v[:total] for k, v in out.items()}
    d_offs = torch.from_numpy(offs).to(device)
    s = torch.cuda.current_stream() if stream is None else stream
    rc = lib().synth_region_points(seed, region.x0_cm, region.y0_cm, region.tile_cm, region.tiles_x,
                                   d_offs.data_ptr(), len(counts), total,
                                   *[out[k].data_ptr() for k in "xyzrgb"], s.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_region_points failed ({rc})")
    out["tile_offsets"] = d_offs
    return out


def region_samples(seed, region, counts, chunk=50000, device="cuda", stream=None):
    counts = np.asarray(counts, dtype=np.int64)
    ns = (counts + chunk - 1) // chunk
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(ns)
    total = int(offs[-1])
    out = _alloc(max(total, 1), device)
    out = {k: v[:total] for k, v in out.items()}
    d_counts = torch.from_numpy(counts).to(device)
    d_offs = torch.from_numpy(offs).to(device)
    s = torch.cuda.current_stream() if stream is None else stream
    rc = lib().synth_region_samples(seed, region.x0_cm, region.y0_cm, region.tile_cm, region.tiles_x,
                                    d_counts.data_ptr(), d_offs.data_ptr(), len(counts), chunk, total,
                                    *[out[k].data_ptr() for k in "xyzrgb"], s.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_region_samples failed ({rc})")
    out["tile_offsets"] = d_offs
    return out
