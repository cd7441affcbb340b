"""Plain CPU oracle of the per-tile heightmap build (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg
may import this package.  The product path (paper_2509_20198_b300) never does.

* oracle.c (built to liboracle.so with gcc, no fused multiply-add): serial integer
  binning, sample extraction, FP64 brute-force Gaussian fill, FP64 tile update.
* unet.py: FP64 numpy U-Net forward/backward, loss, AdamW, learned-input raster.
* interp.py: the interpolated heightmaps of Alg. 1 (nearest-neighbour and
  Delaunay-linear maps of a padded patch), exact integer predicates in Python.
* render.py: the point and heightmap rasterizers into a 64-bit depth|colour
  framebuffer and the resolve (numpy float32, one rounding per operation).
* cnn.py: FP64 forward/backward of the paper's own network variant (per-input
  encoders, fully connected merge, two decoders, skip concat, final CNN, crop).

Parity status of each function (what pins it) is listed in the tests under
tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

I64 = ctypes.c_int64
DBL = ctypes.c_double
P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c to liboracle.so (gcc, -O1, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", _SO, src, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.or_bin_points.restype = I64
        L.or_bin_points.argtypes = [P] * 6 + [I64] * 7 + [P] * 7
        L.or_extract_sample_indices.restype = I64
        L.or_extract_sample_indices.argtypes = [P, I64, I64, P, P]
        L.or_fill_sparse.restype = ctypes.c_int
        L.or_fill_sparse.argtypes = ([P] * 6 + [I64] + [I64] * 5 + [DBL, DBL] + [I64, I64, DBL]
                                     + [P, I64] + [P] * 5)
        L.or_update_tile.restype = None
        L.or_update_tile.argtypes = [P] * 5 + [I64, P, I64, DBL, DBL, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def bin_points(pts, region, cells):
    """Serial integer binning of a region at `cells` x `cells` per tile.

    pts: dict of x, y, z (int32), r, g, b (uint16).  Returns dict of the seven
    [T, cells, cells] accumulator arrays plus 'dropped'."""
    T = region.tiles_x * region.tiles_y
    shape = (T, cells, cells)
    out = {"count": np.empty(shape, np.uint32), "zsum": np.empty(shape, np.int64),
           "zmin": np.empty(shape, np.int32), "zmax": np.empty(shape, np.int32),
           "rsum": np.empty(shape, np.uint64), "gsum": np.empty(shape, np.uint64),
           "bsum": np.empty(shape, np.uint64)}
    a = [_c(pts[k], np.int32) for k in "xyz"] + [_c(pts[k], np.uint16) for k in "rgb"]
    n = len(a[0])
    out["dropped"] = lib().or_bin_points(*[_p(v) for v in a], n, region.x0_cm, region.y0_cm,
                                         region.tile_cm, region.tiles_x, region.tiles_y, cells,
                                         *[_p(out[k]) for k in ("count", "zsum", "zmin", "zmax",
                                                                "rsum", "gsum", "bsum")])
    return out


def extract_sample_indices(tile_offsets, chunk=50000):
    offs = _c(tile_offsets, np.int64)
    T = len(offs) - 1
    cap = int(sum((offs[t + 1] - offs[t] + chunk - 1) // chunk for t in range(T)))
    idx = np.empty(max(cap, 1), np.int64)
    soffs = np.empty(T + 1, np.int64)
    n = lib().or_extract_sample_indices(_p(offs), T, chunk, _p(idx), _p(soffs))
    return idx[:n], soffs


def fill_sparse(samples, region, tile_ids=None, res=64, radius_cm=12000, sigma_cm=4000.0):
    """FP64 Gaussian fill of the requested tiles.  Returns dict with height (m),
    rgbf (8-bit scale, unrounded), rgb8, nearest_d2 and nearest_idx."""
    T = region.tiles_x * region.tiles_y
    tid = _c(np.arange(T) if tile_ids is None else tile_ids, np.int64)
    n = len(tid)
    a = [_c(samples[k], np.int32) for k in "xyz"] + [_c(samples[k], np.uint16) for k in "rgb"]
    out = {"height": np.empty((n, res, res)), "rgbf": np.empty((n, res, res, 3)),
           "rgb8": np.empty((n, res, res, 3), np.uint8),
           "nearest_d2": np.empty((n, res, res), np.int64),
           "nearest_idx": np.empty((n, res, res), np.int64)}
    rc = lib().or_fill_sparse(*[_p(v) for v in a], len(a[0]), region.x0_cm, region.y0_cm,
                              region.tile_cm, region.tiles_x, region.tiles_y,
                              region.z_scale, region.z_offset, res, radius_cm, float(sigma_cm),
                              _p(tid), n, _p(out["height"]), _p(out["rgbf"]), _p(out["rgb8"]),
                              _p(out["nearest_d2"]), _p(out["nearest_idx"]))
    if rc != 0:
        raise MemoryError("oracle fill: allocation failed")
    return out


def update_tile(bins, region, tile_ids, height, rgb):
    """FP64 tile update in place on copies of height (float32) and rgb (uint8)."""
    res = bins["count"].shape[-1]
    tid = _c(tile_ids, np.int64)
    h = np.array(height, dtype=np.float32, copy=True, order="C")
    c = np.array(rgb, dtype=np.uint8, copy=True, order="C")
    lib().or_update_tile(_p(_c(bins["count"], np.uint32)), _p(_c(bins["zsum"], np.int64)),
                         _p(_c(bins["rsum"], np.uint64)), _p(_c(bins["gsum"], np.uint64)),
                         _p(_c(bins["bsum"], np.uint64)), res, _p(tid), len(tid),
                         region.z_scale, region.z_offset, _p(h), _p(c))
    return h, c
