"""B300-native (sm_103a) per-tile heightmap build of LidarScout (HPG 2025).

Python binding of liblidarscout.so: the functions below only marshal torch CUDA
tensors into the C ABI of include/lidarscout.h; the work runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.

Points are dicts of CUDA tensors x, y, z (int32 centimetres) and r, g, b (uint16
stored as int16 or uint16 tensors), optionally with tile_offsets (int64, CSR by
tile).  A region is any object with x0_cm, y0_cm, tile_cm, tiles_x, tiles_y,
z_scale and z_offset attributes.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N

__all__ = ["bin_points", "extract_samples", "extract_samples_into", "fill_sparse", "update_tile", "last_error",
           "release_workspace", "empty_bins", "BIN_KEYS"]

BIN_KEYS = ("count", "zsum", "zmin", "zmax", "rsum", "gsum", "bsum")
_BIN_DTYPES = {"count": torch.int32, "zsum": torch.int64, "zmin": torch.int32, "zmax": torch.int32,
               "rsum": torch.int64, "gsum": torch.int64, "bsum": torch.int64}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return t


def _region(region):
    return N.LsRegion(int(region.x0_cm), int(region.y0_cm), int(region.tile_cm), int(region.tiles_x),
                      int(region.tiles_y), float(region.z_scale), float(region.z_offset))


def _points(p, need_offsets=False):
    for k in ("x", "y", "z"):
        _dev(p[k], k)
        assert p[k].dtype == torch.int32, f"{k} must be int32"
    for k in ("r", "g", "b"):
        _dev(p[k], k)
        assert p[k].element_size() == 2, f"{k} must be a 16-bit tensor"
    off = p.get("tile_offsets")
    if need_offsets and off is None:
        raise ValueError("tile_offsets (int64 CSR by tile) is required")
    if off is not None:
        _dev(off, "tile_offsets")
        assert off.dtype == torch.int64
    n = p["x"].numel()
    return N.LsPoints(_ptr(p["x"]), _ptr(p["y"]), _ptr(p["z"]), _ptr(p["r"]), _ptr(p["g"]),
                      _ptr(p["b"]), n, _ptr(off))


def empty_bins(n_tiles, cells, device="cuda"):
    """Uninitialised accumulator tensors [T, cells, cells] (uint64 sums in int64 storage,
    uint32 count in int32 storage)."""
    return {k: torch.empty((n_tiles, cells, cells), dtype=_BIN_DTYPES[k], device=device)
            for k in BIN_KEYS}


def _bins_struct(b, cells):
    return N.LsBins(cells, *[_ptr(_dev(b[k], k)) for k in BIN_KEYS])


def bin_points(points, region, levels=(640, 64), out=None, dropped=None, stream=None):
    """Exact per-cell count / z-sum / z-min / z-max / RGB sums at one or two levels.

    Returns (list of bin dicts, dropped tensor int64[1])."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = points["x"].device
    if out is None:
        out = [empty_bins(T, c, dev) for c in levels]
    if dropped is None:
        dropped = torch.empty(1, dtype=torch.int64, device=dev)
    arr = (N.LsBins * len(levels))(*[_bins_struct(b, c) for b, c in zip(out, levels)])
    pts = _points(points)
    reg = _region(region)
    N.check("ls_bin_points", N.lib().ls_bin_points(ctypes.byref(pts), ctypes.byref(reg), arr,
                                                  len(levels), _ptr(dropped), _stream(stream)))
    return out, dropped


def extract_samples(points, chunk=50000, capacity=None, stream=None):
    """First point of every `chunk`-point chunk of every tile (needs tile_offsets).

    Returns a sample dict (x, y, z, r, g, b, tile_offsets) on the same device; the
    arrays are sized by the host-side capacity bound and trimmed after a sync."""
    pts = _points(points, need_offsets=True)
    off = points["tile_offsets"]
    T = off.numel() - 1
    n = points["x"].numel()
    if capacity is None:
        capacity = n // chunk + T
    dev = points["x"].device
    out = {k: torch.empty(max(capacity, 1), dtype=points[k].dtype, device=dev) for k in "xyzrgb"}
    soff = torch.empty(T + 1, dtype=torch.int64, device=dev)
    bufs = N.LsSampleBuffers(*[_ptr(out[k]) for k in "xyzrgb"])
    N.check("ls_extract_samples", N.lib().ls_extract_samples(ctypes.byref(pts), T, chunk, _ptr(soff),
                                                            ctypes.byref(bufs), capacity, _stream(stream)))
    total = int(soff[-1].item())
    out = {k: v[:min(total, capacity)] for k, v in out.items()}
    out["tile_offsets"] = soff
    return out


def extract_samples_into(points, samples, capacity, chunk=50000, stream=None):
    """Like extract_samples, into pre-allocated buffers (x, y, z, r, g, b of `capacity`
    entries and tile_offsets of T+1) without any host synchronisation, so the call can
    be captured in a CUDA graph.  The buffers past samples['tile_offsets'][-1] are
    unused."""
    pts = _points(points, need_offsets=True)
    T = points["tile_offsets"].numel() - 1
    bufs = N.LsSampleBuffers(*[_ptr(_dev(samples[k], k)) for k in "xyzrgb"])
    N.check("ls_extract_samples", N.lib().ls_extract_samples(
        ctypes.byref(pts), T, chunk, _ptr(_dev(samples["tile_offsets"], "tile_offsets")),
        ctypes.byref(bufs), capacity, _stream(stream)))
    return samples


def fill_sparse(samples, region, tile_ids=None, res=64, radius_cm=12000, sigma_cm=4000.0,
                height=None, rgb=None, stream=None):
    """Gaussian-weighted fill of res x res texels per requested tile.

    Returns (height float32 [n, res, res] metres, rgb uint8 [n, res, res, 3])."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = samples["x"].device
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = T if tile_ids is None else tile_ids.numel()
    if height is None:
        height = torch.empty((n, res, res), dtype=torch.float32, device=dev)
    if rgb is None:
        rgb = torch.empty((n, res, res, 3), dtype=torch.uint8, device=dev)
    pts = _points(samples, need_offsets=True)
    reg = _region(region)
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    N.check("ls_fill_sparse", N.lib().ls_fill_sparse(ctypes.byref(pts), ctypes.byref(reg), ctypes.byref(prm),
                                                    _ptr(tile_ids), n, _ptr(_dev(height, "height")),
                                                    _ptr(_dev(rgb, "rgb")), _stream(stream)))
    return height, rgb


def update_tile(bins, region, tile_ids, height, rgb, stream=None):
    """Overwrite texels that hold full-resolution points with their mean (in place)."""
    cells = bins["count"].shape[-1]
    n = height.shape[0]
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=height.device, dtype=torch.int32).contiguous(), "tile_ids")
    b = _bins_struct(bins, cells)
    reg = _region(region)
    N.check("ls_update_tile", N.lib().ls_update_tile(ctypes.byref(b), ctypes.byref(reg), _ptr(tile_ids), n,
                                                    _ptr(_dev(height, "height")), _ptr(_dev(rgb, "rgb")),
                                                    _stream(stream)))
    return height, rgb


def last_error():
    """Synchronise and return (then clear) the library's sticky device status."""
    return N.lib().ls_last_error()


def release_workspace():
    N.check("ls_release_workspace", N.lib().ls_release_workspace())
