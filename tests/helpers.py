"""Shared helpers of the test-suite (inputs from synth/, references from oracle/)."""
from __future__ import annotations

import numpy as np

BIN_KEYS = ("count", "zsum", "zmin", "zmax", "rsum", "gsum", "bsum")
# the library stores uint32 counts / uint64 sums in int32 / int64 tensors
_VIEW = {"count": np.uint32, "rsum": np.uint64, "gsum": np.uint64, "bsum": np.uint64}


def to_device(pts, device="cuda"):
    import torch
    out = {}
    for k in "xyz":
        out[k] = torch.from_numpy(np.ascontiguousarray(pts[k], dtype=np.int32)).to(device)
    for k in "rgb":
        out[k] = torch.from_numpy(np.ascontiguousarray(pts[k], dtype=np.uint16)).to(device)
    if "tile_offsets" in pts:
        out["tile_offsets"] = torch.as_tensor(np.asarray(pts["tile_offsets"], np.int64)).to(device)
    return out


def bins_to_numpy(b):
    out = {}
    for k in BIN_KEYS:
        a = b[k].cpu().numpy()
        out[k] = a.view(_VIEW[k]) if k in _VIEW else a
    return out


def assert_bins_equal(gpu, ref, tiles=None, msg=""):
    g = bins_to_numpy(gpu)
    for k in BIN_KEYS:
        a = g[k] if tiles is None else g[k][tiles]
        np.testing.assert_array_equal(a, ref[k], err_msg=f"{msg} {k}")


def assert_fill_close(h_gpu, rgb_gpu, ref, atol_m=1e-3, msg=""):
    """Height within atol_m of the FP64 oracle; 8-bit colour equal wherever the
    oracle's unrounded value is more than 0.01 level from a rounding boundary (the
    fp32 colour error is far below that), and within 1 level elsewhere."""
    h = np.asarray(h_gpu)
    ok_nan = np.isnan(ref["height"]) == np.isnan(h)
    assert ok_nan.all(), f"{msg} NaN pattern differs"
    fin = ~np.isnan(ref["height"])
    err = np.abs(h[fin] - ref["height"][fin])
    assert err.max(initial=0.0) <= atol_m, f"{msg} max height error {err.max():.3e} m"
    c = np.asarray(rgb_gpu).astype(np.int32)
    r8 = ref["rgb8"].astype(np.int32)
    frac = ref["rgbf"] - np.floor(ref["rgbf"])
    safe = np.abs(frac - 0.5) > 0.01
    assert (c[safe] == r8[safe]).all(), f"{msg} rgb mismatch away from rounding boundaries"
    assert (np.abs(c - r8) <= 1).all(), f"{msg} rgb off by more than one level"
