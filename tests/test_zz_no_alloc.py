"""ls_bin_points_fixed_scratch: the binning entry point for callers that cannot
allocate device memory during the call (its per-row scratch is a fixed array inside
the library).  Called through the C ABI, twice in a row, it must give exactly the
results of ls_bin_points and of the oracle (binning is bit-exact), and the device's
free memory must not change across the two calls.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_bins_equal

pytestmark = pytest.mark.gpu

KEYS = ("count", "zsum", "zmin", "zmax", "rsum", "gsum", "bsum")


def _levels(N, torch, T, cells_list):
    out = []
    for cells in cells_list:
        b = {k: torch.full((T, cells, cells), 7, dtype=torch.int32 if k in ("count", "zmin", "zmax") else torch.int64,
                           device="cuda") for k in KEYS}
        out.append(b)
    arr = (N.LsBins * len(out))(*[N.LsBins(c, *[ctypes.c_void_p(b[k].data_ptr()) for k in KEYS])
                                  for b, c in zip(out, cells_list)])
    return out, arr


def test_fixed_scratch_binning_matches_ls_bin_points_twice():
    import torch
    from paper_2509_20198_b300 import _native as N, build
    build.build_library()
    L = N.lib()
    region = synth.Region(tiles_x=3, tiles_y=2)
    counts = np.array([180_000, 0, 95_001, 7, 300_000, 64_000], dtype=np.int64)
    pts = synth.region_points(17, region, counts)
    d = {k: torch.from_numpy(np.ascontiguousarray(pts[k])).cuda() for k in "xyzrgb"}
    P = N.LsPoints(*[ctypes.c_void_p(d[k].data_ptr()) for k in "xyzrgb"], len(pts["x"]), None)
    R = N.LsRegion(region.x0_cm, region.y0_cm, region.tile_cm, region.tiles_x, region.tiles_y,
                   region.z_scale, region.z_offset)
    T = region.n_tiles
    ref, arr_ref = _levels(N, torch, T, (640, 64))
    dref = torch.zeros(1, dtype=torch.int64, device="cuda")
    N.check("ls_bin_points", L.ls_bin_points(ctypes.byref(P), ctypes.byref(R), arr_ref, 2,
                                            ctypes.c_void_p(dref.data_ptr()), None))
    torch.cuda.synchronize()
    # outputs of both calls allocated up front; the library's own workspace released,
    # so that an allocation inside the calls would show in the device's free memory
    outs = [_levels(N, torch, T, (640, 64)) + (torch.full((1,), 99, dtype=torch.int64, device="cuda"),)
            for _ in range(2)]
    N.check("ls_release_workspace", L.ls_release_workspace())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call, (got, arr, dg) in enumerate(outs):
        N.check("ls_bin_points_fixed_scratch",
                L.ls_bin_points_fixed_scratch(ctypes.byref(P), ctypes.byref(R), arr, 2,
                                              ctypes.c_void_p(dg.data_ptr()), None))
        torch.cuda.synchronize()
        assert L.ls_last_error() == 0
    assert torch.cuda.mem_get_info()[0] == free0, "the fixed-scratch calls allocated device memory"
    for call, (got, arr, dg) in enumerate(outs):
        for lv in range(2):
            for k in KEYS:
                assert torch.equal(got[lv][k], ref[lv][k]), (call, lv, k)
        assert int(dg.item()) == int(dref.item())
    for lv, cells in enumerate((640, 64)):
        assert_bins_equal(outs[1][0][lv], oracle.bin_points(pts, region, cells), msg=f"oracle cells={cells}")


def test_fixed_scratch_rejects_regions_over_the_limit():
    import torch
    from paper_2509_20198_b300 import _native as N, build
    build.build_library()
    L = N.lib()
    # 41 x 40 tiles of 640 rows = 1,049,600 fine rows > 2^20: rejected before any launch
    R = N.LsRegion(0, 0, 64000, 41, 40, 0.01, 0.0)
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = torch.zeros(4, dtype=torch.int16, device="cuda")
    P = N.LsPoints(*[ctypes.c_void_p(t.data_ptr()) for t in (x, x, x, c, c, c)], 4, None)
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    lv = N.LsBins(640, *[ctypes.c_void_p(dummy.data_ptr())] * 7)
    assert L.ls_bin_points_fixed_scratch(ctypes.byref(P), ctypes.byref(R), ctypes.byref(lv), 1, None, None) == -6
