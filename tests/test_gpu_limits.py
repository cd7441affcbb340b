"""The largest sizes each call accepts, against the oracle: binning at the finest fine
level a 640 m tile allows under the 4096-cell cap (4000 cells of 16 cm: a one-row
window, so nearly every point of an 8 m strip slides it or arrives late) and at 2000
cells with a 200-cell coarse level; the Gaussian fill at 1000 texels per side (64 cm);
the Alg. 1 maps at 1000 texels per side of the padded patch (96 cm).  Bars as in the
per-call tests (binning bit-exact, fill within 1e-3 m, maps with the bounds of
test_gpu_interp)."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_bins_equal, assert_fill_close, to_device
from tests.test_gpu_fill import _fill_both
from tests.test_gpu_interp import check_patch, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


@pytest.mark.parametrize("levels,counts", [((4000,), (600_000,)), ((2000, 200), (600_000, 150_001))])
def test_binning_at_the_finest_levels(lsb, levels, counts):
    import torch
    region = synth.Region(tiles_x=len(counts), tiles_y=1)
    counts = np.array(counts, dtype=np.int64)
    pts = synth.region_points(21, region, counts)
    del pts["tile_offsets"]
    out, dropped = lsb.bin_points(to_device(pts), region, levels=levels)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    for b, c in zip(out, levels):
        ref = oracle.bin_points(pts, region, c)
        assert_bins_equal(b, ref, msg=f"cells={c}")
    assert int(dropped.item()) == ref["dropped"] == 0


def test_gaussian_fill_at_the_largest_resolution(lsb):
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = synth.lognormal_counts(22, 9)
    samples = synth.region_samples(22, region, counts)
    h, c, ref, st = _fill_both(lsb, samples, region, tile_ids=[4], res=1000)
    assert st == 0
    assert h.shape[-1] == 1000
    assert_fill_close(h, c, ref, msg="res 1000")


def test_interpolated_maps_at_the_largest_resolution(lsb):
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=12.0)
    counts = synth.lognormal_counts(23, 9, mu=np.log(5.0), sigma=0.5)
    samples = synth.region_samples(23, region, counts)
    got, st = run_gpu(lsb, samples, region, tile_ids=[4], res=1000)
    assert st == 0
    check_patch(got, 0, samples, region, 4, msg="res 1000", res=1000)
