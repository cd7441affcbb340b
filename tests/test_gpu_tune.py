"""Launch shapes on the GPU: every candidate shape of the binning and of the Gaussian
fill gives the same results (binning bit-exact against the oracle; fill maps bit-equal
to each other and within the fill bars of the oracle), and the autotuners return one of
the candidates, store it for the call's key and leave the outputs computed."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_bins_equal, assert_fill_close, to_device
from tests.test_gpu_bin import _small_region

pytestmark = pytest.mark.gpu

BIN_SHAPES = [{"spans_per_cta": s, "prefetch_batches": p} for s in (1, 8, 16, 32, 256) for p in (1, 2, 3, 4)]


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    lsb.tune_clear()
    yield lsb
    lsb.tune_clear()


def test_every_binning_shape_is_exact(lsb):
    import torch
    region, pts = _small_region()
    d = to_device(pts)
    refs = [oracle.bin_points(pts, region, c) for c in (640, 64)]
    for shape in BIN_SHAPES:
        lsb.set_bin_shape(d, shape=shape)
        assert lsb.bin_shape(d) == shape
        out, dropped = lsb.bin_points(d, region)
        torch.cuda.synchronize()
        assert lsb.last_error() == 0
        for b, ref, c in zip(out, refs, (640, 64)):
            assert_bins_equal(b, ref, msg=f"{shape} cells={c}")
        assert int(dropped.item()) == refs[0]["dropped"]
    lsb.set_bin_shape(d, shape=None)


def test_binning_autotuner(lsb):
    import torch
    region, pts = _small_region()
    d = to_device(pts)
    shape, ms, out, dropped = lsb.tune_bin_points(d, region, reps=2)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    assert shape["spans_per_cta"] in (8, 16, 32) and shape["prefetch_batches"] in (1, 2, 3)
    assert 0.0 < ms < 1e4
    assert lsb.bin_shape(d) == shape
    for b, c in zip(out, (640, 64)):
        assert_bins_equal(b, oracle.bin_points(pts, region, c), msg=f"tuned cells={c}")


def _fill_case():
    region = synth.Region(tiles_x=4, tiles_y=3)
    counts = synth.lognormal_counts(31, 12)
    return region, synth.region_samples(31, region, counts)


def test_every_fill_shape_gives_the_same_maps(lsb):
    import torch
    region, samples = _fill_case()
    d = to_device(samples)
    n = region.n_tiles
    ref = oracle.fill_sparse(samples, region, res=64)
    first = None
    for split in (1, 2, 4):
        for ctas in (1, 2, 3, 4):
            shape = {"split": split, "ctas_per_sm": ctas}
            lsb.set_fill_shape(d, n, shape=shape)
            assert lsb.fill_shape(d, n) == shape
            h, c = lsb.fill_sparse(d, region)
            torch.cuda.synchronize()
            assert lsb.last_error() == 0
            h, c = h.cpu().numpy(), c.cpu().numpy()
            if first is None:
                assert_fill_close(h, c, ref, msg=str(shape))
                first = (h, c)
            else:
                np.testing.assert_array_equal(h, first[0], err_msg=str(shape))
                np.testing.assert_array_equal(c, first[1], err_msg=str(shape))
    lsb.set_fill_shape(d, n, shape=None)


def test_fill_autotuner(lsb):
    import torch
    region, samples = _fill_case()
    d = to_device(samples)
    shape, ms, h, c = lsb.tune_fill_sparse(d, region, reps=2)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    assert shape["split"] in (1, 2, 4) and shape["ctas_per_sm"] in (1, 2, 3, 4)
    assert 0.0 < ms < 1e4
    assert lsb.fill_shape(d, region.n_tiles) == shape
    assert_fill_close(h.cpu().numpy(), c.cpu().numpy(), oracle.fill_sparse(samples, region, res=64), msg="tuned")
