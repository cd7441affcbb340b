"""Resolution variants (the texel-size study of the evaluation: 1, 2.5, 5, 10, 20 and
40 m texels) through the same kernels, against the oracle at each size: binning
bit-exact, Gaussian fill within 1e-3 m (colour rule of helpers.assert_fill_close), Alg. 1
maps with the bars of test_gpu_interp (the padded patch keeps its 160 m apron: 1.5 times
the tile's texels per side)."""
import numpy as np
import pytest

import synth
from tests.helpers import assert_fill_close
from tests.test_gpu_bin import _check, _small_region
from tests.test_gpu_fill import _fill_both
from tests.test_gpu_interp import check_patch, run_gpu

pytestmark = pytest.mark.gpu

TEXEL_CM = (100, 250, 500, 1000, 2000, 4000)


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


@pytest.mark.parametrize("texel_cm", TEXEL_CM)
def test_binning_at_texel_size(lsb, texel_cm):
    region, pts = _small_region()
    _check(lsb, region, pts, levels=(region.tile_cm // texel_cm,), msg=f"{texel_cm} cm texels")


@pytest.mark.parametrize("texel_cm", TEXEL_CM)
def test_gaussian_fill_at_texel_size(lsb, texel_cm):
    region = synth.Region(tiles_x=3, tiles_y=2)
    counts = synth.lognormal_counts(8, 6)
    samples = synth.region_samples(8, region, counts)
    tiles = [4, 0] if texel_cm <= 250 else None  # the finest maps on two tiles only
    h, c, ref, st = _fill_both(lsb, samples, region, tile_ids=tiles, res=region.tile_cm // texel_cm)
    assert st == 0
    assert_fill_close(h, c, ref, msg=f"{texel_cm} cm texels")


@pytest.mark.parametrize("texel_cm", TEXEL_CM)
def test_interpolated_maps_at_texel_size(lsb, texel_cm):
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=33.0)
    counts = synth.lognormal_counts(9, 9, mu=np.log(5.0), sigma=0.5)
    samples = synth.region_samples(9, region, counts)
    res = (region.tile_cm + 2 * 16000) // texel_cm
    tiles = [4] if texel_cm <= 250 else [4, 0, 8]
    got, st = run_gpu(lsb, samples, region, tile_ids=tiles, res=res)
    assert st == 0
    for o, t in enumerate(tiles):
        check_patch(got, o, samples, region, t, msg=f"{texel_cm} cm tile {t}", res=res)
