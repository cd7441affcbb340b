"""GPU parity of sample extraction, the Gaussian fill and the tile update against the
oracle: extraction bit-exact, fill within 1e-3 m (and the colour rule of
helpers.assert_fill_close), tile update bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_fill_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


def _fill_both(lsb, samples, region, tile_ids=None, res=64, radius_cm=12000, sigma_cm=4000.0):
    import torch
    d = to_device(samples)
    tid = None if tile_ids is None else torch.as_tensor(np.asarray(tile_ids, np.int32))
    h, c = lsb.fill_sparse(d, region, tile_ids=tid, res=res, radius_cm=radius_cm, sigma_cm=sigma_cm)
    torch.cuda.synchronize()
    st = lsb.last_error()
    ref = oracle.fill_sparse(samples, region, tile_ids=tile_ids, res=res, radius_cm=radius_cm,
                             sigma_cm=sigma_cm)
    return h.cpu().numpy(), c.cpu().numpy(), ref, st


def test_extraction_matches_oracle(lsb):
    region = synth.Region(tiles_x=3, tiles_y=1)
    counts = np.array([2_000_000, 0, 50_001], dtype=np.int64)
    pts = synth.region_points(3, region, counts)
    s = lsb.extract_samples(to_device(pts))
    idx, soffs = oracle.extract_sample_indices(pts["tile_offsets"])
    np.testing.assert_array_equal(s["tile_offsets"].cpu().numpy(), soffs)
    for k in "xyzrgb":
        np.testing.assert_array_equal(s[k].cpu().numpy(), pts[k][idx], err_msg=k)


def test_extraction_capacity_overflow_sets_status(lsb):
    region = synth.Region(tiles_x=1, tiles_y=1)
    pts = synth.region_points(3, region, np.array([200_000], np.int64))
    s = lsb.extract_samples(to_device(pts), capacity=2)
    assert lsb.last_error() == -3
    assert s["x"].numel() == 2


def test_single_tile_forty_samples(lsb, single_tile_points):
    region, counts, pts = single_tile_points
    samples = synth.region_samples(1, region, counts)
    h, c, ref, st = _fill_both(lsb, samples, region)
    assert st == 0
    assert_fill_close(h, c, ref, msg="single tile")


@pytest.mark.parametrize("density", [4.0, 0.6])
def test_overview_region_all_tiles(lsb, density):
    """12x12 tiles; at 0.6 pts/m^2 (5 samples per tile) many texels have no sample
    within 120 m and take the nearest one."""
    region = synth.Region(tiles_x=12, tiles_y=12)
    counts = synth.uniform_counts(144, density)
    samples = synth.region_samples(4, region, counts)
    h, c, ref, st = _fill_both(lsb, samples, region)
    assert st == 0
    assert_fill_close(h, c, ref, msg=f"density {density}")


def test_tile_subset_and_far_nearest_fallback(lsb):
    """Samples only in two corner tiles of a 7x7 region: most texels' nearest sample
    is several tiles away (ring search beyond the staged 3x3 neighbourhood)."""
    region = synth.Region(tiles_x=7, tiles_y=7)
    counts = np.zeros(49, np.int64)
    counts[0] = 400_000
    counts[48] = 100_000
    samples = synth.region_samples(8, region, counts)
    tiles = [24, 0, 48, 6, 42, 17]
    h, c, ref, st = _fill_both(lsb, samples, region, tile_ids=tiles)
    assert st == 0
    assert_fill_close(h, c, ref, msg="far")


def test_no_samples_gives_nan(lsb):
    region = synth.Region(tiles_x=2, tiles_y=2)
    samples = synth.region_samples(8, region, np.zeros(4, np.int64))
    h, c, ref, st = _fill_both(lsb, samples, region)
    assert np.isnan(h).all() and (c == 0).all()


def test_constant_terrain_exact_on_gpu(lsb):
    import torch
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=-12.5)
    counts = synth.uniform_counts(9, 4.0)
    s = synth.region_samples(6, region, counts)
    s["z"][:] = 43210
    d = to_device(s)
    h, _ = lsb.fill_sparse(d, region)
    torch.cuda.synchronize()
    assert (h.cpu().numpy() == np.float32(43210 * 0.01 - 12.5)).all()


def test_dense_neighbourhood_beyond_stage_capacity(lsb):
    """3000 samples in one tile: more than the shared-memory stage holds, so the
    kernel reads the neighbourhood from global memory."""
    region = synth.Region(tiles_x=2, tiles_y=1)
    counts = np.array([3000 * 50_000, 20 * 50_000], np.int64)
    s = synth.region_samples(10, region, counts)
    h, c, ref, st = _fill_both(lsb, s, region)
    assert st == 0
    assert_fill_close(h, c, ref, msg="dense")


@pytest.mark.parametrize("res,radius,sigma", [(32, 30000, 9000.0), (128, 6000, 2500.0), (8, 64000, 20000.0)])
def test_other_resolutions_and_radii(lsb, res, radius, sigma):
    region = synth.Region(tiles_x=4, tiles_y=3)
    counts = synth.uniform_counts(12, 3.0)
    s = synth.region_samples(12, region, counts)
    h, c, ref, st = _fill_both(lsb, s, region, res=res, radius_cm=radius, sigma_cm=sigma)
    assert st == 0
    assert_fill_close(h, c, ref, msg=f"res {res}")


def test_sample_in_wrong_bucket_sets_status(lsb):
    import torch
    region = synth.Region(tiles_x=2, tiles_y=1)
    s = synth.region_samples(13, region, np.array([100_000, 100_000], np.int64))
    s["tile_offsets"] = np.array([0, 3, 4], np.int64)  # sample 2 belongs to tile 1
    d = to_device(s)
    lsb.fill_sparse(d, region)
    torch.cuda.synchronize()
    assert lsb.last_error() == -1


def test_full_size_overview_seeded_subset(lsb):
    """The 200x200-tile overview (4 pts/m^2, 33 samples per tile) filled in one
    launch on the GPU; the FP64 oracle checks a seeded 1% subset (400 tiles)."""
    import torch
    import synth.gpu as sg
    region, counts = synth.overview_workload()
    d = sg.region_samples(3, region, counts)
    h, c = lsb.fill_sparse(d, region)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    tiles = np.sort(np.random.default_rng(400).choice(region.n_tiles, 400, replace=False))
    samples = synth.region_samples(3, region, counts)
    ref = oracle.fill_sparse(samples, region, tile_ids=tiles)
    assert_fill_close(h[tiles].cpu().numpy(), c[tiles].cpu().numpy(), ref, msg="overview")


def test_update_tile_bit_exact(lsb, single_tile_points):
    import torch
    region, counts, pts = single_tile_points
    d = to_device(pts)
    (b64,), _ = lsb.bin_points(d, region, levels=(64,))
    h0 = torch.full((1, 64, 64), 7.25, device="cuda")
    c0 = torch.full((1, 64, 64, 3), 3, dtype=torch.uint8, device="cuda")
    # empty some texels to check they are kept
    b64["count"][0, 5:9, 5:9] = 0
    lsb.update_tile(b64, region, None, h0, c0)
    torch.cuda.synchronize()
    bins = {k: v.cpu().numpy() for k, v in b64.items()}
    bins["count"] = bins["count"].view(np.uint32)
    for k in ("rsum", "gsum", "bsum"):
        bins[k] = bins[k].view(np.uint64)
    hr, cr = oracle.update_tile(bins, region, [0], np.full((1, 64, 64), 7.25, np.float32),
                                np.full((1, 64, 64, 3), 3, np.uint8))
    np.testing.assert_array_equal(h0.cpu().numpy(), hr)
    np.testing.assert_array_equal(c0.cpu().numpy(), cr)
    assert (h0[0, 5:9, 5:9] == 7.25).all()
