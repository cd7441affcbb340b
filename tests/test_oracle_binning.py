"""Pins of the oracle's binning and sample extraction against hand values,
invariants and an independent numpy formulation (no GPU)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("count", "zsum", "zmin", "zmax", "rsum", "gsum", "bsum")


def _pts(rows):
    a = np.array(rows, dtype=np.int64)
    return {"x": a[:, 0].astype(np.int32), "y": a[:, 1].astype(np.int32),
            "z": a[:, 2].astype(np.int32), "r": a[:, 3].astype(np.uint16),
            "g": a[:, 4].astype(np.uint16), "b": a[:, 5].astype(np.uint16)}


def test_hand_computed_tile():
    fx = json.load(open(os.path.join(GOLD, "bin_points_hand.json")))
    region = synth.Region(**fx["region"])
    pts = _pts(fx["points"])
    for cells, cases in fx["expect"].items():
        bins = oracle.bin_points(pts, region, int(cells))
        assert bins["dropped"] == fx["dropped"]
        seen = np.zeros(bins["count"].shape, bool)
        for c in cases:
            for k in KEYS:
                assert bins[k][c["tile"], c["i"], c["j"]] == c[k], (cells, c, k)
            seen[c["tile"], c["i"], c["j"]] = True
        # every other cell is empty with the sentinels
        assert (bins["count"][~seen] == 0).all()
        assert (bins["zsum"][~seen] == 0).all()
        assert (bins["zmin"][~seen] == np.iinfo(np.int32).max).all()
        assert (bins["zmax"][~seen] == np.iinfo(np.int32).min).all()
        for k in ("rsum", "gsum", "bsum"):
            assert (bins[k][~seen] == 0).all()


def _numpy_bins(pts, region, cells):
    """Independent formulation with numpy scatter primitives (bincount, minimum.at)."""
    lx = pts["x"].astype(np.int64) - region.x0_cm
    ly = pts["y"].astype(np.int64) - region.y0_cm
    ok = (lx >= 0) & (ly >= 0) & (lx < region.tiles_x * region.tile_cm) & (ly < region.tiles_y * region.tile_cm)
    cell = region.tile_cm // cells
    tx, ty = lx[ok] // region.tile_cm, ly[ok] // region.tile_cm
    j = (lx[ok] % region.tile_cm) // cell
    i = (ly[ok] % region.tile_cm) // cell
    flat = ((ty * region.tiles_x + tx) * cells + i) * cells + j
    n = region.tiles_x * region.tiles_y * cells * cells
    out = {"count": np.bincount(flat, minlength=n).astype(np.uint32)}
    z = pts["z"][ok].astype(np.int64)
    zs = np.zeros(n, np.int64)
    np.add.at(zs, flat, z)
    out["zsum"] = zs
    mn = np.full(n, np.iinfo(np.int32).max, np.int64)
    mx = np.full(n, np.iinfo(np.int32).min, np.int64)
    np.minimum.at(mn, flat, z)
    np.maximum.at(mx, flat, z)
    out["zmin"], out["zmax"] = mn.astype(np.int32), mx.astype(np.int32)
    for k in "rgb":
        s = np.zeros(n, np.uint64)
        np.add.at(s, flat, pts[k][ok].astype(np.uint64))
        out[k + "sum"] = s
    shape = (region.tiles_x * region.tiles_y, cells, cells)
    return {k: v.reshape(shape) for k, v in out.items()}, int((~ok).sum())


@pytest.fixture(scope="module")
def small_region():
    region = synth.Region(tiles_x=3, tiles_y=2)
    counts = np.array([40_000, 0, 123_457, 5, 80, 60_001], dtype=np.int64)
    pts = synth.region_points(7, region, counts)
    # a few points outside the region (dropped) and on the outer edges
    extra = _pts([[region.x0_cm - 1, region.y0_cm, 1, 1, 1, 1],
                  [region.x0_cm + 3 * 64000, region.y0_cm, 1, 1, 1, 1],
                  [region.x0_cm + 3 * 64000 - 1, region.y0_cm + 2 * 64000 - 1, 9, 2, 2, 2],
                  [region.x0_cm, region.y0_cm + 2 * 64000, 1, 1, 1, 1]])
    for k in extra:
        pts[k] = np.concatenate([pts[k], extra[k]])
    del pts["tile_offsets"]
    return region, pts


@pytest.mark.parametrize("cells", [64, 640])
def test_matches_independent_numpy(small_region, cells):
    region, pts = small_region
    bins = oracle.bin_points(pts, region, cells)
    ref, dropped = _numpy_bins(pts, region, cells)
    assert bins["dropped"] == dropped == 3
    for k in KEYS:
        np.testing.assert_array_equal(bins[k], ref[k], err_msg=k)


@pytest.mark.parametrize("cells", [64, 640])
def test_count_sum_and_min_mean_max(small_region, cells):
    region, pts = small_region
    bins = oracle.bin_points(pts, region, cells)
    n = len(pts["x"])
    assert int(bins["count"].sum(dtype=np.int64)) + bins["dropped"] == n
    ne = bins["count"] > 0
    mean = bins["zsum"][ne] / bins["count"][ne]
    assert (bins["zmin"][ne] <= mean).all() and (mean <= bins["zmax"][ne]).all()
    assert (bins["zmin"][~ne] == np.iinfo(np.int32).max).all()


def test_permutation_invariance(small_region):
    region, pts = small_region
    perm = np.random.default_rng(3).permutation(len(pts["x"]))
    a = oracle.bin_points(pts, region, 640)
    b = oracle.bin_points({k: pts[k][perm] for k in "xyzrgb"}, region, 640)
    for k in KEYS + ("dropped",):
        np.testing.assert_array_equal(a[k], b[k])


def test_coarse_level_is_block_reduction_of_fine(small_region):
    """10 m cells are exact 10x10 reductions of 1 m cells (integer sums)."""
    region, pts = small_region
    f = oracle.bin_points(pts, region, 640)
    c = oracle.bin_points(pts, region, 64)
    T = region.tiles_x * region.tiles_y
    blk = lambda a: a.reshape(T, 64, 10, 64, 10)  # noqa: E731
    np.testing.assert_array_equal(c["count"], blk(f["count"]).sum(axis=(2, 4)))
    np.testing.assert_array_equal(c["zsum"], blk(f["zsum"]).sum(axis=(2, 4)))
    np.testing.assert_array_equal(c["zmin"], blk(f["zmin"]).min(axis=(2, 4)))
    np.testing.assert_array_equal(c["zmax"], blk(f["zmax"]).max(axis=(2, 4)))
    for k in ("rsum", "gsum", "bsum"):
        np.testing.assert_array_equal(c[k], blk(f[k]).sum(axis=(2, 4)))


def test_extract_sample_indices_first_point_of_each_chunk():
    # Sec. 3.1/3.2: the first point of every 50,000-point chunk is the sample
    offs = np.array([0, 2_000_000, 2_000_000, 2_050_001, 2_050_002], dtype=np.int64)
    idx, soffs = oracle.extract_sample_indices(offs)
    np.testing.assert_array_equal(soffs, [0, 40, 40, 42, 43])
    np.testing.assert_array_equal(idx[:3], [0, 50_000, 100_000])
    np.testing.assert_array_equal(idx[39:], [1_950_000, 2_000_000, 2_050_000, 2_050_001])


def test_generator_samples_are_the_chunk_heads():
    region = synth.Region(tiles_x=2, tiles_y=1)
    counts = np.array([120_000, 50_000], dtype=np.int64)
    pts = synth.region_points(5, region, counts)
    s = synth.region_samples(5, region, counts)
    idx, soffs = oracle.extract_sample_indices(pts["tile_offsets"])
    np.testing.assert_array_equal(soffs, s["tile_offsets"])
    for k in "xyzrgb":
        np.testing.assert_array_equal(pts[k][idx], s[k])
