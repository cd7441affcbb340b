"""GPU parity of ls_bin_points against the serial oracle: bit-exact on every
accumulator, both levels, for stream order, shuffled order, unaligned pointers,
empty input, points split over several accumulating calls, and sampled tiles of the
full-size 16x16-tile lognormal region."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import BIN_KEYS, assert_bins_equal, bins_to_numpy, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


def _small_region():
    region = synth.Region(tiles_x=3, tiles_y=2)
    counts = np.array([140_000, 0, 123_457, 5, 80, 260_001], dtype=np.int64)
    pts = synth.region_points(7, region, counts)
    extra = {"x": np.array([region.x0_cm - 1, region.x0_cm + 3 * 64000, region.x0_cm + 3 * 64000 - 1], np.int32),
             "y": np.array([region.y0_cm, region.y0_cm, region.y0_cm + 2 * 64000 - 1], np.int32),
             "z": np.array([1, 1, 9], np.int32), "r": np.array([1, 1, 2], np.uint16),
             "g": np.array([1, 1, 2], np.uint16), "b": np.array([1, 1, 2], np.uint16)}
    for k in extra:
        pts[k] = np.concatenate([pts[k], extra[k]])
    del pts["tile_offsets"]
    return region, pts


def _check(lsb, region, pts, levels=(640, 64), msg=""):
    import torch
    d = to_device(pts)
    out, dropped = lsb.bin_points(d, region, levels=levels)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    ref0 = None
    for b, c in zip(out, levels):
        ref = oracle.bin_points(pts, region, c)
        assert_bins_equal(b, ref, msg=f"{msg} cells={c}")
        ref0 = ref
    assert int(dropped.item()) == ref0["dropped"]
    return out


def test_small_region_two_levels(lsb):
    region, pts = _small_region()
    _check(lsb, region, pts, msg="stream order")


@pytest.mark.parametrize("levels", [(640,), (64,), (320, 32), (128, 64)])
def test_other_level_sets(lsb, levels):
    region, pts = _small_region()
    _check(lsb, region, pts, levels=levels, msg=str(levels))


def test_shuffled_order_is_still_exact(lsb):
    region, pts = _small_region()
    perm = np.random.default_rng(11).permutation(len(pts["x"]))
    _check(lsb, region, {k: pts[k][perm] for k in "xyzrgb"}, msg="shuffled")


def test_reversed_strips_and_partial_shuffle(lsb):
    region, pts = _small_region()
    n = len(pts["x"])
    idx = np.arange(n)[::-1].copy()
    rng = np.random.default_rng(12)
    sw = rng.integers(0, n, (2000, 2))
    idx[sw[:, 0]], idx[sw[:, 1]] = idx[sw[:, 1]], idx[sw[:, 0]]
    _check(lsb, region, {k: pts[k][idx] for k in "xyzrgb"}, msg="reversed")


def test_unaligned_pointers_use_scalar_path(lsb):
    import torch
    region, pts = _small_region()
    d = to_device(pts)
    sub = {k: v[1:] for k, v in d.items()}  # 4- and 2-byte aligned only
    out, dropped = lsb.bin_points(sub, region)
    torch.cuda.synchronize()
    ref = oracle.bin_points({k: pts[k][1:] for k in "xyzrgb"}, region, 640)
    assert_bins_equal(out[0], ref, msg="unaligned")
    assert int(dropped.item()) == ref["dropped"]


def _accumulate_parts(lsb, region, parts, levels=(640, 64), out=None, dropped=None):
    import torch
    for i, part in enumerate(parts):
        d = to_device(part)
        if out is None:
            out, dropped = lsb.bin_points(d, region, levels=levels)
        else:
            lsb.bin_points(d, region, levels=levels, out=out, dropped=dropped, accumulate=True)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    return out, dropped


@pytest.mark.parametrize("cuts", [(0.3, 0.71), (0.5,), (1e-6, 0.999999)])
def test_accumulate_over_split_calls_equals_one_call(lsb, cuts):
    """Points that arrive over several calls (the first overwrites, the rest add):
    the bins equal the oracle over the union of the points, bit for bit, at both
    levels; splits fall inside strips, one part is empty and one holds a single point."""
    region, pts = _small_region()
    n = len(pts["x"])
    idx = [0] + [int(c * n) for c in cuts] + [n]
    parts = [{k: pts[k][a:b] for k in "xyzrgb"} for a, b in zip(idx[:-1], idx[1:])]
    out, dropped = _accumulate_parts(lsb, region, parts)
    for b, c in zip(out, (640, 64)):
        ref = oracle.bin_points(pts, region, c)
        assert_bins_equal(b, ref, msg=f"cuts={cuts} cells={c}")
    assert int(dropped.item()) == ref["dropped"]


def test_accumulate_shuffled_parts_onto_empty_bins(lsb):
    """Accumulating into bins that hold the empty-cell values (and a dropped counter
    that starts at 5) equals one call over all points; the parts are shuffled, so
    rows are touched by several calls and late points occur within a call."""
    import torch
    region, pts = _small_region()
    perm = np.random.default_rng(13).permutation(len(pts["x"]))
    sh = {k: pts[k][perm] for k in "xyzrgb"}
    T = region.n_tiles
    out = []
    for c in (640, 64):
        b = lsb.empty_bins(T, c)
        b["count"].zero_(); b["zsum"].zero_(); b["rsum"].zero_(); b["gsum"].zero_(); b["bsum"].zero_()
        b["zmin"].fill_(np.iinfo(np.int32).max); b["zmax"].fill_(np.iinfo(np.int32).min)
        out.append(b)
    dropped = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    n = len(sh["x"])
    parts = [{k: sh[k][a:b] for k in "xyzrgb"} for a, b in ((0, n // 3), (n // 3, n))]
    out, dropped = _accumulate_parts(lsb, region, parts, out=out, dropped=dropped)
    for b, c in zip(out, (640, 64)):
        ref = oracle.bin_points(pts, region, c)
        assert_bins_equal(b, ref, msg=f"shuffled parts cells={c}")
    assert int(dropped.item()) == ref["dropped"] + 5


def test_empty_input_gives_sentinels(lsb):
    import torch
    region = synth.Region(tiles_x=2, tiles_y=2)
    e = {k: np.zeros(0, np.int32 if k in "xyz" else np.uint16) for k in "xyzrgb"}
    d = {k: torch.from_numpy(v).cuda() for k, v in e.items()}
    out, dropped = lsb.bin_points(d, region)
    torch.cuda.synchronize()
    for b, c in zip(out, (640, 64)):
        assert_bins_equal(b, oracle.bin_points(e, region, c), msg="empty")
    assert int(dropped.item()) == 0


def test_single_tile_two_million_points(lsb, single_tile_points):
    region, counts, pts = single_tile_points
    _check(lsb, region, {k: pts[k] for k in "xyzrgb"}, msg="single tile")


def test_dense_tile_forces_window_residency_limit(lsb):
    """A 64 m tile with 1.5M points sorted by y: every window of rows receives far
    more than 65536 points, so rows must leave the window early and merge later."""
    region = synth.Region(tile_cm=6400, tiles_x=2, tiles_y=1)
    rng = np.random.default_rng(21)
    n = 1_500_000
    x = region.x0_cm + rng.integers(0, 2 * 6400, n)
    y = np.sort(region.y0_cm + rng.integers(0, 6400, n))
    pts = {"x": x.astype(np.int32), "y": y.astype(np.int32),
           "z": rng.integers(-2**31, 2**31 - 1, n).astype(np.int32),
           "r": rng.integers(0, 65536, n).astype(np.uint16),
           "g": np.full(n, 65535, np.uint16), "b": rng.integers(0, 65536, n).astype(np.uint16)}
    _check(lsb, region, pts, levels=(64, 8), msg="dense")


def test_gpu_generator_matches_numpy_generator(lsb):
    import synth.gpu as sg
    region = synth.Region(tiles_x=3, tiles_y=2)
    counts = np.array([70_001, 0, 3, 50_000, 10, 99_999], dtype=np.int64)
    d = sg.region_points(9, region, counts)
    h = synth.region_points(9, region, counts)
    for k in "xyzrgb":
        np.testing.assert_array_equal(d[k].cpu().numpy(), h[k], err_msg=k)
    ds = sg.region_samples(9, region, counts)
    hs = synth.region_samples(9, region, counts)
    for k in list("xyzrgb") + ["tile_offsets"]:
        np.testing.assert_array_equal(ds[k].cpu().numpy(), hs[k], err_msg=k)


def test_full_size_lognormal_region_sampled_tiles(lsb):
    """The 16x16-tile lognormal region at full size, in the launch configuration the
    benchmark times: invariants on the whole output, bit-exact oracle parity on three
    tiles regenerated on the host (smallest, median and a seeded random tile)."""
    import torch
    import synth.gpu as sg
    region, counts = synth.batched_region_workload()
    d = sg.region_points(2, region, counts)
    lsb.bin_stats(reset=True)
    out, dropped = lsb.bin_points(d, region, levels=(640, 64))
    torch.cuda.synchronize()
    st = lsb.bin_stats(reset=True)
    print("bin stats", st)
    assert lsb.last_error() == 0
    # strip-ordered input: no point arrives after its row left a window
    assert st["late_points"] == 0 and st["wait_timeouts"] == 0
    n = int(counts.sum())
    assert int(dropped.item()) == 0
    fine, coarse = out
    assert int(fine["count"].to(torch.int64).sum().item()) == n
    assert int(coarse["count"].to(torch.int64).sum().item()) == n
    # coarse level equals the 10x10 block reduction of the fine level
    T = region.n_tiles
    blk = lambda a: a.reshape(T, 64, 10, 64, 10)  # noqa: E731
    assert torch.equal(coarse["count"], blk(fine["count"]).sum(dim=(2, 4), dtype=torch.int64).to(torch.int32))
    assert torch.equal(coarse["zsum"], blk(fine["zsum"]).sum(dim=(2, 4)))
    assert torch.equal(coarse["zmin"], blk(fine["zmin"]).amin(dim=(2, 4)))
    assert torch.equal(coarse["zmax"], blk(fine["zmax"]).amax(dim=(2, 4)))
    order = np.argsort(counts)
    tiles = [int(order[0]), int(order[len(order) // 2]), int(np.random.default_rng(5).integers(0, T))]
    for t in tiles:
        one = synth.Region(x0_cm=region.x0_cm + (t % region.tiles_x) * region.tile_cm,
                           y0_cm=region.y0_cm + (t // region.tiles_x) * region.tile_cm)
        pts = synth.tile_points(2, region, t, int(counts[t]))
        p = dict(zip("xyzrgb", pts))
        for b, c in zip(out, (640, 64)):
            ref = oracle.bin_points(p, one, c)
            g = {k: b[k][t:t + 1] for k in BIN_KEYS}
            assert_bins_equal(g, ref, msg=f"tile {t} cells={c}")
