"""GPU parity of the interpolated heightmaps of Alg. 1 (Sec. 3.3) against the oracle:
triangle sets equal, NN maps and inside mask bit-exact, 8-bit colours bit-exact, linear
heights within the float32 bound derived in check_patch (bit-exact outside the real
triangles, where they are the NN values)."""
import numpy as np
import pytest

import oracle.interp as oi
import synth
from tests.helpers import to_device

pytestmark = pytest.mark.gpu

RES, PAD = 96, 16000


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


def _canon(tri):
    """A triangle as its rotation that starts at the smallest id (orientation kept)."""
    k = int(np.argmin(tri))
    return tuple(int(tri[(k + i) % 3]) for i in range(3))


def _round8(x):
    return np.minimum(np.floor(x + 0.5), 255).astype(np.uint8)


def run_gpu(lsb, samples, region, tile_ids=None, tri_cap=4096, res=RES):
    import torch
    d = to_device(samples)
    tid = None if tile_ids is None else torch.as_tensor(np.asarray(tile_ids, np.int32))
    out = lsb.fill_interp(d, region, tile_ids=tid, res=res, pad_cm=PAD, tri_cap=tri_cap)
    torch.cuda.synchronize()
    st = lsb.last_error()
    return {k: v.cpu().numpy() for k, v in out.items()}, st


def check_patch(got, o, samples, region, t, msg="", res=RES):
    ref = oi.interp_tile(samples, region, t, res=res, pad_cm=PAD)
    # triangulation: the same set of counter-clockwise triangles
    cnt = int(got["tri_count"][o])
    assert cnt == len(ref["triangles"]), f"{msg} triangle count {cnt} vs {len(ref['triangles'])}"
    g = sorted(_canon(tr) for tr in got["triangles"][o][:cnt])
    r = sorted(_canon(tr) for tr in ref["triangles"])
    assert g == r, f"{msg} triangle sets differ"
    # NN maps and inside mask: bit-exact
    ref_nn = ref["nn_height"].astype(np.float32)
    np.testing.assert_array_equal(got["nn_height"][o], ref_nn, err_msg=f"{msg} nn height")
    np.testing.assert_array_equal(got["nn_rgb"][o], _round8(ref["nn_rgb8"]), err_msg=f"{msg} nn rgb")
    np.testing.assert_array_equal(got["inside"][o], ref["inside"], err_msg=f"{msg} inside")
    np.testing.assert_array_equal(got["lin_rgb"][o], _round8(ref["lin_rgb8"]), err_msg=f"{msg} lin rgb")
    ins = ref["inside"].astype(bool)
    lin = got["lin_height"][o]
    np.testing.assert_array_equal(lin[~ins], ref["lin_height"][~ins].astype(np.float32),
                                  err_msg=f"{msg} lin height outside")
    # inside: h = fma(zc, fl(z_scale), fl(z_offset)), zc the exact quotient rounded to
    # float: |error| <= 2^-24 (2.01 |zc z_scale| + |z_offset| + |h|), with
    # |zc z_scale| <= |h| + |z_offset|
    zo = abs(region.z_offset)
    tol = 4.0 * 2.0 ** -24 * (np.abs(ref["lin_height"][ins]) + zo) + 1e-7
    err = np.abs(lin[ins].astype(np.float64) - ref["lin_height"][ins])
    assert (err <= tol).all(), f"{msg} lin height error {err.max():.3e} m (tol {tol.max():.3e})"
    return ref


def bucket(region, x, y, z, rgb=None, seed=0):
    """Samples bucketed by tile (stable: the given order inside a tile)."""
    x = np.asarray(x, np.int64)
    y = np.asarray(y, np.int64)
    lx, ly = x - region.x0_cm, y - region.y0_cm
    t = (ly // region.tile_cm) * region.tiles_x + lx // region.tile_cm
    order = np.argsort(t, kind="stable")
    if rgb is None:
        rgb = np.random.default_rng(seed).integers(0, 65536, size=(len(x), 3))
    rgb = np.asarray(rgb)
    out = {"x": x[order].astype(np.int32), "y": y[order].astype(np.int32),
           "z": np.asarray(z, np.int64)[order].astype(np.int32)}
    for c, k in enumerate("rgb"):
        out[k] = rgb[order, c].astype(np.uint16)
    off = np.zeros(region.n_tiles + 1, np.int64)
    np.add.at(off, t + 1, 1)
    out["tile_offsets"] = np.cumsum(off)
    return out


def test_region_3x3_synthetic_samples(lsb):
    """9 tiles of the chunk-sample workload (about 2M points per tile, 40 samples per
    tile, 60-140 per padded window): the 96- and 192-sample tiers run."""
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=120.25)
    counts = synth.lognormal_counts(5, 9, mu=np.log(5.0), sigma=0.5)
    samples = synth.region_samples(7, region, counts)
    got, st = run_gpu(lsb, samples, region)
    assert st == 0
    for t in range(9):
        check_patch(got, t, samples, region, t, msg=f"tile {t}")


def test_big_tier_dense_windows(lsb):
    """Windows of 250-450 samples (the 384- and 1536-sample tiers), tile subset in
    reverse order."""
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = np.full(9, 9_000_000, np.int64)
    samples = synth.region_samples(11, region, counts)
    tiles = [4, 0, 5]
    got, st = run_gpu(lsb, samples, region, tile_ids=tiles)
    assert st == 0
    for o, t in enumerate(tiles):
        check_patch(got, o, samples, region, t, msg=f"tile {t}")


@pytest.mark.parametrize("n", [96, 97, 192, 193, 384, 385])
def test_tier_edges(lsb, n):
    """A window holding exactly n samples, at and just past each tier's capacity (96,
    192, 384 window samples; the next tier takes the patch from a device queue): the
    centre tile of a 3x3 region holds all n samples, and its neighbours' windows see
    the 160 m of it next to them."""
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=7.5)
    rng = np.random.default_rng(n)
    x = region.x0_cm + region.tile_cm + rng.integers(0, region.tile_cm, n)
    y = region.y0_cm + region.tile_cm + rng.integers(0, region.tile_cm, n)
    z = rng.integers(-20000, 90000, n)
    samples = bucket(region, x, y, z, seed=n)
    tiles = [4, 1, 5]
    got, st = run_gpu(lsb, samples, region, tile_ids=tiles)
    assert st == 0
    for o, t in enumerate(tiles):
        check_patch(got, o, samples, region, t, msg=f"n={n} tile {t}")


def _lattice_case(step, jitter_seed=None, dup=0, shuffle_seed=1):
    """Points of a square lattice over the 3x3 region's centre window (co-circular
    quadruples everywhere, points on texel centres, on the window's edges and on its
    corners), shuffled, with optional duplicates."""
    region = synth.Region(tiles_x=3, tiles_y=3, z_offset=-3.5)
    X0 = region.x0_cm + region.tile_cm - PAD
    W = region.tile_cm + 2 * PAD
    g = np.arange(0, W + 1, step)
    gx, gy = np.meshgrid(g, g)
    x = (X0 + gx.ravel()).astype(np.int64)
    y = (region.y0_cm + region.tile_cm - PAD + gy.ravel()).astype(np.int64)
    rng = np.random.default_rng(shuffle_seed)
    z = rng.integers(30000, 60000, size=len(x))
    p = rng.permutation(len(x))
    x, y, z = x[p], y[p], z[p]
    if dup:
        k = rng.integers(0, len(x), size=dup)
        x, y = np.concatenate([x, x[k]]), np.concatenate([y, y[k]])
        z = np.concatenate([z, rng.integers(30000, 60000, size=dup)])
    return region, bucket(region, x, y, z, seed=shuffle_seed)


@pytest.mark.parametrize("step,dup", [(24000, 0), (12000, 5), (8000, 20)])
def test_lattice_cocircular_duplicates_and_window_edges(lsb, step, dup):
    region, samples = _lattice_case(step, dup=dup)
    got, st = run_gpu(lsb, samples, region, tile_ids=[4, 1, 3])
    assert st == 0
    for o, t in enumerate([4, 1, 3]):
        check_patch(got, o, samples, region, t, msg=f"step {step} tile {t}")


def test_texel_centred_points_and_planar_field(lsb):
    """Points on texel centres with a planar height field: the linear map reproduces
    the plane at every inside texel (within the float bound)."""
    region = synth.Region(tiles_x=1, tiles_y=1, z_offset=50.0)
    rng = np.random.default_rng(3)
    n = 70
    j = rng.integers(16, 80, size=n)
    i = rng.integers(16, 80, size=n)
    lx = 1000 * j + 500 - PAD
    ly = 1000 * i + 500 - PAD
    ok = (lx >= 0) & (lx < region.tile_cm) & (ly >= 0) & (ly < region.tile_cm)
    lx, ly = lx[ok], ly[ok]
    z = 2 * lx + 3 * ly + 1000
    samples = bucket(region, region.x0_cm + lx, region.y0_cm + ly, z, seed=3)
    got, st = run_gpu(lsb, samples, region)
    assert st == 0
    ref = check_patch(got, 0, samples, region, 0, msg="texel-centred")
    ins = ref["inside"].astype(bool)
    assert ins.sum() > 500
    c = 1000 * np.arange(RES) + 500
    GX, GY = np.meshgrid(c, c)
    plane = (2 * (GX - PAD) + 3 * (GY - PAD) + 1000) * region.z_scale + region.z_offset
    err = np.abs(got["lin_height"][0][ins] - plane[ins])
    assert err.max() <= 4.0 * 2.0 ** -24 * (np.abs(plane).max() + 50.0) + 1e-7


def test_degenerate_windows(lsb):
    """No sample, one sample, collinear samples (no real triangle: lin = nn, inside 0)."""
    region = synth.Region(tiles_x=3, tiles_y=1)
    x0, y0, tc = region.x0_cm, region.y0_cm, region.tile_cm
    xs = [x0 + 2 * tc + 20000, x0 + 2 * tc + 21000, x0 + 2 * tc + 22000, x0 + 2 * tc + 23000]
    ys = [y0 + 500, y0 + 1500, y0 + 2500, y0 + 3500]  # collinear, in tile 2
    xs = [x0 + tc // 2] + xs  # one sample in tile 0
    ys = [y0 + tc // 2] + ys
    zs = [40000, 41000, 42000, 43000, 44000]
    samples = bucket(region, xs, ys, zs, seed=9)
    # tile 1's window reaches neither tile 0's sample (320 m away, pad 160 m) nor tile 2's
    got, st = run_gpu(lsb, samples, region)
    assert st == 0
    assert np.isnan(got["nn_height"][1]).all() and np.isnan(got["lin_height"][1]).all()
    assert (got["nn_rgb"][1] == 0).all() and (got["inside"][1] == 0).all()
    assert int(got["tri_count"][1]) == 2
    for t in range(3):
        ref = check_patch(got, t, samples, region, t, msg=f"tile {t}")
        assert ref["inside"].sum() == 0
    assert np.unique(got["nn_height"][0]).size == 1


def test_window_over_capacity_reports_and_writes_nan(lsb):
    region = synth.Region(tiles_x=1, tiles_y=1)
    rng = np.random.default_rng(4)
    n = 1700
    x = region.x0_cm + rng.integers(0, region.tile_cm, n)
    y = region.y0_cm + rng.integers(0, region.tile_cm, n)
    samples = bucket(region, x, y, rng.integers(0, 50000, n), seed=4)
    got, st = run_gpu(lsb, samples, region)
    assert st == -3
    assert np.isnan(got["nn_height"][0]).all() and int(got["tri_count"][0]) == -1


def test_deterministic(lsb):
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = np.full(9, 4_000_000, np.int64)
    samples = synth.region_samples(13, region, counts)
    a, _ = run_gpu(lsb, samples, region)
    b, _ = run_gpu(lsb, samples, region)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_overview_full_size_sampled(lsb):
    """The 200 x 200-tile overview (4 pts/m^2, 33 samples per tile), all 40,000 tiles
    in one call; 8 seeded tiles checked against the oracle."""
    import torch
    from synth import gpu as sg
    region, counts = synth.overview_workload()
    s = sg.region_samples(3, region, counts, device="cuda")
    out = lsb.fill_interp(s, region, res=RES, pad_cm=PAD, tri_cap=512)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    host = {k: v.cpu().numpy() for k, v in s.items()}
    got = {k: v.cpu().numpy() for k, v in out.items()}
    rng = np.random.default_rng(21)
    tiles = list(rng.choice(region.n_tiles, size=6, replace=False)) + [0, region.n_tiles - 1]
    for t in tiles:
        check_patch(got, int(t), host, region, int(t), msg=f"overview tile {t}")


def test_slivers_and_extreme_heights(lsb):
    """Nearly collinear clusters (sliver triangles whose height and colour steps per
    texel are huge) with heights near +-2^27 cm and extreme colours."""
    region = synth.Region(tiles_x=1, tiles_y=1, z_offset=7.0)
    rng = np.random.default_rng(17)
    n = 60
    t = rng.integers(0, region.tile_cm, n)
    lx = t
    # around the texel-centre row at y = 31500 (window y 47500)
    ly = 31500 + (t // 7) % 3 - 1 + rng.integers(-2, 3, n) * (rng.random(n) < 0.2)
    z = rng.choice([-(2 ** 27) + 5, 2 ** 27 - 5, 0, 12345], size=n)
    rgb = rng.choice([0, 65535, 32768, 127], size=(n, 3))
    samples = bucket(region, region.x0_cm + lx, region.y0_cm + ly, z, rgb=rgb)
    got, st = run_gpu(lsb, samples, region)
    assert st == 0
    ref = check_patch(got, 0, samples, region, 0, msg="slivers")
    assert ref["inside"].sum() > 0
