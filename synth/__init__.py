"""Seeded synthetic LiDAR-like inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the heightmap method itself (no binning, no fill,
no network).  It only draws the inputs: int32-quantised LAS-style points
(x, y, z in centimetres, 16-bit RGB) on fBm terrain, ordered the way a LAZ tile
stores them, and the per-tile point counts of the workloads.

Every value is computed in integer arithmetic from a counter-based hash, so this
numpy implementation and the CUDA generator in ``synth/synth_gpu.cu`` produce
bit-identical points for the same (seed, tile, point index).  The definition:

* ``mix64`` is the SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014;
  public constants 0xBF58476D1CE4E5B9, 0x94D049BB133111EB, 0x9E3779B97F4A7C15).
  ``H(s, v) = mix64(s + mix64(v))`` with wrap-around 64-bit arithmetic.
* Terrain: value-noise fBm with 6 octaves, total amplitude 80 m (8000 cm for
  octave 0, halved per octave: gain 0.5), base wavelength 2 km (200000 cm, halved
  per octave: lacunarity 2).  Lattice value of octave o at lattice point (i, j):
  ``(H(H(H(seed ^ SALT_TERRAIN, o), i), j) >> 48) - 32768``.  Interpolation uses the
  cubic fade ``f(t) = t^2 (3 - 2t)`` in Q16 fixed point and floor shifts.
  ``z = 50000 + sum_o ((8000 >> o) * n_o >> 15) + scan_noise`` with
  ``scan_noise`` uniform in [-16, 15] cm.
* Tile point stream (the order of a LAZ file): tile t with N_t points is cut into
  80 row strips of 8 m; strip s holds ``N_t // 80`` points (+1 for the first
  ``N_t % 80`` strips), and point k of the stream lies uniformly at random in its
  strip.  Chunks are 50,000 consecutive points of that stream.
* RGB: a height ramp ``q = clip(z - 34000, 0, 32000) * 65535 // 32000`` with
  R = q, G = q // 2 + 16384, B = 65535 - q, each plus Irwin-Hall (n = 12) noise
  with standard deviation 2000, clamped to [0, 65535].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
C1 = np.uint64(0xBF58476D1CE4E5B9)
C2 = np.uint64(0x94D049BB133111EB)

SALT_TERRAIN = 0x5445525241494E31  # "TERRAIN1"
SALT_POINTS = 0x504F494E54535F31   # "POINTS_1"

TILE_CM = 64000        # 640 m tiles
STRIPS = 80            # 8 m row strips per tile
STRIP_CM = 800
CHUNK = 50000          # LAZ chunk size in points
Z_BASE = 50000         # 500 m base elevation
OCTAVES = 6
AMP0 = 8000            # 80 m
LAMBDA0 = 200000       # 2 km

# hash lanes per point
LANE_X, LANE_Y, LANE_ZN, LANE_RGB = 0, 1, 2, 3   # LANE_RGB .. LANE_RGB + 8 (9 lanes)


def _u64(a):
    return np.asarray(a).astype(np.uint64, copy=False)


def mix64(z):
    """SplitMix64 output function on uint64 arrays (wrap-around)."""
    z = _u64(z)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * C1
        z = (z ^ (z >> np.uint64(27))) * C2
        z = z ^ (z >> np.uint64(31))
    return z


def H(s, v):
    """Two-argument counter hash: mix64(s + mix64(v))."""
    with np.errstate(over="ignore"):
        return mix64(_u64(s) + mix64(v))


def _as_u64_signed(a):
    """int64 -> uint64 two's-complement view (for hashing lattice indices)."""
    return np.asarray(a, dtype=np.int64).view(np.uint64)


def _lattice(seed: int, octave: int, ix, iy):
    h = H(H(H(np.uint64(seed) ^ np.uint64(SALT_TERRAIN), np.uint64(octave)),
            _as_u64_signed(ix)), _as_u64_signed(iy))
    return (h >> np.uint64(48)).astype(np.int64) - 32768


def _fade_q16(t):
    # t in [0, 65536): f = t^2 (3*65536 - 2t) >> 32, fits int64
    return (t * t * (3 * 65536 - 2 * t)) >> 32


def terrain_z(seed: int, x, y):
    """fBm terrain height (cm, int64) at global integer coordinates (cm)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    z = np.zeros(np.broadcast(x, y).shape, dtype=np.int64)
    for o in range(OCTAVES):
        lam = LAMBDA0 >> o
        ix = np.floor_divide(x, lam)
        iy = np.floor_divide(y, lam)
        fx = _fade_q16(((x - ix * lam) << 16) // lam)
        fy = _fade_q16(((y - iy * lam) << 16) // lam)
        v00 = _lattice(seed, o, ix, iy)
        v10 = _lattice(seed, o, ix + 1, iy)
        v01 = _lattice(seed, o, ix, iy + 1)
        v11 = _lattice(seed, o, ix + 1, iy + 1)
        a = v00 + (((v10 - v00) * fx) >> 16)
        b = v01 + (((v11 - v01) * fx) >> 16)
        n = a + (((b - a) * fy) >> 16)
        z += ((AMP0 >> o) * n) >> 15
    return z


@dataclasses.dataclass(frozen=True)
class Region:
    """Regular grid of square tiles; integer centimetre coordinates."""
    x0_cm: int = 50_000_000       # 500 km easting, UTM-like
    y0_cm: int = 400_000_000      # 4000 km northing
    tile_cm: int = TILE_CM
    tiles_x: int = 1
    tiles_y: int = 1
    z_scale: float = 0.01
    z_offset: float = 0.0

    @property
    def n_tiles(self) -> int:
        return self.tiles_x * self.tiles_y


def strip_of(idx, n_points: int):
    """Strip index (0..79) of stream position idx in a tile holding n_points."""
    idx = np.asarray(idx, dtype=np.int64)
    q, rem = divmod(int(n_points), STRIPS)
    big = rem * (q + 1)
    if q == 0:
        return idx.copy()
    return np.where(idx < big, idx // (q + 1), rem + (idx - big) // q)


def _irwin_hall_noise(h3):
    """Sum of 12 16-bit uniforms from three 64-bit hashes -> N(0, 2000)-like int."""
    s = np.zeros(h3[0].shape, dtype=np.int64)
    for h in h3:
        for k in range(4):
            s += ((h >> np.uint64(16 * k)) & np.uint64(0xFFFF)).astype(np.int64)
    return np.floor_divide((s - 393210) * 2000, 65536)


def tile_points(seed: int, region: Region, tile: int, n_points: int,
                start: int = 0, count: int | None = None):
    """Points [start, start+count) of tile `tile`'s stream (LAZ storage order).

    Returns int32 x, y, z (cm) and uint16 r, g, b arrays."""
    if count is None:
        count = n_points - start
    return _points_at(seed, region, tile, n_points,
                      np.arange(start, start + count, dtype=np.int64))


def region_points(seed: int, region: Region, counts):
    """All points of a region, tiles in row-major order, each in stream order.

    Returns dict with x, y, z, r, g, b arrays and tile_offsets (int64, T+1)."""
    counts = np.asarray(counts, dtype=np.int64)
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    parts = [tile_points(seed, region, t, int(n)) for t, n in enumerate(counts)]
    out = {k: np.concatenate([p[i] for p in parts]) if parts else np.zeros(0)
           for i, k in enumerate(("x", "y", "z", "r", "g", "b"))}
    out["tile_offsets"] = offs
    return out


def chunk_sample_count(n_points: int, chunk: int = CHUNK) -> int:
    return (int(n_points) + chunk - 1) // chunk


def region_samples(seed: int, region: Region, counts, chunk: int = CHUNK):
    """First point of every chunk of every tile, generated directly (no full points).

    Sample k of tile t is stream point chunk*k of tile t.  Returns the same dict
    layout as region_points, with tile_offsets giving the CSR of samples by tile."""
    counts = np.asarray(counts, dtype=np.int64)
    ns = (counts + chunk - 1) // chunk
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(ns)
    total = int(offs[-1])
    tile = np.repeat(np.arange(len(counts), dtype=np.int64), ns)
    k = np.arange(total, dtype=np.int64) - offs[tile]
    out = {}
    names = ("x", "y", "z", "r", "g", "b")
    step = 1 << 20
    parts = [_points_at(seed, region, tile[a:a + step], counts[tile[a:a + step]], k[a:a + step] * chunk)
             for a in range(0, total, step)]
    dt = {"x": np.int32, "y": np.int32, "z": np.int32, "r": np.uint16, "g": np.uint16, "b": np.uint16}
    for i, name in enumerate(names):
        out[name] = np.concatenate([p[i] for p in parts]) if parts else np.zeros(0, dtype=dt[name])
    out["tile_offsets"] = offs
    return out


def _strip_of_multi(idx, n_points):
    """strip_of for per-point stream positions and per-point tile sizes."""
    q, rem = np.divmod(n_points, STRIPS)
    big = rem * (q + 1)
    qs = np.maximum(q, 1)
    return np.where(q == 0, idx, np.where(idx < big, idx // (q + 1), rem + (idx - big) // qs))


def _points_at(seed: int, region: Region, tile, n_points, idx):
    """Stream points at positions idx of tiles `tile` holding n_points points each
    (tile and n_points may be scalars or arrays broadcast against idx)."""
    idx = np.asarray(idx, dtype=np.int64)
    tile = np.broadcast_to(np.asarray(tile, dtype=np.int64), idx.shape)
    n_points = np.broadcast_to(np.asarray(n_points, dtype=np.int64), idx.shape)
    tx, ty = tile % region.tiles_x, tile // region.tiles_x
    key = H(np.uint64(seed) ^ np.uint64(SALT_POINTS), tile.astype(np.uint64))
    base = H(key, idx.view(np.uint64))
    lane = lambda k: H(base, np.uint64(k))        # noqa: E731
    s = _strip_of_multi(idx, n_points)
    lx = (lane(LANE_X) % np.uint64(region.tile_cm)).astype(np.int64)
    ly = s * STRIP_CM + (lane(LANE_Y) % np.uint64(STRIP_CM)).astype(np.int64)
    gx = region.x0_cm + tx * region.tile_cm + lx
    gy = region.y0_cm + ty * region.tile_cm + ly
    zn = (lane(LANE_ZN) >> np.uint64(59)).astype(np.int64) - 16
    z = Z_BASE + terrain_z(seed, gx, gy) + zn
    q = np.clip(z - 34000, 0, 32000) * 65535 // 32000
    ramps = (q, q // 2 + 16384, 65535 - q)
    rgb = []
    for c in range(3):
        hs = [lane(LANE_RGB + 3 * c + k) for k in range(3)]
        rgb.append(np.clip(ramps[c] + _irwin_hall_noise(hs), 0, 65535).astype(np.uint16))
    return (gx.astype(np.int32), gy.astype(np.int32), z.astype(np.int32),
            rgb[0], rgb[1], rgb[2])


def lognormal_counts(seed: int, n_tiles: int, mu: float = math.log(4.0),
                     sigma: float = 0.8, tile_m: float = 640.0):
    """Per-tile point counts: density ~ lognormal(mu, sigma) points/m^2."""
    rng = np.random.default_rng(seed)
    dens = np.exp(mu + sigma * rng.standard_normal(n_tiles))
    return np.rint(dens * tile_m * tile_m).astype(np.int64)


def uniform_counts(n_tiles: int, density: float, tile_m: float = 640.0):
    return np.full(n_tiles, int(round(density * tile_m * tile_m)), dtype=np.int64)


# --------------------------------------------------------------------------------
# Workloads (sizes and structure of the heightmap-build configurations)
# --------------------------------------------------------------------------------

def single_tile_workload(seed: int = 1):
    """One 640 m tile, 2,000,000 points (4.88 pts/m^2), 40 chunks of 50,000."""
    region = Region(tiles_x=1, tiles_y=1)
    return region, np.array([2_000_000], dtype=np.int64)


def batched_region_workload(seed: int = 2, tiles: int = 16):
    """16x16 tiles (10.24 km square), density lognormal(ln 4, 0.8) pts/m^2."""
    region = Region(tiles_x=tiles, tiles_y=tiles)
    return region, lognormal_counts(seed, tiles * tiles)


def overview_workload(tiles: int = 200, density: float = 4.0):
    """200x200 tiles (128 km square) at 4 pts/m^2: 1,638,400 points and 33 chunk
    samples per tile."""
    region = Region(tiles_x=tiles, tiles_y=tiles)
    return region, uniform_counts(tiles * tiles, density)
