/*
 * lidarscout.h -- C ABI of the B300 (sm_103a) per-tile heightmap build.
 *
 * The calls follow the problem statement of LidarScout (Erler, Herzberger, Wimmer,
 * Schuetz, HPG 2025): chunk points P with heights h and optional colours rgb, a grid
 * resolution res, and 64x64 height + 64x64x3 texture outputs per 640 m patch
 * (Algorithm 1 inputs; Sec. 3.2-3.4), full-resolution points updating the heightmap
 * textures (abstract; Sec. 3.5).
 *
 * Terminology: a "tile" here is the paper's "patch": a square of side tile_cm on a
 * regular grid of tiles_x * tiles_y tiles, tile index t = ty * tiles_x + tx.
 * A per-tile grid is [cells][cells], row i along y, column j along x.
 *
 * Conventions for every call:
 *  - Coordinates are int32 centimetres (LAS integers at scale 0.01); colours are
 *    16-bit LAS RGB.  z in metres = z_cm * z_scale + z_offset.
 *  - Every data pointer is a DEVICE pointer owned by the caller (e.g. a PyTorch
 *    tensor); the library never frees caller memory.  Opaque handles (ls_model)
 *    are owned by the library and released with their destroy call.
 *  - Calls are asynchronous on the given CUDA stream.  Arguments are validated on
 *    the host before anything is launched; a bad argument returns an error code
 *    and launches nothing.  Conditions found on the device (a bounded wait that ran
 *    out, a capacity exceeded) are recorded in a per-device sticky status word that
 *    ls_last_error() reads (it synchronises the device) and clears.
 *  - Some calls use a library-owned scratch workspace, allocated with cudaMalloc on
 *    the first call that needs it (per device) and grown when a larger size is
 *    needed.  Make one call of each kind with the largest sizes before capturing
 *    calls into a CUDA graph.  ls_release_workspace() frees it.
 *  - No C++ exception crosses this interface.
 */
#ifndef LIDARSCOUT_H
#define LIDARSCOUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ls_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef int32_t ls_status;
#define LS_OK 0
#define LS_ERR_INVALID_ARG (-1)  /* bad pointer, size, alignment or parameter          */
#define LS_ERR_CUDA (-2)         /* a CUDA runtime call failed                          */
#define LS_ERR_OUT_OF_RANGE (-3) /* an output capacity was exceeded on the device       */
#define LS_ERR_TIMEOUT (-4)      /* a bounded device-side wait ran out                  */
#define LS_ERR_NO_MEMORY (-5)    /* workspace allocation failed                         */
#define LS_ERR_UNSUPPORTED (-6)  /* valid but unsupported configuration                 */

/* Point set, structure of arrays, n points (device pointers, 4-byte and 2-byte
 * aligned).  Points of one tile are expected to be stored together and, within a
 * tile, in the scanner's strip order (LAZ storage order, Sec. 3.1): the binning is
 * exact for any order, but fastest for that one.  tile_offsets (optional, int64[T+1],
 * device) is a CSR that lists, for each tile, the range of its points (or, for a
 * sample set, of its samples). */
typedef struct {
  const int32_t *x, *y, *z;
  const uint16_t *r, *g, *b;
  int64_t n;
  const int64_t *tile_offsets;
} ls_points;

/* Regular tile grid.  A point with x - x0_cm outside [0, tiles_x * tile_cm) (or the
 * same for y) lies outside the region.  tiles_x * tile_cm and tiles_y * tile_cm must
 * be below 2^31. */
typedef struct {
  int64_t x0_cm, y0_cm;
  int32_t tile_cm;  /* 64000 for 640 m tiles */
  int32_t tiles_x, tiles_y;
  double z_scale;   /* 0.01 */
  double z_offset;
} ls_region;

/* Per-cell accumulators of one grid level, [T][cells][cells] each (device).
 * Empty cell: count 0, zsum 0, zmin INT32_MAX, zmax INT32_MIN, colour sums 0. */
typedef struct {
  int32_t cells;    /* cells per tile side; tile_cm must be divisible by it */
  uint32_t *count;
  int64_t *zsum;
  int32_t *zmin, *zmax;
  uint64_t *rsum, *gsum, *bsum;
} ls_bins;

/* Gaussian-fill parameters (radius 120 m, sigma 40 m in the reference workload). */
typedef struct {
  int32_t res;       /* texels per tile side, tile_cm divisible by it, 8..256   */
  int32_t radius_cm; /* splat radius R, 1..tile_cm (inclusive d <= R)          */
  float sigma_cm;    /* Gaussian sigma, > 0                                      */
} ls_fill_params;

/* ---------------------------------------------------------------------------------
 * ls_bin_points -- exact full-resolution binning (Sec. 3.4: ground truth is the mean
 * of all points falling onto a texel; Sec. 3.5 and abstract: full-resolution points
 * update the heightmap textures).  For every cell of every tile of the region:
 * count, sum z (int64), min z, max z, sums of R, G, B (uint64).  Bit-exact for any
 * point order.
 *
 * levels[0..n_levels-1]: one or two grid levels; with two, levels[1].cells must
 * divide levels[0].cells (e.g. 640 = 1 m cells and 64 = 10 m cells); the coarse
 * level is reduced exactly from the fine one.  All outputs are overwritten.
 * dropped: device uint64[1] or NULL; receives the number of points outside the
 * region.  pts->tile_offsets is not needed and ignored.
 * Uses library scratch (per-row states) of 4 bytes per fine row of the region.
 * Errors: LS_ERR_INVALID_ARG (null pointer, cells not dividing tile_cm, > 2 levels,
 * fine level over 4096 cells), LS_ERR_NO_MEMORY, LS_ERR_CUDA.  A bounded device wait
 * that ran out sets LS_ERR_TIMEOUT in the sticky status.
 * ------------------------------------------------------------------------------- */
ls_status ls_bin_points(const ls_points *pts, const ls_region *region, const ls_bins *levels,
                        int32_t n_levels, uint64_t *dropped, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * ls_extract_samples -- the chunk points (Sec. 3.1, 3.2): LAZ stores points in
 * chunks of `chunk` (50,000) consecutive points whose first point is uncompressed;
 * sample k of tile t is point tile_offsets[t] + chunk * k.
 * pts->tile_offsets (int64[n_tiles+1], device) is required.
 * Writes sample_offsets (int64[n_tiles+1], device): the CSR of samples by tile, and
 * the samples themselves into the six arrays of *out (capacity entries each).
 * If the total exceeds capacity, only the first `capacity` samples are written and
 * the sticky status gets LS_ERR_OUT_OF_RANGE.  A capacity of
 * pts->n / chunk + n_tiles always suffices.
 * ------------------------------------------------------------------------------- */
typedef struct {
  int32_t *x, *y, *z;
  uint16_t *r, *g, *b;
} ls_sample_buffers;

ls_status ls_extract_samples(const ls_points *pts, int64_t n_tiles, int32_t chunk,
                             int64_t *sample_offsets, const ls_sample_buffers *out,
                             int64_t capacity, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * ls_fill_sparse -- Gaussian-weighted neighbourhood fill of res x res texels per
 * tile from the sparse samples (the High-Quality Splatting baseline of Sec. 4.2:
 * fixed-size splats blended with a Gaussian).  Texel centre c; candidates are
 * samples with |s - c|^2 <= R^2 (exact integer distance); w = exp(-|s-c|^2/(2 sigma^2));
 * height = z_ref + sum w (z - z_ref) / sum w with z_ref the nearest sample's z;
 * colour = (sum w c / sum w) / 256, rounded half up to 8 bits.  With no candidate, the
 * texel copies its nearest sample (ties: lowest sample index).  No sample at all:
 * height NaN, colour 0.
 *
 * samples: bucketed by tile: samples->tile_offsets (int64[T+1], device) is required
 *   and every sample of bucket t must lie in tile t (samples outside the region must
 *   not be listed).  Sample order inside a bucket is the tie-break order.
 * tile_ids: int32[n_out] (device) tiles to fill, or NULL for all T tiles (n_out = T).
 * height: float[n_out][res][res] metres; rgb: uint8[n_out][res][res][3] (device).
 * Uses library scratch of 16 bytes per sample.  A sample found outside its bucket's
 * tile sets LS_ERR_INVALID_ARG in the sticky status.
 * ------------------------------------------------------------------------------- */
ls_status ls_fill_sparse(const ls_points *samples, const ls_region *region,
                         const ls_fill_params *params, const int32_t *tile_ids, int64_t n_out,
                         float *height, uint8_t *rgb, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * ls_update_tile -- tile update with full-resolution data (abstract; Sec. 3.5).
 * For each requested tile and texel with count > 0 in bins (one level, cells = res of
 * the maps): height = (float)((double)zsum / count * z_scale + z_offset) and
 * colour = min(255, floor((double)csum / count / 256 + 0.5)); texels with count 0
 * keep their value.  Bit-exact (IEEE fp64 division, no contraction).
 * tile_ids: int32[n] (device), or NULL for tiles 0..n-1; height/rgb are [n] maps.
 * ------------------------------------------------------------------------------- */
ls_status ls_update_tile(const ls_bins *bins, const ls_region *region, const int32_t *tile_ids,
                         int64_t n, float *height, uint8_t *rgb, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Status helpers.
 * ------------------------------------------------------------------------------- */
const char *ls_status_string(ls_status s);
/* Synchronises the current device, returns and clears its sticky device status. */
ls_status ls_last_error(void);
/* Frees the library scratch workspace of the current device (synchronises it). */
ls_status ls_release_workspace(void);
/* Library version as major * 10000 + minor * 100 + patch. */
int32_t ls_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIDARSCOUT_H */
