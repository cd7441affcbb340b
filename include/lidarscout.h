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
  int32_t res;       /* texels per tile side, tile_cm divisible by it, 8..1024
                        (multiple of 8)                                          */
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
 * Uses library scratch of 4 bytes per fine row of the region (per-row states) plus a
 * 4-byte work counter.
 * Errors: LS_ERR_INVALID_ARG (null pointer, cells not dividing tile_cm, > 2 levels,
 * fine level over 4096 cells), LS_ERR_NO_MEMORY, LS_ERR_CUDA.  A bounded device wait
 * that ran out sets LS_ERR_TIMEOUT in the sticky status.
 * ------------------------------------------------------------------------------- */
ls_status ls_bin_points(const ls_points *pts, const ls_region *region, const ls_bins *levels,
                        int32_t n_levels, uint64_t *dropped, ls_stream_t stream);

/* ls_bin_points_fixed_scratch -- the same binning and results as ls_bin_points, for
 * callers that cannot allocate device memory during the call: an interactive viewer
 * that bins streamed full-resolution tiles between frames must not pay the device
 * synchronisation of cudaMalloc/cudaFree, and an application whose device memory is
 * fully reserved by its own allocator has none to give.  The paper has no
 * counterpart; this is a service of this library.  The per-row scratch is a fixed
 * array of 2^20 rows (4 MiB) compiled into the library, held by every GPU that loads
 * it until the process exits; regions with more than 2^20 fine rows (tiles *
 * levels[0].cells) are rejected with LS_ERR_UNSUPPORTED.  Nothing is allocated: the
 * first call on a device looks up the array's device address and caches it (make
 * that first call before any stream capture; ls_release_workspace drops the cache,
 * which a device reset makes stale).  All calls share the array, which keeps the last
 * call's contents (every call clears the states it uses): calls that overlap on the
 * GPU, on any streams, race and must be serialised by the caller. */
ls_status ls_bin_points_fixed_scratch(const ls_points *pts, const ls_region *region,
                                      const ls_bins *levels, int32_t n_levels, uint64_t *dropped,
                                      ls_stream_t stream);

/* ls_bin_points_accumulate -- ls_bin_points for points that arrive over several calls
 * (Sec. 3.5: the full-resolution points of a tile reach the viewer chunk by chunk while
 * it is on screen, and each chunk refines the tile's texels).  Adds this call's points
 * into the existing accumulators of both levels: counts and the z and colour sums
 * add, zmin / zmax take the minimum / maximum; cells without new points keep their
 * values.  The bins must hold valid accumulators (an earlier ls_bin_points or
 * ls_bin_points_accumulate call, or the empty-cell values).  The result equals one
 * ls_bin_points call over the union of the points, bit for bit, in any split and
 * order.  dropped: device uint64[1] or NULL, incremented by the number of this call's
 * points outside the region.  Every touched row is merged with global atomics, so a
 * call costs more per point than ls_bin_points.  Scratch and errors as ls_bin_points. */
ls_status ls_bin_points_accumulate(const ls_points *pts, const ls_region *region,
                                   const ls_bins *levels, int32_t n_levels, uint64_t *dropped,
                                   ls_stream_t stream);

/* Diagnostics of ls_bin_points, cumulative over calls (synchronous copy):
 * out[0] points that arrived after their row left the CTA's window (merged with
 * global atomics), out[1] waits on a row another CTA was writing, out[2] such waits
 * that ran out, out[3] in-place window flushes forced by the residency bound.
 * reset != 0 clears the counters after reading. */
ls_status ls_bin_stats(uint64_t *out, int32_t reset);

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
 * Launch shapes and their autotuner.  The paper processes its patches in batches
 * because batching pays off (Sec. 4.2); the batched launches here have shape
 * parameters whose best values depend on the workload, chosen by measurement.
 *
 * A call's key is made of the arguments that decide its best shape: for binning the
 * number of levels, their cell counts and floor(log2(n points)); for the fill the
 * resolution, the radius, floor(log2(n_out)) and floor(log2(n samples)).  A table
 * (per process, up to 256 keys, the oldest replaced) maps keys to shapes; a call whose
 * key has no entry uses the default shape.  Lookups are host-only: calls stay
 * asynchronous and capturable in CUDA graphs.
 * ------------------------------------------------------------------------------- */
typedef struct {
  int32_t spans_per_cta;     /* work spans per CTA of the binning launch, 1..256 (default 16) */
  int32_t prefetch_batches;  /* L2 prefetch distance of the point stream, in 4096-point
                                batches, 1..4 (default 2) */
} ls_bin_shape;

typedef struct {
  int32_t split;        /* CTAs per tile, each a band of res / split texel rows: 1, or 2
                           or 4 when res is a multiple of 16 * split (default 4 for fewer
                           than 592 tiles and res a multiple of 64, else 1) */
  int32_t ctas_per_sm;  /* resident CTAs per SM the persistent grid is sized for: 1..4
                           (default 4), capped at what fits next to the launch's sample
                           stage (sized from the average samples per tile) */
} ls_fill_shape;

/* The shape a binning call with these arguments uses (the table's entry or the
 * default).  Only pts->n, the levels' cells and n_levels are read (host memory). */
ls_status ls_bin_shape_get(const ls_points *pts, const ls_bins *levels, int32_t n_levels,
                           ls_bin_shape *out);
/* Pins a shape for the key of these arguments; shape NULL removes the entry.
 * LS_ERR_INVALID_ARG for a shape outside the ranges above. */
ls_status ls_bin_shape_set(const ls_points *pts, const ls_bins *levels, int32_t n_levels,
                           const ls_bin_shape *shape);
/* The same for the fill (samples->n, params->res, params->radius_cm and n_out are read). */
ls_status ls_fill_shape_get(const ls_points *samples, const ls_fill_params *params, int64_t n_out,
                            ls_fill_shape *out);
ls_status ls_fill_shape_set(const ls_points *samples, const ls_fill_params *params, int64_t n_out,
                            const ls_fill_shape *shape);
/* Removes every entry. */
ls_status ls_tune_clear(void);

/* Autotuners: time the call on the caller's own data with every candidate shape
 * (binning: spans per CTA 8, 16, 32 x prefetch 1, 2, 3 batches; fill: split 1, 2, 4 x
 * 1, 2 CTAs per SM, the valid ones), store the best for the call's key and return it
 * with its median time in ms per call (best / best_ms may be NULL).  Each candidate
 * runs once untimed, then the candidates are timed round-robin for `reps` rounds of
 * two calls (CUDA events on `stream`), so drifts of clocks or cache state hit all of
 * them alike; the score is the median over the rounds, and a candidate replaces the
 * default shape only when its median is at least 1 % lower.  The outputs end as one
 * call computes them: every shape gives the same results, bit for bit.  Synchronises
 * the stream; LS_ERR_INVALID_ARG while the stream is being captured or for reps
 * outside 1..1000; otherwise the errors of the tuned call. */
ls_status ls_tune_bin_points(const ls_points *pts, const ls_region *region, const ls_bins *levels,
                             int32_t n_levels, uint64_t *dropped, int32_t reps, ls_stream_t stream,
                             ls_bin_shape *best, float *best_ms);
ls_status ls_tune_fill_sparse(const ls_points *samples, const ls_region *region,
                              const ls_fill_params *params, const int32_t *tile_ids, int64_t n_out,
                              float *height, uint8_t *rgb, int32_t reps, ls_stream_t stream,
                              ls_fill_shape *best, float *best_ms);

/* ---------------------------------------------------------------------------------
 * ls_fill_interp -- the interpolated heightmaps of Alg. 1 (Sec. 3.3): for each
 * requested tile, the nearest-neighbour (NN) and the Delaunay-linear maps of the
 * samples in a padded patch, the network inputs of the paper's filler.
 *
 * Patch of tile t: the window of side W = tile_cm + 2 * pad_cm centred on the tile
 * (96 x 96 texels of 10 m around a 640 m tile: pad_cm = 16000, res = 96); texel (i, j)
 * has the centre (cell * j + cell / 2, cell * i + cell / 2) in window coordinates,
 * cell = W / res.  Its points are the samples inside the closed window, in sample
 * order, plus four padding points without data at the window corners.
 *  - Delaunay triangulation of corners and points, inserted in that order
 *    (Bowyer-Watson, exact integer predicates, a point equal to an earlier one is
 *    skipped; with co-circular points the insertion order decides the diagonals).
 *  - lin: in a triangle of three real points, height and colour are the barycentric
 *    interpolation of its vertices (height within a few float ulps of the exact
 *    value, the same value from every triangle containing the texel; colour the exact
 *    round-half-up of the 8-bit value); every other texel takes its NN value.
 *  - nn: height (float)(z * z_scale + z_offset) (IEEE double, no contraction) and
 *    colour round-half-up(c / 256) of the nearest sample (exact squared distance,
 *    ties to the lowest sample index).  A patch without samples gets NaN and 0.
 *  - inside: 1 where the linear map interpolates.
 *
 * samples: bucketed by tile as for ls_fill_sparse (tile_offsets required, every
 *   sample inside its bucket's tile, sample order the tie-break order).
 * tile_ids: int32[n_out] (device), or NULL for all T tiles (n_out = T).
 * out: every map pointer may be NULL (not written):
 *   nn_height, lin_height float[n_out][res][res] metres; nn_rgb, lin_rgb
 *   uint8[n_out][res][res][3]; inside uint8[n_out][res][res] (these three 4-byte
 *   aligned);
 *   triangles int32[n_out][tri_cap][3]: the first tri_cap triangles (counter-
 *   clockwise global sample indices; -1 - c for window corner c, c = 0..3 at
 *   (0, 0), (W, 0), (W, W), (0, W)), tri_count int32[n_out]: the number of triangles
 *   (corner triangles included), -1 for a patch not triangulated.
 * Limits: res a multiple of 8 in [8, 1024]; 0 <= pad_cm <= tile_cm; W divisible by
 *   res and at most 131072 cm (INVALID_ARG / UNSUPPORTED otherwise); |z| < 2^28 (a
 *   patch with a larger |z| gets LS_ERR_UNSUPPORTED in the sticky status, tri_count
 *   -1 and lin = nn); at most 1536 samples per window (more: LS_ERR_OUT_OF_RANGE in
 *   the sticky status and NaN maps for that patch).
 * Uses library scratch of 32 bytes per sample and 12 bytes per requested tile.
 * ------------------------------------------------------------------------------- */
typedef struct {
  int32_t res;    /* texels per patch side (96) */
  int32_t pad_cm; /* padding on every side of the tile (16000) */
} ls_interp_params;

typedef struct {
  float *nn_height;
  uint8_t *nn_rgb;
  float *lin_height;
  uint8_t *lin_rgb;
  uint8_t *inside;
  int32_t *triangles;
  int32_t *tri_count;
  int32_t tri_cap;
} ls_interp_outputs;

ls_status ls_fill_interp(const ls_points *samples, const ls_region *region,
                         const ls_interp_params *params, const int32_t *tile_ids, int64_t n_out,
                         const ls_interp_outputs *out, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * The paper's own network variant (Sec. 3.4): the linear and NN heightmaps and textures
 * of Alg. 1 (ls_fill_interp) on a res x res patch, encoded independently by four
 * encoders, merged by fully connected layers in two steps, decoded by separate height
 * and texture CNNs, concatenated with the original inputs (the one skip connection),
 * reduced by a final CNN to 5 outputs (height, R, G, B in patch space, and an error
 * bound) and cropped to the centre res/2 x res/2.  The text fixes no layer sizes; the
 * ones used (2,481,733 parameters at res 128, the paper's 2.5M):
 *   encoder (per input: lin height, NN height, lin RGB, NN RGB): 3x3 conv + ReLU + 2x2
 *     max pool with 16, 32, 64, 64 channels, then 3x3 conv + ReLU to 16 at res/16;
 *   fc1 (per input): 16 (res/16)^2 -> 256 + ReLU; fc2: 1024 -> 16 (res/16)^2 + ReLU;
 *   decoder (height, texture): 3x3 conv + ReLU with 64, 32, 32, 16 channels, each
 *     followed by 2x nearest upsampling, then 3x3 conv + ReLU to 16 at res;
 *   final: concat [input 8, height 16, texture 16], 3x3 conv + ReLU to 32 and to 16,
 *     1x1 head to 5.
 * Flat fp32 parameters in that layer order (ls_cnn_layer_info gives kind 0 = 3x3 conv
 * [C_out][3][3][C_in], 1 = fully connected [out][in], 2 = 1x1 head [5][16], each weight
 * block followed by its bias).  x: bf16 [n][res][res][8] (ls_cnn_inputs); y: fp32
 * [n][res/2][res/2][5].  res is 32, 64 or 128; n (and max_batch) a multiple of
 * 128 / (res/16)^2 (2 at res 128).  Every 3x3 convolution, forward and backward, runs on
 * the tensor-core kernels (bf16 operands, fp32 accumulation); the fully connected
 * layers in fp32.  ls_cnn_backward needs a model created with training != 0 and the
 * activations of the last forward (same n).  Loss and optimiser: ls_filler_loss with a
 * zero base, ls_adamw_step.
 * ------------------------------------------------------------------------------- */
typedef struct ls_cnn ls_cnn;

ls_status ls_cnn_create(int32_t res, int32_t max_batch, int32_t training, ls_cnn **out);
void ls_cnn_destroy(ls_cnn *model);
int64_t ls_cnn_param_count(const ls_cnn *model);
int32_t ls_cnn_layer_count(const ls_cnn *model);
ls_status ls_cnn_layer_info(const ls_cnn *model, int32_t layer, int32_t *kind, int32_t *cin, int32_t *cout,
                            int64_t *w_offset, int64_t *b_offset);
/* Pack the conv weights of params into the model's tensor-core operands. */
ls_status ls_cnn_load(ls_cnn *model, const float *params, ls_stream_t stream);
ls_status ls_cnn_forward(ls_cnn *model, const float *params, const uint16_t *x, int32_t n, float *y,
                         ls_stream_t stream);
/* grads (fp32, n_params) = dL/dparams given dy = dL/dy of the last forward.  Reads the
 * x of that forward again (the first layers' weight gradients): the caller keeps it
 * unchanged until this call. */
ls_status ls_cnn_backward(ls_cnn *model, const float *params, const float *dy, int32_t n, float *grads,
                          ls_stream_t stream);
/* Network input from the Alg. 1 maps of n patches (lin/nn height float [n][res][res]
 * metres, lin/nn rgb uint8 [n][res][res][3]): heights (h - c_z) / r_m with c_z the mean of
 * the linear map's 4 central texels (cz fp32 [n] out), colours / 255, NaN heights 0;
 * x bf16 [n][res][res][8] (16-byte aligned). */
ls_status ls_cnn_inputs(const float *lin_height, const float *nn_height, const uint8_t *lin_rgb,
                        const uint8_t *nn_rgb, int64_t n, int32_t res, float r_m, uint16_t *x, float *cz,
                        ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Software rasterizers into a headless framebuffer (Sec. 3.5, rendering): points
 * with a 64-bit depth|colour atomicMin per pixel, heightmaps as triangle meshes with
 * the same per-fragment atomicMin, and a resolve pass that extracts the colours into
 * an RGBA8 image (the paper resolves into an OpenGL texture; here a device buffer).
 *
 * Framebuffer: uint64[height][width], row 0 at the bottom (screen y upwards).  A word
 * is (float bits of the depth d in [0, 1]) << 32 | R | G << 8 | B << 16 | 255 << 24;
 * ls_render_clear sets every word to UINT64_MAX (empty).  The smallest word wins: the
 * nearest fragment, equal depths the smaller colour word.  The result does not
 * depend on the order of the fragments (bit-exact).
 *
 * Vertex arithmetic, float32 with one IEEE rounding per operation and no fused
 * operations, in this order:
 *  - camera frame (cm): q = ((float)(x - ox), (float)(y - oy), (float)(z - oz)) for a
 *    point with LAS integers x, y, z (int64 differences); for heightmap texel (i, j)
 *    of tile t with height h (metres): x = x0_cm + tx * tile_cm + cell * j + cell / 2
 *    and y likewise (integers, cell = tile_cm / res), q.z = ((h - (float)z_offset) *
 *    (float)(1 / z_scale)) - (float)oz; a NaN height drops the texel's triangles;
 *  - clip c_r = ((M[r][0] q.x + M[r][1] q.y) + M[r][2] q.z) + M[r][3], M row-major;
 *  - visible iff c_w > 0; ndc = c_xyz / c_w (three IEEE quotients); screen
 *    sx = (ndc_x * 0.5 + 0.5) * width,
 *    sy = (ndc_y * 0.5 + 0.5) * height; depth d = ndc_z * 0.5 + 0.5, kept iff
 *    0 <= d <= 1;
 *  - colours: 16-bit point colours round half up to 8 bits; heightmap colours as given.
 * Points: the pixel (floor(sx), floor(sy)) if inside the framebuffer.
 * Heightmap triangles: each quad of adjacent texel centres (i, j), (i, j + 1),
 *   (i + 1, j + 1), (i + 1, j) gives the triangles (v00, v01, v11) and (v00, v11, v10);
 *   a triangle is drawn when its three vertices are kept.  With A = (x1 - x0)(y2 - y0)
 *   - (y1 - y0)(x2 - x0) (A = 0: nothing) and the pixel centre p = (ix + 0.5, iy + 0.5):
 *   e0 = (x2 - x1)(py - y1) - (y2 - y1)(px - x1), e1 = (x0 - x2)(py - y2) - (y0 - y2)(px - x2),
 *   e2 = (x1 - x0)(py - y0) - (y1 - y0)(px - x0), all negated with A when A < 0; the
 *   pixel is covered iff e0, e1, e2 >= 0 (pixels with floor(min x) <= ix <= floor(max x),
 *   likewise for y, inside the framebuffer, are tested).  l_k = e_k / A; depth
 *   (l0 d0 + l1 d1) + l2 d2; colour channel floor(((l0 c0 + l1 c1) + l2 c2) + 0.5)
 *   clamped to [0, 255].
 * ------------------------------------------------------------------------------- */
typedef struct {
  int64_t origin_cm[3];  /* camera-frame origin in LAS centimetres                  */
  float view_proj[16];   /* row-major 4x4: camera frame (cm) to clip space           */
  int32_t width, height; /* framebuffer size in pixels, 1..16384                      */
} ls_camera;

/* Every framebuffer word to UINT64_MAX. */
ls_status ls_render_clear(uint64_t *fb, int32_t width, int32_t height, ls_stream_t stream);

/* Points (e.g. the chunk samples or full-resolution points): pts->tile_offsets is
 * ignored.  fb: uint64[camera->height][camera->width] (device, 8-byte aligned).  The
 * origin must lie in the int32 range and every point within 2^31 - 1 cm of it on each
 * axis (the differences are taken in 32 bits). */
ls_status ls_render_points(const ls_points *pts, const ls_camera *camera, uint64_t *fb,
                           ls_stream_t stream);

/* Heightmaps: height float[n][res][res] (metres, NaN = no data) and rgb
 * uint8[n][res][res][3] of the tiles tile_ids[n] (device int32, or NULL for 0..n-1) of
 * the region; res in [2, 1024] dividing tile_cm.  Triangles covering more than 1024
 * candidate pixels are drawn by a whole CTA from a shared queue, the others by one
 * thread each. */
ls_status ls_render_heightmaps(const float *height, const uint8_t *rgb, const int32_t *tile_ids,
                               int64_t n, int32_t res, const ls_region *region,
                               const ls_camera *camera, uint64_t *fb, ls_stream_t stream);

/* RGBA8 image uint8[height][width][4] (device, 4-byte aligned) from the framebuffer:
 * the colour word of covered pixels, background (R | G << 8 | B << 16 | A << 24)
 * elsewhere. */
ls_status ls_render_resolve(const uint64_t *fb, int32_t width, int32_t height, uint32_t background,
                            uint8_t *rgba, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Tensor-core 3x3 convolution of the learned filler (Sec. 3.4: a U-Net-inspired CNN
 * refines the heightmaps).  Stride 1, zero padding 1, NHWC BF16 activations, FP32
 * accumulation (tcgen05 kind::f16, M = 128 pixels, N = c_out, K = 9 * c_in).
 * Shapes: c_in a multiple of 8; c_out a multiple of 16 in [16, 256]; w a power of
 * two <= 128; either w*h >= 128 and 128/w divides h, or 128/(w*h) divides n; n*h*w a
 * multiple of 128.  All device pointers 16-byte aligned.
 * ------------------------------------------------------------------------------- */
typedef struct {
  int32_t n, h, w, cin, cout;
} ls_conv_shape;

/* bf16 elements of the packed weight operand of a (cin -> cout) 3x3 conv, -1 if the
 * channel counts are unsupported. */
int64_t ls_conv3x3_packed_elems(int32_t cin, int32_t cout);

/* Pack fp32 weights w[cout][3][3][cin] (OHWI) into the operand layout of
 * ls_conv3x3_forward.  transpose_flip = 1 packs the input-gradient convolution of a
 * layer whose weights are w[cin][3][3][cout] (here cin/cout are the channels of the
 * gradient conv): W'[o][ky][kx][i] = W[i][2-ky][2-kx][o]. */
ls_status ls_conv3x3_pack(const float *w, int32_t cin, int32_t cout, int32_t transpose_flip,
                          uint16_t *packed, ls_stream_t stream);

/* y[p][o] = act(sum_k x_shift[p][k] W[o][k] + bias[o]); act = ReLU if relu != 0; if
 * mask is non-NULL (bf16, same shape as y) outputs whose mask value is not > 0 are
 * zeroed (the ReLU derivative of the backward pass).  bias may be NULL. */
ls_status ls_conv3x3_forward(const uint16_t *x, const uint16_t *packed, const float *bias,
                             const uint16_t *mask, int32_t relu, const ls_conv_shape *shape,
                             uint16_t *y, ls_stream_t stream);

/* Weight and bias gradients of a 3x3 conv (c_in -> c_out <= 128) on the tensor cores:
 * dw[(tap * c_in + i) * c_out + o] += sum_p x_shift(tap)[p][i] * dz[p][o] with tap =
 * 3 * ky + kx (zero padding), db[o] += sum_p dz[p][o] (db may be NULL).  x: layer
 * input bf16 [n][h][w][c_in]; dz: output gradient bf16 [n][h][w][c_out].  dw and db are
 * fp32 and accumulated into (zero them first).  Shapes: c_in a multiple of 8; c_out a
 * multiple of 16 in [16, 128]; w a power of two <= 128; h * w a multiple of 64, or a
 * divisor of 64 whose quotient divides n (64-pixel stages: half rows at w = 128, whole
 * rows, or whole images). */
ls_status ls_conv3x3_wgrad(const uint16_t *x, const uint16_t *dz, const ls_conv_shape *shape,
                           float *dw, float *db, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Learned filler (Sec. 3.4): a U-Net of `levels` levels with widths[l] channels (two
 * 3x3 conv + ReLU per level, 2x2 max pooling, 2x nearest upsampling, skip concatenation
 * [upsampled, skip], 1x1 head with 5 outputs: height, R, G, B residuals added to the
 * Gaussian fill, and a predicted absolute height error).  Input: 5 channels stored as
 * bf16 [n][res][res][8] (channels 5..7 zero).  Parameters are a caller-owned flat fp32
 * device vector: per layer (order e1a, e1b, ..., eLa, eLb, d(L-1)a, d(L-1)b, ..., d1a,
 * d1b, head) W[c_out][k][k][c_in] then b[c_out]; ls_model_layer_info gives offsets.
 * The model handle owns packed bf16 weights and activations for max_batch tiles
 * (allocated by ls_model_create).  Widths: multiples of 16 in [16, 128].
 * ------------------------------------------------------------------------------- */
typedef struct ls_model ls_model;

ls_status ls_model_create(int32_t levels, const int32_t *widths, int32_t res, int32_t max_batch,
                          ls_model **out);
/* ls_model_create with options.  LS_MODEL_RECOMPUTE: activation recomputation per
 * level, to bound the training memory at large batches (batch 256 in the workload).
 * The first conv output of every level (e{l}a, d{l}a) lives in one buffer shared by
 * all levels; ls_filler_forward consumes it at once and ls_filler_backward recomputes
 * it from the level's stored input, one extra conv per level.  The kernels are
 * deterministic, so outputs and gradients are bit-identical to those without the flag.
 * Other flag bits: LS_ERR_INVALID_ARG. */
#define LS_MODEL_RECOMPUTE 1
ls_status ls_model_create_opts(int32_t levels, const int32_t *widths, int32_t res, int32_t max_batch,
                               int32_t flags, ls_model **out);
/* Device memory the model holds (packed weights, activations, gradient buffers). */
size_t ls_model_device_bytes(const ls_model *model);
void ls_model_destroy(ls_model *model);
int64_t ls_model_param_count(const ls_model *model);
int32_t ls_model_layer_count(const ls_model *model);
ls_status ls_model_layer_info(const ls_model *model, int32_t layer, int32_t *cin, int32_t *cout,
                              int32_t *ksize, int64_t *w_offset, int64_t *b_offset);
/* Pack the tensor-core operands from params; call after every parameter update. */
ls_status ls_model_load(ls_model *model, const float *params, ls_stream_t stream);
/* y: fp32 [n][res][res][5].  Keeps the activations for ls_filler_backward. */
ls_status ls_filler_forward(ls_model *model, const float *params, const uint16_t *x, int32_t n,
                            float *y, ls_stream_t stream);
/* Gradients of all parameters (overwrites grads, flat fp32 like params) given
 * dL/dy of the last forward call (same n).  Reads the x of that forward again (the
 * first layer's weight gradient): the caller keeps it unchanged until this call. */
ls_status ls_filler_backward(ls_model *model, const float *params, const float *dy, int32_t n,
                             float *grads, ls_stream_t stream);
/* Loss of Sec. 3.4: masked MSE of height and colour (each squared error clipped to 1),
 * the two averaged, plus bound_weight * mean((y4 - b)^2) with the detached bound target
 * b = |e| (the height error e = base + y0 - target), or, bound_excess = 1, the excess
 * b = max(|e| - |base - target|, 0) of the learned height's error over the base fill's
 * (the bound then predicts how much the learned fill may be worse than its base; the
 * paper has no bound, this is the library's reading).  base, target:
 * [n_px][4] (normalised height, R, G, B in 0..1); mask [n_px] (0: texel without truth).
 * sums: device double[4] scratch; loss: device float[4] (total, height, colour,
 * bound) or NULL; dy: fp32 [n_px][5]. */
ls_status ls_filler_loss(const float *y, const float *base, const float *target, const uint8_t *mask,
                         int64_t n_px, float bound_weight, int32_t bound_excess, double *sums, float *loss,
                         float *dy, ls_stream_t stream);
/* AdamW with decoupled weight decay (Sec. 3.4 uses lr 1e-4, betas 0.9/0.999, eps 1e-5,
 * weight decay 1e-2); step counts from 1. */
ls_status ls_adamw_step(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                        float beta2, float eps, float weight_decay, int32_t step, ls_stream_t stream);

/* Input raster of n tiles (Sec. 3.3/3.4 patch-space normalisation, r = tile_cm/2 in
 * metres, c_z = mean Gaussian-fill height of the 4 central texels): x bf16
 * [n][res][res][8]; base fp32 [n][res][res][4] (normalised fill height, fill R, G, B in
 * 0..1); cz [n]; fill_height/fill_rgb: the Gaussian fill itself; aux: fp32 scratch of
 * 5 * n * res * res.  res <= 128. */
ls_status ls_learned_inputs(const ls_points *samples, const ls_region *region,
                            const ls_fill_params *params, const int32_t *tile_ids, int64_t n,
                            uint16_t *x, float *base, float *cz, float *fill_height, uint8_t *fill_rgb,
                            float *aux, ls_stream_t stream);
/* Training targets from full-resolution bins (cells = res): per texel (mean height in
 * patch space with the tile's cz, mean R, G, B / 65535), mask = count > 0. */
ls_status ls_learned_targets(const ls_bins *bins, const ls_region *region, const int32_t *tile_ids,
                             int64_t n, const float *cz, float *target, uint8_t *mask, ls_stream_t stream);
/* Step a11 (Sec. 3.3/3.4 de-normalisation; the bound is this library's reading, the
 * paper has none).  height = (base + y0) * r + cz, colour = floor(clamp(base + y1..3,
 * 0, 1) * 255 + 0.5); tile bound = RMS(max(y4, 0)) * r metres, where a NaN in y4 makes
 * the bound NaN; tiles whose bound is not <= max_err_m (above it, or NaN) take the
 * Gaussian fill (fill_height, fill_rgb) unchanged.  y: fp32 [n][res][res][5]; base:
 * fp32 [n][res][res][4] (Gaussian height in patch space, colour in 0..1); cz [n] metres;
 * height/rgb may alias fill_height/fill_rgb.  err_bound [n] and used_fallback [n] may
 * be NULL. */
ls_status ls_learned_finish(const float *y, const float *base, const float *cz, int64_t n, int32_t res,
                            const ls_region *region, float max_err_m, const float *fill_height,
                            const uint8_t *fill_rgb, float *height, uint8_t *rgb, float *err_bound,
                            uint8_t *used_fallback, ls_stream_t stream);
/* Whole learned fill of n tiles in batches of the model's max_batch: input raster,
 * network, finish with Gaussian fallback.  scratch: caller-owned device memory of at
 * least ls_fill_learned_scratch_bytes(model) bytes.  tile_ids may be NULL only when
 * n = T <= max_batch. */
size_t ls_fill_learned_scratch_bytes(const ls_model *model);
ls_status ls_fill_learned(ls_model *model, const float *params, const ls_points *samples,
                          const ls_region *region, const ls_fill_params *params_fill,
                          const int32_t *tile_ids, int64_t n, float max_err_m, float *height,
                          uint8_t *rgb, float *err_bound, uint8_t *used_fallback, void *scratch,
                          size_t scratch_bytes, ls_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Status helpers.
 * ------------------------------------------------------------------------------- */
const char *ls_status_string(ls_status s);
/* Synchronises the current device, returns and clears its sticky device status. */
ls_status ls_last_error(void);
/* Failure detection without a GPU fault (the paper has no counterpart).  Every wait
 * of the library's kernels on another thread's progress (binning row states, the
 * fill's and the tensor-core kernels' mbarriers) gives up after a number of polls,
 * sets LS_ERR_TIMEOUT in the sticky status and lets the kernel return.
 * ls_set_spin_limit sets that number for the current device (polls <= 0 restores the
 * default, 2^22); it synchronises the device first, so no kernel of the library runs
 * while the limit changes.  A short limit is meant for tests only: with it, an
 * ordinary wait can run out, and the results of that call are then undefined (the
 * status says so).  Only binning and ls_probe_wait, whose waits poll global memory
 * with no copy in flight, should run under a short limit.
 * ls_probe_wait runs the binning's row wait once, in one thread, on the caller's
 * device flag (4-byte aligned): it returns when *flag == 2, or sets LS_ERR_TIMEOUT
 * when the limit runs out first.  Either way the kernel ends and the context stays
 * usable; the wait counts in ls_bin_stats (out[1], and out[2] when it ran out). */
ls_status ls_set_spin_limit(int32_t polls);
ls_status ls_probe_wait(const uint32_t *flag, ls_stream_t stream);
/* Frees the library scratch workspace of the current device (synchronises it) and
 * forgets the cached device address of the fixed binning scratch.  After a device
 * reset (cudaDeviceReset) every device pointer the library cached is stale: call this
 * before the next library call on that device. */
ls_status ls_release_workspace(void);
/* Library version as major * 10000 + minor * 100 + patch. */
int32_t ls_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIDARSCOUT_H */
