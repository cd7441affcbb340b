/*
 * Plain, slow CPU oracle for the per-tile heightmap build.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no code, header,
 * table or constant with the CUDA path; its inputs come from the seeded generators
 * in synth/ or from literal fixtures, never from the CUDA path.
 *
 * Arithmetic: integers for binning (exact), IEEE fp64 for the fill and the tile
 * update.  Compile with -O1 -ffp-contract=off so that no multiply-add is fused.
 *
 * Conventions (all coordinates are int32 centimetres, as in LAS with scale 0.01):
 *   region: origin (x0, y0), square tiles of side `tile` cm, tiles_x * tiles_y tiles,
 *   tile index t = ty * tiles_x + tx; per-tile grids are [cells][cells], row i = y,
 *   column j = x.  A point with local coordinate lx = x - x0 outside
 *   [0, tiles_x * tile) (same for y) is outside the region.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------
 * Full-resolution binning.
 * The paper builds ground-truth heightmaps as the mean of all points falling onto a
 * texel (Sec. 3.4) and updates the heightmap textures from full-resolution points
 * (abstract; Sec. 3.5).  The per-cell reduction below keeps exact integer sums so
 * the mean can be formed later: count, sum of z, min z, max z, sums of R, G, B.
 * Empty cells: count 0, zsum 0, zmin INT32_MAX, zmax INT32_MIN, colour sums 0.
 * Returns the number of points outside the region (dropped).
 * ------------------------------------------------------------------------------ */
int64_t or_bin_points(const int32_t *x, const int32_t *y, const int32_t *z,
                      const uint16_t *r, const uint16_t *g, const uint16_t *b, int64_t n,
                      int64_t x0, int64_t y0, int64_t tile, int64_t tiles_x, int64_t tiles_y,
                      int64_t cells,
                      uint32_t *count, int64_t *zsum, int32_t *zmin, int32_t *zmax,
                      uint64_t *rsum, uint64_t *gsum, uint64_t *bsum)
{
    const int64_t cell_cm = tile / cells;
    const int64_t ncell = tiles_x * tiles_y * cells * cells;
    for (int64_t c = 0; c < ncell; ++c) {
        count[c] = 0; zsum[c] = 0; zmin[c] = INT32_MAX; zmax[c] = INT32_MIN;
        rsum[c] = 0; gsum[c] = 0; bsum[c] = 0;
    }
    int64_t dropped = 0;
    for (int64_t p = 0; p < n; ++p) {
        const int64_t lx = (int64_t)x[p] - x0;
        const int64_t ly = (int64_t)y[p] - y0;
        if (lx < 0 || ly < 0 || lx >= tiles_x * tile || ly >= tiles_y * tile) {
            ++dropped;
            continue;
        }
        const int64_t tx = lx / tile, ty = ly / tile;          /* non-negative: floor */
        const int64_t j = (lx - tx * tile) / cell_cm;
        const int64_t i = (ly - ty * tile) / cell_cm;
        const int64_t c = ((ty * tiles_x + tx) * cells + i) * cells + j;
        count[c] += 1;
        zsum[c] += z[p];
        if (z[p] < zmin[c]) zmin[c] = z[p];
        if (z[p] > zmax[c]) zmax[c] = z[p];
        rsum[c] += r[p];
        gsum[c] += g[p];
        bsum[c] += b[p];
    }
    return dropped;
}

/* ------------------------------------------------------------------------------
 * Sample extraction: the chunk points.  LAZ compresses a tile's points in chunks of
 * 50,000 and the first point of each chunk is stored uncompressed (Sec. 3.1, 3.2);
 * sample k of a tile is therefore stream point chunk * k of that tile.  Writes the
 * indices of the samples (global point indices) in tile order and returns how many.
 * ------------------------------------------------------------------------------ */
int64_t or_extract_sample_indices(const int64_t *tile_offsets, int64_t n_tiles, int64_t chunk,
                                  int64_t *sample_index, int64_t *sample_offsets)
{
    int64_t s = 0;
    for (int64_t t = 0; t < n_tiles; ++t) {
        sample_offsets[t] = s;
        for (int64_t k = tile_offsets[t]; k < tile_offsets[t + 1]; k += chunk)
            sample_index[s++] = k;
    }
    sample_offsets[n_tiles] = s;
    return s;
}

/* ------------------------------------------------------------------------------
 * Gaussian-weighted neighbourhood fill (the High-Quality Splatting baseline of
 * Sec. 4.2: each chunk point is a fixed-size splat, heights and colours are blended
 * with a Gaussian weight).  For the centre c of texel (i, j) of tile t:
 *   candidates = samples s with |s - c|^2 <= R^2 (exact integer distance, inclusive),
 *   w_s = exp(-|s - c|^2 / (2 sigma^2)),
 *   z_ref = z of the nearest sample (ties: lowest sample index),
 *   height = (z_ref + sum w (z - z_ref) / sum w) * z_scale + z_offset,
 *   rgb = (sum w c / sum w) / 256 per channel (16-bit LAS colour to 8 bits).
 * With no candidate the texel copies the nearest sample (height and colour).
 * Texel centre: x0 + tx*tile + cell*j + cell/2 (and the same for y).  Samples
 * outside the region are ignored.  With no sample at all the height is NaN, the
 * colour 0 and the nearest distance +inf.
 * Outputs per requested tile k: height[k][res][res], rgbf[k][res][res][3] (unrounded
 * 8-bit scale), rgb8 (min(255, floor(rgbf + 0.5))), nearest_d2 (int64 squared
 * distance to the nearest sample, -1 if none) and nearest_idx (-1 if none).
 * ------------------------------------------------------------------------------ */
typedef struct {
    int64_t *start;   /* [T+1] */
    int64_t *items;   /* sample indices, grouped by tile, increasing index inside */
} tile_index_t;

static int build_tile_index(const int32_t *sx, const int32_t *sy, int64_t S, int64_t x0, int64_t y0,
                            int64_t tile, int64_t tiles_x, int64_t tiles_y, tile_index_t *ix)
{
    const int64_t T = tiles_x * tiles_y;
    ix->start = (int64_t *)calloc((size_t)(T + 1), sizeof(int64_t));
    ix->items = (int64_t *)malloc((size_t)(S > 0 ? S : 1) * sizeof(int64_t));
    int64_t *fillp = (int64_t *)calloc((size_t)(T + 1), sizeof(int64_t));
    if (!ix->start || !ix->items || !fillp) { free(fillp); return -1; }
    for (int64_t s = 0; s < S; ++s) {
        const int64_t lx = (int64_t)sx[s] - x0, ly = (int64_t)sy[s] - y0;
        if (lx < 0 || ly < 0 || lx >= tiles_x * tile || ly >= tiles_y * tile) continue;
        ix->start[(ly / tile) * tiles_x + lx / tile + 1] += 1;
    }
    for (int64_t t = 0; t < T; ++t) ix->start[t + 1] += ix->start[t];
    for (int64_t s = 0; s < S; ++s) {
        const int64_t lx = (int64_t)sx[s] - x0, ly = (int64_t)sy[s] - y0;
        if (lx < 0 || ly < 0 || lx >= tiles_x * tile || ly >= tiles_y * tile) continue;
        const int64_t t = (ly / tile) * tiles_x + lx / tile;
        ix->items[ix->start[t] + fillp[t]++] = s;
    }
    free(fillp);
    return 0;
}

/* nearest sample to (cx, cy): scan Chebyshev rings of tiles around (tx, ty); after
 * ring m every unscanned sample is at least m*tile away, so stop once the best
 * squared distance is <= (m*tile)^2. */
static void nearest_sample(const int32_t *sx, const int32_t *sy, const tile_index_t *ix,
                           int64_t tile, int64_t tiles_x, int64_t tiles_y,
                           int64_t tx, int64_t ty, int64_t cx, int64_t cy,
                           int64_t *best_d2, int64_t *best_idx)
{
    *best_d2 = -1; *best_idx = -1;
    const int64_t mmax = (tiles_x > tiles_y ? tiles_x : tiles_y);
    for (int64_t m = 0; m <= mmax; ++m) {
        for (int64_t uy = ty - m; uy <= ty + m; ++uy) {
            for (int64_t ux = tx - m; ux <= tx + m; ++ux) {
                const int64_t cheb = llabs(ux - tx) > llabs(uy - ty) ? llabs(ux - tx) : llabs(uy - ty);
                if (cheb != m) continue;
                if (ux < 0 || uy < 0 || ux >= tiles_x || uy >= tiles_y) continue;
                const int64_t u = uy * tiles_x + ux;
                for (int64_t q = ix->start[u]; q < ix->start[u + 1]; ++q) {
                    const int64_t s = ix->items[q];
                    const int64_t dx = (int64_t)sx[s] - cx, dy = (int64_t)sy[s] - cy;
                    const int64_t d2 = dx * dx + dy * dy;
                    if (*best_idx < 0 || d2 < *best_d2 || (d2 == *best_d2 && s < *best_idx)) {
                        *best_d2 = d2; *best_idx = s;
                    }
                }
            }
        }
        if (*best_idx >= 0 && *best_d2 <= (m * tile) * (m * tile)) return;
    }
}

int or_fill_sparse(const int32_t *sx, const int32_t *sy, const int32_t *sz,
                   const uint16_t *sr, const uint16_t *sg, const uint16_t *sb, int64_t S,
                   int64_t x0, int64_t y0, int64_t tile, int64_t tiles_x, int64_t tiles_y,
                   double z_scale, double z_offset,
                   int64_t res, int64_t radius_cm, double sigma_cm,
                   const int64_t *tile_ids, int64_t n_out,
                   double *height, double *rgbf, uint8_t *rgb8,
                   int64_t *nearest_d2, int64_t *nearest_idx)
{
    tile_index_t ix;
    if (build_tile_index(sx, sy, S, x0, y0, tile, tiles_x, tiles_y, &ix) != 0) return -1;
    const int64_t cell = tile / res;
    const int64_t R2 = radius_cm * radius_cm;
    const int64_t k = (radius_cm + tile - 1) / tile;       /* tile window holding all candidates */
    const double two_sigma2 = 2.0 * sigma_cm * sigma_cm;
    for (int64_t o = 0; o < n_out; ++o) {
        const int64_t t = tile_ids[o];
        const int64_t tx = t % tiles_x, ty = t / tiles_x;
        for (int64_t i = 0; i < res; ++i) {
            for (int64_t j = 0; j < res; ++j) {
                const int64_t cx = x0 + tx * tile + cell * j + cell / 2;
                const int64_t cy = y0 + ty * tile + cell * i + cell / 2;
                const int64_t e = (o * res + i) * res + j;
                int64_t nd2, ni;
                nearest_sample(sx, sy, &ix, tile, tiles_x, tiles_y, tx, ty, cx, cy, &nd2, &ni);
                if (nearest_d2) nearest_d2[e] = nd2;
                if (nearest_idx) nearest_idx[e] = ni;
                if (ni < 0) {
                    height[e] = NAN;
                    for (int c = 0; c < 3; ++c) { rgbf[e * 3 + c] = 0.0; rgb8[e * 3 + c] = 0; }
                    continue;
                }
                double col[3];
                if (nd2 <= R2) {
                    const double zref = (double)sz[ni];
                    double sw = 0.0, swz = 0.0, swc[3] = {0.0, 0.0, 0.0};
                    for (int64_t uy = ty - k; uy <= ty + k; ++uy) {
                        for (int64_t ux = tx - k; ux <= tx + k; ++ux) {
                            if (ux < 0 || uy < 0 || ux >= tiles_x || uy >= tiles_y) continue;
                            const int64_t u = uy * tiles_x + ux;
                            for (int64_t q = ix.start[u]; q < ix.start[u + 1]; ++q) {
                                const int64_t s = ix.items[q];
                                const int64_t dx = (int64_t)sx[s] - cx, dy = (int64_t)sy[s] - cy;
                                const int64_t d2 = dx * dx + dy * dy;
                                if (d2 > R2) continue;
                                const double w = exp(-(double)d2 / two_sigma2);
                                sw += w;
                                swz += w * ((double)sz[s] - zref);
                                swc[0] += w * (double)sr[s];
                                swc[1] += w * (double)sg[s];
                                swc[2] += w * (double)sb[s];
                            }
                        }
                    }
                    height[e] = (zref + swz / sw) * z_scale + z_offset;
                    for (int c = 0; c < 3; ++c) col[c] = swc[c] / sw / 256.0;
                } else {
                    height[e] = (double)sz[ni] * z_scale + z_offset;
                    col[0] = (double)sr[ni] / 256.0;
                    col[1] = (double)sg[ni] / 256.0;
                    col[2] = (double)sb[ni] / 256.0;
                }
                for (int c = 0; c < 3; ++c) {
                    rgbf[e * 3 + c] = col[c];
                    const double v = floor(col[c] + 0.5);
                    rgb8[e * 3 + c] = (uint8_t)(v > 255.0 ? 255.0 : v);
                }
            }
        }
    }
    free(ix.start);
    free(ix.items);
    return 0;
}

/* ------------------------------------------------------------------------------
 * Tile update with full-resolution data (abstract; Sec. 3.5): texels with at least
 * one full-resolution point take the mean height and mean colour of their points;
 * texels without points keep the value they have.
 *   height = (float)(((double)zsum / count) * z_scale + z_offset)
 *   rgb8   = min(255, floor((double)csum / count / 256 + 0.5))
 * Bins are the region-wide [T][res][res] arrays; outputs are per requested tile.
 * ------------------------------------------------------------------------------ */
void or_update_tile(const uint32_t *count, const int64_t *zsum,
                    const uint64_t *rsum, const uint64_t *gsum, const uint64_t *bsum,
                    int64_t res, const int64_t *tile_ids, int64_t n_out,
                    double z_scale, double z_offset, float *height, uint8_t *rgb)
{
    for (int64_t o = 0; o < n_out; ++o) {
        const int64_t t = tile_ids[o];
        for (int64_t c = 0; c < res * res; ++c) {
            const int64_t src = t * res * res + c;
            const int64_t dst = o * res * res + c;
            if (count[src] == 0) continue;
            const double n = (double)count[src];
            const double mean = (double)zsum[src] / n;
            height[dst] = (float)(mean * z_scale + z_offset);
            const uint64_t sums[3] = {rsum[src], gsum[src], bsum[src]};
            for (int k = 0; k < 3; ++k) {
                const double v = floor((double)sums[k] / n / 256.0 + 0.5);
                rgb[dst * 3 + k] = (uint8_t)(v > 255.0 ? 255.0 : v);
            }
        }
    }
}
