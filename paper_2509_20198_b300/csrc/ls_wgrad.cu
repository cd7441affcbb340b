// Weight and bias gradients of a 3x3 convolution on the tensor cores (training of the
// learned filler, Sec. 3.4).  dW^T[k][o] = sum_p X_shift(k)[p] dZ[p][o] with
// k = tap * C_in + c_in: a GEMM with M = 9*C_in, N = C_out and K = pixels.  Three forms:
//  k_wgrad_halo     input channels in blocks of 32, images 16..128 wide: one input box
//                   per chunk of rows serves all nine taps (ky as dZ row shifts in N,
//                   kx as input pixel shifts in M);
//  k_wgrad_halo_c8  eight input channels: the same with the operands swapped;
//  k_wgrad          the per-tap form below for every other shape.
// Each CTA stores the partial sums of its slice of pixels; k_wsum adds them to the FP32
// gradient in a fixed order, so the result does not depend on CTA scheduling (training
// is reproducible).
//
// Per-tap form: M tiles of 128 rows, K = 64 pixels per stage; each CTA owns one tile
// and one slice of pixels.
// Both operands are stored pixel-minor (NHWC): for a pixel (the GEMM's K index) the
// channels (its M or N index) are contiguous.  That is the MN-major operand layout, so
// the MMA reads the TMA boxes as they land, with no transposition:
//  warp 0     TMA producer: the M tile's rows are 128 / cw blocks of cw channels of one
//             tap (cw = 64, 32, 16 or 8 dividing C_in): one 4-D tiled load per block of the
//             tap-shifted input (cw channels x 64 pixels: whole rows, or half a row of a
//             128-wide image; zero-filled outside the image: the padding; rows of
//             128 / 64 / 32 bytes written with the matching swizzle), and dZ in blocks of
//             cwb output channels, into a ring of stages;
//  warp 5     issues tcgen05.mma kind::f16 (M=128, N=C_out, K=16) with both operands
//             MN-major and commits each stage back to the producer;
//  warps 1-4  read the accumulator from TMEM at the end (one row per thread).
// The bias gradient is a column sum of dZ.  When 9*C_in leaves padding rows in the last
// M tile, the first padding row of every stage is set to ones once (no load writes the
// padding blocks), so the same MMAs sum dZ over the pixels into that row and k_wsum
// passes it on as the bias gradient; otherwise k_colsum (per-block partials) and k_dbsum
// (in block order) compute it.
#include <cuda_bf16.h>

#include "ls_tc.cuh"

namespace ls {
namespace {

constexpr int kWgThreads = 192;
// Four stages: at C_out <= 64 a CTA needs at most 96 KB of shared memory and two or
// three CTAs share an SM, whose independent pipelines hide the load latency better than
// deeper rings in one CTA
constexpr int kWgStages = 4;
constexpr int kWgPix = 64;  // pixels (K) per stage
constexpr int kWgABytes = 128 * kWgPix * 2;

// Byte offset in a stage of channel ch (multiple of 8) of pixel px, the stage being
// a sequence of blocks of cw channels x 64 pixels as the TMA wrote them: pixel rows of
// 2*cw bytes; 16-byte chunk c of row px sits at chunk c ^ (px & 7) (128B swizzle, cw 64),
// c ^ ((px >> 1) & 3) (64B swizzle, cw 32) or c ^ ((px >> 2) & 1) (32B swizzle, cw 16);
// cw 8 rows are plain 16-byte rows.
__device__ __forceinline__ uint32_t raw_off(int ch, int px, int cw) {
  const int blk = ch / cw, c = (ch - blk * cw) >> 3;
  const uint32_t base = (uint32_t)blk * (kWgPix * cw * 2) + (uint32_t)px * (uint32_t)(cw * 2);
  const int sc = cw == 64 ? (c ^ (px & 7)) : cw == 32 ? (c ^ ((px >> 1) & 3)) : cw == 16 ? (c ^ ((px >> 2) & 1)) : c;
  return base + (uint32_t)sc * 16u;
}

struct WgArgs {
  float* __restrict__ part;  // [CTAs][128][cout] fp32 partial sums (CTA = slice * n_mtiles + tile)
  int32_t cw, cwb;                // channel block widths of the x and dZ loads
  int32_t h, w, cin, cout, rows;  // rows = 9*cin
  int32_t rows_per_step;          // image rows per 64-pixel stage (64 / w, 1, or h)
  int32_t cols_per_step;          // pixels of a row per stage (w, or 64 when w = 128)
  int32_t imgs_per_step;          // images per stage (1, or 64 / (h * w))
  int64_t pix_total, pix_per_cta;
  int32_t n_mtiles;
  int32_t ones_row;  // row k = rows of the last tile set to ones (bias gradient), or -1
  uint32_t idesc, tmem_cols, b_bytes;
};

__global__ void __launch_bounds__(kWgThreads, 1)
    k_wgrad(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dzmap, const WgArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_bytes = kWgABytes + a.b_bytes;
  const int mt = blockIdx.x % a.n_mtiles;
  const int64_t slice = blockIdx.x / a.n_mtiles;
  const int64_t p_begin = slice * a.pix_per_cta;
  const int64_t p_end = min(p_begin + a.pix_per_cta, a.pix_total);
  const int n_steps = (int)((p_end - p_begin + kWgPix - 1) / kWgPix);
  const int m0 = mt * 128;
  const int blk_a = kWgPix * a.cw * 2, blk_b = kWgPix * a.cwb * 2;  // bytes per block load
  // blocks of cw channels of the tile inside the 9*C_in rows (a block never straddles
  // two taps: cw divides C_in); the rest of the tile is padding that no load writes
  const int n_blocks = 128 / a.cw;
  int n_valid = (a.rows - m0) / a.cw;
  if (n_valid > n_blocks) n_valid = n_blocks;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kWgStages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    tc::prefetch_tmap(&dzmap);
  }
  if (n_valid < n_blocks && warp >= 1 && warp <= 4) {
    // padding blocks of every stage, once: zeros, and, for the bias gradient, the ones
    // row (the tile's row `rows`: channel 0 of the first padding block) for all pixels
    const int t = threadIdx.x - 32;
    for (int s = 0; s < kWgStages; ++s) {
      uint32_t* pad = reinterpret_cast<uint32_t*>(smem + (size_t)s * stage_bytes + (size_t)n_valid * blk_a);
      const int words = (n_blocks - n_valid) * blk_a / 4;
      for (int i = t; i < words; i += 128) pad[i] = 0u;
    }
    __syncwarp();
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the four padding warps
    if (a.ones_row == a.rows && a.ones_row >= m0 && a.ones_row < m0 + 128) {
      for (int i = t; i < kWgStages * kWgPix; i += 128) {
        const int s = i / kWgPix, px = i - s * kWgPix;
        uint16_t* one = reinterpret_cast<uint16_t*>(smem + (size_t)s * stage_bytes +
                                                    raw_off(n_valid * a.cw, px, a.cw));
        *one = 0x3F80u;  // bf16 1.0
      }
    }
    tc::fence_proxy_async_smem();
  }
  if (warp == 5) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: the tile's block coordinates are fixed, the
      // pixel position advances by one stage (64 pixels) at a time
      const int64_t hw = (int64_t)a.h * a.w;
      int bc[16], bx[16], by[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = m0 + i * a.cw;
        bc[i] = bx[i] = by[i] = 0;
        if (i < n_valid) {
          const int tap = k / a.cin;
          bc[i] = k - tap * a.cin;
          by[i] = tap / 3 - 1;
          bx[i] = tap - (tap / 3) * 3 - 1;
        }
      }
      const int n_ob = a.cout / a.cwb;
      const uint32_t bytes = (uint32_t)(n_valid * blk_a + n_ob * blk_b);
      int n0 = (int)(p_begin / hw);
      const int64_t in_img = p_begin - (int64_t)n0 * hw;  // a multiple of the stage
      int y0 = a.imgs_per_step > 1 ? 0 : (int)(in_img / a.w);
      int x0 = a.imgs_per_step > 1 ? 0 : (int)(in_img - (int64_t)y0 * a.w);
      int slot = 0;
      uint32_t ph = 0;
      for (int s = 0; s < n_steps && !abort_flag; ++s) {
        if (!tc::mbar_wait(&empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
        uint8_t* RA = smem + (size_t)slot * stage_bytes;
        uint8_t* RB = RA + kWgABytes;
        tc::mbar_arrive_expect_tx(&full[slot], bytes);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < n_valid)
            tc::tma_load_4d(RA + i * blk_a, &xmap, bc[i], x0 + bx[i], y0 + by[i], n0, &full[slot]);
        for (int ob = 0; ob < n_ob; ++ob)
          tc::tma_load_4d(RB + ob * blk_b, &dzmap, ob * a.cwb, x0, y0, n0, &full[slot]);
        // next 64 pixels: the rest of this row, more rows of this image, or the next
        // image(s)
        if (a.imgs_per_step > 1) {
          n0 += a.imgs_per_step;
        } else {
          x0 += a.cols_per_step;
          if (x0 >= a.w) {
            x0 = 0;
            y0 += a.rows_per_step;
            if (y0 >= a.h) { y0 = 0; ++n0; }
          }
        }
        if (++slot == kWgStages) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (warp <= 4) {
    // ---------------- epilogue: TMEM row per thread into this CTA's partial block
    if (n_steps > 0 && tc::mbar_wait(&done, 0) && !abort_flag) {
      tc::fence_after();
      const int q = warp & 3;
      const int row = q * 32 + lane;
      float* out = a.part + ((size_t)blockIdx.x * 128 + row) * a.cout;
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (m0 + row < a.rows || m0 + row == a.ones_row) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4*>(out + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer (warp 5): both operands MN-major, straight from the
    // TMA boxes (NHWC: channels contiguous); K = 16 pixels per MMA is two 8-row groups
    const uint32_t s0 = tc::saddr(smem);
    const uint32_t mode_a = a.cw == 64 ? 2u : a.cw == 32 ? 4u : a.cw == 16 ? 6u : 0u;
    const uint32_t mode_b = a.cwb == 64 ? 2u : a.cwb == 32 ? 4u : a.cwb == 16 ? 6u : 0u;
    const uint32_t kgrp_a = 16u * (uint32_t)a.cw, kgrp_b = 16u * (uint32_t)a.cwb;  // bytes per 8 K rows
    const uint64_t adesc0 = a.cw == 8 ? tc::sdesc_mn(s0, kgrp_a, (uint32_t)blk_a, 0u)
                                      : tc::sdesc_mn(s0, (uint32_t)blk_a, kgrp_a, mode_a);
    const uint64_t bdesc0 = a.cwb == 8 ? tc::sdesc_mn(s0 + kWgABytes, kgrp_b, (uint32_t)blk_b, 0u)
                                       : tc::sdesc_mn(s0 + kWgABytes, (uint32_t)blk_b, kgrp_b, mode_b);
    int slot = 0;
    uint32_t ph = 0;
    for (int s = 0; s < n_steps && !abort_flag; ++s) {
      if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
      tc::fence_after();
      const uint64_t so = (uint64_t)((slot * stage_bytes) >> 4);
#pragma unroll
      for (int j = 0; j < kWgPix / 16; ++j)
        tc::mma_bf16(taddr, adesc0 + so + (uint64_t)((j * 2 * kgrp_a) >> 4),
                     bdesc0 + so + (uint64_t)((j * 2 * kgrp_b) >> 4), a.idesc, (s > 0 || j > 0) ? 1u : 0u);
      tc::mma_commit(&empty[slot]);
      if (++slot == kWgStages) { slot = 0; ph ^= 1u; }
    }
    if (n_steps > 0) tc::mma_commit(&done);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 5) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, a.tmem_cols);
  }
}

// ---------------------------------------------------------------------------------
// Halo form for input channels in blocks of 32 on images 16 to 128 wide (a power of
// two).  With q = p + (ky - 1, 0) the sum becomes
//   dW^T[(ky, kx, c)][o] = sum_q X(q + (0, kx - 1))[c] dZ(q - (ky - 1, 0))[o],
// so the horizontal tap kx shifts the input along its row and the vertical tap ky
// shifts dZ by whole rows.  A stage is one chunk of R image rows (R * W = 128 pixels q)
// of one image: per block of 32 input channels a TMA box of rows y0 .. y0+R-1 and
// columns -1 .. W (P = W + 2 pixels per row, zero outside the image; 64-byte pixel rows,
// 64-byte swizzle), and per block of cwb = 32 or 64 output channels the dZ box of rows
// y0-1 .. y0+R (zero outside the image).  The K index is q, 16 per MMA within a row.
//  A (M = 128): blocks kx = 0..3 of 32 channels, the same input box seen one pixel row
//    apart (LBO = one 64-byte row), starting at box pixel row r * P + x0; block kx = 3
//    is not a tap (its rows are computed and dropped: 3/4 of the M rows are used; it
//    reads at most one pixel row past the box, inside the box's slack).
//  B (N = 3 * cwb): blocks j = 0..2 of cwb channels, dZ rows r + j of the box
//    (LBO = one dZ image row), j = 2 - ky.
// One MMA thus serves all nine taps of a channel block and cwb outputs: the A operand
// (4 KB per MMA, the bulk of the shared-memory reads) is read once for three taps.
// An issuing warp owns the accumulator of one (channel block, dZ block) unit and takes
// every nk-th of the chunk's eight 16-pixel steps: with nk > 1 (TMEM permitting) the
// unit has nk accumulator copies that the epilogue adds in order (one thread waits
// about 150 cycles per MMA, so the issue rate grows with the number of issuers).
// TMEM: copy-major, per channel block 3 * C_out columns, [ob][j][cwb].
// With the bias gradient, the four epilogue warps of the group-0 CTAs sum dZ over the
// chunk pixels of every stage meanwhile (they release the stage too).  At the end the
// epilogue warp of TMEM lane quadrant q stores the rows of tap column kx = q.
// Partials land in k_wsum's layout: [slice][9 * C_in + 1][C_out], the last row the bias
// partial.
constexpr int kWhMaxIssuers = 9;
constexpr int kWhMaxStages = 8;
constexpr int kWhSteps = 8;  // 16-pixel steps per 128-pixel block of a chunk
constexpr int kWhThreads = 32 * (1 + kWhMaxIssuers + 4);
constexpr size_t kWhSmemBudget = 226 * 1024;  // with the 1 KB of static shared memory: the 227 KB limit

struct WhArgs {
  float* __restrict__ part;
  int32_t bias;  // the group-0 CTAs store the bias partial as row 9 * C_in
  int32_t w, p, r, cin, cout, cwb, n_dzb, gblocks, groups, nissue, nk;
  int32_t chunks_per_img, n_chunks, chunks_per_cta, stages;
  int32_t cp;             // chunk pixels: R * W = 128, 256 or 512
  uint32_t a_h, b_h;      // descriptor start-address steps (16-byte units) per 128-pixel block
  uint32_t box_stride, xbox_bytes, dz_blk_bytes, dz_rowb, dz_mode, stage_bytes, idesc, tmem_cols;
  int32_t part_rows;
};

__global__ void __launch_bounds__(kWhThreads, 1)
    k_wgrad_halo(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dzmap, const WhArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kWhMaxStages], empty[kWhMaxStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x % a.groups, slice = blockIdx.x / a.groups;
  const int c_begin = slice * a.chunks_per_cta;
  const int c_end = min(c_begin + a.chunks_per_cta, a.n_chunks);
  const int nissue = a.nissue;
  const bool bias = a.bias && g == 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.stages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], nissue + (bias ? 4 : 0));
    }
    tc::mbar_init(&done, nissue);
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    tc::prefetch_tmap(&dzmap);
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;
  const int first_epi = 1 + nissue;
  const uint32_t dz_off = (uint32_t)a.gblocks * a.box_stride;  // dZ blocks after the input boxes
  const int blk_cols = 3 * a.cout;                             // TMEM columns per channel block

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: per chunk the input boxes of the group's channel
      // blocks and the dZ boxes (one row of halo above and below)
      const uint32_t bytes = (uint32_t)a.gblocks * a.xbox_bytes + (uint32_t)a.n_dzb * a.dz_blk_bytes;
      int slot = 0;
      uint32_t ph = 0;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        const int n = c / a.chunks_per_img, y0 = (c - n * a.chunks_per_img) * a.r;
        if (!tc::mbar_wait(&empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
        uint8_t* st = smem + (size_t)slot * a.stage_bytes;
        tc::mbar_arrive_expect_tx(&full[slot], bytes);
        for (int lb = 0; lb < a.gblocks; ++lb)
          tc::tma_load_4d(st + (size_t)lb * a.box_stride, &xmap, (g * a.gblocks + lb) * 32, -1, y0, n, &full[slot]);
        for (int ob = 0; ob < a.n_dzb; ++ob)
          tc::tma_load_4d(st + dz_off + (size_t)ob * a.dz_blk_bytes, &dzmap, ob * a.cwb, 0, y0 - 1, n, &full[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (warp <= nissue) {
    if (lane == 0) {
      // ---------------- MMA issuer of unit (channel block lb, dZ block ob), steps kp,
      // kp + nk, ... of each chunk into accumulator copy kp
      const int u = (warp - 1) / a.nk, kp = (warp - 1) - u * a.nk;
      const int lb = u / a.n_dzb, ob = u - lb * a.n_dzb;
      const uint32_t s0 = tc::saddr(smem);
      const uint32_t d = taddr + (uint32_t)(kp * a.gblocks * blk_cols + lb * blk_cols + ob * 3 * a.cwb);
      const int ksteps = a.w / 16;
      // descriptors of the chunk's eight 16-pixel steps in stage 0, built once; a stage
      // adds its offset to the start-address field (shared addresses stay below 256 KB)
      uint64_t adsc[kWhSteps], bdsc[kWhSteps];
#pragma unroll
      for (int i = 0; i < kWhSteps; ++i) {
        const int rr = i / ksteps, x0 = (i - rr * ksteps) * 16;
        adsc[i] = tc::sdesc_mn(s0 + (uint32_t)lb * a.box_stride + (uint32_t)(rr * a.p + x0) * 64u, 64u, 512u, 4u);
        bdsc[i] = tc::sdesc_mn(s0 + dz_off + (uint32_t)ob * a.dz_blk_bytes + (uint32_t)(rr * a.w + x0) * a.dz_rowb,
                               (uint32_t)a.w * a.dz_rowb, 8u * a.dz_rowb, a.dz_mode);
      }
      const uint32_t idesc = a.idesc;
      const int kmask = a.nk - 1;
      int slot = 0;
      uint32_t ph = 0;
      uint32_t acc = 0u;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
        tc::fence_after();
        const uint64_t so = (uint64_t)(((uint32_t)slot * a.stage_bytes) >> 4);
        for (int h = 0; h < a.cp; h += 128) {  // 128-pixel blocks: R * 128 / cp rows each
          const uint64_t sa = so + (uint64_t)((uint32_t)(h >> 7) * a.a_h);
          const uint64_t sb = so + (uint64_t)((uint32_t)(h >> 7) * a.b_h);
#pragma unroll
          for (int i = 0; i < kWhSteps; ++i) {
            if ((i & kmask) == kp) {
              tc::mma_bf16(d, adsc[i] + sa, bdsc[i] + sb, idesc, acc);
              acc = 1u;
            }
          }
        }
        tc::mma_commit(&empty[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
      tc::mma_commit(&done);
    }
  } else if (warp < first_epi + 4) {
    const int q = warp & 3;
    const int et = (warp - first_epi) * 32 + lane;  // 0..127
    float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int nch = a.cout / 8;                  // 16-byte channel chunks per pixel
    const int lanes = 128 / nch, bj = et % nch;  // pixel lanes; this thread's chunk
    const int bl = et / nch < lanes ? et / nch : (1 << 20);  // threads past the last lane idle
    if (bias) {
      // ---------------- bias gradient: dZ over the chunk's pixels (box rows 1 .. R),
      // channels of chunk bj, pixels bl, bl + lanes, ...
      const int ob = bj / (a.cwb / 8), cj = bj - ob * (a.cwb / 8);
      int slot = 0;
      uint32_t ph = 0;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
        const uint8_t* zb = smem + (size_t)slot * a.stage_bytes + dz_off + (size_t)ob * a.dz_blk_bytes;
        for (int px = bl; px < a.cp; px += lanes) {
          const int row = a.w + px;  // box row 0 is the halo row above the chunk
          const int sc = a.cwb == 64 ? (cj ^ (row & 7)) : (cj ^ ((row >> 1) & 3));
          const uint4 v = *reinterpret_cast<const uint4*>(zb + (size_t)row * a.dz_rowb + sc * 16);
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            bsum[2 * i] += __uint_as_float(wv[i] << 16);
            bsum[2 * i + 1] += __uint_as_float(wv[i] & 0xffff0000u);
          }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
    }
    // ---------------- epilogue: TMEM lane quadrant q of every channel block = tap
    // column kx = q; column (ob, j, o') = tap row ky = 2 - j, output ob * cwb + o'
    const bool ok = c_end > c_begin && tc::mbar_wait(&done, 0) && !abort_flag;
    if (ok) {
      tc::fence_after();
      float* out = a.part + (size_t)slice * a.part_rows * a.cout;
      for (int lb = 0; lb < a.gblocks; ++lb) {
        const int cbase = (g * a.gblocks + lb) * 32 + lane;
        for (int col = 0; col < blk_cols; col += 16) {
          const int ob = col / (3 * a.cwb), rem = col - ob * 3 * a.cwb;
          const int j = rem / a.cwb, o0 = ob * a.cwb + (rem - j * a.cwb);
          const uint32_t ta = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(lb * blk_cols + col);
          float v[16];
          tc::tmem_ld16(ta, v);
          for (int kp = 1; kp < a.nk; ++kp) {  // accumulator copies in order
            float v2[16];
            tc::tmem_ld16(ta + (uint32_t)(kp * a.gblocks * blk_cols), v2);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += v2[i];
          }
          if (q < 3) {
            const int k = ((2 - j) * 3 + q) * a.cin + cbase;
            float* o = out + (size_t)k * a.cout + o0;
#pragma unroll
            for (int i = 0; i < 16; i += 4)
              *reinterpret_cast<float4*>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          }
        }
      }
    }
    if (bias) {
      // fixed-order combination of the pixel lanes through shared memory (the ring is
      // idle: every load was consumed by the finished MMAs)
      asm volatile("bar.sync 1, 128;" ::: "memory");
      float* red = reinterpret_cast<float*>(smem);
      if (ok) {
#pragma unroll
        for (int i = 0; i < 8; ++i) red[et * 8 + i] = bsum[i];
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (ok && et < a.cout) {
        const int cc = et / 8, i = et - cc * 8;
        float s = 0.f;
        for (int l = 0; l < lanes; ++l) s += red[(l * nch + cc) * 8 + i];
        a.part[((size_t)slice * a.part_rows + 9 * a.cin) * a.cout + et] = s;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, a.tmem_cols);
  }
}

// ---------------------------------------------------------------------------------
// Halo form for eight input channels (one 16-byte pixel row) and C_out = 32 or 64: the
// roles of the operands swap.  The chunk, boxes and bias sums are those of
// k_wgrad_halo (the input box has 16-byte rows, no swizzle); per 16-pixel step:
//  A (M = 128): dZ rows r + j of the box, blocks j of cwb = C_out channels (LBO = one
//    dZ image row): j = 0..3 in one tile at C_out = 32 (j = 3 is not a tap: dropped),
//    j = 0, 1 and j = 2, 3 in two tiles at C_out = 64;
//  B (N = 32): the input box seen at four pixel offsets kx = 0..3 (8-element groups one
//    16-byte pixel row apart: SBO = 16 B, LBO = 8 pixel rows; kx = 3 dropped).
// D[(j, o)][(kx, c)] accumulates dW^T[((2 - j) * 3 + kx) * 8 + c][o].  Issuers as in
// k_wgrad_halo: one per (M tile, accumulator copy).
__global__ void __launch_bounds__(kWhThreads, 1)
    k_wgrad_halo_c8(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dzmap,
                    const WhArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kWhMaxStages], empty[kWhMaxStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = blockIdx.x;
  const int c_begin = slice * a.chunks_per_cta;
  const int c_end = min(c_begin + a.chunks_per_cta, a.n_chunks);
  const int nissue = a.nissue;
  const bool bias = a.bias != 0;
  const int mtiles = a.cout / 32;  // M tiles per step
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.stages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], nissue + (bias ? 4 : 0));
    }
    tc::mbar_init(&done, nissue);
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    tc::prefetch_tmap(&dzmap);
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;
  const int first_epi = 1 + nissue;
  const uint32_t dz_off = a.box_stride;  // the dZ block after the input box

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t bytes = a.xbox_bytes + a.dz_blk_bytes;
      int slot = 0;
      uint32_t ph = 0;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        const int n = c / a.chunks_per_img, y0 = (c - n * a.chunks_per_img) * a.r;
        if (!tc::mbar_wait(&empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
        uint8_t* st = smem + (size_t)slot * a.stage_bytes;
        tc::mbar_arrive_expect_tx(&full[slot], bytes);
        tc::tma_load_4d(st, &xmap, 0, -1, y0, n, &full[slot]);
        tc::tma_load_4d(st + dz_off, &dzmap, 0, 0, y0 - 1, n, &full[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (warp <= nissue) {
    if (lane == 0) {
      // ---------------- MMA issuer of M tile t (dZ rows j = t * jt ..), steps kp, kp + nk, ...
      const int t = (warp - 1) / a.nk, kp = (warp - 1) - t * a.nk;
      const int jt = 128 / a.cout;  // dZ row blocks per M tile
      const uint32_t s0 = tc::saddr(smem);
      const uint32_t d = taddr + (uint32_t)((kp * mtiles + t) * 32);
      const int ksteps = a.w / 16;
      uint64_t adsc[kWhSteps], bdsc[kWhSteps];
#pragma unroll
      for (int i = 0; i < kWhSteps; ++i) {
        const int rr = i / ksteps, x0 = (i - rr * ksteps) * 16;
        adsc[i] = tc::sdesc_mn(s0 + dz_off + (uint32_t)((rr + t * jt) * a.w + x0) * a.dz_rowb,
                               (uint32_t)a.w * a.dz_rowb, 8u * a.dz_rowb, a.dz_mode);
        bdsc[i] = tc::sdesc_mn(s0 + (uint32_t)(rr * a.p + x0) * 16u, 128u, 16u, 0u);
      }
      const uint32_t idesc = a.idesc;
      const int kmask = a.nk - 1;
      int slot = 0;
      uint32_t ph = 0;
      uint32_t acc = 0u;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
        tc::fence_after();
        const uint64_t so = (uint64_t)(((uint32_t)slot * a.stage_bytes) >> 4);
        for (int h = 0; h < a.cp; h += 128) {  // 128-pixel blocks: R * 128 / cp rows each
          const uint64_t sa = so + (uint64_t)((uint32_t)(h >> 7) * a.a_h);
          const uint64_t sb = so + (uint64_t)((uint32_t)(h >> 7) * a.b_h);
#pragma unroll
          for (int i = 0; i < kWhSteps; ++i) {
            if ((i & kmask) == kp) {
              tc::mma_bf16(d, adsc[i] + sa, bdsc[i] + sb, idesc, acc);
              acc = 1u;
            }
          }
        }
        tc::mma_commit(&empty[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
      tc::mma_commit(&done);
    }
  } else if (warp < first_epi + 4) {
    const int q = warp & 3;
    const int et = (warp - first_epi) * 32 + lane;
    float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int nch = a.cout / 8;
    const int lanes = 128 / nch, bj = et % nch;
    const int bl = et / nch < lanes ? et / nch : (1 << 20);
    if (bias) {
      // bias gradient: dZ over the chunk's pixels (box rows 1 .. R), as in k_wgrad_halo
      int slot = 0;
      uint32_t ph = 0;
      for (int c = c_begin; c < c_end && !abort_flag; ++c) {
        if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
        const uint8_t* zb = smem + (size_t)slot * a.stage_bytes + dz_off;
        for (int px = bl; px < a.cp; px += lanes) {
          const int row = a.w + px;
          const int sc = a.cwb == 64 ? (bj ^ (row & 7)) : (bj ^ ((row >> 1) & 3));
          const uint4 v = *reinterpret_cast<const uint4*>(zb + (size_t)row * a.dz_rowb + sc * 16);
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            bsum[2 * i] += __uint_as_float(wv[i] << 16);
            bsum[2 * i + 1] += __uint_as_float(wv[i] & 0xffff0000u);
          }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[slot]);
        if (++slot == a.stages) { slot = 0; ph ^= 1u; }
      }
    }
    // ---------------- epilogue: TMEM lane 32 q + lane of tile t is (j, o) with
    // j = t * jt + (32 q + lane) / cout; columns kx * 8 + c, kx < 3 stored
    const bool ok = c_end > c_begin && tc::mbar_wait(&done, 0) && !abort_flag;
    if (ok) {
      tc::fence_after();
      float* out = a.part + (size_t)slice * a.part_rows * a.cout;
      const int jt = 128 / a.cout;
      const int m = q * 32 + lane, jl = m / a.cout, o = m - jl * a.cout;
      for (int t = 0; t < mtiles; ++t) {
        const int j = t * jt + jl;
        const uint32_t ta = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * 32);
        float v0[16], v1[16];  // columns 0-15 (kx 0, 1) and 16-31 (kx 2, 3)
        tc::tmem_ld16(ta, v0);
        tc::tmem_ld16(ta + 16u, v1);
        for (int kp = 1; kp < a.nk; ++kp) {  // accumulator copies in order
          float v2[16];
          const uint32_t tk = ta + (uint32_t)(kp * mtiles * 32);
          tc::tmem_ld16(tk, v2);
#pragma unroll
          for (int i = 0; i < 16; ++i) v0[i] += v2[i];
          tc::tmem_ld16(tk + 16u, v2);
#pragma unroll
          for (int i = 0; i < 16; ++i) v1[i] += v2[i];
        }
        if (j < 3) {
          float* rowp = out + (size_t)((2 - j) * 3) * 8 * a.cout + o;  // tap (ky, kx = 0), channel 0
#pragma unroll
          for (int n = 0; n < 16; ++n) rowp[(size_t)n * a.cout] = v0[n];
#pragma unroll
          for (int n = 0; n < 8; ++n) rowp[(size_t)(16 + n) * a.cout] = v1[n];
        }
      }
    }
    if (bias) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      float* red = reinterpret_cast<float*>(smem);
      if (ok) {
#pragma unroll
        for (int i = 0; i < 8; ++i) red[et * 8 + i] = bsum[i];
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (ok && et < a.cout) {
        const int cc = et / 8, i = et - cc * 8;
        float s = 0.f;
        for (int l = 0; l < lanes; ++l) s += red[(l * nch + cc) * 8 + i];
        a.part[((size_t)slice * a.part_rows + 9 * a.cin) * a.cout + et] = s;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, a.tmem_cols);
  }
}

// dW^T[k][o] += sum over slices of the CTA partials ([slice][stride] floats, element
// e = k * cout + o).  A block takes 32 consecutive elements; warp g adds slices g, g + 8,
// ... in increasing order (loads four ahead), then warp 0 adds the eight warp sums in
// order: a fixed order, so the result does not depend on scheduling.  With db, row
// `rows` of the partials is the bias gradient: into db.
constexpr int kWsumGroups = 8;
__global__ void __launch_bounds__(32 * kWsumGroups) k_wsum(const float* __restrict__ part, int slices,
                                                            int64_t stride, int rows, int cout,
                                                            float* __restrict__ dwt, float* __restrict__ db) {
  __shared__ float red[kWsumGroups][32];
  const int total = (rows + (db ? 1 : 0)) * cout;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (e < total) {
    const float* p = part + e;
    int sl = g;
    for (; sl + 3 * kWsumGroups < slices; sl += 4 * kWsumGroups) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = p[(size_t)(sl + i * kWsumGroups) * stride];
#pragma unroll
      for (int i = 0; i < 4; ++i) s += v[i];
    }
    for (; sl < slices; sl += kWsumGroups) s += p[(size_t)sl * stride];
  }
  red[g][lane] = s;
  __syncthreads();
  if (g == 0 && e < total) {
    float t = red[0][lane];
#pragma unroll
    for (int k = 1; k < kWsumGroups; ++k) t += red[k][lane];
    if (e < rows * cout) dwt[e] += t;
    else db[e - rows * cout] += t;
  }
}

constexpr int kColsumBlocks = 2 * kSmCount;
// Column sums of dz [P][cout] per block: thread = (pixel lane, group of 8 channels),
// 16-byte loads; lanes combined in a fixed order through shared memory.
__global__ void __launch_bounds__(256) k_colsum(const uint16_t* __restrict__ dz, int64_t pix, int cout,
                                                float* __restrict__ part /* [blocks][cout] */) {
  __shared__ float red[256 * 8];
  const int ng = cout / 8, lanes = blockDim.x / ng;
  const int g = threadIdx.x % ng, pl = threadIdx.x / ng;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t p = (int64_t)blockIdx.x * lanes + pl; p < pix; p += (int64_t)gridDim.x * lanes) {
    const uint4 v = *reinterpret_cast<const uint4*>(dz + p * cout + g * 8);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[2 * i] += __uint_as_float(w[i] << 16);
      acc[2 * i + 1] += __uint_as_float(w[i] & 0xffff0000u);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) red[threadIdx.x * 8 + i] = acc[i];
  __syncthreads();
  for (int c = threadIdx.x; c < cout; c += blockDim.x) {
    const int gg = c / 8, i = c - gg * 8;
    float s = 0.f;
    for (int l = 0; l < lanes; ++l) s += red[(l * ng + gg) * 8 + i];
    part[(size_t)blockIdx.x * cout + c] = s;
  }
}

// db[o] += sum over blocks of the column-sum partials: one block per channel, thread t
// sums blocks t, t + 256, ... in order, then a fixed-shape tree over the threads.
__global__ void __launch_bounds__(256) k_dbsum(const float* __restrict__ part, int blocks, int cout,
                                               float* __restrict__ db) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) s += part[(size_t)b * cout + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] += red[0];
}

}  // namespace

// Launch of k_wgrad_halo_c8 (eight input channels, C_out = 32 or 64) with its partial
// sums; the chunking, slicing and workspace follow wgrad_halo_launch.
static ls_status wgrad_halo_c8_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cout, float* dwt,
                                      float* db, cudaStream_t stream) {
  WhArgs a = {};
  a.w = w; a.p = w + 2; a.cin = 8; a.cout = cout;
  a.cwb = cout;
  a.n_dzb = 1;
  a.gblocks = 1;
  a.groups = 1;
  const int mtiles = cout / 32;
  a.nk = 1;
  while (a.nk < kWhSteps && mtiles * a.nk * 2 <= kWhMaxIssuers) a.nk *= 2;
  a.nissue = mtiles * a.nk;
  a.idesc = tc::idesc_bf16_mn(128, 32);
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < a.nk * mtiles * 32) a.tmem_cols <<= 1;
  // input box: R rows of P 16-byte pixels plus one pixel of slack (the dropped kx = 3);
  // dZ box: R + 2 rows plus one image row of slack (the dropped row block j = 3); the
  // chunk size as in wgrad_halo_launch
  a.dz_rowb = (uint32_t)cout * 2u;
  a.dz_mode = cout == 64 ? 2u : 4u;
  for (int cp = 512; cp >= 128; cp >>= 1) {
    a.cp = cp;
    a.r = cp / w;
    a.xbox_bytes = (uint32_t)(a.r * a.p * 16);
    a.box_stride = (a.xbox_bytes + 16u + 1023u) & ~1023u;
    a.dz_blk_bytes = (uint32_t)(a.r + 2) * (uint32_t)w * a.dz_rowb;
    a.stage_bytes = a.box_stride + ((a.dz_blk_bytes + (uint32_t)w * a.dz_rowb + 1023u) & ~1023u);
    if (cp == 128 || (a.r <= h && 3 * (size_t)a.stage_bytes <= kWhSmemBudget)) break;
  }
  a.a_h = (uint32_t)((128 / w) * w) * (a.dz_rowb >> 4);  // A: 128 / w dZ rows
  a.b_h = (uint32_t)((128 / w) * a.p);                    // B: 128 / w input rows of P 16-byte pixels
  a.chunks_per_img = (h + a.r - 1) / a.r;
  const int64_t n_chunks = (int64_t)n * a.chunks_per_img;
  if (n_chunks > INT32_MAX / 2) return LS_ERR_UNSUPPORTED;
  a.n_chunks = (int)n_chunks;
  a.stages = (int)(kWhSmemBudget / a.stage_bytes);
  if (a.stages > kWhMaxStages) a.stages = kWhMaxStages;
  if (a.stages < 2) return LS_ERR_UNSUPPORTED;
  a.part_rows = 73;  // 9 * 8 rows and the bias row
  int64_t slices = kSmCount;
  if (slices > n_chunks) slices = n_chunks;
  a.chunks_per_cta = (int)((n_chunks + slices - 1) / slices);
  slices = (n_chunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
  const size_t smem = (size_t)a.stages * a.stage_bytes;
  CUtensorMap xmap, dzmap;
  const uint32_t xbox[4] = {8u, (uint32_t)a.p, (uint32_t)a.r, 1u};
  const uint32_t zbox[4] = {(uint32_t)cout, (uint32_t)w, (uint32_t)(a.r + 2), 1u};
  const uint64_t xd[4] = {8u, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t xs[3] = {16u, (uint64_t)w * 16, (uint64_t)h * w * 16};
  const uint64_t zd[4] = {(uint64_t)cout, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t zs[3] = {(uint64_t)cout * 2, (uint64_t)w * cout * 2, (uint64_t)h * w * cout * 2};
  if (!encode_tmap_bf16_4d(&xmap, x, xd, xs, xbox, 0) || !encode_tmap_bf16_4d(&dzmap, dz, zd, zs, zbox, cout * 2))
    return LS_ERR_CUDA;
  const size_t part_bytes = (size_t)slices * a.part_rows * cout * 4;
  uint8_t* ws = static_cast<uint8_t*>(workspace(kWsGradPart, part_bytes));
  if (!ws) return LS_ERR_NO_MEMORY;
  a.part = reinterpret_cast<float*>(ws);
  a.bias = db ? 1 : 0;
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_once(once, dev, [] {
        return cudaFuncSetAttribute(k_wgrad_halo_c8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kWhSmemBudget) == cudaSuccess;
      }))
    return LS_ERR_CUDA;
  k_wgrad_halo_c8<<<(unsigned)slices, kWhThreads, smem, stream>>>(xmap, dzmap, a);
  k_wsum<<<(73 * cout + 31) / 32, 32 * kWsumGroups, 0, stream>>>(a.part, (int)slices, (int64_t)a.part_rows * cout, 72,
                                                                  cout, dwt, db);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// The halo form (k_wgrad_halo) when the shapes allow it; LS_ERR_UNSUPPORTED otherwise
// (the caller falls back to the per-tap form).
static ls_status wgrad_halo_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cin, int cout,
                                   float* dwt, float* db, cudaStream_t stream) {
  const bool c8 = cin == 8 && (cout == 32 || cout == 64);
  if ((cin % 32 && !c8) || cout % 32 || cout > 128 || w < 16 || w > 128 || (w & (w - 1))) return LS_ERR_UNSUPPORTED;
  if (c8) return wgrad_halo_c8_launch(x, dz, n, h, w, cout, dwt, db, stream);
  WhArgs a = {};
  a.w = w; a.p = w + 2; a.cin = cin; a.cout = cout;
  a.cwb = cout % 64 == 0 ? 64 : 32;
  a.n_dzb = cout / a.cwb;
  const int cblocks = cin / 32;
  // channel blocks per CTA: all nine taps of a block in TMEM (3 * cout columns each),
  // at most nine issuing units, a divisor of the block count
  int gmax = 512 / (3 * cout);
  while (gmax > 1 && gmax * a.n_dzb > kWhMaxIssuers) --gmax;
  a.gblocks = 1;
  for (int gb = gmax; gb >= 1; --gb)
    if (cblocks % gb == 0) { a.gblocks = gb; break; }
  a.groups = cblocks / a.gblocks;
  const int units = a.gblocks * a.n_dzb;
  // accumulator copies: as many as TMEM and the issuing warps allow, dividing the eight
  // 16-pixel steps of a chunk
  a.nk = 1;
  while (a.nk < 8 && units * a.nk * 2 <= kWhMaxIssuers && a.gblocks * 3 * cout * a.nk * 2 <= 512) a.nk *= 2;
  a.nissue = units * a.nk;
  a.idesc = tc::idesc_bf16_mn(128, 3 * a.cwb);
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < a.nk * a.gblocks * 3 * cout) a.tmem_cols <<= 1;
  // input box: R rows of P pixels of 64 bytes, plus one pixel row of slack for the
  // dropped block kx = 3, rounded up to the 1024-byte swizzle alignment; dZ boxes of
  // R + 2 rows (a multiple of 1024 bytes: w >= 16).  The chunk is the largest of 512,
  // 256 and 128 pixels (rows within the image) with three stages in shared memory: a
  // TMA unit keeps a bounded number of boxes in flight, so larger boxes stream faster,
  // and the dZ halo rows are a smaller share.
  a.dz_rowb = (uint32_t)a.cwb * 2u;
  a.dz_mode = a.cwb == 64 ? 2u : 4u;
  for (int cp = 512; cp >= 128; cp >>= 1) {
    a.cp = cp;
    a.r = cp / w;
    a.xbox_bytes = (uint32_t)(a.r * a.p * 64);
    a.box_stride = (a.xbox_bytes + 64u + 1023u) & ~1023u;
    a.dz_blk_bytes = (uint32_t)(a.r + 2) * (uint32_t)w * a.dz_rowb;
    a.stage_bytes = (uint32_t)a.gblocks * a.box_stride + (uint32_t)a.n_dzb * a.dz_blk_bytes;
    if (cp == 128 || (a.r <= h && 3 * (size_t)a.stage_bytes <= kWhSmemBudget)) break;
  }
  a.a_h = (uint32_t)((128 / w) * a.p * 4);                    // 128 / w input rows of P 64-byte pixels
  a.b_h = (uint32_t)((128 / w) * w) * (a.dz_rowb >> 4);       // 128 / w dZ rows
  a.chunks_per_img = (h + a.r - 1) / a.r;
  const int64_t n_chunks = (int64_t)n * a.chunks_per_img;
  if (n_chunks > INT32_MAX / 2) return LS_ERR_UNSUPPORTED;
  a.n_chunks = (int)n_chunks;
  a.stages = (int)(kWhSmemBudget / a.stage_bytes);
  if (a.stages > kWhMaxStages) a.stages = kWhMaxStages;
  if (a.stages < 2) return LS_ERR_UNSUPPORTED;
  a.part_rows = 9 * cin + 1;  // the dW^T rows and the bias row
  // one CTA per SM over all groups (more than 256 TMEM columns keep a CTA alone on its
  // SM; the shared-memory request below makes sure of it); every slice non-empty
  int64_t slices = kSmCount / a.groups > 0 ? kSmCount / a.groups : 1;
  if (slices > n_chunks) slices = n_chunks;
  a.chunks_per_cta = (int)((n_chunks + slices - 1) / slices);
  slices = (n_chunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
  size_t smem = (size_t)a.stages * a.stage_bytes;
  if (a.tmem_cols > 256 && smem < 120 * 1024) smem = 120 * 1024;
  CUtensorMap xmap, dzmap;
  const uint32_t xbox[4] = {32u, (uint32_t)a.p, (uint32_t)a.r, 1u};
  const uint32_t zbox[4] = {(uint32_t)a.cwb, (uint32_t)w, (uint32_t)(a.r + 2), 1u};
  const uint64_t xd[4] = {(uint64_t)cin, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t xs[3] = {(uint64_t)cin * 2, (uint64_t)w * cin * 2, (uint64_t)h * w * cin * 2};
  const uint64_t zd[4] = {(uint64_t)cout, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t zs[3] = {(uint64_t)cout * 2, (uint64_t)w * cout * 2, (uint64_t)h * w * cout * 2};
  if (!encode_tmap_bf16_4d(&xmap, x, xd, xs, xbox, 64) || !encode_tmap_bf16_4d(&dzmap, dz, zd, zs, zbox, a.cwb * 2))
    return LS_ERR_CUDA;
  const size_t part_bytes = (size_t)slices * a.part_rows * cout * 4;
  uint8_t* ws = static_cast<uint8_t*>(workspace(kWsGradPart, part_bytes));
  if (!ws) return LS_ERR_NO_MEMORY;
  a.part = reinterpret_cast<float*>(ws);
  a.bias = db ? 1 : 0;
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_once(once, dev, [] {
        return cudaFuncSetAttribute(k_wgrad_halo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kWhSmemBudget) == cudaSuccess;
      }))
    return LS_ERR_CUDA;
  k_wgrad_halo<<<(unsigned)(slices * a.groups), kWhThreads, smem, stream>>>(xmap, dzmap, a);
  const int rows = 9 * cin;
  k_wsum<<<((rows + 1) * cout + 31) / 32, 32 * kWsumGroups, 0, stream>>>(
      a.part, (int)slices, (int64_t)a.part_rows * cout, rows, cout, dwt, db);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// Accumulates into dwt ([9*cin][cout], fp32) and db ([cout], may be NULL).
ls_status wgrad_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cin, int cout, float* dwt,
                       float* db, cudaStream_t stream) {
  if (!x || !dz || !dwt || n <= 0 || h <= 0 || w <= 0) return LS_ERR_INVALID_ARG;
  if (cin % 8 || cout < 16 || cout > 128 || cout % 16) return LS_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)dz) % 16) return LS_ERR_INVALID_ARG;
  if (ls_status st = wgrad_halo_launch(x, dz, n, h, w, cin, cout, dwt, db, stream); st != LS_ERR_UNSUPPORTED)
    return st;
  // per-tap form: a stage is 64 pixels: half a row (w = 128), whole image rows of one image, or
  // whole images
  const int64_t hw = (int64_t)h * w;
  if ((w > kWgPix && w != 2 * kWgPix) || (w <= kWgPix && kWgPix % w) || (hw % kWgPix && kWgPix % hw))
    return LS_ERR_UNSUPPORTED;
  if (hw < kWgPix && n % (kWgPix / hw)) return LS_ERR_UNSUPPORTED;
  WgArgs a = {};
  a.h = h; a.w = w; a.cin = cin; a.cout = cout; a.rows = 9 * cin;
  a.rows_per_step = hw >= kWgPix ? (w >= kWgPix ? 1 : kWgPix / w) : h;
  a.cols_per_step = w > kWgPix ? kWgPix : w;
  a.imgs_per_step = hw >= kWgPix ? 1 : (int32_t)(kWgPix / hw);
  a.pix_total = (int64_t)n * h * w;
  a.n_mtiles = (a.rows + 127) / 128;
  a.ones_row = (db && a.rows % 128) ? a.rows : -1;
  // about 3 CTAs per SM (two or three are resident at once), slices a multiple of the
  // stage (measured: 2 per SM 13.9 ms, 3 per SM 13.5 ms, 4 per SM 13.6 ms for a U-Net
  // step plus a paper-network backward)
  int64_t slices = (3 * kSmCount + a.n_mtiles - 1) / a.n_mtiles;
  int64_t per = (a.pix_total + slices - 1) / slices;
  per = (per + kWgPix - 1) / kWgPix * kWgPix;
  if (per < 1024) per = 1024;
  a.pix_per_cta = per;
  slices = (a.pix_total + per - 1) / per;
  a.idesc = tc::idesc_bf16_mn(128, cout);
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < cout) a.tmem_cols <<= 1;
  a.b_bytes = (uint32_t)cout * kWgPix * 2;
  // widest channel blocks per TMA load (fewer, longer rows), dividing the channel counts
  a.cw = cin % 64 == 0 ? 64 : cin % 32 == 0 ? 32 : cin % 16 == 0 ? 16 : 8;
  a.cwb = cout % 64 == 0 ? 64 : cout % 32 == 0 ? 32 : cout % 16 == 0 ? 16 : 8;
  CUtensorMap xmap, dzmap;
  const uint32_t box[4] = {(uint32_t)a.cw, (uint32_t)a.cols_per_step, (uint32_t)a.rows_per_step,
                           (uint32_t)a.imgs_per_step};
  const uint32_t boxb[4] = {(uint32_t)a.cwb, (uint32_t)a.cols_per_step, (uint32_t)a.rows_per_step,
                            (uint32_t)a.imgs_per_step};
  const uint64_t xd[4] = {(uint64_t)cin, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t xs[3] = {(uint64_t)cin * 2, (uint64_t)w * cin * 2, (uint64_t)h * w * cin * 2};
  const uint64_t zd[4] = {(uint64_t)cout, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t zs[3] = {(uint64_t)cout * 2, (uint64_t)w * cout * 2, (uint64_t)h * w * cout * 2};
  if (!encode_tmap_bf16_4d(&xmap, x, xd, xs, box, a.cw == 8 ? 0 : a.cw * 2) ||
      !encode_tmap_bf16_4d(&dzmap, dz, zd, zs, boxb, a.cwb == 8 ? 0 : a.cwb * 2))
    return LS_ERR_CUDA;
  const size_t smem = (size_t)kWgStages * (kWgABytes + a.b_bytes);
  const int64_t ctas = slices * a.n_mtiles;
  const size_t part_bytes = (size_t)ctas * 128 * cout * 4, db_bytes = (size_t)kColsumBlocks * cout * 4;
  uint8_t* ws = static_cast<uint8_t*>(workspace(kWsGradPart, part_bytes + db_bytes));
  if (!ws) return LS_ERR_NO_MEMORY;
  a.part = reinterpret_cast<float*>(ws);
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_once(once, dev, [] {
        return cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kWgStages * (kWgABytes + 128 * kWgPix * 2)) == cudaSuccess;
      }))
    return LS_ERR_CUDA;
  k_wgrad<<<(unsigned)ctas, kWgThreads, smem, stream>>>(xmap, dzmap, a);
  const bool ones = a.ones_row >= 0;
  k_wsum<<<((a.rows + 1) * cout + 31) / 32, 32 * kWsumGroups, 0, stream>>>(
      a.part, (int)slices, (int64_t)a.n_mtiles * 128 * cout, a.rows, cout, dwt, ones ? db : nullptr);
  if (db && !ones) {
    float* dbp = reinterpret_cast<float*>(ws + part_bytes);
    const int threads = 256 - 256 % (cout / 8);  // whole pixel lanes of cout/8 threads
    k_colsum<<<kColsumBlocks, threads, 0, stream>>>(dz, a.pix_total, cout, dbp);
    k_dbsum<<<cout, 256, 0, stream>>>(dbp, kColsumBlocks, cout, db);
  }
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace ls

extern "C" ls_status ls_conv3x3_wgrad(const uint16_t* x, const uint16_t* dz, const ls_conv_shape* shape, float* dw,
                                      float* db, ls_stream_t stream) {
  if (!shape) return LS_ERR_INVALID_ARG;
  return ls::wgrad_launch(x, dz, shape->n, shape->h, shape->w, shape->cin, shape->cout, dw, db,
                          reinterpret_cast<cudaStream_t>(stream));
}
