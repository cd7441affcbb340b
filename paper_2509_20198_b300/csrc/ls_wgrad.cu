// Weight and bias gradients of a 3x3 convolution on the tensor cores (training of the
// learned filler, Sec. 3.4).  dW^T[k][o] = sum_p X_shift(k)[p] dZ[p][o] with
// k = tap * C_in + c_in: a GEMM with M = 9*C_in (tiles of 128 rows), N = C_out and
// K = pixels (64 per stage).  Each CTA owns one 128-row tile and one slice of pixels
// and stores its partial sums; k_wsum adds them to the FP32 gradient in a fixed order,
// so the result does not depend on CTA scheduling (training is reproducible).
//
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

// dW^T[k][o] += sum over slices of the CTA partials, slices in increasing order (loads
// issued eight ahead of the in-order additions).
// With db, row `rows` of the partials (the ones row) is the bias gradient: into db.
__global__ void k_wsum(const float* __restrict__ part, int slices, int n_mtiles, int rows, int cout,
                       float* __restrict__ dwt, float* __restrict__ db) {
  const int total = (rows + (db ? 1 : 0)) * cout;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k = e / cout, o = e - k * cout;
    const int mt = k >> 7, row = k & 127;
    const size_t stride = (size_t)n_mtiles * 128 * cout;
    const float* p = part + ((size_t)mt * 128 + row) * cout + o;
    float s = 0.f;
    int sl = 0;
    for (; sl + 8 <= slices; sl += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = p[(size_t)(sl + i) * stride];
#pragma unroll
      for (int i = 0; i < 8; ++i) s += v[i];
    }
    for (; sl < slices; ++sl) s += p[(size_t)sl * stride];
    if (k < rows) dwt[e] += s;
    else db[o] += s;
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

// Accumulates into dwt ([9*cin][cout], fp32) and db ([cout], may be NULL).
ls_status wgrad_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cin, int cout, float* dwt,
                       float* db, cudaStream_t stream) {
  if (!x || !dz || !dwt || n <= 0 || h <= 0 || w <= 0) return LS_ERR_INVALID_ARG;
  if (cin % 8 || cout < 16 || cout > 128 || cout % 16) return LS_ERR_UNSUPPORTED;
  // a stage is 64 pixels: half a row (w = 128), whole image rows of one image, or
  // whole images
  const int64_t hw = (int64_t)h * w;
  if ((w > kWgPix && w != 2 * kWgPix) || (w <= kWgPix && kWgPix % w) || (hw % kWgPix && kWgPix % hw))
    return LS_ERR_UNSUPPORTED;
  if (hw < kWgPix && n % (kWgPix / hw)) return LS_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)dz) % 16) return LS_ERR_INVALID_ARG;
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
  k_wsum<<<grid_cap(((a.rows + 1) * cout + 255) / 256, kSmCount * 4), 256, 0, stream>>>(
      a.part, (int)slices, a.n_mtiles, a.rows, cout, dwt, ones ? db : nullptr);
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
