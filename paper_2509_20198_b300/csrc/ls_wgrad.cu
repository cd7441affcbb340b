// Weight and bias gradients of a 3x3 convolution on the tensor cores (training of the
// learned filler, Sec. 3.4).  dW^T[k][o] = sum_p X_shift(k)[p] dZ[p][o] with
// k = tap * C_in + c_in: a GEMM with M = 9*C_in (tiles of 128 rows), N = C_out and
// K = pixels (64 per stage).  Each CTA owns one 128-row tile and one slice of pixels
// and stores its partial sums; k_wsum adds them to the FP32 gradient in a fixed order,
// so the result does not depend on CTA scheduling (training is reproducible).
//
// Both operands are stored pixel-minor (NHWC), while the MMA reads K-major tiles
// (pixels contiguous), so every stage is transposed once in shared memory:
//  warp 0     TMA producer: the M tile's rows are 128 / cw blocks of cw channels of one
//             tap (cw = 64, 32, 16 or 8 dividing C_in): one 4-D tiled load per block of the
//             tap-shifted input (cw channels x 64 pixels: whole rows, or half a row of a
//             128-wide image; zero-filled outside the image: the padding; rows of 128 / 64 bytes are written with the 128B / 64B
//             swizzle), and dZ in blocks of cwb output channels, into a raw ring;
//  warps 1-4  transpose raw -> K-major core matrices with ldmatrix (8x8 b16 blocks:
//             8 pixel rows of one 16-byte channel chunk, un-swizzled by address) and
//             stmatrix.trans, 4 blocks per instruction pair, then make the tile visible
//             to the tensor core (fence.proxy.async);
//             at the end they read the accumulator from TMEM (one row per thread);
//  warp 5     issues tcgen05.mma kind::f16 (M=128, N=C_out, K=16) and commits.
// The bias gradient is a column sum of dZ.  When 9*C_in leaves padding rows in the last
// M tile, the first padding row of every A stage is set to ones, so the same MMAs sum
// dZ over the pixels into that row and k_wsum passes it on as the bias gradient;
// otherwise k_colsum (per-block partials) and k_dbsum (in block order) compute it.
#include <cuda_bf16.h>

#include "ls_tc.cuh"

namespace ls {
namespace {

constexpr int kWgThreads = 192;
// Two raw and two operand stages: at C_out <= 64 a CTA then needs at most 96 KB of
// shared memory and two or three CTAs share an SM, whose independent pipelines hide the
// load and transpose latency better than deeper rings in one CTA (measured: 3 + 3
// stages, one CTA per SM, made the weight gradients 25 % slower)
constexpr int kWgRaw = 2;   // raw (TMA) stages
constexpr int kWgOps = 2;   // operand (K-major) stages
constexpr int kWgPix = 64;  // pixels (K) per stage
constexpr int kWgABytes = 128 * kWgPix * 2;

// Byte offset in a raw stage of channel ch (multiple of 8) of pixel px, the stage being
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
  __shared__ __align__(8) uint64_t raw_full[kWgRaw], raw_empty[kWgRaw], op_full[kWgOps], op_empty[kWgOps], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_bytes = kWgABytes + a.b_bytes;
  uint8_t* raw = smem;
  uint8_t* ops = smem + (size_t)kWgRaw * stage_bytes;
  const int mt = blockIdx.x % a.n_mtiles;
  const int64_t slice = blockIdx.x / a.n_mtiles;
  const int64_t p_begin = slice * a.pix_per_cta;
  const int64_t p_end = min(p_begin + a.pix_per_cta, a.pix_total);
  const int n_steps = (int)((p_end - p_begin + kWgPix - 1) / kWgPix);
  const int m0 = mt * 128;
  const int n_og = a.cout / 8;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kWgRaw; ++i) {
      tc::mbar_init(&raw_full[i], 1);
      tc::mbar_init(&raw_empty[i], 4);
    }
    for (int i = 0; i < kWgOps; ++i) {
      tc::mbar_init(&op_full[i], 4);
      tc::mbar_init(&op_empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    tc::prefetch_tmap(&dzmap);
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
      const int blk_a = kWgPix * a.cw * 2, blk_b = kWgPix * a.cwb * 2;  // bytes per block load
      int n_valid = 0;  // blocks of the tile inside the 9*C_in rows
      int bc[16], bx[16], by[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = m0 + i * a.cw;  // a block never straddles two taps: cw divides C_in
        bc[i] = bx[i] = by[i] = 0;
        if (i < 128 / a.cw && k < a.rows) {
          const int tap = k / a.cin;
          bc[i] = k - tap * a.cin;
          by[i] = tap / 3 - 1;
          bx[i] = tap - (tap / 3) * 3 - 1;
          ++n_valid;
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
        if (!tc::mbar_wait(&raw_empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
        uint8_t* RA = raw + (size_t)slot * stage_bytes;
        uint8_t* RB = RA + kWgABytes;
        tc::mbar_arrive_expect_tx(&raw_full[slot], bytes);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < n_valid)
            tc::tma_load_4d(RA + i * blk_a, &xmap, bc[i], x0 + bx[i], y0 + by[i], n0, &raw_full[slot]);
        for (int ob = 0; ob < n_ob; ++ob)
          tc::tma_load_4d(RB + ob * blk_b, &dzmap, ob * a.cwb, x0, y0, n0, &raw_full[slot]);
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
        if (++slot == kWgRaw) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (warp <= 4) {
    // ---------------- transposers (warps 1-4), then epilogue
    const int tw = warp - 1;
    const int mi = lane >> 3, mj = lane & 7;  // matrix of this lane's row address, row within it
    const int n_aitems = 32;                  // 16 row groups x 2 quads of pixel groups
    const int n_items = n_aitems + n_og * 2;
    // this warp's items (at most 8 of A and 8 of B): lane offsets from the raw stage's
    // and the operand stage's bases, computed once
    uint32_t src[16], dst[16];
    int mine = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int it = tw + 4 * q;
      src[q] = dst[q] = 0u;
      if (it < n_items) {
        ++mine;
        if (it < n_aitems) {
          // A block (row group g, pixel group pg): raw rows = pixels, K-major core
          // matrix rows = channels (16 B = 8 pixels)
          const int g = it >> 1, pg = (it & 1) * 4 + mi;
          src[q] = raw_off(g * 8, pg * 8 + mj, a.cw);
          dst[q] = g * 128 + pg * 2048 + mj * 16;
        } else {
          const int u = it - n_aitems, og = u >> 1, pg = (u & 1) * 4 + mi;
          src[q] = kWgABytes + raw_off(og * 8, pg * 8 + mj, a.cwb);
          dst[q] = kWgABytes + og * 128 + pg * (a.cout * 16) + mj * 16;
        }
      }
    }
    // the ones row (local row lr of this tile): its two halves of 4 pixel groups belong
    // to items 2 g1 and 2 g1 + 1, written by the warps that transpose those items
    const int lr = a.ones_row - m0;
    const bool has_ones = a.ones_row >= 0 && lr >= 0 && lr < 128;
    const int g1 = lr >> 3, rr = lr & 7;
    int ones_h = -1;  // half (pixel groups 4 h .. 4 h + 3) this warp writes
    if (has_ones) {
      if ((2 * g1) % 4 == tw) ones_h = 0;
      else if ((2 * g1 + 1) % 4 == tw) ones_h = 1;
    }
    for (int s = 0; s < n_steps && !abort_flag; ++s) {
      const int rs = s % kWgRaw, os = s % kWgOps;
      if (!tc::mbar_wait(&raw_full[rs], (uint32_t)(s / kWgRaw) & 1u)) { abort_flag = 1; break; }
      if (!tc::mbar_wait(&op_empty[os], ((uint32_t)(s / kWgOps) & 1u) ^ 1u)) { abort_flag = 1; break; }
      const uint32_t RA = tc::saddr(raw + (size_t)rs * stage_bytes);
      const uint32_t OA = tc::saddr(ops + (size_t)os * stage_bytes);
      // four loads in flight before their stores
#pragma unroll
      for (int q0 = 0; q0 < 16; q0 += 4) {
        if (q0 < mine) {
          uint32_t r[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q0 + q < mine) tc::ldmatrix_x4(RA + src[q0 + q], r[q]);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q0 + q < mine) tc::stmatrix_x4_trans(OA + dst[q0 + q], r[q]);
        }
      }
      if (ones_h >= 0) {
        __syncwarp();
        if (lane < 4) {
          const uint32_t one2 = 0x3F803F80u;  // two bf16 1.0
          const uint32_t adr = OA + (uint32_t)(g1 * 128 + (ones_h * 4 + lane) * 2048 + rr * 16);
          asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(adr), "r"(one2) : "memory");
        }
        __syncwarp();
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&raw_empty[rs]);
        tc::mbar_arrive(&op_full[os]);
      }
    }
    // ---------------- epilogue: TMEM row per thread into this CTA's partial block
    if (n_steps > 0 && !abort_flag && tc::mbar_wait(&done, 0)) {
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
    // ---------------- MMA issuer (warp 5): descriptors are the stage's base + offsets
    const uint32_t o0 = tc::saddr(ops);
    const uint64_t adesc0 = tc::sdesc(o0, 2048, 128);
    const uint64_t bdesc0 = tc::sdesc(o0 + kWgABytes, a.cout * 16, 128);
    for (int s = 0; s < n_steps && !abort_flag; ++s) {
      const int os = s % kWgOps;
      if (!tc::mbar_wait(&op_full[os], (uint32_t)(s / kWgOps) & 1u)) { abort_flag = 1; break; }
      tc::fence_after();
      const uint64_t so = (uint64_t)((os * stage_bytes) >> 4);
#pragma unroll
      for (int j = 0; j < kWgPix / 16; ++j)
        tc::mma_bf16(taddr, adesc0 + so + (uint64_t)(j * 4096 >> 4), bdesc0 + so + (uint64_t)((j * 2 * a.cout * 16) >> 4),
                     a.idesc, (s > 0 || j > 0) ? 1u : 0u);
      tc::mma_commit(&op_empty[os]);
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
  a.idesc = tc::idesc_bf16(128, cout);
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
  const size_t smem = (size_t)(kWgRaw + kWgOps) * (kWgABytes + a.b_bytes);
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
                                    (kWgRaw + kWgOps) * (kWgABytes + 128 * kWgPix * 2)) == cudaSuccess;
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
