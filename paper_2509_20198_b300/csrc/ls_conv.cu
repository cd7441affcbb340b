// 3x3 convolution (stride 1, zero padding 1) on the 5th-generation tensor cores as an
// implicit GEMM: M = 128 output pixels, N = C_out, K = 9 * C_in, BF16 operands, FP32
// accumulation in TMEM.  This is the convolution of the learned heightmap filler
// (Sec. 3.4: a U-Net-inspired CNN refines the heightmaps) in its forward pass and,
// with transposed and flipped weights, in the input-gradient pass of training.
//
// Per CTA (persistent over 128-pixel tiles, 6 warps, a ring of up to 8 operand stages):
// three CTAs per SM with about 70 KB of stages each where their accumulator pairs fit
// the TMEM together (C_out <= 64), two with about 108 KB (C_out <= 128), else one with
// about 200 KB.  Independent pipelines per SM hide the TMA and epilogue latency better
// than one deeper ring (four CTAs per SM measured slower than three).
//  warp 0  TMA producer: per 8-channel chunk of one tap, one 4-D tiled TMA load of
//          the shifted 128-pixel slab (out-of-range rows/columns are zero-filled by
//          the TMA unit: that is the padding) and one 1-D bulk copy of the
//          pre-packed weight block of the stage;
//  warp 1  MMA issuer: tcgen05.mma kind::f16 (M=128, N=C_out, K=16) per chunk pair,
//          tcgen05.commit to free the stage and to publish a finished accumulator;
//  warps 2-5 epilogue: tcgen05.ld of the accumulator (one pixel per thread), bias,
//          ReLU or a ReLU-derivative mask, BF16 store (NHWC).
// Two TMEM accumulators let the epilogue of tile i overlap the MMAs of tile i+1.
// Operands are K-major without swizzle: an A stage holds up to 8 chunks of
// 128 rows x 16 bytes (LBO 2048 B between chunks, SBO 128 B between 8-row groups);
// the packed weights of a stage are C_out rows x 8 chunks (LBO C_out*16 B, SBO 128 B).
// Images 64 or 128 pixels wide (H a multiple of 64) take the halo form further down
// (k_conv3x3_halo): one box per tile and channel block serves all nine taps.
#include <cuda_bf16.h>

#include <algorithm>

#include "ls_tc.cuh"

namespace ls {

bool encode_tmap_bf16_4d(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides[3],
                         const uint32_t box[4], int swizzle_bytes) {
  // looked up once (a function-local static: thread-safe initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  if (!fn) return false;
  cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t s[3] = {strides[0], strides[1], strides[2]};
  cuuint32_t b[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t e[4] = {1, 1, 1, 1};
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), d, s, b, e,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

constexpr int kConvThreads = 192;
constexpr int kConvStages = 8;            // most stages; a launch uses as many as fit
constexpr size_t kConvSmemBudget = 200 * 1024;
constexpr size_t kConvSmemBudget2 = 108 * 1024;  // per CTA with two CTAs per SM
constexpr size_t kConvSmemBudget3 = 70 * 1024;   // per CTA with three CTAs per SM
constexpr int kChunksPerStage = 8;
constexpr int kAStageBytes = kChunksPerStage * 2048;
constexpr int kMaxLoads = 9 * 256 / 8;  // TMA loads per 128-pixel tile at most (C_in <= 256)

struct ConvArgs {
  const uint16_t* __restrict__ wpk;
  const float* __restrict__ bias;
  const uint16_t* __restrict__ mask;
  uint16_t* __restrict__ y;
  int32_t cin, cout, cpt, kc_real, kc, n_stages, n_mtiles;
  int32_t tiles_per_img, rows_per_tile, imgs_per_tile;
  int32_t relu;
  // output: channel group g (ygroup channels, a multiple of 16) of every pixel goes to
  // tensor g, ygstride elements after tensor g - 1 (one tensor: ygroup = cout)
  int32_t ygroup;
  int64_t ygstride;
  uint32_t acc_cols, tmem_cols, stage_bytes, idesc;
  int32_t ring;  // stages in use (<= kConvStages)
  // A operand: cw-channel blocks of one tap per TMA load (cw = 64, 32 or 16: rows of
  // 128 / 64 / 32 bytes, 128B / 64B / 32B swizzle; cw = 8: 8 unswizzled chunks per stage)
  int32_t cw, cblocks, blocks_per_stage, n_blocks;
  uint32_t blk_bytes, sbo_a, swz;
  // input channels [0, c_split) come from the first tensor map, the rest from the second
  // (an upsampled tensor and its skip connection read without a concatenated copy)
  int32_t c_split;
  int32_t wide;  // outputs 32-byte aligned: 256-bit stores
  // up2: y is the 2x nearest-neighbour upsampling of the output ([n][2h][2w][cout])
  int32_t up2, img_h, img_w;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// The values a BF16 store of v keeps (v rounded to bf16 and back), packed as stored
__device__ __forceinline__ void round_bf16_16(float (&v)[16], uint4& o0, uint4& o1) {
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    w[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
  o0 = make_uint4(w[0], w[1], w[2], w[3]);
  o1 = make_uint4(w[4], w[5], w[6], w[7]);
}

// 32 bytes of BF16 at yp: one 256-bit store (a whole L2 sector per thread, half the
// store instructions and L1 wavefronts of two 16-byte stores) when yp is 32-byte aligned
__device__ __forceinline__ void store32(uint16_t* yp, const uint4& o0, const uint4& o1, bool wide) {
  if (wide) {
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(yp), "r"(o0.x), "r"(o0.y), "r"(o0.z),
                 "r"(o0.w), "r"(o1.x), "r"(o1.y), "r"(o1.z), "r"(o1.w)
                 : "memory");
  } else {
    *reinterpret_cast<uint4*>(yp) = o0;
    *reinterpret_cast<uint4*>(yp + 8) = o1;
  }
}

// 16 accumulator columns of one output pixel: + bias, ReLU or the ReLU-derivative mask
// (a bf16 mask value > 0 keeps the gradient), BF16 store of 32 bytes
__device__ __forceinline__ void epilogue16(float (&v)[16], const float* bias, int relu, const uint16_t* mp,
                                           uint16_t* yp, bool wide) {
  if (bias) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] += __ldg(bias + i);
  }
  if (relu) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
  }
  if (mp) {
    const uint4 m0 = *reinterpret_cast<const uint4*>(mp);
    const uint4 m1 = *reinterpret_cast<const uint4*>(mp + 8);
    const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      // bf16 > 0: sign bit clear and not +0
      const uint32_t lo = mw[i] & 0xffffu, hi = mw[i] >> 16;
      if (!(lo != 0u && !(lo & 0x8000u))) v[2 * i] = 0.f;
      if (!(hi != 0u && !(hi & 0x8000u))) v[2 * i + 1] = 0.f;
    }
  }
  uint4 o0, o1;
  o0.x = pack_bf16x2(v[0], v[1]); o0.y = pack_bf16x2(v[2], v[3]);
  o0.z = pack_bf16x2(v[4], v[5]); o0.w = pack_bf16x2(v[6], v[7]);
  o1.x = pack_bf16x2(v[8], v[9]); o1.y = pack_bf16x2(v[10], v[11]);
  o1.z = pack_bf16x2(v[12], v[13]); o1.w = pack_bf16x2(v[14], v[15]);
  store32(yp, o0, o1, wide);
}

// kUp2: the epilogue stores the output as its 2x upsampling (ConvArgs::up2), a
// separate instance
template <bool kUp2>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv3x3(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap xmap2,
              const ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kConvStages], empty[kConvStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  // per TMA load of a tile: channel offset | (kx << 16) | (ky << 20), in load order
  __shared__ uint32_t ktab[kMaxLoads];
  __shared__ float s_bias[256];  // the epilogue's bias (C_out <= 256)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < a.cout; i += blockDim.x) s_bias[i] = a.bias ? a.bias[i] : 0.f;
  const int n_loads = a.cw == 8 ? a.kc : a.n_blocks;
  for (int i = threadIdx.x; i < n_loads; i += blockDim.x) {
    int ci, tap;
    if (a.cw == 8) {
      const int c = i < a.kc_real ? i : 0;  // padding chunk: any finite data, its weights are zero
      tap = c / a.cpt;
      ci = (c - tap * a.cpt) * 8;
    } else {
      tap = i / a.cblocks;
      ci = (i - tap * a.cblocks) * a.cw;
    }
    const int ky = tap / 3, kx = tap - ky * 3;
    ktab[i] = (uint32_t)ci | ((uint32_t)kx << 16) | ((uint32_t)ky << 20);
  }

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.ring; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], 128);
    }
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    if (a.c_split < a.cin) tc::prefetch_tmap(&xmap2);
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int slot = 0;
    uint32_t ph = 0;
    const int per_stage = a.cw == 8 ? kChunksPerStage : a.blocks_per_stage;
    const uint32_t load_bytes = a.cw == 8 ? 2048u : a.blk_bytes;
    for (int m = blockIdx.x; m < a.n_mtiles && !abort_flag; m += gridDim.x) {
      int n0, y0;
      if (a.imgs_per_tile == 1) {
        n0 = m / a.tiles_per_img;
        y0 = (m - n0 * a.tiles_per_img) * a.rows_per_tile;
      } else {
        n0 = m * a.imgs_per_tile;
        y0 = 0;
      }
      int li = 0;  // next TMA load of this tile
      for (int s = 0; s < a.n_stages; ++s) {
        if (!tc::mbar_wait(&empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
        const int c0 = s * kChunksPerStage;
        const int nc = min(kChunksPerStage, a.kc - c0);
        const int nl = min(per_stage, n_loads - li);
        uint8_t* A = smem + (size_t)slot * a.stage_bytes;
        uint8_t* B = A + kAStageBytes;
        tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)nl * load_bytes + (uint32_t)(nc * a.cout * 16));
        for (int k = 0; k < nl; ++k, ++li) {
          const uint32_t e = ktab[li];
          const int ci = (int)(e & 0xffffu);
          const bool second = ci >= a.c_split;
          tc::tma_load_4d(A + k * load_bytes, second ? &xmap2 : &xmap, second ? ci - a.c_split : ci,
                          (int)((e >> 16) & 15u) - 1,
                          y0 + (int)(e >> 20) - 1, n0, &full[slot]);
        }
        tc::bulk_load(B, a.wpk + (size_t)c0 * a.cout * 8, (uint32_t)(nc * a.cout * 16), &full[slot]);
        if (++slot == a.ring) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: descriptors are the stage's base plus fixed offsets,
    // so each MMA costs one add (a single thread feeds the tensor core)
    uint32_t aoff[4], boff[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      aoff[j] = a.cw == 8 ? (uint32_t)j * 4096u
                          : (uint32_t)((j * 16) / a.cw) * a.blk_bytes + (uint32_t)(((j * 16) % a.cw) / 16) * 32u;
      boff[j] = (uint32_t)(j * 2 * a.cout * 16);
    }
    const uint32_t s0 = tc::saddr(smem);
    const uint64_t adesc0 = a.cw == 8 ? tc::sdesc(s0, 2048, 128) : tc::sdesc_sw(s0, a.sbo_a, a.swz);
    const uint64_t bdesc0 = tc::sdesc(s0 + kAStageBytes, a.cout * 16, 128);
    const int last_nk = (a.kc - (a.n_stages - 1) * kChunksPerStage) / 2;
    int slot = 0, ai = 0;
    uint32_t ph = 0;
    for (int m = blockIdx.x; m < a.n_mtiles && !abort_flag; m += gridDim.x, ++ai) {
      const int acc = ai & 1;
      const uint32_t aph = (uint32_t)(ai >> 1) & 1u;
      if (!tc::mbar_wait(&tempty[acc], aph ^ 1u)) { abort_flag = 1; break; }
      tc::fence_after();
      const uint32_t d = taddr + (uint32_t)acc * a.acc_cols;
      for (int s = 0; s < a.n_stages; ++s) {
        if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
        tc::fence_after();
        const uint64_t so = (uint64_t)((slot * a.stage_bytes) >> 4);
        const int nk = s == a.n_stages - 1 ? last_nk : 4;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < nk)
            tc::mma_bf16(d, adesc0 + so + (aoff[j] >> 4), bdesc0 + so + (boff[j] >> 4), a.idesc,
                         (s > 0 || j > 0) ? 1u : 0u);
        tc::mma_commit(&empty[slot]);
        if (++slot == a.ring) { slot = 0; ph ^= 1u; }
      }
      tc::mma_commit(&tfull[acc]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: one output pixel per thread
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int ai = 0;
    for (int m = blockIdx.x; m < a.n_mtiles && !abort_flag; m += gridDim.x, ++ai) {
      const int acc = ai & 1;
      const uint32_t aph = (uint32_t)(ai >> 1) & 1u;
      if (!tc::mbar_wait(&tfull[acc], aph)) { abort_flag = 1; break; }
      tc::fence_after();
      const size_t pix = (size_t)m * 128 + row;
      const uint16_t* mp = a.mask ? a.mask + pix * a.cout : nullptr;
      for (int c32 = 0; c32 < a.cout; c32 += 32) {
        // 32 accumulator columns with one wait (columns past cout are inside acc_cols, a
        // power of two >= 32)
        float v32[32];
        tc::tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * a.acc_cols + (uint32_t)c32, v32);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int c0 = c32 + hh * 16;
          if (c0 >= a.cout) break;
          const int g = a.ygroup == a.cout ? 0 : c0 / a.ygroup;  // no division for one group
          uint16_t* yp = a.y + ((int64_t)g * a.ygstride + (int64_t)pix * a.ygroup + (c0 - g * a.ygroup));
          float v[16];
          if (a.bias) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = v32[hh * 16 + i] + s_bias[c0 + i];
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = v32[hh * 16 + i];
          }
          if (kUp2) {
            // output pixel (nn, yy, xx) at its four positions of the 2x upsampling
            const size_t hw = (size_t)a.img_h * a.img_w;
            const size_t nn = pix / hw, r = pix - nn * hw;
            const int yy = (int)(r / (size_t)a.img_w), xx = (int)(r - (size_t)yy * a.img_w);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
            uint4 o0, o1;
            round_bf16_16(v, o0, o1);
            uint16_t* up = a.y + (((nn * 2 * a.img_h + 2 * yy) * (2 * a.img_w) + 2 * xx) * a.cout + c0);
            const size_t row = (size_t)2 * a.img_w * a.cout;
            store32(up, o0, o1, a.wide != 0);
            store32(up + a.cout, o0, o1, a.wide != 0);
            store32(up + row, o0, o1, a.wide != 0);
            store32(up + row + a.cout, o0, o1, a.wide != 0);
          } else {
            epilogue16(v, nullptr, a.relu, mp ? mp + c0 : nullptr, yp, a.wide != 0);
          }
        }
      }
      tc::fence_before();
      tc::mbar_arrive(&tempty[acc]);
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
// Halo form for images W = 32, 64 or 128 wide: the output is computed on a grid of
// P = W + 2 slots per row (two junk slots per row, discarded; an image's slots are
// padded to whole 128-slot tiles, the slots beyond its last row junk too), so that the
// input pixel of output slot s under tap (ky, kx) is padded-input slot s + ky*P + kx,
// a fixed row offset.  One TMA box of the padded rows around a 128-slot tile (x from
// -1 to W, rows y0-1 .. y0+bh-2, zero-filled outside the image) then serves all nine
// taps of one channel block: each MMA's A operand starts a whole number of 2*cw-byte
// rows into the box (the swizzle is a function of the absolute shared address, so any
// row offset reads the rows that the TMA wrote).  The packed weights of the layer stay
// in shared memory for the whole launch, and the CTA runs up to four independent
// pipelines that share them, one tcgen05.mma issuer each (one issuing thread is
// accepted about one M=128 MMA per 150 cycles whatever N; the SM takes about four):
//  warp 6g      TMA producer of pipeline g (one box per tile and channel block);
//  warp 6g + 1  MMA issuer: 9 taps x cw/16 MMAs per box (8-channel inputs: two taps
//               per K=16 MMA, the second tap's rows LBO bytes after the first's);
//  warps 6g+2.. epilogue of pipeline g (one slot per thread; junk slots not stored).
constexpr int kHaloMaxPipes = 4;
constexpr int kHaloRingMax = 8;  // ring slots declared per pipeline
constexpr int kHaloRingUse = 4;  // boxes per pipeline a launch uses at most (as many as fit)
constexpr int kHaloThreadsPerPipe = 192;
constexpr size_t kHaloSmemBudget = 223 * 1024;  // + the static bias and head copies: the 227 KB limit
constexpr int kHaloMaxCout = 64;                 // four pipelines of two accumulators

struct HaloArgs {
  const uint16_t* __restrict__ wpk;
  const float* __restrict__ bias;
  const uint16_t* __restrict__ mask;
  uint16_t* __restrict__ y;
  int32_t cin, cout, cpt, cw, cblocks, relu, ygroup;
  int64_t ygstride;
  int32_t w, h, p, bh;          // image width, height, slots per row (w + 2), box rows
  // a box serves tpb consecutive 128-slot tiles of an image, one per pipeline of a team
  // of tpb pipelines (npipes / tpb teams, each with one producer and one ring)
  int32_t tpb, teams, spi, n_super, slots_img;  // boxes per image, in all, slots per image
  int32_t npipes, ring;
  // optional 1x1 head fused into the epilogue: head_y[pixel][o] = head[head_out * cout + o]
  // + sum_c head[o * cout + c] * out[c] over the bf16-rounded outputs (store_y: also
  // store the BF16 output itself)
  const float* __restrict__ head;
  float* __restrict__ head_y;
  int32_t head_out, store_y;
  uint32_t wbytes, box_bytes, box_stride, acc_cols, tmem_cols, idesc, swz, rowb;
  int32_t c_split;  // input channels [0, c_split) from the first map, the rest from the second
  int32_t wide;     // outputs 32-byte aligned: 256-bit stores
  // streamed weights (wstage > 0, wbytes = 0): each stage holds, wofs bytes after its
  // box, the nine taps' weights of its channel block (wtap bytes per tap)
  uint32_t wstage, wtap, wofs;
  // multiply-shift divisions by p and by spi (spi > 1) instead of a division routine in
  // the per-tile index arithmetic of the three roles
  FastDiv31 f_p, f_spi;
  // up2: y is the 2x nearest-neighbour upsampling of the output ([n][2h][2w][cout]):
  // each output pixel's values are stored at its four positions there
  int32_t up2;
};

__device__ __forceinline__ int halo_img(const HaloArgs& a, int st) {
  return a.spi > 1 ? (int)fdiv31((uint32_t)st, a.f_spi) : st;
}

// kUp2: the epilogue stores the output as its 2x upsampling (HaloArgs::up2); a separate
// instance, so that the plain one keeps its registers
template <bool kUp2>
__global__ void __launch_bounds__(kHaloMaxPipes * kHaloThreadsPerPipe, 1)
    k_conv3x3_halo(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap xmap2,
                   const HaloArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kHaloMaxPipes][kHaloRingMax], empty[kHaloMaxPipes][kHaloRingMax];
  __shared__ __align__(8) uint64_t tfull[kHaloMaxPipes][2], tempty[kHaloMaxPipes][2], wbar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  // the epilogue's bias and head weights, read from shared memory instead of one global
  // load per element and pixel
  __shared__ float s_bias[kHaloMaxCout], s_head[8 * kHaloMaxCout + 8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // pipeline g and role (0 producer, 1 issuer, 2-5 epilogue): warps [0, np) issue the
  // MMAs, [np, 2np) produce, the rest are the epilogues, four consecutive warps per
  // pipeline (their warp index mod 4 selects the TMEM lane quadrant).  With np = 4 each
  // SM sub-partition (warp index mod 4) runs one issuer, one producer and four epilogue
  // warps; pipelines of consecutive warps put two issuers on each of two sub-partitions.
  const int np_ = a.npipes;
  const int g = warp < np_ ? warp : warp < 2 * np_ ? warp - np_ : (warp - 2 * np_) >> 2;
  const int role = warp < np_ ? 1 : warp < 2 * np_ ? 0 : 2 + ((warp - 2 * np_) & 3);
  for (int i = threadIdx.x; i < a.cout; i += blockDim.x) s_bias[i] = a.bias ? a.bias[i] : 0.f;
  if (a.head)
    for (int i = threadIdx.x; i < a.head_out * (a.cout + 1); i += blockDim.x) s_head[i] = a.head[i];
  uint8_t* wsm = smem;                          // packed weights (a.wbytes)
  uint8_t* boxes = smem + ((a.wbytes + 1023u) & ~1023u);  // 1024-aligned: the swizzle atoms
  if (threadIdx.x == 0) {
    for (int q = 0; q < a.teams; ++q) {
      for (int i = 0; i < a.ring; ++i) {
        tc::mbar_init(&full[q][i], 1);
        tc::mbar_init(&empty[q][i], (uint32_t)a.tpb);  // released by each issuer of the team
      }
    }
    for (int q = 0; q < a.npipes; ++q) {
      for (int i = 0; i < 2; ++i) {
        tc::mbar_init(&tfull[q][i], 1);
        tc::mbar_init(&tempty[q][i], 128);
      }
    }
    tc::mbar_init(&wbar, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
    tc::prefetch_tmap(&xmap);
    if (a.c_split < a.cin) tc::prefetch_tmap(&xmap2);
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;
  if (threadIdx.x == 0 && a.wbytes) {  // the layer's weights, once (unless streamed)
    tc::mbar_arrive_expect_tx(&wbar, a.wbytes);
    tc::bulk_load(wsm, a.wpk, a.wbytes, &wbar);
  }
  // boxes are dealt out team by team; pipeline g takes tile r of each box of its team
  const int team = g / a.tpb, r = g - team * a.tpb;
  const int stride = gridDim.x * a.teams;
  const int first = blockIdx.x * a.teams + team;
  uint8_t* ring = boxes + (size_t)team * a.ring * a.box_stride;

  if (role == 0 && lane == 0 && r == 0) {
    // ---------------- TMA producer of the team
    int slot = 0;
    uint32_t ph = 0;
    for (int st = first; st < a.n_super && !abort_flag; st += stride) {
      const int n = halo_img(a, st);
      const int y0 = (int)fdiv31((uint32_t)((st - n * a.spi) * a.tpb * 128), a.f_p);  // first slot row
      for (int b = 0; b < a.cblocks; ++b) {
        if (!tc::mbar_wait(&empty[team][slot], ph ^ 1u)) { abort_flag = 1; break; }
        tc::mbar_arrive_expect_tx(&full[team][slot], a.box_bytes + a.wstage);
        // padded rows y0 .. y0 + bh - 1 = image rows y0 - 1 .. y0 + bh - 2, columns -1 .. w
        const int c0 = b * a.cw;
        const bool second = c0 >= a.c_split;
        uint8_t* stage = ring + (size_t)slot * a.box_stride;
        tc::tma_load_4d(stage, second ? &xmap2 : &xmap, second ? c0 - a.c_split : c0, -1, y0 - 1, n,
                        &full[team][slot]);
        if (a.wstage) {
          // the block's packed chunks of each tap: cw / 8 consecutive chunks per tap
          const int cpb = a.cw / 8;
          for (int tap = 0; tap < 9; ++tap)
            tc::bulk_load(stage + a.wofs + (size_t)tap * a.wtap,
                          a.wpk + (size_t)(tap * a.cpt + b * cpb) * a.cout * 8, a.wtap, &full[team][slot]);
        }
        if (++slot == a.ring) { slot = 0; ph ^= 1u; }
      }
    }
  } else if (role == 1 && lane == 0) {
    // ---------------- MMA issuer of pipeline g.  A descriptor is linear in its start
    // address (16-byte units in the low bits), so the taps' descriptors are a base plus
    // offsets computed once: one thread's dependent integer work per MMA is what limits
    // the issue rate, not the tensor core.
    if (a.wbytes && !tc::mbar_wait(&wbar, 0)) abort_flag = 1;
    tc::fence_after();
    const uint32_t wb = tc::saddr(wsm), rb = tc::saddr(ring);
    const uint32_t chunkb = (uint32_t)a.cout * 16u;  // one packed chunk: C_out rows x 8 K
    uint64_t a0[9], b0[9];
    if (a.cw == 8) {
      // one 8-channel block (C_in = 8): chunk c is tap c, so a K=16 MMA takes taps 2i
      // and 2i + 1 (the second 8 K-elements LBO bytes after the first); tap 9 is the zero
      // chunk of the pack, read against tap 8's rows
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const int t0 = 2 * i, t1 = t0 + 1 < 9 ? t0 + 1 : t0;
        const int r0 = (t0 / 3) * a.p + (t0 % 3), r1 = (t1 / 3) * a.p + (t1 % 3);
        a0[i] = tc::sdesc(rb + (uint32_t)r0 * 16u, (uint32_t)(r1 - r0) * 16u, 128);
        b0[i] = tc::sdesc(wb + (uint32_t)t0 * chunkb, chunkb, 128);
      }
    } else {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        a0[tap] = tc::sdesc_sw(rb + (uint32_t)((tap / 3) * a.p + (tap % 3)) * a.rowb, 8u * a.rowb, a.swz);
        // resident: tap's chunks in the layer pack; streamed: in stage 0 (slot added below)
        b0[tap] = a.wstage ? tc::sdesc(rb + a.wofs + (uint32_t)tap * a.wtap, chunkb, 128)
                           : tc::sdesc(wb + (uint32_t)(tap * a.cpt) * chunkb, chunkb, 128);
      }
    }
    const uint32_t bstep = (2u * chunkb) >> 4;                        // next 16 K in B
    const uint32_t bblk = ((uint32_t)(a.cw / 8) * chunkb) >> 4;       // next channel block
    const uint32_t slot_u = a.box_stride >> 4;
    int slot = 0, ai = 0;
    uint32_t ph = 0;
    for (int st = first; st < a.n_super && !abort_flag; st += stride) {
      const int n = halo_img(a, st);
      const int sbox = (st - n * a.spi) * a.tpb * 128;  // first slot of the box's tiles
      const int s0 = sbox + r * 128;
      if (s0 >= a.slots_img) {
        // a tile past the image (the last box of an image): release its boxes unread
        for (int b = 0; b < a.cblocks; ++b) {
          if (!tc::mbar_wait(&full[team][slot], ph)) { abort_flag = 1; break; }
          tc::mbar_arrive(&empty[team][slot]);
          if (++slot == a.ring) { slot = 0; ph ^= 1u; }
        }
        continue;
      }
      const int o = s0 - (int)fdiv31((uint32_t)sbox, a.f_p) * a.p;  // first slot from the box's first row
      const uint32_t ao = ((uint32_t)o * (a.cw == 8 ? 16u : a.rowb)) >> 4;
      const int acc = ai & 1;
      const uint32_t aph = (uint32_t)(ai >> 1) & 1u;
      ++ai;
      if (!tc::mbar_wait(&tempty[g][acc], aph ^ 1u)) { abort_flag = 1; break; }
      tc::fence_after();
      const uint32_t d = taddr + (uint32_t)(g * 2 + acc) * a.acc_cols;
      uint32_t accf = 0u;
      for (int b = 0; b < a.cblocks; ++b) {
        if (!tc::mbar_wait(&full[team][slot], ph)) { abort_flag = 1; break; }
        tc::fence_after();
        const uint32_t sa = (uint32_t)slot * slot_u + ao;
        const uint32_t sb = a.wstage ? (uint32_t)slot * slot_u : (uint32_t)b * bblk;
        if (a.cw == 8) {
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            tc::mma_bf16(d, a0[i] + sa, b0[i], a.idesc, accf);
            accf = 1u;
          }
        } else if (a.cw == 32) {
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            tc::mma_bf16(d, a0[tap] + sa, b0[tap] + sb, a.idesc, accf);
            tc::mma_bf16(d, a0[tap] + sa + 2u, b0[tap] + sb + bstep, a.idesc, 1u);
            accf = 1u;
          }
        } else {
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            for (int j = 0; j < a.cw / 16; ++j) {
              tc::mma_bf16(d, a0[tap] + sa + 2u * j, b0[tap] + sb + bstep * j, a.idesc, accf);
              accf = 1u;
            }
          }
        }
        tc::mma_commit(&empty[team][slot]);
        if (++slot == a.ring) { slot = 0; ph ^= 1u; }
      }
      tc::mma_commit(&tfull[g][acc]);
    }
  } else if (role >= 2) {
    // ---------------- epilogue of pipeline g: slot 32q + lane of the tile per thread
    const int q = warp & 3;
    const int m = q * 32 + lane;
    int ai = 0;
    for (int st = first; st < a.n_super && !abort_flag; st += stride) {
      const int n = halo_img(a, st);
      const int s0 = ((st - n * a.spi) * a.tpb + r) * 128;
      if (s0 >= a.slots_img) continue;  // a tile past the image: no accumulator
      const int acc = ai & 1;
      const uint32_t aph = (uint32_t)(ai >> 1) & 1u;
      ++ai;
      if (!tc::mbar_wait(&tfull[g][acc], aph)) { abort_flag = 1; break; }
      tc::fence_after();
      const int s = s0 + m;
      const int yy = (int)fdiv31((uint32_t)s, a.f_p), xx = s - yy * a.p;
      const bool real = xx < a.w && yy < a.h;  // slots w, w + 1 of a row and rows >= h: junk
      const size_t pix = ((size_t)n * a.h + (real ? yy : 0)) * a.w + (real ? xx : 0);
      const uint16_t* mp = a.mask ? a.mask + pix * a.cout : nullptr;
      float hacc[8];
      if (a.head) {
#pragma unroll
        for (int o = 0; o < 8; ++o) hacc[o] = o < a.head_out ? s_head[a.head_out * a.cout + o] : 0.f;
      }
      for (int c32 = 0; c32 < a.cout; c32 += 32) {
        // 32 accumulator columns with one wait (columns past cout are inside acc_cols)
        float v32[32];
        tc::tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 2 + acc) * a.acc_cols + (uint32_t)c32,
                      v32);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int c0 = c32 + hh * 16;
          if (c0 >= a.cout || !real) continue;
          float v[16];
          if (a.bias) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = v32[hh * 16 + i] + s_bias[c0 + i];
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = v32[hh * 16 + i];
          }
          const int gi = a.ygroup == a.cout ? 0 : c0 / a.ygroup;
          uint16_t* yp = a.y ? a.y + ((int64_t)gi * a.ygstride + (int64_t)pix * a.ygroup + (c0 - gi * a.ygroup))
                             : nullptr;
          if (kUp2) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
            uint4 o0, o1;
            round_bf16_16(v, o0, o1);
            const size_t up = (((size_t)n * 2 * a.h + 2 * yy) * (2 * a.w) + 2 * xx) * a.cout + c0;
            const size_t row = (size_t)2 * a.w * a.cout;
            store32(a.y + up, o0, o1, a.wide != 0);
            store32(a.y + up + a.cout, o0, o1, a.wide != 0);
            store32(a.y + up + row, o0, o1, a.wide != 0);
            store32(a.y + up + row + a.cout, o0, o1, a.wide != 0);
          } else if (!a.head) {
            epilogue16(v, nullptr, a.relu, mp ? mp + c0 : nullptr, yp, a.wide != 0);
          } else {
            // ReLU, then the head over the values the BF16 output holds, channel by
            // channel in order (the arithmetic of the separate 1x1 head)
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
            uint4 o0, o1;
            round_bf16_16(v, o0, o1);
            if (a.store_y) store32(yp, o0, o1, a.wide != 0);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
              if (o >= a.head_out) break;
              const float* hw = s_head + o * a.cout + c0;
#pragma unroll
              for (int i = 0; i < 16; ++i) hacc[o] = fmaf(v[i], hw[i], hacc[o]);
            }
          }
        }
      }
      if (a.head && real) {
        float* hy = a.head_y + pix * a.head_out;
#pragma unroll
        for (int o = 0; o < 8; ++o)
          if (o < a.head_out) hy[o] = hacc[o];
      }
      tc::fence_before();
      tc::mbar_arrive(&tempty[g][acc]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, a.tmem_cols);
  }
}


// elements of one tap) is a block of C_out rows x 16 bytes, 8-row groups of 128 bytes.
__device__ __forceinline__ uint16_t pack_elem(const float* __restrict__ w, int cin, int cout, int tflip, int64_t e) {
  const int cpt = cin / 8;
  const int c = (int)(e / (cout * 8));
  const int r = (int)(e - (int64_t)c * cout * 8);
  const int o = (r >> 6) * 8 + ((r & 63) >> 3);
  const int ee = r & 7;
  float v = 0.f;
  if (c < 9 * cpt) {
    const int tap = c / cpt, ci = (c - tap * cpt) * 8 + ee;
    const int ky = tap / 3, kx = tap - ky * 3;
    if (!tflip) {
      v = w[(((int64_t)o * 3 + ky) * 3 + kx) * cin + ci];
    } else {
      // input-gradient conv: W'[o][ky][kx][ci] = W[ci][2-ky][2-kx][o], W is [cin][3][3][cout]
      v = w[(((int64_t)ci * 3 + (2 - ky)) * 3 + (2 - kx)) * cout + o];
    }
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&h);
}

__global__ void k_pack_weights(const float* __restrict__ w, int cin, int cout, int tflip, int kc,
                               uint16_t* __restrict__ out) {
  const int64_t total = (int64_t)kc * cout * 8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = pack_elem(w, cin, cout, tflip, e);
}

// Several packs in one launch (a model's layers, each step of a training): job j covers
// elements [begin[j], begin[j + 1]) of the concatenated outputs
struct PackBatch {
  PackJob job[kMaxPackJobs];
  int64_t begin[kMaxPackJobs + 1];
  int32_t n;
};
__global__ void k_pack_batch(const __grid_constant__ PackBatch b) {
  const int64_t total = b.begin[b.n];
  int j = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    while (e >= b.begin[j + 1]) ++j;  // e only grows in a thread's loop
    const PackJob& J = b.job[j];
    const int64_t le = e - b.begin[j];
    J.out[le] = pack_elem(J.w, J.cin, J.cout, J.tflip, le);
  }
}

int chunk_count(int cin) {
  const int kc = 9 * (cin / 8);
  return kc + (kc & 1);
}

// All packs of `jobs` with as few launches as the job table allows (kMaxPackJobs each)
ls_status conv3x3_pack_batch(const PackJob* jobs, int n, cudaStream_t stream) {
  for (int j0 = 0; j0 < n; j0 += kMaxPackJobs) {
    PackBatch b = {};
    b.n = std::min(kMaxPackJobs, n - j0);
    b.begin[0] = 0;
    for (int j = 0; j < b.n; ++j) {
      const PackJob& J = jobs[j0 + j];
      if (!J.w || !J.out || J.cin < 8 || J.cin % 8 || J.cout < 16 || J.cout % 16) return LS_ERR_INVALID_ARG;
      b.job[j] = J;
      b.begin[j + 1] = b.begin[j] + (int64_t)chunk_count(J.cin) * J.cout * 8;
    }
    k_pack_batch<<<grid_cap((b.begin[b.n] + 255) / 256, kSmCount * 8), 256, 0, stream>>>(b);
    LS_CUDA_TRY(cudaGetLastError());
  }
  return LS_OK;
}

}  // namespace

// The tensor maps of the input: channels [0, cs) of x (cs channels per pixel) and, when
// x2 is given, channels [cs, cin) from x2 (cin - cs per pixel); without x2 the second
// map repeats the first.  Boxes of cw channels x bx x by x 1.
bool encode_input_maps(CUtensorMap* m1, CUtensorMap* m2, const uint16_t* x, const uint16_t* x2, int cs, int cin,
                       int n, int h, int w, int cw, uint32_t bx, uint32_t by, uint32_t bn) {
  const uint32_t box[4] = {(uint32_t)cw, bx, by, bn};
  const int sw = cw == 8 ? 0 : cw * 2;
  const int c1 = x2 ? cs : cin;
  const uint64_t d1[4] = {(uint64_t)c1, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t s1[3] = {(uint64_t)c1 * 2, (uint64_t)w * c1 * 2, (uint64_t)h * w * c1 * 2};
  if (!encode_tmap_bf16_4d(m1, x, d1, s1, box, sw)) return false;
  if (!x2) {
    *m2 = *m1;
    return true;
  }
  const int c2 = cin - cs;
  const uint64_t d2[4] = {(uint64_t)c2, (uint64_t)w, (uint64_t)h, (uint64_t)n};
  const uint64_t s2[3] = {(uint64_t)c2 * 2, (uint64_t)w * c2 * 2, (uint64_t)h * w * c2 * 2};
  return encode_tmap_bf16_4d(m2, x2, d2, s2, box, sw);
}

// The halo form (k_conv3x3_halo) when the shape allows it: W = 32, 64 or 128 (narrower
// rows would waste too many junk slots), 8-channel inputs only as a single block, and
// the layer's packed weights plus two pipelines' box rings within the shared memory.
// LS_ERR_UNSUPPORTED: use the per-tap form.
ls_status conv3x3_halo_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, const uint16_t* mask,
                              int relu, int n, int h, int w, int cin, int cout, uint16_t* y, int ygroup,
                              int64_t ygstride, cudaStream_t stream, const float* head = nullptr,
                              float* head_y = nullptr, int head_out = 0, int store_y = 1,
                              const uint16_t* x2 = nullptr, int c_split = 0, int up2 = 0) {
  if (!(w == 32 || w == 64 || w == 128)) return LS_ERR_UNSUPPORTED;
  HaloArgs a = {};
  a.up2 = up2;
  a.c_split = x2 ? c_split : cin;
  a.head = head; a.head_y = head_y; a.head_out = head_out; a.store_y = head ? store_y : 1;
  a.cin = cin; a.cout = cout; a.cpt = cin / 8;
  a.relu = relu; a.ygroup = ygroup; a.ygstride = ygstride;
  a.wpk = wpk; a.bias = bias; a.mask = mask; a.y = y;
  a.wide = (uintptr_t)y % 32 == 0 && (ygroup == cout || (ygstride * 2) % 32 == 0);
  a.w = w; a.h = h; a.p = w + 2;
  a.slots_img = h * a.p;
  a.wbytes = (uint32_t)chunk_count(cin) * (uint32_t)cout * 16u;
  const size_t wsz = ((size_t)a.wbytes + 1023) & ~(size_t)1023;
  a.acc_cols = 32;
  while ((int)a.acc_cols < cout) a.acc_cols <<= 1;
  // pipelines: as many as the TMEM holds (two accumulators each), up to four (more
  // issuers gain nothing: at C_out <= 64 four already saturate the shared-memory operand
  // reads of the MMAs); boxes of 32 channels (64-byte rows) where C_in allows, 16 or 8
  // otherwise (measured: 64-channel boxes and narrower ones were both slower); a ring
  // of up to four boxes per team (deeper measured no faster)
  int np = kHaloMaxPipes;
  while (np > 1 && (uint32_t)np * 2u * a.acc_cols > 512u) np >>= 1;
  const int cw = (cin % 32 == 0 && a.c_split % 32 == 0) ? 32 : (cin % 16 == 0 && a.c_split % 16 == 0) ? 16 : 8;
  if (cw == 8 && (cin != 8 || x2)) return LS_ERR_UNSUPPORTED;
  // tiles per box T: a box holds the padded rows around T consecutive tiles (the first
  // starts at most p - 1 slots into the box's first row and the last needs 128 + 2p + 2
  // slots from its start), shared by a team of T pipelines
  auto bh_of = [&](int T) { return ((a.p - 1) + 128 * T + 1 + 2 * a.p) / a.p + 1; };
  auto stride_of = [&](int T) {
    return ((uint32_t)bh_of(T) * (uint32_t)a.p * (uint32_t)(2 * cw) + 1023u) & ~1023u;
  };
  auto ring_of = [&](int T) {
    const size_t per = (size_t)(np / T) * stride_of(T);
    return wsz >= kHaloSmemBudget ? 0 : (int)std::min<size_t>(kHaloRingUse, (kHaloSmemBudget - wsz) / per);
  };
  int tpb = 0;
  // resident weights: one tile per box (measured: sharing boxes between pipelines
  // saved L2 traffic but no time when the weights are resident)
  if (ring_of(1) >= 2) tpb = 1;
  int ring = tpb ? ring_of(tpb) : 0;
  uint32_t stride = tpb ? stride_of(tpb) : 0;
  // two pipelines where C_out is 65-128 (measured: d1a's input gradient, 32 -> 96
  // channels, 174 -> 143 us at 512 tiles against the per-tap form); one pipeline (C_out >
  // 128) is left to the per-tap form, which runs several CTAs per SM
  if (np < 2) return LS_ERR_UNSUPPORTED;
  if (!tpb && cw == 32) {
    // weights too large to stay resident: each stage carries its channel block's nine
    // tap slices beside the box, shared by the T pipelines of a team.  Candidates (pipes,
    // tiles per box) by the fewest stage bytes per image among those with two stages;
    // three pipelines of three tiles cover a 32 x 32 image's 1,088 slots exactly
    a.wtap = (uint32_t)(cw / 8) * (uint32_t)cout * 16u;
    a.wstage = 9u * a.wtap;
    const int cand[4][2] = {{4, 4}, {3, 3}, {4, 2}, {2, 2}};
    int64_t best = 0;
    for (const auto& c : cand) {
      const int P = c[0], T = c[1];
      if ((uint32_t)P * 2u * a.acc_cols > 512u) continue;
      const uint32_t wofs = ((uint32_t)bh_of(T) * (uint32_t)a.p * (uint32_t)(2 * cw) + 1023u) & ~1023u;
      const uint32_t st = (wofs + a.wstage + 1023u) & ~1023u;
      const int rg = (int)std::min<size_t>(kHaloRingUse, kHaloSmemBudget / ((size_t)(P / T) * st));
      if (rg < 2) continue;
      const int64_t bytes = (int64_t)((a.slots_img + 128 * T - 1) / (128 * T)) * st;
      if (!best || bytes < best) {
        best = bytes; np = P; tpb = T; ring = rg; stride = st; a.wofs = wofs;
      }
    }
    if (!tpb) return LS_ERR_UNSUPPORTED;
    a.wbytes = 0;
  }
  if (!tpb) return LS_ERR_UNSUPPORTED;
  a.tpb = tpb;
  a.teams = np / tpb;
  a.spi = (a.slots_img + 128 * tpb - 1) / (128 * tpb);
  a.f_p = make_fastdiv31((uint32_t)a.p);
  if (a.spi > 1) a.f_spi = make_fastdiv31((uint32_t)a.spi);
  const int64_t ns = (int64_t)n * a.spi;
  if (ns > INT32_MAX) return LS_ERR_UNSUPPORTED;
  a.n_super = (int32_t)ns;
  a.bh = bh_of(tpb);
  a.cw = cw;
  a.cblocks = cin / cw;
  a.npipes = np;
  a.ring = ring;
  a.rowb = (uint32_t)(2 * cw);
  a.swz = cw == 64 ? 2u : cw == 32 ? 4u : cw == 16 ? 6u : 0u;
  a.box_bytes = (uint32_t)a.bh * (uint32_t)a.p * a.rowb;
  a.box_stride = stride;
  a.tmem_cols = 32;  // an allocation is a power of two (three pipelines: 384 -> 512)
  while (a.tmem_cols < (uint32_t)np * 2u * a.acc_cols) a.tmem_cols <<= 1;
  a.idesc = tc::idesc_bf16(128, cout);
  const size_t smem = (a.wbytes ? wsz : 0) + (size_t)a.teams * a.ring * a.box_stride;
  CUtensorMap map, map2;
  if (!encode_input_maps(&map, &map2, x, x2, a.c_split, cin, n, h, w, a.cw, (uint32_t)a.p, (uint32_t)a.bh, 1))
    return LS_ERR_CUDA;
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_once(once, dev, [] {
        return cudaFuncSetAttribute(k_conv3x3_halo<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kHaloSmemBudget) == cudaSuccess &&
               cudaFuncSetAttribute(k_conv3x3_halo<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kHaloSmemBudget) == cudaSuccess;
      }))
    return LS_ERR_CUDA;
  const int grid = grid_cap(((int64_t)a.n_super + a.teams - 1) / a.teams, kSmCount);
  if (a.up2)
    k_conv3x3_halo<true><<<grid, np * kHaloThreadsPerPipe, smem, stream>>>(map, map2, a);
  else
    k_conv3x3_halo<false><<<grid, np * kHaloThreadsPerPipe, smem, stream>>>(map, map2, a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// Convolution + bias + ReLU with a 1x1 head (head_out <= 8 outputs, FP32) fused into
// its epilogue, computed over the BF16-rounded outputs in channel order (the same
// arithmetic as a separate head over the stored output); the BF16 output is stored
// only when store_y.  LS_ERR_UNSUPPORTED when the shape has no halo form: the caller
// runs the convolution and the head separately.
ls_status conv3x3_head_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, int n, int h, int w, int cin,
                              int cout, uint16_t* y, const float* head, float* head_y, int head_out, int store_y,
                              cudaStream_t stream) {
  if (!x || !wpk || !head || !head_y || (store_y && !y) || n <= 0 || h <= 0 || w <= 0) return LS_ERR_INVALID_ARG;
  if (head_out < 1 || head_out > 8) return LS_ERR_UNSUPPORTED;
  if (cin < 8 || cin % 8 || cin > 256 || cout < 16 || cout > 256 || cout % 16) return LS_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)wpk | (uintptr_t)y) % 16) return LS_ERR_INVALID_ARG;
  return conv3x3_halo_launch(x, wpk, bias, nullptr, 1, n, h, w, cin, cout, store_y ? y : nullptr, cout, 0, stream,
                             head, head_y, head_out, store_y);
}

// Shared with the model code: validated launch of one convolution whose output
// channels go to cout / ygroup tensors of ygroup channels each, ygstride elements apart
// (ygroup = cout: one NHWC tensor).  Without a mask only (a mask is one NHWC tensor).
// x2 (optional): input channels [c_split, cin) come from x2 (cin - c_split per pixel)
// and [0, c_split) from x (c_split per pixel), as if the two were concatenated.
ls_status conv3x3_launch_groups(const uint16_t* x, const uint16_t* wpk, const float* bias, const uint16_t* mask,
                                int relu, int n, int h, int w, int cin, int cout, uint16_t* y, int ygroup,
                                int64_t ygstride, cudaStream_t stream, const uint16_t* x2 = nullptr,
                                int c_split = 0, int up2 = 0) {
  if (!x || !wpk || !y || n <= 0 || h <= 0 || w <= 0) return LS_ERR_INVALID_ARG;
  if (x2 && (c_split <= 0 || c_split >= cin || c_split % 8 || (uintptr_t)x2 % 16)) return LS_ERR_INVALID_ARG;
  if (cin < 8 || cin % 8 || cin > 256 || cout < 16 || cout > 256 || cout % 16) return LS_ERR_UNSUPPORTED;
  if (ygroup < 16 || ygroup % 16 || cout % ygroup ||
      (ygroup != cout && (mask || ygstride % 8 || ygstride < (int64_t)n * h * w * ygroup)))
    return LS_ERR_INVALID_ARG;
  if (w > 128 || 128 % w) return LS_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)wpk | (uintptr_t)y | (uintptr_t)mask) % 16) return LS_ERR_INVALID_ARG;
  {
    const ls_status hs = conv3x3_halo_launch(x, wpk, bias, mask, relu, n, h, w, cin, cout, y, ygroup,
                                             ygroup == cout ? 0 : ygstride, stream, nullptr, nullptr, 0, 1, x2,
                                             c_split, up2);
    if (hs != LS_ERR_UNSUPPORTED) return hs;  // else the shape is not one for the halo form
  }
  ConvArgs a = {};
  a.c_split = x2 ? c_split : cin;
  uint32_t box[4] = {8, (uint32_t)w, 1, 1};
  if (w * h >= 128) {
    const int rpt = 128 / w;
    if (h % rpt) return LS_ERR_UNSUPPORTED;
    a.rows_per_tile = rpt;
    a.tiles_per_img = h / rpt;
    a.imgs_per_tile = 1;
    box[2] = (uint32_t)rpt;
  } else {
    if (128 % (w * h)) return LS_ERR_UNSUPPORTED;
    const int ipt = 128 / (w * h);
    if (n % ipt) return LS_ERR_UNSUPPORTED;
    a.rows_per_tile = h;
    a.tiles_per_img = 1;
    a.imgs_per_tile = ipt;
    box[2] = (uint32_t)h;
    box[3] = (uint32_t)ipt;
  }
  const int64_t P = (int64_t)n * h * w;
  if (P % 128 || P / 128 > (int64_t)INT32_MAX) return LS_ERR_UNSUPPORTED;
  a.n_mtiles = (int32_t)(P / 128);
  a.wpk = wpk; a.bias = bias; a.mask = mask; a.y = y; a.relu = relu;
  a.up2 = up2; a.img_h = h; a.img_w = w;
  a.wide = (uintptr_t)y % 32 == 0 && (ygroup == cout || (ygstride * 2) % 32 == 0);
  a.ygroup = ygroup; a.ygstride = ygroup == cout ? 0 : ygstride;
  a.cin = cin; a.cout = cout; a.cpt = cin / 8;
  a.kc_real = 9 * a.cpt;
  a.kc = chunk_count(cin);
  a.n_stages = (a.kc + kChunksPerStage - 1) / kChunksPerStage;
  // widest channel block per TMA load: fewer, longer rows for the TMA unit
  // (a channel block never straddles the two inputs)
  a.cw = 64;
  while (a.cw > 8 && (cin % a.cw || a.c_split % a.cw)) a.cw >>= 1;
  a.cblocks = cin / a.cw;
  a.blocks_per_stage = 64 / a.cw;
  a.n_blocks = 9 * a.cblocks;
  a.blk_bytes = (uint32_t)(128 * a.cw * 2);
  a.sbo_a = (uint32_t)(8 * a.cw * 2);  // 8 rows of one swizzle atom
  a.swz = a.cw == 64 ? 2u : a.cw == 32 ? 4u : a.cw == 16 ? 6u : 0u;  // 128B, 64B, 32B swizzle
  box[0] = (uint32_t)a.cw;
  a.acc_cols = 32;
  while ((int)a.acc_cols < cout) a.acc_cols <<= 1;
  a.tmem_cols = 2 * a.acc_cols;
  a.stage_bytes = (uint32_t)(kAStageBytes + cout * 8 * 16);
  a.idesc = tc::idesc_bf16(128, cout);
  CUtensorMap map, map2;
  if (!encode_input_maps(&map, &map2, x, x2, a.c_split, cin, n, h, w, a.cw, box[1], box[2], box[3]))
    return LS_ERR_CUDA;
  // two CTAs per SM where their accumulators fit the TMEM together (tmem_cols <= 256):
  // each gets half the shared-memory budget
  const size_t budget = a.tmem_cols <= 128 ? kConvSmemBudget3 : a.tmem_cols <= 256 ? kConvSmemBudget2 : kConvSmemBudget;
  a.ring = (int32_t)std::min<size_t>(kConvStages, budget / a.stage_bytes);
  if (a.ring < 2) return LS_ERR_UNSUPPORTED;
  const size_t smem = (size_t)a.ring * a.stage_bytes;
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (!device_once(once, dev, [] {
        return cudaFuncSetAttribute(k_conv3x3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kConvSmemBudget) == cudaSuccess &&
               cudaFuncSetAttribute(k_conv3x3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kConvSmemBudget) == cudaSuccess;
      }))
    return LS_ERR_CUDA;
  const int per_sm = a.tmem_cols <= 128 ? 3 : a.tmem_cols <= 256 ? 2 : 1;
  if (a.up2)
    k_conv3x3<true><<<grid_cap(a.n_mtiles, (int64_t)kSmCount * per_sm), kConvThreads, smem, stream>>>(map, map2, a);
  else
    k_conv3x3<false><<<grid_cap(a.n_mtiles, (int64_t)kSmCount * per_sm), kConvThreads, smem, stream>>>(map, map2, a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// Convolution + bias + ReLU whose output is stored only as its 2x nearest-neighbour
// upsampling y_up ([n][2h][2w][cout]), for a convolution whose output feeds the next
// decoder level's upsampling alone.  LS_ERR_UNSUPPORTED when the shape has neither form
// (the caller stores the output and upsamples it).
ls_status conv3x3_up2_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, int n, int h, int w, int cin,
                             int cout, uint16_t* y_up, cudaStream_t stream) {
  if (!x || !wpk || !y_up || n <= 0 || h <= 0 || w <= 0) return LS_ERR_INVALID_ARG;
  if (cin < 8 || cin % 8 || cin > 256 || cout < 16 || cout > 256 || cout % 16) return LS_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)wpk | (uintptr_t)y_up) % 16) return LS_ERR_INVALID_ARG;
  return conv3x3_launch_groups(x, wpk, bias, nullptr, 1, n, h, w, cin, cout, y_up, cout, 0, stream, nullptr, 0, 1);
}

ls_status conv3x3_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, const uint16_t* mask, int relu,
                         int n, int h, int w, int cin, int cout, uint16_t* y, cudaStream_t stream) {
  return conv3x3_launch_groups(x, wpk, bias, mask, relu, n, h, w, cin, cout, y, cout, 0, stream);
}

}  // namespace ls

extern "C" int64_t ls_conv3x3_packed_elems(int32_t cin, int32_t cout) {
  if (cin < 8 || cin % 8 || cout < 16 || cout % 16) return -1;
  return (int64_t)ls::chunk_count(cin) * cout * 8;
}

extern "C" ls_status ls_conv3x3_pack(const float* w, int32_t cin, int32_t cout, int32_t transpose_flip,
                                     uint16_t* packed, ls_stream_t stream) {
  if (!w || !packed || cin < 8 || cin % 8 || cout < 16 || cout % 16) return LS_ERR_INVALID_ARG;
  const int kc = ls::chunk_count(cin);
  const int64_t total = (int64_t)kc * cout * 8;
  ls::k_pack_weights<<<ls::grid_cap((total + 255) / 256, ls::kSmCount * 8), 256, 0,
                       reinterpret_cast<cudaStream_t>(stream)>>>(w, cin, cout, transpose_flip, kc, packed);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_conv3x3_forward(const uint16_t* x, const uint16_t* packed, const float* bias,
                                        const uint16_t* mask, int32_t relu, const ls_conv_shape* shape, uint16_t* y,
                                        ls_stream_t stream) {
  if (!shape) return LS_ERR_INVALID_ARG;
  return ls::conv3x3_launch(x, packed, bias, mask, relu, shape->n, shape->h, shape->w, shape->cin, shape->cout, y,
                            reinterpret_cast<cudaStream_t>(stream));
}
