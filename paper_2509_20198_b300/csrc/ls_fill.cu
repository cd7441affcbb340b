// Chunk-point extraction, Gaussian-weighted sparse fill and full-resolution tile
// update.
//
//  * Extraction (Sec. 3.1, 3.2): the first point of every 50,000-point LAZ chunk is
//    stored uncompressed; sample k of tile t is point tile_offsets[t] + chunk * k.
//  * Gaussian fill (the High-Quality Splatting baseline of Sec. 4.2): each sample is
//    a fixed-radius splat, heights and colours are blended with a Gaussian weight;
//    a texel reached by no splat copies its nearest sample.
//  * Tile update (abstract, Sec. 3.5): texels with full-resolution points take their
//    mean height and colour.
//
// Fill design (B300): one CTA per output tile.  The samples of the 3x3 tile
// neighbourhood (three contiguous CSR ranges) are packed 32-byte records that one
// thread stages into shared memory with three cp.async.bulk copies completing on an
// mbarrier.  Each warp owns 8x4-texel blocks: lanes test 32 staged samples at a time
// against the block's box grown by R, a ballot lists the hits, and every lane
// weighs each hit for its own texel with an exact 64-bit squared distance and
// __expf.  Results are staged in shared memory and written with 16-byte stores.
#include <climits>
#include <cmath>

#include "ls_internal.cuh"

namespace ls {
namespace {

// Packed sample record (32 bytes): coordinates relative to the region origin.
struct __align__(16) Rec {
  int32_t lx, ly, z, idx;
  uint32_t rg;  // R | G << 16
  uint32_t b;
  uint32_t pad0, pad1;
};
static_assert(sizeof(Rec) == 32, "record size");

constexpr int kFillThreads = 256;
constexpr int kStageCap = 2048;  // most staged samples per tile (64 KB)
constexpr int kOutStageRes = 64; // texel maps up to 64x64 are staged in shared memory
constexpr int kCandCap = 256;    // candidate list of a block row (indices into the stage)
constexpr int kFillMaxCtasPerSm = 4;

// ---------------------------------------------------------------------------------
// extraction
// ---------------------------------------------------------------------------------
__global__ void k_sample_offsets(const int64_t* __restrict__ toff, int64_t n_tiles, int64_t chunk,
                                 int64_t* __restrict__ soff) {
  // single CTA exclusive scan of per-tile chunk counts
  __shared__ int64_t carry;
  __shared__ int64_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    int64_t v = 0;
    if (t < n_tiles) {
      const int64_t np = toff[t + 1] - toff[t];
      v = np > 0 ? (np + chunk - 1) / chunk : 0;
    }
    // inclusive warp scan
    int64_t s = v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
      int64_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      wsum[lane] = w;  // inclusive prefix of warp sums
    }
    __syncthreads();
    const int64_t excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + s - v;
    if (t < n_tiles) soff[t] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) soff[n_tiles] = carry;
}

__global__ void k_extract(ls_points p, int64_t n_tiles, int64_t chunk, const int64_t* __restrict__ soff,
                          ls_sample_buffers out, int64_t capacity) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < n_tiles; t += warps) {
    const int64_t p0 = p.tile_offsets[t], p1 = p.tile_offsets[t + 1];
    const int64_t s0 = soff[t];
    for (int64_t k = lane; p0 + k * chunk < p1; k += 32) {
      const int64_t src = p0 + k * chunk, dst = s0 + k;
      if (dst >= capacity) {
        set_status(LS_ERR_OUT_OF_RANGE);
        break;
      }
      out.x[dst] = p.x[src]; out.y[dst] = p.y[src]; out.z[dst] = p.z[src];
      out.r[dst] = p.r[src]; out.g[dst] = p.g[src]; out.b[dst] = p.b[src];
    }
  }
}

// ---------------------------------------------------------------------------------
// fill
// ---------------------------------------------------------------------------------
struct FillArgs {
  const int64_t* __restrict__ toff;  // sample CSR by tile [T+1]
  const Rec* __restrict__ recs;      // packed samples
  const int32_t* __restrict__ tile_ids;
  int64_t n_out;
  int64_t n_samples;  // records in recs
  int32_t tiles_x, tiles_y, tile_cm, res, cell_cm;
  uint32_t R2u;  // R^2 (R < 65536)
  int32_t R;
  float k2;     // log2(e) / (2 sigma^2): w = 2^(-d^2 k2)
  float zs_f;   // z_scale in FP32
  int32_t stage_cap;  // records the dynamic shared stage holds
  double z_scale, z_offset;
  float* height;
  uint8_t* rgb;
  float4* aux_hc;  // optional per texel: height (m), R, G, B (0..1, unrounded)
  float* aux_d;    // optional per texel: distance to the nearest sample (cm)
  int32_t split;   // CTAs per tile, each a band of res / split texel rows (few tiles: more CTAs)
};

__global__ void k_pack(ls_points s, int64_t n_tiles, int64_t x0, int64_t y0, int32_t tile_cm,
                       int32_t tiles_x, Rec* __restrict__ recs) {
  // samples outside [0, s.n) (an inconsistent CSR) are reported, never touched
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < n_tiles; t += warps) {
    const int64_t q0 = s.tile_offsets[t], q1 = s.tile_offsets[t + 1];
    const int64_t tx = t % tiles_x, ty = t / tiles_x;
    if (q0 < 0 || q1 < q0 || q1 > s.n) {
      if (lane == 0) set_status(LS_ERR_INVALID_ARG);
      continue;
    }
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const int64_t lx = (int64_t)s.x[q] - x0, ly = (int64_t)s.y[q] - y0;
      if (lx < tx * tile_cm || lx >= (tx + 1) * tile_cm || ly < ty * tile_cm || ly >= (ty + 1) * tile_cm)
        set_status(LS_ERR_INVALID_ARG);
      Rec rc;
      rc.lx = (int32_t)lx; rc.ly = (int32_t)ly; rc.z = s.z[q]; rc.idx = (int32_t)q;
      rc.rg = (uint32_t)s.r[q] | ((uint32_t)s.g[q] << 16);
      rc.b = s.b[q];
      rc.pad0 = rc.pad1 = 0u;
      recs[q] = rc;
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

struct LaneAcc {
  float sw, swz, swr, swg, swb;
  long long bd2;  // nearest squared distance (LLONG_MAX: none yet)
  int bidx;       // its sample index (records are indexed by sample)
};

// One sample for this lane's texel: the nearest by exact squared distance (ties: lower
// sample index), and, within R, the Gaussian weight on height (relative to the tile's
// reference zref) and colour.  R^2 <= tile_cm^2 < 2^32, so an in-radius d2 converts
// to float from 32 bits.
__device__ __forceinline__ void weigh(const Rec& q, int cx, int cy, int zref, uint32_t R2, float k2, LaneAcc& a) {
  const int dx = q.lx - cx, dy = q.ly - cy;
  const long long d2 = (long long)dx * dx + (long long)dy * dy;
  if (d2 < a.bd2 || (d2 == a.bd2 && q.idx < a.bidx)) {
    a.bd2 = d2;
    a.bidx = q.idx;
  }
  if (d2 <= (long long)R2) {
    const float w = exp2f(-__uint2float_rn((uint32_t)d2) * k2);
    a.sw += w;
    a.swz = fmaf(w, (float)(q.z - zref), a.swz);
    a.swr = fmaf(w, (float)(q.rg & 0xffffu), a.swr);
    a.swg = fmaf(w, (float)(q.rg >> 16), a.swg);
    a.swb = fmaf(w, (float)q.b, a.swb);
  }
}

// A staged record after the per-tile conversion: height relative to the tile's
// reference and colours as floats, so that a hit needs no integer conversions.
struct __align__(16) StRec {
  int32_t lx, ly;
  float fz;     // z - zref (cm)
  int32_t idx;  // sample index
  float fr, fg, fb;
  uint32_t pad;
};
static_assert(sizeof(StRec) == sizeof(Rec), "staged records are converted in place");

// Nearest of the staged samples as one 64-bit key: squared distance above the stage
// index (stage order is sample order, so the smaller key also breaks ties by the
// lower sample index).
constexpr int kKeyShift = 11;  // stage indices < kStageCap = 2^11
static_assert((1 << kKeyShift) >= kStageCap, "stage index field");

struct LaneAccS {
  float sw, swz, swr, swg, swb;
  unsigned long long key;  // ~0: none yet
};

// A lane owns two texels of one column, 4 rows apart (an 8 x 8 block per warp): one
// sample's x distance serves both.
constexpr int kTexPerLane = 2;

// One staged sample for this lane's texels (rows cy and cy + dyt).  kSmall: the
// squared distance of every sample in the block's box fits 32 bits (checked on the
// host).  Weights are branch-free: a sample beyond R gets weight 0 (the lanes of a warp
// disagree often).
template <bool kSmall>
__device__ __forceinline__ void weigh_st(const StRec& q, int si, int cx, int cy, int dyt, uint32_t R2, float k2,
                                         LaneAccS (&a)[kTexPerLane]) {
  const int dx = q.lx - cx;
#pragma unroll
  for (int t = 0; t < kTexPerLane; ++t) {
    const int dy = q.ly - cy - t * dyt;
    unsigned long long d2;
    if (kSmall) {
      d2 = (uint32_t)dx * (uint32_t)dx + (uint32_t)dy * (uint32_t)dy;
    } else {
      d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
    }
    const unsigned long long key = (d2 << kKeyShift) | (unsigned)si;
    a[t].key = key < a[t].key ? key : a[t].key;
    float w = exp2f(-__uint2float_rn((uint32_t)d2) * k2);
    w = d2 <= (unsigned long long)R2 ? w : 0.f;
    a[t].sw += w;
    a[t].swz = fmaf(w, q.fz, a[t].swz);
    a[t].swr = fmaf(w, q.fr, a[t].swr);
    a[t].swg = fmaf(w, q.fg, a[t].swg);
    a[t].swb = fmaf(w, q.fb, a[t].swb);
  }
}

// The staged samples of a candidate list (or of the whole stage, cand == nullptr) that
// fall in the warp's box, for this lane's texels.
template <bool kSmall>
__device__ __forceinline__ void splat_st(const StRec* stage, const uint16_t* cand, int n, int bx0, int bx1, int by0,
                                         int by1, int cx, int cy, int dyt, uint32_t R2, float k2,
                                         LaneAccS (&a)[kTexPerLane]) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    bool in = false;
    int k = base + lane;
    if (base + lane < n) {
      if (cand) k = cand[base + lane];
      const int2 xy = *reinterpret_cast<const int2*>(&stage[k]);
      in = xy.x >= bx0 && xy.x <= bx1 && xy.y >= by0 && xy.y <= by1;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int si = __shfl_sync(0xffffffffu, k, src);
      weigh_st<kSmall>(stage[si], si, cx, cy, dyt, R2, k2, a);
    }
  }
}

// Nearest staged sample for the lane's texels that need it (need bit t), within the
// warp's block box grown by the caller.
__device__ __forceinline__ void nearest_st(const StRec* stage, int n, unsigned need, int cx, int cy, int dyt,
                                           int bx0, int bx1, int by0, int by1, LaneAccS (&a)[kTexPerLane]) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    bool in = false;
    if (base + lane < n) {
      const int2 xy = *reinterpret_cast<const int2*>(&stage[base + lane]);
      in = xy.x >= bx0 && xy.x <= bx1 && xy.y >= by0 && xy.y <= by1;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int2 xy = *reinterpret_cast<const int2*>(&stage[base + src]);
#pragma unroll
      for (int t = 0; t < kTexPerLane; ++t) {
        if (need & (1u << t)) {
          const int dx = xy.x - cx, dy = xy.y - cy - t * dyt;
          const unsigned long long d2 = (unsigned long long)((long long)dx * dx + (long long)dy * dy);
          const unsigned long long key = (d2 << kKeyShift) | (unsigned)(base + src);
          a[t].key = key < a[t].key ? key : a[t].key;
        }
      }
    }
  }
}

// Weigh, for this lane's texel, the samples recs[0..n) that fall in the warp's box.
__device__ __forceinline__ void splat_range(const Rec* recs, int n, int bx0, int bx1, int by0, int by1, int cx,
                                            int cy, int zref, uint32_t R2, float k2, LaneAcc& a) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    bool in = false;
    if (base + lane < n) {
      const int2 xy = *reinterpret_cast<const int2*>(&recs[base + lane]);
      in = xy.x >= bx0 && xy.x <= bx1 && xy.y >= by0 && xy.y <= by1;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      weigh(recs[base + src], cx, cy, zref, R2, k2, a);
    }
  }
}

// Nearest sample among recs[0..n) for lanes that need it (no candidate within R),
// testing only samples inside the warp's block box grown by `grow` (every sample
// nearer than a lane's current best lies there when grow >= that best distance).
__device__ __forceinline__ void nearest_range(const Rec* recs, int n, bool need, int cx, int cy, int bx0, int bx1,
                                              int by0, int by1, LaneAcc& a) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    bool in = false;
    if (base + lane < n) {
      const int2 xy = *reinterpret_cast<const int2*>(&recs[base + lane]);
      in = xy.x >= bx0 && xy.x <= bx1 && xy.y >= by0 && xy.y <= by1;
    }
    unsigned mask = __ballot_sync(0xffffffffu, in);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const Rec q = recs[base + src];
      if (need) {
        const int dx = q.lx - cx, dy = q.ly - cy;
        const long long d2 = (long long)dx * dx + (long long)dy * dy;
        if (d2 < a.bd2 || (d2 == a.bd2 && q.idx < a.bidx)) {
          a.bd2 = d2;
          a.bidx = q.idx;
        }
      }
    }
  }
}

// Rings of tiles at Chebyshev distance >= 2 (rare: only when the 3x3 block holds no
// sample within one tile size of the texel).
__device__ void nearest_far(const FillArgs& f, int tx, int ty, int cx, int cy, LaneAcc& a) {
  const int mmax = f.tiles_x > f.tiles_y ? f.tiles_x : f.tiles_y;
  for (int m = 2; m <= mmax; ++m) {
    for (int uy = ty - m; uy <= ty + m; ++uy) {
      if (uy < 0 || uy >= f.tiles_y) continue;
      const bool edge_row = (uy == ty - m || uy == ty + m);
      for (int ux = tx - m; ux <= tx + m; ux += (edge_row ? 1 : 2 * m)) {
        if (ux < 0 || ux >= f.tiles_x) continue;
        const int64_t u = (int64_t)uy * f.tiles_x + ux;
        const int64_t q1 = f.toff[u + 1] < f.n_samples ? f.toff[u + 1] : f.n_samples;
        for (int64_t q = f.toff[u] < 0 ? 0 : f.toff[u]; q < q1; ++q) {
          const Rec rc = f.recs[q];
          const int dx = rc.lx - cx, dy = rc.ly - cy;
          const long long d2 = (long long)dx * dx + (long long)dy * dy;
          if (d2 < a.bd2 || (d2 == a.bd2 && rc.idx < a.bidx)) {
            a.bd2 = d2;
            a.bidx = rc.idx;
          }
        }
      }
    }
    if (a.bd2 != LLONG_MAX && a.bd2 <= (long long)m * f.tile_cm * (long long)m * f.tile_cm) return;
  }
}

// One CTA per tile (or per band of a tile when f.split > 1), 8 warps.  Each warp takes
// whole rows of 8 x 8-texel blocks, two texels of a column per lane.  For a block row it
// lists once the staged samples within R of the row's texels (a candidate list in shared
// memory, ~25 samples in the overview against ~300 staged), and each block of the row
// ballots over that list only.
// Heights are blended relative to the tile's reference z (the first staged sample), so
// the per-texel arithmetic is FP32; the tile's base height z_ref * z_scale + z_offset
// is formed once in FP64.
template <bool kSmall>
__global__ void __launch_bounds__(kFillThreads, kFillMaxCtasPerSm) k_fill(FillArgs f) {
  extern __shared__ __align__(128) unsigned char fill_dyn[];
  Rec* stage = reinterpret_cast<Rec*>(fill_dyn);  // f.stage_cap records (dynamic)
  StRec* st = reinterpret_cast<StRec*>(fill_dyn);  // the same records once converted
  __shared__ __align__(16) float out_h[kOutStageRes * kOutStageRes];
  __shared__ __align__(16) uint8_t out_c[kOutStageRes * kOutStageRes * 3];
  __shared__ __align__(16) uint16_t cand_all[kFillThreads / 32][kCandCap];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int64_t rng_lo[3], rng_n[3];
  __shared__ int stage_n, staged, zref_s;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int res = f.res, cell = f.cell_cm;
  const bool stage_out = res <= kOutStageRes;
  uint16_t* cand = cand_all[warp];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;

  for (int64_t item = blockIdx.x; item < f.n_out * f.split; item += gridDim.x) {
    const int64_t o = item / f.split;
    const int part = (int)(item - o * f.split);
    const int t = f.tile_ids ? f.tile_ids[o] : (int)o;
    if (t < 0 || t >= f.tiles_x * f.tiles_y) {  // uniform across the CTA
      if (threadIdx.x == 0) set_status(LS_ERR_INVALID_ARG);
      continue;
    }
    const int tx = t % f.tiles_x, ty = t / f.tiles_x;
    // ---- stage the 3x3 neighbourhood (three contiguous CSR ranges)
    if (threadIdx.x == 0) {
      int64_t total = 0;
      const int xa = tx > 0 ? tx - 1 : 0, xb = tx + 1 < f.tiles_x ? tx + 1 : tx;
      for (int k = 0; k < 3; ++k) {
        const int uy = ty - 1 + k;
        rng_lo[k] = 0; rng_n[k] = 0;
        if (uy < 0 || uy >= f.tiles_y) continue;
        int64_t a0 = f.toff[(int64_t)uy * f.tiles_x + xa];
        int64_t a1 = f.toff[(int64_t)uy * f.tiles_x + xb + 1];
        if (a0 < 0 || a1 < a0 || a1 > f.n_samples) {  // inconsistent CSR: use nothing
          set_status(LS_ERR_INVALID_ARG);
          a0 = a1 = 0;
        }
        rng_lo[k] = a0; rng_n[k] = a1 - a0;
        total += a1 - a0;
      }
      stage_n = (int)(total < f.stage_cap ? total : f.stage_cap);
      staged = total <= f.stage_cap;
      // the tile's height reference: the first sample of its neighbourhood
      int zr = 0;
      for (int k = 0; k < 3; ++k)
        if (rng_n[k] > 0) { zr = f.recs[rng_lo[k]].z; break; }
      zref_s = zr;
      if (staged && total > 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar, (uint32_t)(total * sizeof(Rec)));
        int64_t d = 0;
        for (int k = 0; k < 3; ++k) {
          if (rng_n[k] > 0) bulk_g2s(&stage[d], &f.recs[rng_lo[k]], (uint32_t)(rng_n[k] * sizeof(Rec)), &bar);
          d += rng_n[k];
        }
      }
    }
    __syncthreads();
    const bool use_stage = staged;
    const int zref = zref_s;
    // base height of the tile, FP64 once; texels add (blended z - zref) * z_scale in FP32
    const float base_h = (float)((double)zref * f.z_scale + f.z_offset);
    if (use_stage && stage_n > 0) {
      int it = 0, limit = 0;
      while (!mbar_try_wait(&bar, phase)) {
        if (it == 0) limit = spin_limit();
        if (++it > limit) { set_status(LS_ERR_TIMEOUT); break; }
      }
      phase ^= 1u;
      // convert the staged records in place: heights relative to zref and colours as
      // floats (each thread its own records)
      for (int k = threadIdx.x; k < stage_n; k += blockDim.x) {
        const Rec r = stage[k];
        StRec v;
        v.lx = r.lx; v.ly = r.ly; v.fz = (float)(r.z - zref); v.idx = r.idx;
        v.fr = (float)(r.rg & 0xffffu); v.fg = (float)(r.rg >> 16); v.fb = (float)r.b; v.pad = 0u;
        st[k] = v;
      }
      __syncthreads();
    }
    // ---- rows of 8 x 8-texel blocks, one row per warp at a time; lane (r, c) of a
    // block owns the texels (r, c) and (r + 4, c)
    const int bw = res / 8, nbr = res / 8;
    const int br0 = part * (nbr / f.split), br1 = br0 + nbr / f.split;  // this part's block rows
    const int dyt = 4 * cell;
    for (int br = br0 + warp; br < br1; br += kFillThreads / 32) {
      const int bi = br * 8;
      const int y0b = ty * f.tile_cm + cell * bi + cell / 2;
      const int rx0 = tx * f.tile_cm + cell / 2 - f.R, rx1 = tx * f.tile_cm + (res - 1) * cell + cell / 2 + f.R;
      const int ry0 = y0b - f.R, ry1 = y0b + 7 * cell + f.R;
      // candidate list of the row (staged samples within R of any of its texels' box)
      int n_cand = 0;
      if (use_stage) {
        for (int base = 0; base < stage_n; base += 32) {
          bool in = false;
          if (base + lane < stage_n) {
            const int2 xy = *reinterpret_cast<const int2*>(&stage[base + lane]);
            in = xy.x >= rx0 && xy.x <= rx1 && xy.y >= ry0 && xy.y <= ry1;
          }
          const unsigned m = __ballot_sync(0xffffffffu, in);
          const int pos = n_cand + __popc(m & ((1u << lane) - 1u));
          if (in && pos < kCandCap) cand[pos] = (uint16_t)(base + lane);
          n_cand += __popc(m);
        }
        __syncwarp();
      }
      const bool use_list = use_stage && n_cand <= kCandCap;
      for (int bj8 = 0; bj8 < bw; ++bj8) {
        const int bj = bj8 * 8;
        const int j = bj + (lane & 7), i0 = bi + (lane >> 3);
        const int cx = tx * f.tile_cm + cell * j + cell / 2;
        const int cy = ty * f.tile_cm + cell * i0 + cell / 2;
        const int x0b = tx * f.tile_cm + cell * bj + cell / 2;
        const int bx0 = x0b - f.R, bx1 = x0b + 7 * cell + f.R;
        LaneAcc a[kTexPerLane];
        unsigned need = 0;
#pragma unroll
        for (int t = 0; t < kTexPerLane; ++t) a[t] = LaneAcc{0.f, 0.f, 0.f, 0.f, 0.f, LLONG_MAX, INT_MAX};
        if (use_stage) {
          LaneAccS as[kTexPerLane];
#pragma unroll
          for (int t = 0; t < kTexPerLane; ++t) as[t] = LaneAccS{0.f, 0.f, 0.f, 0.f, 0.f, ~0ull};
          splat_st<kSmall>(st, use_list ? cand : nullptr, use_list ? n_cand : stage_n, bx0, bx1, ry0, ry1, cx, cy,
                           dyt, f.R2u, f.k2, as);
#pragma unroll
          for (int t = 0; t < kTexPerLane; ++t) need |= (as[t].sw > 0.f) ? 0u : (1u << t);
          if (__any_sync(0xffffffffu, need != 0)) {
            // grow the box to the largest current best distance of the texels in need
            // (in-box samples were all considered above); a texel without any in-box
            // sample makes the search unbounded
            bool unbounded = false;
            long long wmax = 0;
#pragma unroll
            for (int t = 0; t < kTexPerLane; ++t) {
              if (!(need & (1u << t))) continue;
              if (as[t].key == ~0ull) unbounded = true;
              else wmax = max(wmax, (long long)(as[t].key >> kKeyShift));
            }
            for (int off = 16; off > 0; off >>= 1) {
              const long long ov = __shfl_xor_sync(0xffffffffu, wmax, off);
              wmax = ov > wmax ? ov : wmax;
            }
            int grow = (int)ceilf(sqrtf((float)wmax)) + 1;
            if (__any_sync(0xffffffffu, unbounded) || grow > 2 * f.tile_cm) grow = 2 * f.tile_cm;
            nearest_st(st, stage_n, need, cx, cy, dyt, x0b - grow, x0b + 7 * cell + grow, y0b - grow,
                       y0b + 7 * cell + grow, as);
          }
#pragma unroll
          for (int t = 0; t < kTexPerLane; ++t) {
            a[t].sw = as[t].sw; a[t].swz = as[t].swz; a[t].swr = as[t].swr; a[t].swg = as[t].swg;
            a[t].swb = as[t].swb;
            if (as[t].key != ~0ull) {
              a[t].bd2 = (long long)(as[t].key >> kKeyShift);
              // the sample index is needed only for a nearest-sample texel
              if (need & (1u << t)) a[t].bidx = st[as[t].key & ((1u << kKeyShift) - 1)].idx;
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < kTexPerLane; ++t) {
            for (int k = 0; k < 3; ++k)
              splat_range(f.recs + rng_lo[k], (int)rng_n[k], bx0, bx1, ry0, ry1, cx, cy + t * dyt, zref, f.R2u,
                          f.k2, a[t]);
            need |= (a[t].sw > 0.f) ? 0u : (1u << t);
          }
          if (__any_sync(0xffffffffu, need != 0)) {
            bool unbounded = false;
            long long wmax = 0;
#pragma unroll
            for (int t = 0; t < kTexPerLane; ++t) {
              if (!(need & (1u << t))) continue;
              if (a[t].bd2 == LLONG_MAX) unbounded = true;
              else wmax = max(wmax, a[t].bd2);
            }
            for (int off = 16; off > 0; off >>= 1) {
              const long long ov = __shfl_xor_sync(0xffffffffu, wmax, off);
              wmax = ov > wmax ? ov : wmax;
            }
            int grow = (int)ceilf(sqrtf((float)wmax)) + 1;
            if (__any_sync(0xffffffffu, unbounded) || grow > 2 * f.tile_cm) grow = 2 * f.tile_cm;
            const int gx0 = x0b - grow, gx1 = x0b + 7 * cell + grow;
            const int gy0 = y0b - grow, gy1 = y0b + 7 * cell + grow;
#pragma unroll
            for (int t = 0; t < kTexPerLane; ++t)
              for (int k = 0; k < 3; ++k)
                nearest_range(f.recs + rng_lo[k], (int)rng_n[k], (need >> t) & 1u, cx, cy + t * dyt, gx0, gx1, gy0,
                              gy1, a[t]);
          }
        }
#pragma unroll
        for (int t = 0; t < kTexPerLane; ++t) {
          const int i = i0 + 4 * t;
          const int cyt = cy + t * dyt;
          const bool nd = (need >> t) & 1u;
          if (nd && !(a[t].bd2 != LLONG_MAX && a[t].bd2 <= (long long)f.tile_cm * f.tile_cm))
            nearest_far(f, tx, ty, cx, cyt, a[t]);
          float h;
          float c3[3];
          if (!nd) {
            const float inv = 1.0f / a[t].sw;
            h = fmaf(a[t].swz * inv, f.zs_f, base_h);
            c3[0] = a[t].swr * inv * (1.0f / 256.0f);
            c3[1] = a[t].swg * inv * (1.0f / 256.0f);
            c3[2] = a[t].swb * inv * (1.0f / 256.0f);
          } else if (a[t].bd2 != LLONG_MAX) {
            const Rec q = f.recs[a[t].bidx];  // records are indexed by sample
            h = fmaf((float)(q.z - zref), f.zs_f, base_h);
            c3[0] = (float)(q.rg & 0xffffu) * (1.0f / 256.0f);
            c3[1] = (float)(q.rg >> 16) * (1.0f / 256.0f);
            c3[2] = (float)q.b * (1.0f / 256.0f);
          } else {
            h = __int_as_float(0x7fc00000);
            c3[0] = c3[1] = c3[2] = 0.f;
          }
          if (f.aux_hc) {
            const size_t ae = (size_t)o * res * res + (size_t)i * res + j;
            f.aux_hc[ae] = make_float4(h, c3[0] * (256.0f / 65535.0f), c3[1] * (256.0f / 65535.0f),
                                       c3[2] * (256.0f / 65535.0f));
            f.aux_d[ae] = a[t].bd2 != LLONG_MAX ? sqrtf((float)a[t].bd2) : __int_as_float(0x7f800000);
          }
          uint8_t q8[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float v = floorf(c3[c] + 0.5f);
            q8[c] = (uint8_t)(v > 255.f ? 255.f : v);
          }
          const int e = i * res + j;
          if (stage_out) {
            out_h[e] = h;
            out_c[3 * e] = q8[0]; out_c[3 * e + 1] = q8[1]; out_c[3 * e + 2] = q8[2];
          } else {
            f.height[o * res * res + e] = h;
            uint8_t* dst = f.rgb + (o * res * res + e) * 3;
            dst[0] = q8[0]; dst[1] = q8[1]; dst[2] = q8[2];
          }
        }
      }
      __syncwarp();  // the next row's list overwrites this one
    }
    __syncthreads();
    if (stage_out) {
      // this part's band of rows; its bytes (rows * res * 4 and * 3) are multiples of 16
      // for res % 16 == 0
      const int rows = res / f.split, r0 = part * rows;
      const int h0 = r0 * res / 4, nh = rows * res / 4, c0 = r0 * res * 3 / 16, nc = rows * res * 3 / 16;
      float4* gh = reinterpret_cast<float4*>(f.height + o * res * res);
      int4* gc = reinterpret_cast<int4*>(f.rgb + o * res * res * 3);
      for (int k = threadIdx.x; k < nh; k += blockDim.x) gh[h0 + k] = reinterpret_cast<const float4*>(out_h)[h0 + k];
      for (int k = threadIdx.x; k < nc; k += blockDim.x) gc[c0 + k] = reinterpret_cast<const int4*>(out_c)[c0 + k];
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------
// tile update
// ---------------------------------------------------------------------------------
__global__ void k_update(ls_bins bins, const int32_t* __restrict__ tile_ids, int64_t n, int64_t n_tiles,
                         double z_scale, double z_offset, float* __restrict__ height, uint8_t* __restrict__ rgb) {
  const int64_t cpt = (int64_t)bins.cells * bins.cells;
  const int64_t total = n * cpt;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e / cpt, c = e - o * cpt;
    const int64_t t = tile_ids ? (int64_t)tile_ids[o] : o;
    if (t < 0 || t >= n_tiles) {
      set_status(LS_ERR_INVALID_ARG);
      continue;
    }
    const int64_t src = t * cpt + c;
    const uint32_t cnt = bins.count[src];
    if (cnt == 0u) continue;
    const double nd = (double)cnt;
    const double mean = __ddiv_rn((double)bins.zsum[src], nd);
    height[e] = (float)__dadd_rn(__dmul_rn(mean, z_scale), z_offset);
    const uint64_t sums[3] = {bins.rsum[src], bins.gsum[src], bins.bsum[src]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = floor(__dadd_rn(__ddiv_rn(__ddiv_rn((double)sums[k], nd), 256.0), 0.5));
      rgb[e * 3 + k] = (uint8_t)(v > 255.0 ? 255.0 : v);
    }
  }
}

}  // namespace
}  // namespace ls

using namespace ls;

extern "C" ls_status ls_extract_samples(const ls_points* pts, int64_t n_tiles, int32_t chunk,
                                        int64_t* sample_offsets, const ls_sample_buffers* out,
                                        int64_t capacity, ls_stream_t stream) {
  if (!pts || !out || !sample_offsets || n_tiles <= 0 || chunk <= 0 || capacity < 0) return LS_ERR_INVALID_ARG;
  if (!pts->tile_offsets) return LS_ERR_INVALID_ARG;
  if (pts->n > 0 && (!pts->x || !pts->y || !pts->z || !pts->r || !pts->g || !pts->b)) return LS_ERR_INVALID_ARG;
  if (capacity > 0 && (!out->x || !out->y || !out->z || !out->r || !out->g || !out->b)) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_sample_offsets<<<1, 1024, 0, s>>>(pts->tile_offsets, n_tiles, chunk, sample_offsets);
  k_extract<<<grid_cap((n_tiles + 7) / 8, kSmCount * 8), 256, 0, s>>>(*pts, n_tiles, chunk, sample_offsets, *out,
                                                                     capacity);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

namespace ls {
// Validated launch of the Gaussian fill (optionally with the per-texel auxiliary
// outputs of the learned filler's input raster).  Returns the packed records.
ls_status fill_launch(const ls_points* samples, const ls_region* region, const ls_fill_params* params,
                      const int32_t* tile_ids, int64_t n_out, float* height, uint8_t* rgb, float4* aux_hc,
                      float* aux_d, cudaStream_t s, const void** recs_out) {
  if (!samples || !region || !params || !height || !rgb || n_out < 0) return LS_ERR_INVALID_ARG;
  if (!samples->tile_offsets) return LS_ERR_INVALID_ARG;
  if (samples->n > 0 && (!samples->x || !samples->y || !samples->z || !samples->r || !samples->g || !samples->b))
    return LS_ERR_INVALID_ARG;
  if (samples->n >= (int64_t(1) << 31)) return LS_ERR_UNSUPPORTED;
  if (region->tile_cm <= 0 || region->tiles_x <= 0 || region->tiles_y <= 0) return LS_ERR_INVALID_ARG;
  if ((int64_t)region->tiles_x * region->tile_cm >= (int64_t(1) << 31) ||
      (int64_t)region->tiles_y * region->tile_cm >= (int64_t(1) << 31))
    return LS_ERR_INVALID_ARG;
  const int64_t T = (int64_t)region->tiles_x * region->tiles_y;
  if (!tile_ids && n_out != T) return LS_ERR_INVALID_ARG;
  if (params->res < 8 || params->res > 1024 || params->res % 8 || region->tile_cm % params->res)
    return LS_ERR_INVALID_ARG;
  if (params->radius_cm < 1 || params->radius_cm > region->tile_cm || params->radius_cm > 65535)
    return LS_ERR_UNSUPPORTED;
  if (!(params->sigma_cm > 0.f)) return LS_ERR_INVALID_ARG;
  if (n_out == 0) return LS_OK;
  Rec* recs = static_cast<Rec*>(workspace(kWsFillPacked, (size_t)(samples->n > 0 ? samples->n : 1) * sizeof(Rec)));
  if (!recs) return LS_ERR_NO_MEMORY;
  if (recs_out) *recs_out = recs;
  if (samples->n > 0)
    k_pack<<<grid_cap((T + 7) / 8, kSmCount * 16), 256, 0, s>>>(*samples, T, region->x0_cm, region->y0_cm,
                                                                 region->tile_cm, region->tiles_x, recs);
  FillArgs f;
  f.toff = samples->tile_offsets;
  f.recs = recs;
  f.tile_ids = tile_ids;
  f.n_out = n_out;
  f.n_samples = samples->n;
  f.tiles_x = region->tiles_x;
  f.tiles_y = region->tiles_y;
  f.tile_cm = region->tile_cm;
  f.res = params->res;
  f.cell_cm = region->tile_cm / params->res;
  f.R = params->radius_cm;
  f.R2u = (uint32_t)params->radius_cm * (uint32_t)params->radius_cm;
  f.k2 = (float)(1.4426950408889634 / (2.0 * (double)params->sigma_cm * (double)params->sigma_cm));
  f.zs_f = (float)region->z_scale;
  // stage: room for 1.5 x the average 3 x 3 neighbourhood (a power of two, 256..2048
  // records); a tile whose neighbourhood does not fit reads it from global memory
  {
    const int64_t want = (samples->n * 27 + 2 * T - 1) / (2 * T);
    int cap = 256;
    while (cap < want && cap < kStageCap) cap *= 2;
    f.stage_cap = cap;
  }
  f.z_scale = region->z_scale;
  f.z_offset = region->z_offset;
  f.height = height;
  f.rgb = rgb;
  f.aux_hc = aux_hc;
  f.aux_d = aux_d;
  static DeviceOnce once;
  static int occ[kMaxDevicesOnce + 1][5] = {};  // resident CTAs per SM by stage size (256 << k)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ERR_CUDA;
  const int di = dev >= 0 && dev < kMaxDevicesOnce ? dev : kMaxDevicesOnce;
  if (!device_once(once, dev, [&] {
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(k_fill<true>, attr, (int)(kStageCap * sizeof(Rec))) != cudaSuccess ||
            cudaFuncSetAttribute(k_fill<false>, attr, (int)(kStageCap * sizeof(Rec))) != cudaSuccess)
          return false;
        for (int k = 0; k < 5; ++k) {
          int b = 0, b2 = 0;
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fill<true>, kFillThreads,
                                                            (size_t)(256 << k) * sizeof(Rec)) != cudaSuccess ||
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_fill<false>, kFillThreads,
                                                            (size_t)(256 << k) * sizeof(Rec)) != cudaSuccess)
            return false;
          b = b2 < b ? b2 : b;
          occ[di][k] = b > 0 ? b : 1;
        }
        return true;
      }))
    return LS_ERR_CUDA;
  int ks = 0;
  while ((256 << ks) < f.stage_cap) ++ks;
  // launch shape: tuned for this key (ls_tune_fill_sparse / ls_fill_shape_set), else the
  // default: few tiles are split over 4 CTAs (bands of res / 4 texel rows, whole 8-row
  // blocks), and the persistent grid is sized for the CTAs that fit on an SM
  FillShape shape;
  fill_shape_lookup(fill_shape_key(samples->n, n_out, params), params->res, n_out, &shape);
  f.split = shape.split;
  const int per_sm = shape.ctas_per_sm < occ[di][ks] ? shape.ctas_per_sm : occ[di][ks];
  // 32-bit squared distances for every sample in a block's box: |dx|, |dy| <= R + 7
  // cells from either texel of a lane
  const uint64_t ex = (uint64_t)f.R + 7 * (uint64_t)f.cell_cm, ey = ex;
  const bool small = ex * ex + ey * ey < (uint64_t(1) << 32);
  const dim3 grid(grid_cap(n_out * f.split, (int64_t)kSmCount * per_sm));
  const size_t smem = (size_t)f.stage_cap * sizeof(Rec);
  if (small)
    k_fill<true><<<grid, kFillThreads, smem, s>>>(f);
  else
    k_fill<false><<<grid, kFillThreads, smem, s>>>(f);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
}  // namespace ls

extern "C" ls_status ls_fill_sparse(const ls_points* samples, const ls_region* region,
                                    const ls_fill_params* params, const int32_t* tile_ids, int64_t n_out,
                                    float* height, uint8_t* rgb, ls_stream_t stream) {
  return ls::fill_launch(samples, region, params, tile_ids, n_out, height, rgb, nullptr, nullptr,
                         reinterpret_cast<cudaStream_t>(stream), nullptr);
}

extern "C" ls_status ls_update_tile(const ls_bins* bins, const ls_region* region, const int32_t* tile_ids,
                                    int64_t n, float* height, uint8_t* rgb, ls_stream_t stream) {
  if (!bins || !region || !height || !rgb || n < 0) return LS_ERR_INVALID_ARG;
  if (!bins->count || !bins->zsum || !bins->rsum || !bins->gsum || !bins->bsum || bins->cells <= 0)
    return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  if (!tile_ids && n > (int64_t)region->tiles_x * region->tiles_y) return LS_ERR_INVALID_ARG;
  const int64_t total = n * bins->cells * bins->cells;
  k_update<<<grid_cap((total + 255) / 256, kSmCount * 16), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      *bins, tile_ids, n, (int64_t)region->tiles_x * region->tiles_y, region->z_scale, region->z_offset,
      height, rgb);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
