// Exact full-resolution binning of int32-quantised points into per-tile cell grids
// (count, sum z, min z, max z, sums of R, G, B per cell).  Ground-truth heightmaps
// are the mean of all points falling onto a texel (Sec. 3.4) and full-resolution
// points update the heightmap textures (abstract, Sec. 3.5); these exact integer
// sums are what both need.
//
// Design (B300, one CTA per SM, HBM-bound):
//  * The points arrive in LAZ storage order: tile after tile, and inside a tile in
//    8 m scan strips.  "Global fine row" G = tile * cells + row is therefore almost
//    monotone along the stream.  Each CTA streams a contiguous span of points with
//    128-bit loads and accumulates into a shared-memory ring of W fine rows
//    (32 bytes per cell: packed R|G, B|count, z-sum, z-min, z-max) with shared
//    atomics.  When a point lands above the window, the window slides and the rows
//    that leave are flushed.
//  * Flush protocol per row (per-row state word in scratch: 0 free, 1 being
//    written, 2 written): the first CTA to flush a row claims it (0 -> 1), writes
//    all its cells with plain coalesced stores (empty cells get the sentinels),
//    fences and publishes 2.  Any later contribution to that row (another CTA's
//    part of a strip, or a late point) merges with global atomics after seeing 2.
//    So every output byte is written once by a plain store in the common case and
//    no memset pass is needed.  Rows that nobody touched get sentinels in a final
//    pass.  Result is exact for ANY point order; only speed depends on the order.
//  * Coarse level (e.g. 64x64 from 640x640): reduced exactly from the fine cells
//    while they are flushed, accumulated in a small shared ring of coarse rows and
//    merged with global atomics into the (L2-resident) coarse arrays, which a
//    prologue kernel initialises.
//  * Packed 32-bit colour sums in shared memory cannot overflow: a row is forced out
//    of the window before it can have absorbed 65536 points (65536 * 65535 < 2^32).
#include <climits>
#include <mutex>

#include "ls_internal.cuh"

namespace ls {
namespace {

constexpr int kBinThreads = 512;
constexpr int kPtsPerThread = 4;
constexpr int kBatch = kBinThreads * kPtsPerThread;  // 2048 points per batch
constexpr int kResidLimitBatches = 65536 / kBatch;     // residency bound (batches)
constexpr int kMaxW = 64;
constexpr int kCW = 4;  // coarse ring rows

struct BinArgs {
  const int32_t* __restrict__ x;
  const int32_t* __restrict__ y;
  const int32_t* __restrict__ z;
  const uint16_t* __restrict__ r;
  const uint16_t* __restrict__ g;
  const uint16_t* __restrict__ b;
  int64_t n;
  int64_t x0, y0;
  uint32_t ext_x, ext_y;
  FastDiv div_tile, div_cell, div_f;
  uint32_t tile_cm, cell_cm;
  int32_t tiles_x, cells, W, f, ccells, has_coarse;
  int32_t n_rows;  // T * cells
  // fine level
  uint32_t* count;
  int64_t* zsum;
  int32_t* zmin;
  int32_t* zmax;
  uint64_t *rsum, *gsum, *bsum;
  // coarse level
  uint32_t* ccount;
  int64_t* czsum;
  int32_t* czmin;
  int32_t* czmax;
  uint64_t *crsum, *cgsum, *cbsum;
  uint32_t* row_state;
  uint64_t* dropped;
  int64_t span;
  int64_t n_items;
  int vec;
  int narrow;            // x0 and y0 fit int32: 32-bit region-local coordinates
  int32_t x0_32, y0_32;
  // shared-memory row layout: the f fine cells of a coarse cell occupy gs >= f slots
  // (gs odd), so one thread per coarse cell reads its fine cells without bank conflicts
  int32_t gs, rstride;
};

// shared-memory layout (dynamic).  Every fine accumulator is a 32-bit word (32-bit
// shared atomics are several times cheaper than 64-bit ones): z is split into its low
// 16 bits (unsigned) and its high bits (signed), zsum = 65536 * sum(hi) + sum(lo),
// both sums exact while a cell absorbs at most 65536 points.
struct Smem {
  unsigned* cnt;  // [W*rstride]
  unsigned* rs;
  unsigned* gs;
  unsigned* bs;
  unsigned* zlo;
  int* zhi;
  int* mn;
  int* mx;
  unsigned long long* crs;  // [kCW*ccells] coarse sums
  unsigned long long* cgs;
  unsigned long long* cbs;
  unsigned long long* czs;
  unsigned* ccnt;
  int* cmn;
  int* cmx;
};

struct Meta {
  int touched[kMaxW];
  int enter[kMaxW];  // batch index at which the row entered the window
  int mode[kMaxW];   // 0 none, 1 store, 2 merge
  int red[kBinThreads / 32];
  int redx[kBinThreads / 32];
  int bcast, bcastx;
  int clo_old, clo_new;  // coarse ring scratch of evict_rows (not shared with block_min)
  int n_inplace;
  int oldest;  // lowest entry batch over the window's slots
  unsigned long long dropped;
  unsigned long long n_late;
};

__device__ __forceinline__ Smem carve(unsigned char* base, int WC, int CC) {
  Smem s;
  s.crs = reinterpret_cast<unsigned long long*>(base);
  s.cgs = s.crs + CC;
  s.cbs = s.cgs + CC;
  s.czs = s.cbs + CC;
  s.cnt = reinterpret_cast<unsigned*>(s.czs + CC);
  s.rs = s.cnt + WC;
  s.gs = s.rs + WC;
  s.bs = s.gs + WC;
  s.zlo = s.bs + WC;
  s.zhi = reinterpret_cast<int*>(s.zlo + WC);
  s.mn = s.zhi + WC;
  s.mx = s.mn + WC;
  s.ccnt = reinterpret_cast<unsigned*>(s.mx + WC);
  s.cmn = reinterpret_cast<int*>(s.ccnt + CC);
  s.cmx = s.cmn + CC;
  return s;
}

__host__ __device__ constexpr size_t smem_bytes(int WC, int CC) {
  return (size_t)WC * (8 * 4) + (size_t)CC * (4 * 8 + 3 * 4);
}

// one fine cell, reassembled from its shared words
struct Cell {
  unsigned cnt;
  long long zsum;
  int zmin, zmax;
  unsigned r, g, b;
};

__device__ __forceinline__ Cell read_cell(const Smem& s, int si) {
  Cell c;
  c.cnt = s.cnt[si];
  c.zsum = (long long)s.zhi[si] * 65536 + (long long)s.zlo[si];
  c.zmin = s.mn[si];
  c.zmax = s.mx[si];
  c.r = s.rs[si];
  c.g = s.gs[si];
  c.b = s.bs[si];
  return c;
}

__device__ __forceinline__ void reset_cell(Smem& s, int si) {
  s.cnt[si] = 0u; s.rs[si] = 0u; s.gs[si] = 0u; s.bs[si] = 0u;
  s.zlo[si] = 0u; s.zhi[si] = 0; s.mn[si] = INT_MAX; s.mx[si] = INT_MIN;
}

// Diagnostics of the last calls (cumulative until read): late points, waits on a
// row another CTA was writing, waits that ran out, rows flushed in place by the
// residency bound.
__device__ unsigned long long g_bin_stats[4];

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait (bounded) until a row state is 2.
__device__ void wait_written(const uint32_t* state) {
  if (ld_acquire(state) == 2u) return;
  atomicAdd(&g_bin_stats[1], 1ull);
  int it = 0;
  while (ld_acquire(state) != 2u) {
    if (++it > kSpinLimit) {
      set_status(LS_ERR_TIMEOUT);
      atomicAdd(&g_bin_stats[2], 1ull);
      return;
    }
    __nanosleep(64);
  }
}

__device__ __forceinline__ void store_empty_cell(const BinArgs& a, int64_t o) {
  a.count[o] = 0u;
  a.zsum[o] = 0;
  a.zmin[o] = INT_MAX;
  a.zmax[o] = INT_MIN;
  a.rsum[o] = 0ull;
  a.gsum[o] = 0ull;
  a.bsum[o] = 0ull;
}

__device__ __forceinline__ void merge_fine(const BinArgs& a, int64_t o, uint32_t cnt, long long zsum,
                                           int zmin, int zmax, unsigned long long rs,
                                           unsigned long long gs, unsigned long long bs) {
  atomicAdd(&a.count[o], cnt);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.zsum[o]), (unsigned long long)zsum);
  atomicMin(&a.zmin[o], zmin);
  atomicMax(&a.zmax[o], zmax);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.rsum[o]), rs);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.gsum[o]), gs);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.bsum[o]), bs);
}

__device__ __forceinline__ void merge_coarse(const BinArgs& a, int64_t o, uint32_t cnt, long long zsum,
                                             int zmin, int zmax, unsigned long long rs,
                                             unsigned long long gs, unsigned long long bs) {
  atomicAdd(&a.ccount[o], cnt);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.czsum[o]), (unsigned long long)zsum);
  atomicMin(&a.czmin[o], zmin);
  atomicMax(&a.czmax[o], zmax);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.crsum[o]), rs);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.cgsum[o]), gs);
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.cbsum[o]), bs);
}

__device__ __forceinline__ int coarse_row_of(const BinArgs& a, int G) {
  const int tile = G / a.cells;
  const int row = G - tile * a.cells;
  return tile * a.ccells + (int)fdiv((uint32_t)row, a.div_f);
}

__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory reductions without a returned value (no scoreboard wait)
__device__ __forceinline__ void red_add(unsigned* p, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add(int* p, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_min(int* p, int v) {
  asm volatile("red.shared.min.s32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void red_max(int* p, int v) {
  asm volatile("red.shared.max.s32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}

// shared slot of fine column col in ring slot `slot` (padded layout, see BinArgs)
__device__ __forceinline__ int sidx(const BinArgs& a, int slot, int col) {
  const int cg = (int)fdiv((uint32_t)col, a.div_f);
  return slot * a.rstride + cg * a.gs + (col - cg * a.f);
}

// A point whose row already left this CTA's window: claim the row if nobody has
// written it yet (single thread writes sentinels), then merge with global atomics.
__device__ void late_point(const BinArgs& a, int G, int col, int z, uint32_t r, uint32_t g, uint32_t b) {
  uint32_t* st = &a.row_state[G];
  if (ld_acquire(st) != 2u) {
    if (atomicCAS(st, 0u, 1u) == 0u) {
      const int64_t base = (int64_t)G * a.cells;
      for (int c = 0; c < a.cells; ++c) store_empty_cell(a, base + c);
      __threadfence();
      atomicExch(st, 2u);
    } else {
      wait_written(st);
    }
  }
  merge_fine(a, (int64_t)G * a.cells + col, 1u, z, z, z, r, g, b);
  if (a.has_coarse) {
    const int64_t o = (int64_t)coarse_row_of(a, G) * a.ccells + (int)fdiv((uint32_t)col, a.div_f);
    merge_coarse(a, o, 1u, z, z, z, r, g, b);
  }
}

// Block-wide min and max (every thread gets both).
__device__ __forceinline__ void block_minmax(int vmin, int vmax, Meta& m, int& omin, int& omax) {
  vmin = __reduce_min_sync(0xffffffffu, vmin);
  vmax = __reduce_max_sync(0xffffffffu, vmax);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // m.red may still be read by a previous reduction
  if (lane == 0) { m.red[warp] = vmin; m.redx[warp] = vmax; }
  __syncthreads();
  if (warp == 0) {
    int u = lane < (kBinThreads / 32) ? m.red[lane] : INT_MAX;
    int x = lane < (kBinThreads / 32) ? m.redx[lane] : INT_MIN;
    u = __reduce_min_sync(0xffffffffu, u);
    x = __reduce_max_sync(0xffffffffu, x);
    if (lane == 0) { m.bcast = u; m.bcastx = x; }
  }
  __syncthreads();
  omin = m.bcast;
  omax = m.bcastx;
}

// Flush coarse ring rows [ca, cb) (all inside the ring) to global with atomics.
__device__ void coarse_evict(const BinArgs& a, Smem& s, int ca, int cb) {
  const int n = (cb - ca) * a.ccells;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int rr = i / a.ccells, c = i - rr * a.ccells;
    const int Gc = ca + rr;
    const int si = (Gc % kCW) * a.ccells + c;
    const unsigned cnt = s.ccnt[si];
    if (cnt) {
      merge_coarse(a, (int64_t)Gc * a.ccells + c, cnt, (long long)s.czs[si], s.cmn[si], s.cmx[si],
                   s.crs[si], s.cgs[si], s.cbs[si]);
      s.ccnt[si] = 0u;
      s.czs[si] = 0ull;
      s.crs[si] = 0ull;
      s.cgs[si] = 0ull;
      s.cbs[si] = 0ull;
      s.cmn[si] = INT_MAX;
      s.cmx[si] = INT_MIN;
    }
  }
}

// Evict fine rows [ra, rb) (rb - ra <= W, all inside the ring).  The caller has
// synchronised the block after the last accumulation.
__device__ void evict_rows(const BinArgs& a, Smem& s, Meta& m, int ra, int rb, int& clo) {
  const int nr = rb - ra;
  if (nr <= 0) return;
  const int W = a.W;
  // claim (0 -> 1) without waiting: a CTA never waits while it holds an unpublished
  // claim, so two CTAs flushing overlapping rows cannot wait on each other
  if (threadIdx.x < nr) {
    const int G = ra + threadIdx.x;
    const int slot = G & (W - 1);
    int mode = 0;
    if (m.touched[slot]) mode = (atomicCAS(&a.row_state[G], 0u, 1u) == 0u) ? 1 : 2;
    m.mode[threadIdx.x] = mode;
  }
  // coarse ring: make room for the coarse rows of [ra, rb)
  if (a.has_coarse && threadIdx.x == 0) {
    const int ca = coarse_row_of(a, ra), cb = coarse_row_of(a, rb - 1);
    const int c0 = clo < 0 ? ca : clo;
    m.clo_old = c0;
    m.clo_new = (cb >= c0 + kCW) ? cb - kCW + 1 : c0;
  }
  __syncthreads();
  if (a.has_coarse) {
    const int old_clo = m.clo_old, new_clo = m.clo_new;
    if (new_clo > old_clo) {
      coarse_evict(a, s, old_clo, new_clo < old_clo + kCW ? new_clo : old_clo + kCW);
      __syncthreads();
    }
    clo = new_clo;
    // coarse reduction of the fine rows being evicted: one thread per (fine row,
    // coarse cell) pair sums its f fine cells, then shared atomics merge pairs that
    // fall on the same coarse cell
    for (int e = threadIdx.x; e < nr * a.ccells; e += blockDim.x) {
      const int rr = e / a.ccells, c = e - rr * a.ccells;
      if (m.mode[rr] == 0) continue;
      const int G = ra + rr;
      const int slot = G & (W - 1);
      unsigned cnt = 0;
      long long zsum = 0;
      int zmn = INT_MAX, zmx = INT_MIN;
      unsigned long long rs = 0, gs = 0, bs = 0;
      for (int k = 0; k < a.f; ++k) {
        const int si = slot * a.rstride + c * a.gs + k;
        const unsigned cn = s.cnt[si];
        if (!cn) continue;
        const Cell fc = read_cell(s, si);
        cnt += cn;
        zsum += fc.zsum;
        zmn = min(zmn, fc.zmin);
        zmx = max(zmx, fc.zmax);
        rs += fc.r;
        gs += fc.g;
        bs += fc.b;
      }
      if (!cnt) continue;
      const int Gc = coarse_row_of(a, G);
      if (Gc >= clo && Gc < clo + kCW) {
        const int ci = (Gc % kCW) * a.ccells + c;
        atomicAdd(&s.ccnt[ci], cnt);
        atomicAdd(&s.czs[ci], (unsigned long long)zsum);
        atomicMin(&s.cmn[ci], zmn);
        atomicMax(&s.cmx[ci], zmx);
        atomicAdd(&s.crs[ci], rs);
        atomicAdd(&s.cgs[ci], gs);
        atomicAdd(&s.cbs[ci], bs);
      } else {
        merge_coarse(a, (int64_t)Gc * a.ccells + c, cnt, zsum, zmn, zmx, rs, gs, bs);
      }
    }
    __syncthreads();
  }
  // fine rows claimed here: plain stores of every cell (empty cells get sentinels)
  for (int rr = 0; rr < nr; ++rr) {
    if (m.mode[rr] != 1) continue;
    const int G = ra + rr;
    const int slot = G & (W - 1);
    const int64_t base = (int64_t)G * a.cells;
    for (int c = threadIdx.x; c < a.cells; c += blockDim.x) {
      const int si = sidx(a, slot, c);
      const Cell fc = read_cell(s, si);
      a.count[base + c] = fc.cnt;
      a.zsum[base + c] = fc.zsum;
      a.zmin[base + c] = fc.zmin;
      a.zmax[base + c] = fc.zmax;
      a.rsum[base + c] = fc.r;
      a.gsum[base + c] = fc.g;
      a.bsum[base + c] = fc.b;
      reset_cell(s, si);
    }
  }
  __threadfence();
  __syncthreads();
  // publish, then (holding no claim any more) wait for rows another CTA is writing
  if (threadIdx.x < nr) {
    const int G = ra + threadIdx.x;
    if (m.mode[threadIdx.x] == 1) atomicExch(&a.row_state[G], 2u);
    else if (m.mode[threadIdx.x] == 2) wait_written(&a.row_state[G]);
  }
  __syncthreads();
  // rows written first by another CTA: merge with global atomics
  for (int rr = 0; rr < nr; ++rr) {
    if (m.mode[rr] != 2) continue;
    const int G = ra + rr;
    const int slot = G & (W - 1);
    const int64_t base = (int64_t)G * a.cells;
    for (int c = threadIdx.x; c < a.cells; c += blockDim.x) {
      const int si = sidx(a, slot, c);
      const Cell fc = read_cell(s, si);
      if (fc.cnt) merge_fine(a, base + c, fc.cnt, fc.zsum, fc.zmin, fc.zmax, fc.r, fc.g, fc.b);
      reset_cell(s, si);
    }
  }
  __syncthreads();
  if (threadIdx.x < nr) m.touched[(ra + threadIdx.x) & (W - 1)] = 0;
  __syncthreads();
}

// Raw points of one thread's slot of a batch (kPtsPerThread consecutive points).
struct Raw {
  int x[kPtsPerThread], y[kPtsPerThread], z[kPtsPerThread];
  uint32_t r[kPtsPerThread], g[kPtsPerThread], b[kPtsPerThread];
  int n;
};

__device__ __forceinline__ void load_raw(const BinArgs& a, Raw& v, int64_t i0, int64_t p1) {
  v.n = (int)((p1 - i0) < kPtsPerThread ? (p1 - i0) : kPtsPerThread);
  if (v.n == kPtsPerThread && a.vec) {
    const int4 vx = __ldcs(reinterpret_cast<const int4*>(a.x + i0));
    const int4 vy = __ldcs(reinterpret_cast<const int4*>(a.y + i0));
    const int4 vz = __ldcs(reinterpret_cast<const int4*>(a.z + i0));
    const uint2 vr = __ldcs(reinterpret_cast<const uint2*>(a.r + i0));
    const uint2 vg = __ldcs(reinterpret_cast<const uint2*>(a.g + i0));
    const uint2 vb = __ldcs(reinterpret_cast<const uint2*>(a.b + i0));
    v.x[0] = vx.x; v.x[1] = vx.y; v.x[2] = vx.z; v.x[3] = vx.w;
    v.y[0] = vy.x; v.y[1] = vy.y; v.y[2] = vy.z; v.y[3] = vy.w;
    v.z[0] = vz.x; v.z[1] = vz.y; v.z[2] = vz.z; v.z[3] = vz.w;
    v.r[0] = vr.x & 0xffffu; v.r[1] = vr.x >> 16; v.r[2] = vr.y & 0xffffu; v.r[3] = vr.y >> 16;
    v.g[0] = vg.x & 0xffffu; v.g[1] = vg.x >> 16; v.g[2] = vg.y & 0xffffu; v.g[3] = vg.y >> 16;
    v.b[0] = vb.x & 0xffffu; v.b[1] = vb.x >> 16; v.b[2] = vb.y & 0xffffu; v.b[3] = vb.y >> 16;
  } else {
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
      if (k < v.n) {
        v.x[k] = a.x[i0 + k]; v.y[k] = a.y[i0 + k]; v.z[k] = a.z[i0 + k];
        v.r[k] = a.r[i0 + k]; v.g[k] = a.g[i0 + k]; v.b[k] = a.b[i0 + k];
      } else {
        v.x[k] = v.y[k] = v.z[k] = 0;
        v.r[k] = v.g[k] = v.b[k] = 0u;
      }
    }
  }
}

__device__ __forceinline__ void accumulate(Smem& s, Meta& m, const BinArgs& a, int slot, int col, int z, uint32_t r,
                                           uint32_t g, uint32_t b) {
  const int si = sidx(a, slot, col);
  red_add(&s.cnt[si], 1u);
  red_add(&s.rs[si], r);
  red_add(&s.gs[si], g);
  red_add(&s.bs[si], b);
  red_add(&s.zlo[si], (unsigned)z & 0xffffu);
  red_add(&s.zhi[si], z >> 16);
  red_min(&s.mn[si], z);
  red_max(&s.mx[si], z);
  m.touched[slot] = 1;
}

__global__ void __launch_bounds__(kBinThreads, 1) k_bin_main(BinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Meta m;
  const int WC = a.W * a.rstride;
  const int CC = a.has_coarse ? kCW * a.ccells : 0;
  Smem s = carve(smem_raw, WC, CC);
  for (int i = threadIdx.x; i < WC; i += blockDim.x) reset_cell(s, i);
  for (int i = threadIdx.x; i < CC; i += blockDim.x) {
    s.crs[i] = 0ull; s.cgs[i] = 0ull; s.cbs[i] = 0ull; s.czs[i] = 0ull;
    s.ccnt[i] = 0u; s.cmn[i] = INT_MAX; s.cmx[i] = INT_MIN;
  }
  if (threadIdx.x < kMaxW) { m.touched[threadIdx.x] = 0; m.enter[threadIdx.x] = 0; }
  if (threadIdx.x == 0) { m.dropped = 0ull; m.n_late = 0ull; m.n_inplace = 0; m.oldest = 0; }
  __syncthreads();
  unsigned long long my_dropped = 0, my_late = 0;
  const int W = a.W;

  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int64_t p0 = item * a.span;
    const int64_t p1 = p0 + a.span < a.n ? p0 + a.span : a.n;
    int lo = -1;   // lowest fine row of the window (uniform); -1 = empty
    int clo = -1;  // lowest coarse row of the coarse ring
    int batch = 0;
    Raw cur, nxt;
    load_raw(a, cur, p0 + (int64_t)threadIdx.x * kPtsPerThread, p1);
    for (int64_t b0 = p0; b0 < p1; b0 += kBatch, ++batch) {
      // prefetch the next batch while this one is processed
      if (b0 + kBatch < p1) load_raw(a, nxt, b0 + kBatch + (int64_t)threadIdx.x * kPtsPerThread, p1);
      int G[kPtsPerThread], col[kPtsPerThread];
      unsigned pend = 0;
#pragma unroll
      for (int k = 0; k < kPtsPerThread; ++k) {
        G[k] = INT_MAX;
        col[k] = 0;
        if (k >= cur.n) continue;
        uint32_t ux, uy;
        bool in;
        if (a.narrow) {
          ux = (uint32_t)cur.x[k] - (uint32_t)a.x0_32;
          uy = (uint32_t)cur.y[k] - (uint32_t)a.y0_32;
          in = ux < a.ext_x && uy < a.ext_y;
        } else {
          const int64_t lx = (int64_t)cur.x[k] - a.x0, ly = (int64_t)cur.y[k] - a.y0;
          in = lx >= 0 && ly >= 0 && lx < (int64_t)a.ext_x && ly < (int64_t)a.ext_y;
          ux = (uint32_t)lx;
          uy = (uint32_t)ly;
        }
        if (!in) {
          ++my_dropped;
          continue;
        }
        const uint32_t tx = fdiv(ux, a.div_tile), ty = fdiv(uy, a.div_tile);
        const uint32_t cx = fdiv(ux - tx * a.tile_cm, a.div_cell);
        const uint32_t cy = fdiv(uy - ty * a.tile_cm, a.div_cell);
        G[k] = ((int)ty * a.tiles_x + (int)tx) * a.cells + (int)cy;
        col[k] = (int)cx;
        pend |= 1u << k;
      }
      // ---- common case (one barrier): every point of the block inside the window
      bool outside = false;
#pragma unroll
      for (int k = 0; k < kPtsPerThread; ++k)
        if (pend & (1u << k)) outside |= (lo < 0) || ((unsigned)(G[k] - lo) >= (unsigned)W);
      if (!__syncthreads_or(outside)) {
#pragma unroll
        for (int k = 0; k < kPtsPerThread; ++k) {
          if (!(pend & (1u << k))) continue;
          accumulate(s, m, a, G[k] & (W - 1), col[k], cur.z[k], cur.r[k], cur.g[k], cur.b[k]);
        }
      } else {
        // ---- general case: late points, window slides
        while (true) {
          if (lo >= 0) {
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k) {
              if (!(pend & (1u << k))) continue;
              if (G[k] < lo) {
                late_point(a, G[k], col[k], cur.z[k], cur.r[k], cur.g[k], cur.b[k]);
                ++my_late;
                pend &= ~(1u << k);
              } else if (G[k] < lo + W) {
                accumulate(s, m, a, G[k] & (W - 1), col[k], cur.z[k], cur.r[k], cur.g[k], cur.b[k]);
                pend &= ~(1u << k);
              }
            }
          }
          int mymin = INT_MAX, mymax = INT_MIN;
#pragma unroll
          for (int k = 0; k < kPtsPerThread; ++k)
            if (pend & (1u << k)) { mymin = min(mymin, G[k]); mymax = max(mymax, G[k]); }
          int mn, mx;
          block_minmax(mymin, mymax, m, mn, mx);
          if (mn == INT_MAX) break;
          // Every pending point lies at or above lo + W.  Slide as little as possible:
          // keep the window as low as it can be while covering all pending rows (the
          // lower rows of a strip whose first points are already here come later), or,
          // when the pending rows span more than W rows, start at the lowest of them.
          int nlo = (mx - mn < W) ? mx - W + 1 : mn;
          if (lo >= 0 && nlo < lo + 1) nlo = lo + 1;
          if (lo < 0) nlo = mn;
          if (lo >= 0) {
            const int hi = (nlo < lo + W) ? nlo : lo + W;
            evict_rows(a, s, m, lo, hi, clo);
          }
          if (threadIdx.x == 0) {
            // rows [max(lo + W, nlo), nlo + W) enter; rows kept in the window keep their age
            const int first_new = (lo >= 0 && lo + W > nlo) ? lo + W : nlo;
            for (int G2 = first_new; G2 < nlo + W; ++G2) m.enter[G2 & (W - 1)] = batch;
            int o = INT_MAX;
            for (int k = 0; k < W; ++k) o = min(o, m.enter[k]);
            m.oldest = o;
          }
          lo = nlo;
          __syncthreads();
        }
      }
      // ---- residency bound: before any row can have absorbed 65536 points the
      // window is flushed in place (its rows stay in the window; their next flush
      // merges), so strip-ordered input never produces late points
      if (lo >= 0 && batch - m.oldest + 1 >= kResidLimitBatches) {
        __syncthreads();
        evict_rows(a, s, m, lo, lo + W, clo);
        if (threadIdx.x == 0) {
          for (int k = 0; k < W; ++k) m.enter[k] = batch + 1;
          m.oldest = batch + 1;
          ++m.n_inplace;
        }
        __syncthreads();
      }
      cur = nxt;
    }
    // ---- end of the span: flush everything
    __syncthreads();
    if (lo >= 0) evict_rows(a, s, m, lo, lo + W, clo);
    if (a.has_coarse && clo >= 0) {
      coarse_evict(a, s, clo, clo + kCW);
      __syncthreads();
    }
  }
  {
    const unsigned lt = __reduce_add_sync(0xffffffffu, (unsigned)my_late);
    if ((threadIdx.x & 31) == 0 && lt) atomicAdd((unsigned long long*)&m.n_late, (unsigned long long)lt);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (m.n_late) atomicAdd(&g_bin_stats[0], m.n_late);
      if (m.n_inplace) atomicAdd(&g_bin_stats[3], (unsigned long long)m.n_inplace);
    }
  }
  if (a.dropped) {
    my_dropped = __reduce_add_sync(0xffffffffu, (unsigned)my_dropped);
    if ((threadIdx.x & 31) == 0 && my_dropped) atomicAdd((unsigned long long*)&m.dropped, my_dropped);
    __syncthreads();
    if (threadIdx.x == 0 && m.dropped) atomicAdd((unsigned long long*)a.dropped, m.dropped);
  }
}

// Prologue: clear row states and the dropped counter; give the coarse level its
// empty sentinels (it is only ever merged into with atomics).
__global__ void k_bin_prologue(BinArgs a, int64_t n_coarse) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_rows; i += stride)
    a.row_state[i] = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_coarse; i += stride) {
    a.ccount[i] = 0u; a.czsum[i] = 0; a.czmin[i] = INT_MAX; a.czmax[i] = INT_MIN;
    a.crsum[i] = 0ull; a.cgsum[i] = 0ull; a.cbsum[i] = 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.dropped) *a.dropped = 0ull;
}

// Epilogue: rows that no point reached get the empty sentinels.
__global__ void k_bin_finalize(BinArgs a) {
  for (int64_t G = blockIdx.x; G < a.n_rows; G += gridDim.x) {
    if (a.row_state[G] != 0u) continue;
    const int64_t base = G * a.cells;
    for (int c = threadIdx.x; c < a.cells; c += blockDim.x) store_empty_cell(a, base + c);
  }
}

}  // namespace

// Validates and builds the kernel arguments (shared with the fixed-scratch entry).
ls_status bin_prepare(const ls_points* pts, const ls_region* region, const ls_bins* levels,
                      int32_t n_levels, uint64_t* dropped, BinArgs* out, size_t* smem, int64_t* n_coarse);

ls_status bin_prepare(const ls_points* pts, const ls_region* region, const ls_bins* levels,
                      int32_t n_levels, uint64_t* dropped, BinArgs* out, size_t* smem, int64_t* n_coarse) {
  if (!pts || !region || !levels || n_levels < 1 || n_levels > 2) return LS_ERR_INVALID_ARG;
  if (pts->n < 0) return LS_ERR_INVALID_ARG;
  if (pts->n > 0 && (!pts->x || !pts->y || !pts->z || !pts->r || !pts->g || !pts->b))
    return LS_ERR_INVALID_ARG;
  if (region->tile_cm <= 0 || region->tiles_x <= 0 || region->tiles_y <= 0) return LS_ERR_INVALID_ARG;
  const int64_t ext_x = (int64_t)region->tiles_x * region->tile_cm;
  const int64_t ext_y = (int64_t)region->tiles_y * region->tile_cm;
  if (ext_x >= (int64_t(1) << 31) || ext_y >= (int64_t(1) << 31)) return LS_ERR_INVALID_ARG;
  const ls_bins& L0 = levels[0];
  if (L0.cells <= 0 || L0.cells > 4096 || region->tile_cm % L0.cells) return LS_ERR_INVALID_ARG;
  if (!L0.count || !L0.zsum || !L0.zmin || !L0.zmax || !L0.rsum || !L0.gsum || !L0.bsum)
    return LS_ERR_INVALID_ARG;
  const int64_t T = (int64_t)region->tiles_x * region->tiles_y;
  const int64_t n_rows = T * L0.cells;
  if (n_rows >= (int64_t(1) << 31) - 256) return LS_ERR_INVALID_ARG;
  BinArgs a = {};
  a.x = pts->x; a.y = pts->y; a.z = pts->z; a.r = pts->r; a.g = pts->g; a.b = pts->b;
  a.n = pts->n;
  a.x0 = region->x0_cm; a.y0 = region->y0_cm;
  a.ext_x = (uint32_t)ext_x; a.ext_y = (uint32_t)ext_y;
  a.tile_cm = (uint32_t)region->tile_cm;
  a.cell_cm = (uint32_t)(region->tile_cm / L0.cells);
  a.div_tile = make_fastdiv(a.tile_cm);
  a.div_cell = make_fastdiv(a.cell_cm);
  a.tiles_x = region->tiles_x;
  a.cells = L0.cells;
  a.n_rows = (int32_t)n_rows;
  a.count = L0.count; a.zsum = L0.zsum; a.zmin = L0.zmin; a.zmax = L0.zmax;
  a.rsum = L0.rsum; a.gsum = L0.gsum; a.bsum = L0.bsum;
  a.dropped = dropped;
  a.f = 1;
  a.ccells = 1;
  a.div_f = make_fastdiv(1);
  *n_coarse = 0;
  if (n_levels == 2) {
    const ls_bins& L1 = levels[1];
    if (L1.cells <= 0 || L0.cells % L1.cells) return LS_ERR_INVALID_ARG;
    if (!L1.count || !L1.zsum || !L1.zmin || !L1.zmax || !L1.rsum || !L1.gsum || !L1.bsum)
      return LS_ERR_INVALID_ARG;
    a.has_coarse = 1;
    a.ccells = L1.cells;
    a.f = L0.cells / L1.cells;
    a.div_f = make_fastdiv((uint32_t)a.f);
    a.ccount = L1.count; a.czsum = L1.zsum; a.czmin = L1.zmin; a.czmax = L1.zmax;
    a.crsum = L1.rsum; a.cgsum = L1.gsum; a.cbsum = L1.bsum;
    *n_coarse = T * L1.cells * L1.cells;
  }
  a.gs = (a.f % 2) ? a.f : a.f + 1;
  a.rstride = (a.cells / a.f) * a.gs;
  // window rows: the largest power of two <= 8 whose ring fits in ~196 KB of shared memory
  const size_t budget = 196 * 1024;
  int W = 8;
  const int CC = a.has_coarse ? kCW * a.ccells : 0;
  while (W > 1 && smem_bytes(W * a.rstride, CC) > budget) W >>= 1;
  if (W > a.cells) {
    W = 1;
    while (W * 2 <= a.cells) W *= 2;
  }
  if (smem_bytes(W * a.rstride, CC) > budget) return LS_ERR_UNSUPPORTED;
  a.W = W;
  *smem = smem_bytes(W * a.rstride, CC);
  // vector loads need 16-byte aligned int32 arrays and 8-byte aligned uint16 arrays
  a.narrow = region->x0_cm >= INT32_MIN && region->x0_cm <= INT32_MAX && region->y0_cm >= INT32_MIN &&
             region->y0_cm <= INT32_MAX;
  a.x0_32 = a.narrow ? (int32_t)region->x0_cm : 0;
  a.y0_32 = a.narrow ? (int32_t)region->y0_cm : 0;
  a.vec = (((uintptr_t)a.x | (uintptr_t)a.y | (uintptr_t)a.z) % 16 == 0) &&
          (((uintptr_t)a.r | (uintptr_t)a.g | (uintptr_t)a.b) % 8 == 0);
  // spans: about 4 per CTA, multiples of the batch size
  const int64_t grid = kSmCount;
  int64_t span = (a.n + grid * 4 - 1) / (grid * 4);
  span = (span + kBatch - 1) / kBatch * kBatch;
  if (span < kBatch) span = kBatch;
  a.span = span;
  a.n_items = (a.n + span - 1) / span;
  *out = a;
  return LS_OK;
}

ls_status bin_launch(BinArgs a, size_t smem, int64_t n_coarse, cudaStream_t stream) {
  static bool attr_set[64] = {};
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    LS_CUDA_TRY(cudaFuncSetAttribute(k_bin_main, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     210 * 1024));
    attr_set[dev] = true;
  }
  const int64_t work = a.n_rows > n_coarse ? a.n_rows : n_coarse;
  k_bin_prologue<<<grid_cap((work + 255) / 256, kSmCount * 8), 256, 0, stream>>>(a, n_coarse);
  if (a.n_items > 0) {
    k_bin_main<<<grid_cap(a.n_items, kSmCount), kBinThreads, smem, stream>>>(a);
  }
  k_bin_finalize<<<grid_cap(a.n_rows, kSmCount * 16), 128, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace ls

extern "C" ls_status ls_bin_stats(uint64_t* out, int32_t reset) {
  if (!out) return LS_ERR_INVALID_ARG;
  if (cudaMemcpyFromSymbol(out, ls::g_bin_stats, 4 * sizeof(uint64_t)) != cudaSuccess) return LS_ERR_CUDA;
  if (reset) {
    const uint64_t z[4] = {0, 0, 0, 0};
    if (cudaMemcpyToSymbol(ls::g_bin_stats, z, sizeof(z)) != cudaSuccess) return LS_ERR_CUDA;
  }
  return LS_OK;
}

extern "C" ls_status ls_bin_points(const ls_points* pts, const ls_region* region, const ls_bins* levels,
                                   int32_t n_levels, uint64_t* dropped, ls_stream_t stream) {
  ls::BinArgs a;
  size_t smem = 0;
  int64_t n_coarse = 0;
  ls_status st = ls::bin_prepare(pts, region, levels, n_levels, dropped, &a, &smem, &n_coarse);
  if (st != LS_OK) return st;
  a.row_state = static_cast<uint32_t*>(ls::workspace(ls::kWsBinRows, (size_t)a.n_rows * 4));
  if (!a.row_state) return LS_ERR_NO_MEMORY;
  return ls::bin_launch(a, smem, n_coarse, reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------------
// Variant of ls_bin_points that allocates nothing.  Its per-row claim states live in
// a fixed array compiled into the library instead of the growable workspace, for
// callers that must not allocate device memory while binning, e.g. an interactive
// viewer that streams full-resolution tiles in between frames (cudaMalloc and
// cudaFree can synchronise the device and stall a frame) or an application whose
// device memory is fully reserved by its own allocator.
// ---------------------------------------------------------------------------------
namespace ls {
namespace {
constexpr int64_t kFixedBinRows = int64_t(1) << 20;  // 4 MiB of row states
static __device__ __align__(256) uint32_t g_bin_rows_fixed[kFixedBinRows];
std::mutex g_fixed_mu;
uint32_t* g_fixed_ptr[64] = {};
}  // namespace
}  // namespace ls

extern "C" ls_status ls_bin_points_fixed_scratch(const ls_points* pts, const ls_region* region,
                                                 const ls_bins* levels, int32_t n_levels, uint64_t* dropped,
                                                 ls_stream_t stream) {
  ls::BinArgs a;
  size_t smem = 0;
  int64_t n_coarse = 0;
  ls_status st = ls::bin_prepare(pts, region, levels, n_levels, dropped, &a, &smem, &n_coarse);
  if (st != LS_OK) return st;
  if ((int64_t)a.n_rows > ls::kFixedBinRows) return LS_ERR_UNSUPPORTED;  // tiles * cells rows over 2^20
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ERR_CUDA;
  if (dev < 0 || dev >= 64) return LS_ERR_UNSUPPORTED;
  uint32_t* rows = nullptr;
  {
    // once per device, with that device current: the device address of the array
    // (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(ls::g_fixed_mu);
    if (!ls::g_fixed_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, ls::g_bin_rows_fixed) != cudaSuccess || !p) return LS_ERR_CUDA;
      ls::g_fixed_ptr[dev] = static_cast<uint32_t*>(p);
    }
    rows = ls::g_fixed_ptr[dev];
  }
  a.row_state = rows;  // cleared by the prologue kernel of every call
  return ls::bin_launch(a, smem, n_coarse, reinterpret_cast<cudaStream_t>(stream));
}
