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
//    (eight 32-bit words per cell: count, R, G, B, low and high halves of z, z-min,
//    z-max) with shared atomics.  When a point lands above the window, the window
//    slides and the rows that leave are flushed.
//  * Flush protocol per row (per-row state word in scratch: 0 free, 1 being
//    written, 2 written): the first CTA to flush a row claims it (0 -> 1), writes
//    all its cells with plain coalesced stores (empty cells get the sentinels),
//    fences and publishes 2.  Any later contribution to that row (another CTA's
//    part of a strip, or a late point) merges with global atomics after seeing 2.
//    Late points (rows already below the window) are taken one row at a time by
//    their whole warp: lane 0 claims or waits, the warp writes the row's sentinels.
//    So every output byte is written once by a plain store in the common case and
//    no memset pass is needed.  Rows that nobody touched get sentinels in a final
//    pass.  Result is exact for ANY point order; only speed depends on the order.
//  * Coarse level (e.g. 64x64 from 640x640): reduced exactly from the fine cells
//    while they are flushed, accumulated in a small shared ring of coarse rows and
//    merged with global atomics into the (L2-resident) coarse arrays, which a
//    prologue kernel initialises.
//  * The 32-bit sums in shared memory cannot overflow: no ring row absorbs more than
//    65536 points (65536 * 65535 < 2^32).  The rows are counted when the fullest one
//    could first reach that bound, and the window is flushed in place only when a
//    row is near it.
#include <algorithm>
#include <climits>
#include <mutex>

#include "ls_internal.cuh"

namespace ls {
namespace {

constexpr int kBinThreads = 1024;
constexpr int kPtsPerThread = 4;
constexpr int kBatch = kBinThreads * kPtsPerThread;  // 4096 points per batch
constexpr int kRowLimit = 65536;                      // residency bound: points per ring row
constexpr int kResidLimitBatches = kRowLimit / kBatch;  // batches before the first row check
constexpr int kMaxW = 64;
constexpr int kCW = 4;  // coarse ring rows
constexpr int kMaxWFlush = 8;  // window rows (W <= 8)
constexpr int kBinSmemAttr = 224 * 1024;  // dynamic shared memory allowed (budget + margin)

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
  FastDiv31 d31_tile, d31_cell;  // the same divisions for numerators < 2^31 (cell_cm >= 2)
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
  uint32_t* row_state;    // [n_rows] claim states, then the span counter
  uint64_t* dropped;
  int64_t span;
  int64_t n_items;
  int vec;
  int narrow;            // x0 and y0 fit int32: 32-bit region-local coordinates
  int32_t x0_32, y0_32;
  // shared-memory row layout: the f fine cells of a coarse cell occupy gs >= f slots,
  // rows are rstride slots apart; the coarse partials split a coarse cell's f columns
  // at fh (gs and fh chosen against bank conflicts, see bin_coarse_layout)
  int32_t gs, rstride, fh;
  int32_t accumulate;  // add into the existing bins: every flushed row merges with atomics
  int32_t vec_out;     // rows of 4-cell groups (16-byte shared and global alignment): 128-bit flush
  int32_t pf_dist;     // batches prefetched into L2 ahead of the loads (launch shape, 1..4)
};

// shared-memory layout (dynamic).  Every fine accumulator is a 32-bit word (32-bit
// shared atomics are several times cheaper than 64-bit ones): z is split into its low
// 16 bits (unsigned) and its high bits (signed), zsum = 65536 * sum(hi) + sum(lo),
// both sums exact while a cell absorbs at most 65536 points.
struct Smem {
  uint32_t fa, fs;  // shared address of cnt[0]; byte stride between the eight fine arrays
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
  // per-(row, coarse cell) partials of a flush: [8][SC], SC = W * ccells (32-bit)
  unsigned* sp;
};

struct Meta {
  int touched[kMaxW];
  unsigned rowc[kMaxW];  // points per ring row (scratch of the residency check)
  int mode[kMaxW];   // 0 none, 1 store, 2 merge
  int ckey[kMaxW];   // coarse row of each row being flushed
  int red[kBinThreads / 32];
  int redx[kBinThreads / 32];
  int bcast, bcastx;
  int clo_old, clo_new;  // coarse ring scratch of evict_rows (not shared with block_min)
  int n_inplace;
  int next_check;  // batch after whose accumulation the rows are counted again (per span)
  long long item;  // span taken from the counter
  // rows this CTA claimed and stored in its last flush, published (state 2) later
  int pend_row[kMaxW];  // -1: none
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
  s.sp = reinterpret_cast<unsigned*>(s.cmx + CC);
  s.fa = (uint32_t)__cvta_generic_to_shared(s.cnt);
  s.fs = (uint32_t)WC * 4u;
  return s;
}

// fine ring (8 words per cell), coarse ring (4 x 64-bit + 3 x 32-bit per cell) and
// the flush partials (8 words per (row, coarse cell))
__host__ __device__ constexpr size_t smem_bytes(int WC, int CC, int SC) {
  return (size_t)WC * (8 * 4) + (size_t)CC * (4 * 8 + 3 * 4) + (size_t)SC * (8 * 4);
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

// Store ring slot `slot` as fine row `base / cells` (every cell, empty ones as the
// sentinels) and reset it, four cells per thread with 128-bit shared and global
// accesses (the row's cells are contiguous: no padding; a.vec_out checked the
// alignment).  Threads t0, t0 + nt, ... take part.
__device__ __forceinline__ void store_row_vec(const BinArgs& a, Smem& s, int slot, int64_t base, int t0, int nt) {
  const int o = slot * a.rstride;
  const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
  for (int q = t0; q < a.cells / 4; q += nt) {
    const int si = o + 4 * q;
    const int64_t o4 = base + 4 * q;
    // one array at a time: load the 4 cells, store them, reset them
    {
      uint4* p = reinterpret_cast<uint4*>(s.cnt + si);
      *reinterpret_cast<uint4*>(a.count + o4) = *p;
      *p = z4;
    }
    {
      uint4* pl = reinterpret_cast<uint4*>(s.zlo + si);
      int4* ph = reinterpret_cast<int4*>(s.zhi + si);
      const uint4 zl = *pl;
      const int4 zh = *ph;
      *reinterpret_cast<longlong2*>(a.zsum + o4) =
          make_longlong2((long long)zh.x * 65536 + (long long)zl.x, (long long)zh.y * 65536 + (long long)zl.y);
      *reinterpret_cast<longlong2*>(a.zsum + o4 + 2) =
          make_longlong2((long long)zh.z * 65536 + (long long)zl.z, (long long)zh.w * 65536 + (long long)zl.w);
      *pl = z4;
      *reinterpret_cast<uint4*>(ph) = z4;
    }
    {
      int4* p = reinterpret_cast<int4*>(s.mn + si);
      *reinterpret_cast<int4*>(a.zmin + o4) = *p;
      *p = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
    }
    {
      int4* p = reinterpret_cast<int4*>(s.mx + si);
      *reinterpret_cast<int4*>(a.zmax + o4) = *p;
      *p = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
    }
    unsigned* const src[3] = {s.rs, s.gs, s.bs};
    uint64_t* const dst[3] = {a.rsum, a.gsum, a.bsum};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint4* p = reinterpret_cast<uint4*>(src[j] + si);
      const uint4 v = *p;
      *reinterpret_cast<ulonglong2*>(dst[j] + o4) = make_ulonglong2(v.x, v.y);
      *reinterpret_cast<ulonglong2*>(dst[j] + o4 + 2) = make_ulonglong2(v.z, v.w);
      *p = z4;
    }
  }
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
  const int limit = spin_limit();
  while (ld_acquire(state) != 2u) {
    if (++it > limit) {
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

// shared-memory reductions at a 32-bit shared address, without a returned value (no
// scoreboard wait)
__device__ __forceinline__ void red_add_u(uint32_t p, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_s(uint32_t p, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_min_s(uint32_t p, int v) {
  asm volatile("red.shared.min.s32 [%0], %1;" ::"r"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_max_s(uint32_t p, int v) {
  asm volatile("red.shared.max.s32 [%0], %1;" ::"r"(p), "r"(v) : "memory");
}

// shared slot of fine column col in ring slot `slot` (padded layout, see BinArgs)
__device__ __forceinline__ int sidx(const BinArgs& a, int slot, int col) {
  if (a.gs == a.f) return slot * a.rstride + col;  // groups without padding
  const int cg = (int)fdiv((uint32_t)col, a.div_f);
  return slot * a.rstride + cg * a.gs + (col - cg * a.f);
}

// Rows below this CTA's window (late points), one row at a time for the whole warp
// (called by all 32 lanes, converged): lane 0 claims the row if nobody has written it
// yet, and then the warp writes its empty cells and lane 0 publishes it; when another
// claim holds the row, lane 0 waits (bounded) until it is written.  When accumulating,
// the row already holds valid bins.  Afterwards the late point merges with atomics.
__device__ void late_row_ready(const BinArgs& a, int G) {
  if (a.accumulate) return;
  const int lane = threadIdx.x & 31;
  uint32_t* st = &a.row_state[G];
  int act = 0;  // 0 written, 1 claimed here, 2 being written by another claim
  if (lane == 0 && ld_acquire(st) != 2u) act = atomicCAS(st, 0u, 1u) == 0u ? 1 : 2;
  act = __shfl_sync(0xffffffffu, act, 0);
  if (act == 1) {
    const int64_t base = (int64_t)G * a.cells;
    for (int c = lane; c < a.cells; c += 32) store_empty_cell(a, base + c);
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      atomicExch(st, 2u);
    }
  } else if (act == 2) {
    if (lane == 0) wait_written(st);
  }
  __syncwarp();
}

__device__ __forceinline__ void late_merge(const BinArgs& a, int G, int col, int z, uint32_t r, uint32_t g,
                                           uint32_t b) {
  merge_fine(a, (int64_t)G * a.cells + col, 1u, z, z, z, r, g, b);
  if (a.has_coarse) {
    const int64_t o = (int64_t)coarse_row_of(a, G) * a.ccells + (int)fdiv((uint32_t)col, a.div_f);
    merge_coarse(a, o, 1u, z, z, z, r, g, b);
  }
}

// Largest point count over the W ring rows (every thread gets it; block-wide, with
// barriers before and after).  Thread t sums the count words of row t / (threads / W).
__device__ unsigned row_count_max(const BinArgs& a, const Smem& s, Meta& m) {
  const int W = a.W;
  const int per = (int)blockDim.x / W;  // threads per row (W divides 1024)
  const int r = (int)threadIdx.x / per, t = (int)threadIdx.x - r * per;
  __syncthreads();  // the accumulation before is complete
  if (threadIdx.x < W) m.rowc[threadIdx.x] = 0u;
  __syncthreads();
  unsigned c = 0;
  for (int i = t; i < a.rstride; i += per) c += s.cnt[r * a.rstride + i];  // padding slots hold 0
  c = __reduce_add_sync(0xffffffffu, c);  // per divides into whole warps (per >= 128)
  if ((threadIdx.x & 31) == 0) atomicAdd(&m.rowc[r], c);
  __syncthreads();
  unsigned mx = 0;
  for (int k = 0; k < W; ++k) mx = max(mx, m.rowc[k]);
  __syncthreads();  // m.rowc is read before anyone reuses it
  return mx;
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
__device__ void coarse_evict(const BinArgs& a, Smem& s, int ca, int cb, int nthreads) {
  const int n = (cb - ca) * a.ccells;
  for (int i = threadIdx.x; i < n; i += nthreads) {
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

// Publish (state 2) the rows this CTA stored in its previous flush.  Their stores
// precede at least one block barrier; the fence orders them before the state store.
// Slot t of the pending list belongs to thread t alone.
__device__ __forceinline__ void publish_pending(const BinArgs& a, Meta& m) {
  if (threadIdx.x < kMaxW) {
    const int G = m.pend_row[threadIdx.x];
    if (G >= 0) {
      __threadfence();
      atomicExch(&a.row_state[G], 2u);
      m.pend_row[threadIdx.x] = -1;
    }
  }
}

// Partial coarse cell of one ring row.  32-bit fields suffice for any set of cells of
// one row: the residency bound keeps a row at or below 65536 points, so count, colour
// sums and the sum of the low z halves stay below 2^32 and the sum of the high z
// halves inside int32.  Sums over several rows are only formed in the 64-bit coarse
// ring and arrays.
struct CAcc {
  unsigned cnt, zlo;
  int zhi, mn, mx;
  unsigned r, g, b;
};

__device__ __forceinline__ void cacc_clear(CAcc& v) {
  v.cnt = 0u; v.zlo = 0u; v.zhi = 0; v.mn = INT_MAX; v.mx = INT_MIN; v.r = 0u; v.g = 0u; v.b = 0u;
}

// add fine cell si (an empty cell adds nothing: zero sums, min/max sentinels)
__device__ __forceinline__ void cacc_cell(CAcc& v, const Smem& s, int si) {
  v.cnt += s.cnt[si];
  v.zlo += s.zlo[si];
  v.zhi += s.zhi[si];
  v.mn = min(v.mn, s.mn[si]);
  v.mx = max(v.mx, s.mx[si]);
  v.r += s.rs[si];
  v.g += s.gs[si];
  v.b += s.bs[si];
}

// v += the partner lane's (lane ^ 1) partial
__device__ __forceinline__ void cacc_pair(CAcc& v) {
  v.cnt += __shfl_xor_sync(0xffffffffu, v.cnt, 1);
  v.zlo += __shfl_xor_sync(0xffffffffu, v.zlo, 1);
  v.zhi += __shfl_xor_sync(0xffffffffu, v.zhi, 1);
  v.mn = min(v.mn, __shfl_xor_sync(0xffffffffu, v.mn, 1));
  v.mx = max(v.mx, __shfl_xor_sync(0xffffffffu, v.mx, 1));
  v.r += __shfl_xor_sync(0xffffffffu, v.r, 1);
  v.g += __shfl_xor_sync(0xffffffffu, v.g, 1);
  v.b += __shfl_xor_sync(0xffffffffu, v.b, 1);
}

// Partial of coarse cell (key, c) into the coarse ring (plain read-modify-write: the
// caller is its only writer in this pass) or, for a coarse row outside the ring,
// into the global coarse arrays with atomics.
__device__ __forceinline__ void cacc_emit(const BinArgs& a, Smem& s, int key, int c, int clo, const CAcc& v) {
  if (!v.cnt) return;
  const long long zs = (long long)v.zhi * 65536 + (long long)v.zlo;
  if (key >= clo && key < clo + kCW) {
    const int ci = (key % kCW) * a.ccells + c;
    s.ccnt[ci] += v.cnt;
    s.czs[ci] += (unsigned long long)zs;
    s.cmn[ci] = min(s.cmn[ci], v.mn);
    s.cmx[ci] = max(s.cmx[ci], v.mx);
    s.crs[ci] += v.r;
    s.cgs[ci] += v.g;
    s.cbs[ci] += v.b;
  } else {
    merge_coarse(a, (int64_t)key * a.ccells + c, v.cnt, zs, v.mn, v.mx, v.r, v.g, v.b);
  }
}

constexpr int kCoarseThreads = 64;  // warps 0-1 combine the coarse partials of a flush

// Coarse reduction of a flush, step 1 (all threads): lane pair (2c, 2c + 1) of fine
// row rr sums coarse cell c's f fine columns of that row (split at fh, combined with
// one shuffle) and the even lane stores the partial in sp[.][rr * ccells + c].
__device__ void coarse_partials(const BinArgs& a, Smem& s, const Meta& m, int ra, int nr) {
  const int W = a.W;
  const int SC = W * a.ccells;
  const int n = 2 * SC;
  const int nloop = (n + 31) & ~31;  // whole warps: every lane takes part in the shuffle
  for (int e = threadIdx.x; e < nloop; e += blockDim.x) {
    const int h = e & 1, pc = e >> 1;  // pc = rr * ccells + c
    const int rr = pc / a.ccells, c = pc - rr * a.ccells;
    const bool live = e < n && rr < nr && m.mode[rr] != 0;
    CAcc v;
    cacc_clear(v);
    if (live) {
      const int base = ((ra + rr) & (W - 1)) * a.rstride + c * a.gs;
      const int k1 = h ? a.f : a.fh;
      for (int k = h ? a.fh : 0; k < k1; ++k) cacc_cell(v, s, base + k);
    }
    cacc_pair(v);
    if (h == 0 && live) {
      s.sp[0 * SC + pc] = v.cnt;
      s.sp[1 * SC + pc] = v.zlo;
      s.sp[2 * SC + pc] = (unsigned)v.zhi;
      s.sp[3 * SC + pc] = (unsigned)v.mn;
      s.sp[4 * SC + pc] = (unsigned)v.mx;
      s.sp[5 * SC + pc] = v.r;
      s.sp[6 * SC + pc] = v.g;
      s.sp[7 * SC + pc] = v.b;
    }
  }
}

// Step 2 (threads < kCoarseThreads): one thread per coarse column adds the touched
// rows' partials, one row at a time, to their coarse cells (the 64-bit coarse ring,
// or the global coarse arrays for a coarse row outside it).
__device__ void coarse_combine(const BinArgs& a, Smem& s, const Meta& m, int nr, int clo) {
  const int SC = a.W * a.ccells;
  for (int c = threadIdx.x; c < a.ccells; c += kCoarseThreads) {
#pragma unroll 1
    for (int rr = 0; rr < nr; ++rr) {
      if (m.mode[rr] == 0) continue;
      const int pc = rr * a.ccells + c;
      CAcc v;
      v.cnt = s.sp[0 * SC + pc];
      v.zlo = s.sp[1 * SC + pc];
      v.zhi = (int)s.sp[2 * SC + pc];
      v.mn = (int)s.sp[3 * SC + pc];
      v.mx = (int)s.sp[4 * SC + pc];
      v.r = s.sp[5 * SC + pc];
      v.g = s.sp[6 * SC + pc];
      v.b = s.sp[7 * SC + pc];
      cacc_emit(a, s, m.ckey[rr], c, clo, v);
    }
  }
}

// Reset the cells of ring slot `slot` to empty, all threads, coalesced.
__device__ __forceinline__ void reset_row(const BinArgs& a, Smem& s, int slot) {
  const int o = slot * a.rstride;
  for (int i = threadIdx.x; i < a.rstride; i += blockDim.x) reset_cell(s, o + i);
}

// Evict fine rows [ra, rb) (rb - ra <= W, all inside the ring).  The caller has
// synchronised the block after the last accumulation.
//
// Claimed rows are normally published one flush later (publish_pending at the start of
// the next flush or of the next pass through the general path), so their stores drain
// while the CTA streams on instead of stalling on a fence.  Deadlock freedom: a CTA
// only ever waits on another row while it holds no unpublished claim (pending rows are
// published before any wait; a flush that must merge publishes its own rows first).
__device__ void evict_rows(const BinArgs& a, Smem& s, Meta& m, int ra, int rb, int& clo) {
  const int nr = rb - ra;
  if (nr <= 0) return;
  const int W = a.W;
  publish_pending(a, m);
  // claim (0 -> 1) without waiting
  bool merge_row = false;
  if (threadIdx.x < nr) {
    const int G = ra + threadIdx.x;
    const int slot = G & (W - 1);
    int mode = 0;
    if (m.touched[slot]) {
      mode = (!a.accumulate && atomicCAS(&a.row_state[G], 0u, 1u) == 0u) ? 1 : 2;
      m.touched[slot] = 0;
    }
    m.mode[threadIdx.x] = mode;
    m.ckey[threadIdx.x] = a.has_coarse ? coarse_row_of(a, G) : 0;
    merge_row = mode == 2;
  }
  // coarse ring: make room for the coarse rows of [ra, rb)
  if (a.has_coarse && threadIdx.x == 0) {
    const int ca = coarse_row_of(a, ra), cb = coarse_row_of(a, rb - 1);
    const int c0 = clo < 0 ? ca : clo;
    m.clo_old = c0;
    m.clo_new = (cb >= c0 + kCW) ? cb - kCW + 1 : c0;
  }
  const bool any_merge = __syncthreads_or(merge_row);
  if (a.has_coarse) {
    // coarse ring rows leaving and per-row partials (independent data, all threads)
    const int old_clo = m.clo_old, new_clo = m.clo_new;
    clo = new_clo;
    if (new_clo > old_clo)
      coarse_evict(a, s, old_clo, new_clo < old_clo + kCW ? new_clo : old_clo + kCW, blockDim.x);
    coarse_partials(a, s, m, ra, nr);
    __syncthreads();
  }
  // warps 0-1 combine the coarse partials while the others store the fine rows claimed
  // here (every cell, empty ones as sentinels) and reset their cells
  const int st0 = a.has_coarse ? kCoarseThreads : 0;
  if (a.has_coarse && threadIdx.x < kCoarseThreads) coarse_combine(a, s, m, nr, clo);
  if ((int)threadIdx.x >= st0) {
    const int nst = blockDim.x - st0;
    for (int rr = 0; rr < nr; ++rr) {
      if (m.mode[rr] != 1) continue;
      const int G = ra + rr;
      const int slot = G & (W - 1);
      const int64_t base = (int64_t)G * a.cells;

      for (int c = threadIdx.x - st0; c < a.cells; c += nst) {
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
  }
  if (!any_merge) {
    if (threadIdx.x < nr && m.mode[threadIdx.x] == 1) m.pend_row[threadIdx.x] = ra + threadIdx.x;
  } else {
    // publish this flush's rows, then wait for rows another claim holds, then merge
    __syncthreads();
    if (threadIdx.x < nr) {
      const int G = ra + threadIdx.x;
      if (m.mode[threadIdx.x] == 1) {
        __threadfence();
        atomicExch(&a.row_state[G], 2u);
      } else if (m.mode[threadIdx.x] == 2 && !a.accumulate) {
        wait_written(&a.row_state[G]);
      }
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
      if (m.mode[rr] != 2) continue;
      const int G = ra + rr;
      const int slot = G & (W - 1);
      const int64_t base = (int64_t)G * a.cells;
      for (int c = threadIdx.x; c < a.cells; c += blockDim.x) {
        const int si = sidx(a, slot, c);
        const Cell fc = read_cell(s, si);
        if (fc.cnt) merge_fine(a, base + c, fc.cnt, fc.zsum, fc.zmin, fc.zmax, fc.r, fc.g, fc.b);
      }
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr)
      if (m.mode[rr] == 2) reset_row(a, s, (ra + rr) & (W - 1));
  }
  __syncthreads();
}

// Raw points of one thread's slot of a batch (kPtsPerThread consecutive points).
struct Raw {
  int x[kPtsPerThread], y[kPtsPerThread], z[kPtsPerThread];
  // colours stay packed as loaded, two 16-bit values per word
  uint32_t r[kPtsPerThread / 2], g[kPtsPerThread / 2], b[kPtsPerThread / 2];
  int n;
};

__device__ __forceinline__ uint32_t half16(const uint32_t* w, int k) {
  return (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xffffu);
}

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
    v.r[0] = vr.x; v.r[1] = vr.y;
    v.g[0] = vg.x; v.g[1] = vg.y;
    v.b[0] = vb.x; v.b[1] = vb.y;
  } else {
#pragma unroll
    for (int k = 0; k < kPtsPerThread / 2; ++k) v.r[k] = v.g[k] = v.b[k] = 0u;
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
      if (k < v.n) {
        v.x[k] = a.x[i0 + k]; v.y[k] = a.y[i0 + k]; v.z[k] = a.z[i0 + k];
        const int sh = (k & 1) * 16;
        v.r[k >> 1] |= (uint32_t)a.r[i0 + k] << sh;
        v.g[k >> 1] |= (uint32_t)a.g[i0 + k] << sh;
        v.b[k >> 1] |= (uint32_t)a.b[i0 + k] << sh;
      } else {
        v.x[k] = v.y[k] = v.z[k] = 0;
      }
    }
  }
}

// Prefetch into L2 of the point records [i0, min(i0 + kBatch, p1)): one 128-byte line
// per thread (x, y, z: 128 lines each, r, g, b: 64 each for a full batch), issued
// without waiting.
constexpr int kPfLines = kBatch * 4 / 128 * 3 + kBatch * 2 / 128 * 3;
static_assert(kPfLines <= kBinThreads, "one prefetch line per thread");
__device__ __forceinline__ void prefetch_batch(const BinArgs& a, int64_t i0, int64_t p1) {
  if (i0 >= p1 || threadIdx.x >= kPfLines) return;
  const int64_t cnt = (p1 - i0) < kBatch ? (p1 - i0) : kBatch;
  constexpr int l4 = kBatch * 4 / 128, l2 = kBatch * 2 / 128;
  const int t = threadIdx.x;
  const char* p;
  int64_t off, bytes;
  if (t < 3 * l4) {
    const int arr = t / l4;
    p = reinterpret_cast<const char*>(arr == 0 ? a.x : arr == 1 ? a.y : a.z);
    off = (int64_t)(t - arr * l4) * 128;
    bytes = cnt * 4;
    p += i0 * 4;
  } else {
    const int u = t - 3 * l4, arr = u / l2;
    p = reinterpret_cast<const char*>(arr == 0 ? a.r : arr == 1 ? a.g : a.b);
    off = (int64_t)(u - arr * l2) * 128;
    bytes = cnt * 2;
    p += i0 * 2;
  }
  if (off < bytes) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
}

__device__ __forceinline__ void accumulate(Smem& s, Meta& m, const BinArgs& a, int slot, int col, int z, uint32_t r,
                                           uint32_t g, uint32_t b) {
  // the eight fine arrays lie s.fs bytes apart: cnt, rs, gs, bs, zlo, zhi, mn, mx
  const uint32_t p = s.fa + 4u * (uint32_t)sidx(a, slot, col);
  red_add_u(p, 1u);
  red_add_u(p + s.fs, r);
  red_add_u(p + 2u * s.fs, g);
  red_add_u(p + 3u * s.fs, b);
  red_add_u(p + 4u * s.fs, (unsigned)z & 0xffffu);
  if (z >> 16) red_add_s(p + 5u * s.fs, z >> 16);  // 0 <= z < 65536 cm: nothing to add
  red_min_s(p + 6u * s.fs, z);
  red_max_s(p + 7u * s.fs, z);
  m.touched[slot] = 1;
}

// PF: batches prefetched into L2 ahead of the loads (a launch-shape parameter, compiled
// in so that it costs no register).  kD31: cells of at least 2 cm, so the tile and cell
// divisions take the two-instruction form.
template <int PF, bool kD31>
__global__ void __launch_bounds__(kBinThreads, 1) k_bin_main(BinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Meta m;
  const int WC = a.W * a.rstride;
  const int CC = a.has_coarse ? kCW * a.ccells : 0;
  Smem s = carve(smem_raw, WC, CC);  // partials after the coarse ring
  for (int i = threadIdx.x; i < WC; i += blockDim.x) reset_cell(s, i);
  for (int i = threadIdx.x; i < CC; i += blockDim.x) {
    s.crs[i] = 0ull; s.cgs[i] = 0ull; s.cbs[i] = 0ull; s.czs[i] = 0ull;
    s.ccnt[i] = 0u; s.cmn[i] = INT_MAX; s.cmx[i] = INT_MIN;
  }
  if (threadIdx.x < kMaxW) { m.touched[threadIdx.x] = 0; m.pend_row[threadIdx.x] = -1; }
  if (threadIdx.x == 0) { m.dropped = 0ull; m.n_late = 0ull; m.n_inplace = 0; }
  __syncthreads();
  unsigned my_dropped = 0, my_late = 0;  // per thread: far below 2^32 points
  const int W = a.W;

  // spans are handed out dynamically: their cost depends on how many strips (window
  // slides) they hold, not only on their point count
  uint32_t* span_counter = a.row_state + a.n_rows;
  while (true) {
    if (threadIdx.x == 0) m.item = atomicAdd(span_counter, 1u);
    __syncthreads();
    const int64_t item = m.item;
    if (item >= a.n_items) break;
    const int64_t p0 = item * a.span;
    const int64_t p1 = p0 + a.span < a.n ? p0 + a.span : a.n;
    int lo = -1;   // lowest fine row of the window (uniform); -1 = empty
    int clo = -1;  // lowest coarse row of the coarse ring
    int batch = 0;
    if (threadIdx.x == 0) m.next_check = kResidLimitBatches - 1;  // the window starts empty
    Raw cur;
    for (int d = 1; d < PF; ++d) prefetch_batch(a, p0 + (int64_t)d * kBatch, p1);
    for (int64_t b0 = p0; b0 < p1; b0 += kBatch, ++batch) {
      // keep the L2 PF batches ahead of the loads
      prefetch_batch(a, b0 + (int64_t)PF * kBatch, p1);
      load_raw(a, cur, b0 + (int64_t)threadIdx.x * kPtsPerThread, p1);
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
        uint32_t tx, ty, cx, cy;
        if constexpr (kD31) {  // ux, uy < ext < 2^31
          tx = fdiv31(ux, a.d31_tile);
          ty = fdiv31(uy, a.d31_tile);
          cx = fdiv31(ux - tx * a.tile_cm, a.d31_cell);
          cy = fdiv31(uy - ty * a.tile_cm, a.d31_cell);
        } else {
          tx = fdiv(ux, a.div_tile);
          ty = fdiv(uy, a.div_tile);
          cx = fdiv(ux - tx * a.tile_cm, a.div_cell);
          cy = fdiv(uy - ty * a.tile_cm, a.div_cell);
        }
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
          accumulate(s, m, a, G[k] & (W - 1), col[k], cur.z[k], half16(cur.r, k), half16(cur.g, k), half16(cur.b, k));
        }
      } else {
        // ---- general case: late points, window slides.  Rows of the last flush are
        // published first, so a late point never waits on a claim of this CTA.  Only
        // the first pass can meet late points: every slide keeps the window at or
        // below the lowest pending row.
        publish_pending(a, m);
        while (true) {
          if (lo >= 0) {
            // late points (rows below the window), the warp's one at a time
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k) {
              const bool late = (pend & (1u << k)) && G[k] < lo;
              unsigned todo = __ballot_sync(0xffffffffu, late);
              while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                late_row_ready(a, __shfl_sync(0xffffffffu, G[k], src));
                if ((int)(threadIdx.x & 31) == src)
                  late_merge(a, G[k], col[k], cur.z[k], half16(cur.r, k), half16(cur.g, k), half16(cur.b, k));
              }
              if (late) {
                ++my_late;
                pend &= ~(1u << k);
              }
            }
#pragma unroll
            for (int k = 0; k < kPtsPerThread; ++k) {
              if ((pend & (1u << k)) && G[k] < lo + W) {
                accumulate(s, m, a, G[k] & (W - 1), col[k], cur.z[k], half16(cur.r, k), half16(cur.g, k), half16(cur.b, k));
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
          lo = nlo;  // the rows that enter are empty
          __syncthreads();
        }
      }
      // ---- residency bound: no ring row may absorb more than kRowLimit points (the
      // 32-bit sums of its cells stay exact).  A batch adds at most kBatch points to a
      // row, so after a count of the rows the next one is due once the fullest row
      // could reach the limit; rows that enter are empty.  Only when a row is near the
      // limit is the window flushed in place (its rows stay; their next flush merges).
      if (lo >= 0 && batch >= m.next_check) {
        const int room = kRowLimit - (int)row_count_max(a, s, m);
        if (room < 4 * kBatch) evict_rows(a, s, m, lo, lo + W, clo);
        if (threadIdx.x == 0) {
          m.n_inplace += room < 4 * kBatch;
          m.next_check = batch + (room < 4 * kBatch ? kResidLimitBatches : room / kBatch);
        }
        __syncthreads();
      }
    }
    // ---- end of the span: flush everything
    __syncthreads();
    if (lo >= 0) evict_rows(a, s, m, lo, lo + W, clo);
    if (a.has_coarse && clo >= 0) {
      coarse_evict(a, s, clo, clo + kCW, blockDim.x);
      __syncthreads();
    }
  }
  publish_pending(a, m);
  {
    const unsigned lt = __reduce_add_sync(0xffffffffu, my_late);
    if ((threadIdx.x & 31) == 0 && lt) atomicAdd((unsigned long long*)&m.n_late, (unsigned long long)lt);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (m.n_late) atomicAdd(&g_bin_stats[0], m.n_late);
      if (m.n_inplace) atomicAdd(&g_bin_stats[3], (unsigned long long)m.n_inplace);
    }
  }
  if (a.dropped) {
    my_dropped = __reduce_add_sync(0xffffffffu, my_dropped);
    if ((threadIdx.x & 31) == 0 && my_dropped)
      atomicAdd((unsigned long long*)&m.dropped, (unsigned long long)my_dropped);
    __syncthreads();
    if (threadIdx.x == 0 && m.dropped) atomicAdd((unsigned long long*)a.dropped, m.dropped);
  }
}

// Prologue: clear row states and the dropped counter; give the coarse level its
// empty sentinels (it is only ever merged into with atomics).  When accumulating, the
// bins and the dropped counter keep their contents.
__global__ void k_bin_prologue(BinArgs a, int64_t n_coarse) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_rows; i += stride)
    a.row_state[i] = 0u;
  if (a.accumulate) n_coarse = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_coarse; i += stride) {
    a.ccount[i] = 0u; a.czsum[i] = 0; a.czmin[i] = INT_MAX; a.czmax[i] = INT_MIN;
    a.crsum[i] = 0ull; a.cgsum[i] = 0ull; a.cbsum[i] = 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.row_state[a.n_rows] = 0u;  // span counter
    if (a.dropped && !a.accumulate) *a.dropped = 0ull;
  }
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

// Group stride gs (f <= gs < f + 4) and column split fh (1 <= fh <= f) of the coarse
// partials.  The lanes of a warp (coarse columns c0 + j, j < 16, groups h < 2, one fine
// row) read words j * gs + h * fh + k at step k; while both groups are active a step
// costs as many shared-memory wavefronts as the busiest bank has lanes, afterwards as
// many as the first group alone needs.  Fewest wavefronts win, then fewest steps, then
// the smallest stride.  E.g. f = 10: gs = 10, fh = 5 puts all 32 lanes on distinct banks.
static void bin_coarse_layout(int f, int32_t* gs_out, int32_t* fh_out) {
  int64_t best = INT64_MAX;
  *gs_out = f;
  *fh_out = f;
  for (int gs = f; gs < f + 4; ++gs) {
    int hits1[32] = {};
    int worst1 = 0;
    for (int j = 0; j < 16; ++j) worst1 = std::max(worst1, ++hits1[(j * gs) % 32]);
    for (int split = 1; split <= f; ++split) {
      int hits[32] = {};
      int worst = 0;
      for (int j = 0; j < 16; ++j)
        for (int h = 0; h < 2; ++h) worst = std::max(worst, ++hits[(j * gs + h * split) % 32]);
      const int both = std::min(split, f - split), steps = std::max(split, f - split);
      const int64_t wavefronts = (int64_t)both * worst + (int64_t)(steps - both) * worst1;
      const int64_t score = (wavefronts << 24) + ((int64_t)steps << 4) + (gs - f);
      if (score < best) { best = score; *gs_out = gs; *fh_out = split; }
    }
  }
}

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
  if (a.cell_cm >= 2) {  // then tile_cm >= 2 too; every numerator is below ext < 2^31
    a.d31_tile = make_fastdiv31(a.tile_cm);
    a.d31_cell = make_fastdiv31(a.cell_cm);
  }
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
  bin_coarse_layout(a.f, &a.gs, &a.fh);
  // window rows: the largest power of two <= 8 whose rings fit in ~220 KB of shared memory
  const size_t budget = 220 * 1024;
  int W = 8;
  if (W > a.cells) {
    W = 1;
    while (W * 2 <= a.cells) W *= 2;
  }
  const int CC = a.has_coarse ? kCW * a.ccells : 0;
  a.rstride = (a.cells / a.f) * a.gs;
  auto need = [&](int w) { return smem_bytes(w * a.rstride, CC, a.has_coarse ? w * a.ccells : 0); };
  while (W > 1 && need(W) > budget) W >>= 1;
  if (need(W) > budget) return LS_ERR_UNSUPPORTED;
  // every fine column's slot lies inside its row: sidx(col) < (cells / f) * gs <= rstride
  if (a.rstride < (a.cells / a.f) * a.gs || a.fh < 1 || a.fh > a.f) return LS_ERR_UNSUPPORTED;
  a.W = W;
  *smem = need(W);
  // 128-bit row stores: contiguous rows of whole 4-cell groups, every fine output array
  // and the shared arrays (WC words each, after the 64-bit coarse sums) 16-byte aligned
  a.vec_out = a.gs == a.f && a.cells % 4 == 0 && a.rstride % 4 == 0 && (W * a.rstride) % 4 == 0 &&
              (((uintptr_t)a.count | (uintptr_t)a.zsum | (uintptr_t)a.zmin | (uintptr_t)a.zmax |
                (uintptr_t)a.rsum | (uintptr_t)a.gsum | (uintptr_t)a.bsum) % 16 == 0);
  // vector loads need 16-byte aligned int32 arrays and 8-byte aligned uint16 arrays
  a.narrow = region->x0_cm >= INT32_MIN && region->x0_cm <= INT32_MAX && region->y0_cm >= INT32_MIN &&
             region->y0_cm <= INT32_MAX;
  a.x0_32 = a.narrow ? (int32_t)region->x0_cm : 0;
  a.y0_32 = a.narrow ? (int32_t)region->y0_cm : 0;
  a.vec = (((uintptr_t)a.x | (uintptr_t)a.y | (uintptr_t)a.z) % 16 == 0) &&
          (((uintptr_t)a.r | (uintptr_t)a.g | (uintptr_t)a.b) % 8 == 0);
  // launch shape: tuned for this key (ls_tune_bin_points / ls_bin_shape_set) or the default
  BinShape shape;
  bin_shape_lookup(bin_shape_key(pts->n, levels, n_levels), &shape);
  a.pf_dist = shape.prefetch_batches;
  // spans: about shape.spans_per_cta per CTA, multiples of the batch size
  const int64_t grid = kSmCount;
  int64_t span = (a.n + grid * shape.spans_per_cta - 1) / (grid * shape.spans_per_cta);
  span = (span + kBatch - 1) / kBatch * kBatch;
  if (span < kBatch) span = kBatch;
  a.span = span;
  a.n_items = (a.n + span - 1) / span;
  *out = a;
  return LS_OK;
}

ls_status bin_launch(BinArgs a, size_t smem, int64_t n_coarse, cudaStream_t stream) {
  static DeviceOnce once;
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  const bool ok = device_once(once, dev, [] {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    return cudaFuncSetAttribute(k_bin_main<1, true>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<2, true>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<3, true>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<4, true>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<1, false>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<2, false>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<3, false>, attr, kBinSmemAttr) == cudaSuccess &&
           cudaFuncSetAttribute(k_bin_main<4, false>, attr, kBinSmemAttr) == cudaSuccess;
  });
  if (!ok) return LS_ERR_CUDA;
  const int64_t work = a.n_rows > n_coarse ? a.n_rows : n_coarse;
  k_bin_prologue<<<grid_cap((work + 255) / 256, kSmCount * 8), 256, 0, stream>>>(a, n_coarse);
  if (a.n_items > 0) {
    const int grid = grid_cap(a.n_items, kSmCount);
    const bool d31 = a.cell_cm >= 2;
    switch (a.pf_dist * 2 + (d31 ? 1 : 0)) {
      case 2: k_bin_main<1, false><<<grid, kBinThreads, smem, stream>>>(a); break;
      case 3: k_bin_main<1, true><<<grid, kBinThreads, smem, stream>>>(a); break;
      case 6: k_bin_main<3, false><<<grid, kBinThreads, smem, stream>>>(a); break;
      case 7: k_bin_main<3, true><<<grid, kBinThreads, smem, stream>>>(a); break;
      case 8: k_bin_main<4, false><<<grid, kBinThreads, smem, stream>>>(a); break;
      case 9: k_bin_main<4, true><<<grid, kBinThreads, smem, stream>>>(a); break;
      default:
        if (d31)
          k_bin_main<2, true><<<grid, kBinThreads, smem, stream>>>(a);
        else
          k_bin_main<2, false><<<grid, kBinThreads, smem, stream>>>(a);
        break;
    }
  }
  if (!a.accumulate) k_bin_finalize<<<grid_cap(a.n_rows, kSmCount * 16), 128, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace ls

namespace ls {
namespace {
// One thread runs the binning's bounded row wait on a caller's flag.
__global__ void k_probe_wait(const uint32_t* flag) {
  if (blockIdx.x == 0 && threadIdx.x == 0) wait_written(flag);
}
}  // namespace
}  // namespace ls

extern "C" ls_status ls_probe_wait(const uint32_t* flag, ls_stream_t stream) {
  if (!flag || (reinterpret_cast<uintptr_t>(flag) & 3u)) return LS_ERR_INVALID_ARG;
  ls::k_probe_wait<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(flag);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

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
  a.row_state = static_cast<uint32_t*>(ls::workspace(ls::kWsBinRows, ((size_t)a.n_rows + 1) * 4));
  if (!a.row_state) return LS_ERR_NO_MEMORY;
  return ls::bin_launch(a, smem, n_coarse, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" ls_status ls_bin_points_accumulate(const ls_points* pts, const ls_region* region,
                                              const ls_bins* levels, int32_t n_levels, uint64_t* dropped,
                                              ls_stream_t stream) {
  ls::BinArgs a;
  size_t smem = 0;
  int64_t n_coarse = 0;
  ls_status st = ls::bin_prepare(pts, region, levels, n_levels, dropped, &a, &smem, &n_coarse);
  if (st != LS_OK) return st;
  a.accumulate = 1;
  a.row_state = static_cast<uint32_t*>(ls::workspace(ls::kWsBinRows, ((size_t)a.n_rows + 1) * 4));
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
static __device__ __align__(256) uint32_t g_bin_rows_fixed[kFixedBinRows + 64];  // + span counter
std::mutex g_fixed_mu;
uint32_t* g_fixed_ptr[64] = {};
}  // namespace

void forget_fixed_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_fixed_mu);
  if (dev >= 0 && dev < 64) g_fixed_ptr[dev] = nullptr;
}
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
