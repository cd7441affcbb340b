// Interpolated heightmaps of Alg. 1 (Sec. 3.3): per patch, the nearest-neighbour map
// and the Delaunay-linear map of the chunk samples that fall in a window made of the
// tile grown by a padding on every side (96 x 96 texels of 10 m around a 640 m tile),
// with four padding points (no data) at the window corners.
//
// Design (B300): one warp per patch, its whole state in the warp's slice of shared
// memory, no CTA barrier anywhere.
//  * gather: the window's samples from the 3x3 tile neighbourhood (three contiguous
//    CSR ranges of packed records), compacted with ballots in global sample order;
//  * triangulation: Bowyer-Watson in that order.  For each new point the lanes test
//    every triangle's circumcircle (a float test with a proven error margin, the
//    exact int128 determinant inside the margin), list the cavity's boundary edges
//    with ballots and re-triangulate the cavity in place, keeping neighbour links;
//  * maps: 8 x 4 texel blocks, one texel per lane.  NN: per block the candidates are
//    the points whose distance to the block is at most the smallest farthest-corner
//    distance; every lane takes the exact int64 nearest of them (ties to the lowest
//    index).  lin: the triangle that holds the texel centre, by a visibility walk
//    over the neighbour links from the lane's texel of the block above (exact int64
//    orientations), then the barycentric interpolation from the exact numerator;
//    outputs staged per block and stored as whole rows and 4-byte words.
// Patches whose window holds more samples than the small tier's capacity (96) are
// queued on the device for a second launch with one warp per CTA and room for 192 (about
// nine CTAs per SM), those over that for a third with room for 384 (four per SM), and
// those over that for a fourth with room for 1536 (one per SM).
#include <climits>

#include "ls_internal.cuh"

namespace ls {
namespace {

constexpr int kInterpMaxRes = 1024;
constexpr int kInterpHintRes = 128;  // up to this resolution walks start from the block above
constexpr int kInterpSmallCap = 96;     // window samples per patch, small tier
constexpr int kInterpSmallWarps = 4;    // patches (warps) per CTA, small tier
constexpr int kInterpMid1Cap = 192;     // first medium tier: one warp per CTA
constexpr int kInterpMidCap = 384;      // second medium tier: one warp per CTA, 4 CTAs per SM
constexpr int kInterpBigCap = 1536;     // big tier: one warp per CTA, one CTA per SM
constexpr int kInterpMaxWindow = 1 << 17;  // window side bound of the exact arithmetic
constexpr int kInterpZBound = 1 << 28;     // |z| bound of the exact numerators

// Per-warp state of one patch with up to CAP window samples.  A triangulation of
// CAP + 4 vertices whose hull is the window square has at most 2 * CAP + 2 triangles.
template <int CAP>
struct InterpWarp {
  static constexpr int NV = CAP + 4;
  static constexpr int NT = 2 * CAP + 2;
  float4 circ[NT];       // circumcircle: centre x, y, radius^2, error margin
  int2 P[NV];            // window-local vertex coordinates (0..3: corners)
  ushort4 tv[NT];        // vertices (counter-clockwise), cavity mark
  short4 tn[NT];         // neighbour across (v0,v1), (v1,v2), (v2,v0); -1 none
  ushort4 edge[NT + 2];  // cavity boundary edges: a, b, outside triangle
  int32_t start[NV];     // new triangle whose boundary edge starts at a vertex (stamped)
  int32_t z[CAP];
  float hm[CAP];         // height in metres of each sample
  uint32_t c8[CAP];      // 8-bit colour of each sample, R | G << 8 | B << 16
  uint32_t rg[CAP];      // 16-bit R | G << 16
  uint32_t bl[CAP];      // 16-bit B
  int32_t gidx[CAP];     // global sample index
  uint16_t list[NT];     // cavity triangles; later the NN candidates of a block
  __align__(16) uint8_t bytes[224];  // one texel block's colours (NN, lin) and flags
  uint16_t hints[kInterpHintRes / 8][32];  // per block column and lane: the last triangle
};

struct InterpArgs {
  const int64_t* __restrict__ toff;  // sample CSR by tile [T+1]
  const Rec* __restrict__ recs;      // packed samples (region-relative coordinates)
  const int32_t* __restrict__ tile_ids;
  int64_t n_out, n_samples;
  int32_t tiles_x, tiles_y, tile_cm, res, cell_cm, pad_cm, W;
  double z_scale, z_offset;
  float zs_f, zo_f;
  ls_interp_outputs out;
  // three queues of n_out + 1 words: [0] the number of patches queued for the next
  // tier (the two medium tiers, then big), [1..] their ordinals
  int32_t* queue;
};

__device__ __forceinline__ unsigned lanes_below() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ long long orient2(int2 a, int2 b, int2 c) {
  return (long long)(b.x - a.x) * (c.y - a.y) - (long long)(b.y - a.y) * (c.x - a.x);
}

// Float of a 64-bit integer with |x| < 2^62 from two 32-bit conversions (relative
// error below 2^-23).  The 64-bit conversions run on the FP64 pipe, which is narrow.
__device__ __forceinline__ float ll2f(long long x) {
  const unsigned long long u = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
  const float f = fmaf((float)(uint32_t)(u >> 32), 4294967296.f, (float)(uint32_t)u);
  return x < 0 ? -f : f;
}

// Sign of the lifted in-circle determinant of (a, b, c, d): > 0 iff d lies strictly
// inside the circumcircle of the counter-clockwise triangle (a, b, c).  Coordinate
// differences are below 2^17, so the 2x2 minors fit int64 and the sum int128.
__device__ __noinline__ bool incircle_exact(int2 a, int2 b, int2 c, int2 d) {
  const long long adx = a.x - d.x, ady = a.y - d.y;
  const long long bdx = b.x - d.x, bdy = b.y - d.y;
  const long long cdx = c.x - d.x, cdy = c.y - d.y;
  const long long ad = adx * adx + ady * ady, bd = bdx * bdx + bdy * bdy, cd = cdx * cdx + cdy * cdy;
  const __int128 det = (__int128)adx * (bdy * cd - bd * cdy) - (__int128)ady * (bdx * cd - bd * cdx) +
                       (__int128)ad * (bdx * cdy - bdy * cdx);
  return det > 0;
}

// Circumcircle of the counter-clockwise triangle (a, b, c) in float, with the margin
// m = S^2 / 2^16, S = |cx| + |cy| + 2 W.  The centre comes from exact int64 numerators
// over the exact denominator (two conversions within 2^-23, a division and an add:
// <= 6 * 2^-24 S), so each of |p - c|^2 and r^2 is within 32 * 2^-24 S^2 of its true
// value for any p in the window and their difference within 2^-18 S^2 < m: outside
// the band |d^2 - r^2| <= m the float comparison decides the exact predicate.
__device__ __forceinline__ float4 circumcircle(int2 a, int2 b, int2 c, int W) {
  const long long bx = b.x - a.x, by = b.y - a.y, cx = c.x - a.x, cy = c.y - a.y;
  const long long D = 2 * (bx * cy - by * cx);
  const long long B2 = bx * bx + by * by, C2 = cx * cx + cy * cy;
  const long long Nx = cy * B2 - by * C2, Ny = bx * C2 - cx * B2;
  const float Df = ll2f(D);
  const float ccx = (float)a.x + __fdiv_rn(ll2f(Nx), Df);
  const float ccy = (float)a.y + __fdiv_rn(ll2f(Ny), Df);
  const float rx = (float)a.x - ccx, ry = (float)a.y - ccy;
  const float S = fabsf(ccx) + fabsf(ccy) + 2.f * (float)W;
  return make_float4(ccx, ccy, fmaf(rx, rx, ry * ry), S * S * (1.f / 65536.f));
}

template <int CAP>
__device__ __forceinline__ bool in_circumcircle(const InterpWarp<CAP>& s, int i, int2 p) {
  const float4 c = s.circ[i];
  const float dx = (float)p.x - c.x, dy = (float)p.y - c.y;
  const float d2 = fmaf(dx, dx, dy * dy);
  if (d2 < c.z - c.w) return true;
  if (d2 > c.z + c.w) return false;
  const ushort4 v = s.tv[i];
  return incircle_exact(s.P[v.x], s.P[v.y], s.P[v.z], p);
}

__device__ __forceinline__ short& tn_at(short4& t, int e) { return e == 0 ? t.x : e == 1 ? t.y : t.z; }

// Bowyer-Watson insertion of vertex vi (the whole warp).  Returns false when the
// cavity is not a simple polygon around the point (impossible with exact predicates;
// checked all the same).  T is updated.
template <int CAP>
__device__ bool insert_point(InterpWarp<CAP>& s, int vi, int W, int& T) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanes_below();
  const int2 p = s.P[vi];
  // triangles whose circumcircle holds p strictly inside
  int nb = 0;
  for (int base = 0; base < T; base += 32) {
    const int i = base + lane;
    const bool bad = i < T && in_circumcircle(s, i, p);
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (bad) {
      s.list[nb + __popc(m & lt)] = (uint16_t)i;
      s.tv[i].w = (uint16_t)vi;
    }
    nb += __popc(m);
  }
  __syncwarp();
  if (nb == 0) return true;  // p repeats a vertex
  // boundary edges of the cavity (the neighbour across is not in it), kept when the
  // join with p has positive area (a zero-area join lies on the window's edge)
  int K = 0;
  bool err = false;
  for (int base = 0; base < 3 * nb; base += 32) {
    const int item = base + lane;
    bool keep = false;
    ushort4 ed = make_ushort4(0, 0, 0, 0);
    if (item < 3 * nb) {
      const int tb = s.list[item / 3], e = item % 3;
      const ushort4 v = s.tv[tb];
      const int va = e == 0 ? v.x : e == 1 ? v.y : v.z;
      const int vb = e == 0 ? v.y : e == 1 ? v.z : v.x;
      short4 nn = s.tn[tb];
      const int on = tn_at(nn, e);
      if (on >= T) {
        err = true;  // a broken link (never expected): stop before following it
      } else if (on < 0 || s.tv[on].w != vi) {
        keep = orient2(s.P[va], s.P[vb], p) > 0;
        err = !keep && on >= 0;
      }
      ed = make_ushort4((uint16_t)va, (uint16_t)vb, (uint16_t)on, 0);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int pos = K + __popc(m & lt);
    if (keep && pos < InterpWarp<CAP>::NT + 2) s.edge[pos] = ed;
    K += __popc(m);
  }
  if (__any_sync(0xffffffffu, err) || K <= nb || T + K - nb > InterpWarp<CAP>::NT) return false;
  __syncwarp();
  // new triangles (a, b, p) in the cavity's slots, then in fresh ones
  for (int j = lane; j < K; j += 32) {
    const int slot = j < nb ? s.list[j] : T + j - nb;
    const ushort4 ed = s.edge[j];
    const int on = (int16_t)ed.z;
    s.tv[slot] = make_ushort4(ed.x, ed.y, (uint16_t)vi, 0);
    s.tn[slot] = make_short4((short)on, -1, -1, 0);
    s.circ[slot] = circumcircle(s.P[ed.x], s.P[ed.y], p, W);
    if (on >= 0) {
      const ushort4 ov = s.tv[on];
      short* tp = &s.tn[on].x;
      if (ov.x == ed.y && ov.y == ed.x) tp[0] = (short)slot;
      else if (ov.y == ed.y && ov.z == ed.x) tp[1] = (short)slot;
      else tp[2] = (short)slot;
    }
    s.start[ed.x] = (vi << 16) | slot;
  }
  __syncwarp();
  // link consecutive new triangles: (a, b, p) and (b, c, p) share the edge (b, p)
  for (int j = lane; j < K; j += 32) {
    const int slot = j < nb ? s.list[j] : T + j - nb;
    const int st = s.start[s.edge[j].y];
    if ((st >> 16) == vi) {
      const int t2 = st & 0xffff;
      s.tn[slot].y = (short)t2;
      s.tn[t2].z = (short)slot;
    }
  }
  __syncwarp();
  T += K - nb;
  return true;
}

__device__ __forceinline__ bool real_tri(ushort4 v) { return v.x >= 4 && v.y >= 4 && v.z >= 4; }

// Triangle that contains the point g (closed), by a visibility walk from `hint`: cross
// the first edge that has g strictly on its outer side.  The walk ends on a Delaunay
// triangulation; a scan of all triangles backs up a walk that runs too long.  w gets
// the weights of g in the triangle found: w[k] = twice the area of the sub-triangle
// opposite vertex k.
template <int CAP>
__device__ int locate(const InterpWarp<CAP>& s, int2 g, int hint, int T, long long w[3]) {
  int t = hint >= 0 && hint < T ? hint : 0;
  for (int step = 0; step < 2 * T + 8; ++step) {
    const ushort4 v = s.tv[t];
    short4 nb = s.tn[t];
    const int2 A = s.P[v.x], B = s.P[v.y], C = s.P[v.z];
    w[2] = orient2(A, B, g);
    w[0] = orient2(B, C, g);
    w[1] = orient2(C, A, g);
    const int e = w[2] < 0 ? 0 : (w[0] < 0 ? 1 : (w[1] < 0 ? 2 : -1));
    if (e < 0) return t;
    const int nt = tn_at(nb, e);
    if (nt < 0 || nt >= T) break;
    t = nt;
  }
  for (int i = 0; i < T; ++i) {
    const ushort4 v = s.tv[i];
    const int2 A = s.P[v.x], B = s.P[v.y], C = s.P[v.z];
    w[0] = orient2(B, C, g);
    w[1] = orient2(C, A, g);
    w[2] = orient2(A, B, g);
    if (w[0] >= 0 && w[1] >= 0 && w[2] >= 0) return i;
  }
  return -1;
}

// A triangle of three real points that holds g on its boundary, given the triangle t
// without data that contains g with the weights w (w[k] = 0: g on the edge opposite
// vertex k).  -1 if there is none.
template <int CAP>
__device__ int real_neighbour(const InterpWarp<CAP>& s, int t, const long long w[3], int T) {
  const ushort4 v = s.tv[t];
  const int vid[3] = {v.x, v.y, v.z};
  const int zeros = (w[0] == 0) + (w[1] == 0) + (w[2] == 0);
  if (zeros == 1) {  // on the edge opposite vertex k: edge index (k + 1) % 3
    const int k = w[0] == 0 ? 0 : (w[1] == 0 ? 1 : 2);
    short4 nb = s.tn[t];
    const int n = tn_at(nb, (k + 1) % 3);
    return n >= 0 && n < T && real_tri(s.tv[n]) ? n : -1;
  }
  if (zeros != 2) return -1;
  // g is the vertex with the non-zero weight: turn around it both ways
  const int c = w[0] != 0 ? vid[0] : (w[1] != 0 ? vid[1] : vid[2]);
  if (c < 4) return -1;
  for (int dir = 0; dir < 2; ++dir) {
    int cur = t;
    for (int it = 0; it < T; ++it) {
      const ushort4 u = s.tv[cur];
      const int k = u.x == c ? 0 : (u.y == c ? 1 : 2);
      short4 nb = s.tn[cur];
      const int n = tn_at(nb, dir == 0 ? k : (k + 2) % 3);
      if (n < 0 || n >= T || n == t) break;
      if (real_tri(s.tv[n])) return n;
      cur = n;
    }
  }
  return -1;
}

// Linear height (metres) and 8-bit colour of g in the real triangle t, from the
// weights w (twice the areas of the sub-triangles opposite each vertex).
template <int CAP>
__device__ __forceinline__ void linear_value(const InterpWarp<CAP>& s, const InterpArgs& a, int t,
                                             const long long w[3], float& h, uint32_t& c8) {
  const ushort4 v = s.tv[t];
  const long long wa = w[0], wb = w[1], wc = w[2];
  const long long area = wa + wb + wc;
  const int ka = v.x - 4, kb = v.y - 4, kc = v.z - 4;
  const float inv = __frcp_rn(ll2f(area));
  // q = floor(num / area) and r = num - q * area, exact: a float estimate (within 81
  // of q for |z| < 2^28) corrected in int64.  The product may wrap around in the
  // unsigned arithmetic; the true remainder fits, so the difference is exact.
  const long long num = wa * s.z[ka] + wb * s.z[kb] + wc * s.z[kc];
  int q = (int)floorf(ll2f(num) * inv);
  long long r = (long long)((unsigned long long)num - (unsigned long long)(long long)q * (unsigned long long)area);
  const int dq = (int)floorf(ll2f(r) * inv);
  q += dq;
  r -= (long long)dq * area;
  if (r < 0) {
    q -= 1; r += area;
  } else if (r >= area) {
    q += 1; r -= area;
  }
  h = fmaf((float)q + ll2f(r) * inv, a.zs_f, a.zo_f);  // the fraction within 2^-21
  // colours from float barycentric weights (within 2^-21): the 16-bit value within
  // 0.06, the 8-bit one within 3e-4; near a rounding boundary the exact integers decide
  const float lb = ll2f(wb) * inv, lc = ll2f(wc) * inv;
  const uint32_t ca[3] = {s.rg[ka] & 0xffffu, s.rg[ka] >> 16, s.bl[ka]};
  const uint32_t cb[3] = {s.rg[kb] & 0xffffu, s.rg[kb] >> 16, s.bl[kb]};
  const uint32_t cc[3] = {s.rg[kc] & 0xffffu, s.rg[kc] >> 16, s.bl[kc]};
  c8 = 0u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float ya = (float)ca[ch];
    const float y = fmaf(lb, (float)cb[ch] - ya, fmaf(lc, (float)cc[ch] - ya, ya));
    const float fq = fmaf(y, 1.f / 256.f, 0.5f);
    const float fl = floorf(fq), fr = fq - fl;
    int k = (int)fl;
    if (!(fr > 1e-3f && fr < 1.f - 1e-3f)) {
      const long long numc = wa * ca[ch] + wb * cb[ch] + wc * cc[ch];
      k = (int)((numc + 128 * area) / (256 * area));
    }
    c8 |= (uint32_t)(k > 255 ? 255 : k) << (8 * ch);
  }
}

// All maps over 8 x 4 texel blocks, one texel per lane.
//  * NN: the candidates of a block are the points whose distance to the block is at
//    most U, the smallest farthest-corner distance over all points (every texel's
//    nearest point, and every point tied with it, is one); each lane takes the exact
//    nearest candidate, candidates in sample order.
//  * lin: the triangle that contains the texel centre, found by a walk from the one
//    the same lane found in the block above (4 texels up); a triangle with a padding corner hands the
//    texel to a real triangle that holds it on its boundary, if any (closed triangles,
//    as the inside test of Alg. 1), else the texel takes its NN value.
// Outputs are staged per block and stored as 32-byte rows of heights and 4-byte words
// of colours and inside flags.
template <int CAP>
__device__ void texel_maps(InterpWarp<CAP>& s, const InterpArgs& a, int64_t o, int n, int T) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanes_below();
  const int res = a.res, cell = a.cell_cm, h = cell / 2;
  const int bxn = res / 8, nblk = bxn * (res / 4);
  int hint = 0;
  // blocks row by row (whole 32-byte sectors of every output row are written by
  // consecutive blocks); a lane's walk starts from the triangle it found in the block
  // above (4 texels up), in the first block row and above 128 texels per side from
  // the block to the left
  for (int blk = 0; blk < nblk; ++blk) {
    const int bj = (blk % bxn) * 8, bi = (blk / bxn) * 4;
    const bool keep_hint = res <= kInterpHintRes;
    if (bi > 0 && keep_hint) hint = s.hints[bj >> 3][lane];
    const int jj = bj + (lane & 7), ii = bi + (lane >> 3);
    const int gxa = cell * bj + h, gxb = gxa + 7 * cell, gya = cell * bi + h, gyb = gya + 3 * cell;
    long long U = LLONG_MAX;
    for (int k = lane; k < n; k += 32) {
      const int2 q = s.P[4 + k];
      const int dx = max(abs(q.x - gxa), abs(q.x - gxb)), dy = max(abs(q.y - gya), abs(q.y - gyb));
      const long long d2 = (long long)dx * dx + (long long)dy * dy;
      U = d2 < U ? d2 : U;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const long long u = __shfl_xor_sync(0xffffffffu, U, d);
      U = u < U ? u : U;
    }
    int nc = 0;
    for (int base = 0; base < n; base += 32) {
      const int k = base + lane;
      bool c = false;
      if (k < n) {
        const int2 q = s.P[4 + k];
        const int dx = q.x < gxa ? gxa - q.x : (q.x > gxb ? q.x - gxb : 0);
        const int dy = q.y < gya ? gya - q.y : (q.y > gyb ? q.y - gyb : 0);
        c = (long long)dx * dx + (long long)dy * dy <= U;
      }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      if (c) s.list[nc + __popc(m & lt)] = (uint16_t)k;
      nc += __popc(m);
    }
    __syncwarp();
    const int2 g = make_int2(cell * jj + h, cell * ii + h);
    long long best = LLONG_MAX;
    int bk = -1;
    for (int c = 0; c < nc; ++c) {
      const int k = s.list[c];
      const int2 q = s.P[4 + k];
      const long long d2 = (long long)(q.x - g.x) * (q.x - g.x) + (long long)(q.y - g.y) * (q.y - g.y);
      if (d2 < best) { best = d2; bk = k; }
    }
    const float nn_h = bk >= 0 ? s.hm[bk] : __int_as_float(0x7fc00000);
    const uint32_t nn_c = bk >= 0 ? s.c8[bk] : 0u;
    float lin_h = nn_h;
    uint32_t lin_c = nn_c;
    bool in = false;
    if (T > 0) {
      long long w[3];
      int t = locate(s, g, hint, T, w);
      if (t >= 0) {
        hint = t;
        if (keep_hint) s.hints[bj >> 3][lane] = (uint16_t)t;
        if (!real_tri(s.tv[t])) {
          t = (w[0] == 0 || w[1] == 0 || w[2] == 0) ? real_neighbour(s, t, w, T) : -1;
          if (t >= 0) {
            const ushort4 v = s.tv[t];
            const int2 A = s.P[v.x], B = s.P[v.y], C = s.P[v.z];
            w[0] = orient2(B, C, g);
            w[1] = orient2(C, A, g);
            w[2] = orient2(A, B, g);
          }
        }
        if (t >= 0) {
          in = true;
          linear_value(s, a, t, w, lin_h, lin_c);
        }
      }
    }
    // ---- stores: heights as rows of 8 floats; colours and flags through the stage
    const size_t ge = (size_t)o * res * res + (size_t)ii * res + jj;
    if (a.out.nn_height) a.out.nn_height[ge] = nn_h;
    if (a.out.lin_height) a.out.lin_height[ge] = lin_h;
    __syncwarp();  // the previous block's stage has been stored
    uint8_t* st = s.bytes;
    st[3 * lane] = (uint8_t)nn_c; st[3 * lane + 1] = (uint8_t)(nn_c >> 8); st[3 * lane + 2] = (uint8_t)(nn_c >> 16);
    st[96 + 3 * lane] = (uint8_t)lin_c; st[97 + 3 * lane] = (uint8_t)(lin_c >> 8);
    st[98 + 3 * lane] = (uint8_t)(lin_c >> 16);
    st[192 + lane] = in ? 1 : 0;
    __syncwarp();
    const size_t row0 = (size_t)o * res * res + (size_t)bi * res + bj;  // texel of the block's first row
    if (lane < 24) {  // 4 rows x 6 words of 8 texels' colours
      const int r = lane / 6, w = lane % 6;
      const size_t off = (row0 + (size_t)r * res) * 3 + 4 * w;
      if (a.out.nn_rgb) *reinterpret_cast<uint32_t*>(a.out.nn_rgb + off) = reinterpret_cast<const uint32_t*>(st)[6 * r + w];
      if (a.out.lin_rgb)
        *reinterpret_cast<uint32_t*>(a.out.lin_rgb + off) = reinterpret_cast<const uint32_t*>(st + 96)[6 * r + w];
    } else if (a.out.inside) {  // 4 rows x 2 words of flags
      const int r = (lane - 24) >> 1, w = lane & 1;
      *reinterpret_cast<uint32_t*>(a.out.inside + row0 + (size_t)r * res + 4 * w) =
          reinterpret_cast<const uint32_t*>(st + 192)[2 * r + w];
    }
  }
  __syncwarp();
}

// Alg. 1 for output ordinal o.  Tiers 0, 1 and 2 queue a patch with more than CAP window
// samples for the next tier; the last tier reports it (LS_ERR_OUT_OF_RANGE) and writes
// NaN heights.
template <int CAP, int TIER>
__device__ void interp_patch(InterpWarp<CAP>& s, const InterpArgs& a, int64_t o) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanes_below();
  const int t = a.tile_ids ? a.tile_ids[o] : (int)o;
  if (t < 0 || t >= a.tiles_x * a.tiles_y) {  // uniform across the warp
    if (lane == 0) set_status(LS_ERR_INVALID_ARG);
    return;
  }
  const int tx = t % a.tiles_x, ty = t / a.tiles_x;
  const int64_t X0 = (int64_t)tx * a.tile_cm - a.pad_cm, Y0 = (int64_t)ty * a.tile_cm - a.pad_cm;
  // ---- gather the window's samples in global order
  int n = 0;
  bool zbad = false;
  for (int k = 0; k < 3; ++k) {
    const int uy = ty - 1 + k;
    if (uy < 0 || uy >= a.tiles_y) continue;
    const int xa = tx > 0 ? tx - 1 : 0, xb = tx + 1 < a.tiles_x ? tx + 1 : tx;
    const int64_t q0 = a.toff[(int64_t)uy * a.tiles_x + xa], q1 = a.toff[(int64_t)uy * a.tiles_x + xb + 1];
    if (q0 < 0 || q1 < q0 || q1 > a.n_samples) {  // inconsistent CSR: use nothing
      if (lane == 0) set_status(LS_ERR_INVALID_ARG);
      continue;
    }
    for (int64_t base = q0; base < q1; base += 32) {
      const int64_t q = base + lane;
      bool in = false;
      int4 r0 = make_int4(0, 0, 0, 0);
      int2 r1 = make_int2(0, 0);
      int lx = 0, ly = 0;
      if (q < q1) {
        const int4* rp = reinterpret_cast<const int4*>(a.recs + q);
        r0 = __ldg(rp);
        r1 = __ldg(reinterpret_cast<const int2*>(rp + 1));
        const int64_t wx = (int64_t)r0.x - X0, wy = (int64_t)r0.y - Y0;
        in = wx >= 0 && wx <= a.W && wy >= 0 && wy <= a.W;
        lx = (int)wx; ly = (int)wy;
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      const int pos = n + __popc(m & lt);
      if (in && pos < CAP) {
        s.P[4 + pos] = make_int2(lx, ly);
        s.z[pos] = r0.z;
        s.gidx[pos] = r0.w;
        s.rg[pos] = (uint32_t)r1.x;
        s.bl[pos] = (uint32_t)r1.y;
        zbad |= r0.z >= kInterpZBound || r0.z <= -kInterpZBound;
      }
      n += __popc(m);
    }
  }
  bool failed = false;
  if (n > CAP) {
    if (TIER < 3) {
      if (lane == 0) {
        int32_t* q = a.queue + (size_t)TIER * (a.n_out + 1);
        const int qpos = atomicAdd(q, 1);
        q[1 + qpos] = (int)o;
      }
      return;
    }
    if (lane == 0) set_status(LS_ERR_OUT_OF_RANGE);
    n = 0;  // NaN maps
    failed = true;
  }
  if (__any_sync(0xffffffffu, zbad)) {
    if (lane == 0) set_status(LS_ERR_UNSUPPORTED);
    failed = true;  // nearest-neighbour maps only
  }
  // ---- per-sample values, corners, empty inside mask
  for (int k = lane; k < n; k += 32) {
    s.hm[k] = (float)__dadd_rn(__dmul_rn((double)s.z[k], a.z_scale), a.z_offset);
    uint32_t c8 = 0;
    const uint32_t c16[3] = {s.rg[k] & 0xffffu, s.rg[k] >> 16, s.bl[k]};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const uint32_t v = (c16[ch] + 128u) >> 8;  // round half up of c / 256
      c8 |= (v > 255u ? 255u : v) << (8 * ch);
    }
    s.c8[k] = c8;
  }
  for (int k = lane; k < n + 4; k += 32) s.start[k] = -1;
  if (lane < 4) s.P[lane] = make_int2(lane == 1 || lane == 2 ? a.W : 0, lane >= 2 ? a.W : 0);
  __syncwarp();
  // ---- Delaunay triangulation of corners and samples
  int T = 0;
  if (!failed) {
    if (lane < 2) {
      const int2 P0 = s.P[0], P1 = s.P[lane + 1], P2 = s.P[lane + 2];
      s.tv[lane] = make_ushort4(0, (uint16_t)(lane + 1), (uint16_t)(lane + 2), 0);
      s.tn[lane] = lane == 0 ? make_short4(-1, -1, 1, 0) : make_short4(0, -1, -1, 0);
      s.circ[lane] = circumcircle(P0, P1, P2, a.W);
    }
    __syncwarp();
    T = 2;
    for (int k = 0; k < n; ++k) {
      if (!insert_point(s, 4 + k, a.W, T)) {
        if (lane == 0) set_status(LS_ERR_UNSUPPORTED);
        failed = true;
        T = 0;
        break;
      }
    }
  }
  if (a.out.tri_count && lane == 0) a.out.tri_count[o] = failed ? -1 : T;
  if (a.out.triangles) {
    const int m = T < a.out.tri_cap ? T : a.out.tri_cap;
    int32_t* dst = a.out.triangles + (size_t)o * a.out.tri_cap * 3;
    for (int i = lane; i < m; i += 32) {
      const ushort4 v = s.tv[i];
      dst[3 * i] = v.x >= 4 ? s.gidx[v.x - 4] : -1 - v.x;
      dst[3 * i + 1] = v.y >= 4 ? s.gidx[v.y - 4] : -1 - v.y;
      dst[3 * i + 2] = v.z >= 4 ? s.gidx[v.z - 4] : -1 - v.z;
    }
  }
  // ---- NN map and linear map inside triangles of three real points
  texel_maps(s, a, o, n, T);
}

// Tier 0 takes every requested patch; tiers 1 to 3 the ones the previous tier queued
// (written by the previous launch on the same stream).
template <int CAP, int TIER>
__global__ void __launch_bounds__(TIER > 0 ? 32 : 32 * kInterpSmallWarps) k_interp(InterpArgs a) {
  extern __shared__ __align__(16) unsigned char interp_dyn[];
  InterpWarp<CAP>& s = reinterpret_cast<InterpWarp<CAP>*>(interp_dyn)[threadIdx.x >> 5];
  const int wpc = blockDim.x >> 5;
  int64_t items = a.n_out;
  const int32_t* in = TIER > 0 ? a.queue + (size_t)(TIER - 1) * (a.n_out + 1) : nullptr;
  if (TIER > 0) {
    const int queued = *reinterpret_cast<const volatile int32_t*>(in);
    items = queued < a.n_out ? queued : a.n_out;
  }
  for (int64_t item = (int64_t)blockIdx.x * wpc + (threadIdx.x >> 5); item < items;
       item += (int64_t)gridDim.x * wpc) {
    const int64_t o = TIER > 0 ? (int64_t)in[1 + item] : item;
    interp_patch<CAP, TIER>(s, a, o);
  }
}

}  // namespace
}  // namespace ls

extern "C" ls_status ls_fill_interp(const ls_points* samples, const ls_region* region,
                                    const ls_interp_params* params, const int32_t* tile_ids, int64_t n_out,
                                    const ls_interp_outputs* out, ls_stream_t stream) {
  using namespace ls;
  if (!samples || !region || !params || !out || n_out < 0) return LS_ERR_INVALID_ARG;
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
  const int res = params->res;
  if (res < 8 || res > kInterpMaxRes || res % 8) return LS_ERR_INVALID_ARG;
  // colours and flags are stored as 4-byte words
  if ((reinterpret_cast<uintptr_t>(out->nn_rgb) | reinterpret_cast<uintptr_t>(out->lin_rgb) |
       reinterpret_cast<uintptr_t>(out->inside)) & 3u)
    return LS_ERR_INVALID_ARG;
  if (params->pad_cm < 0 || params->pad_cm > region->tile_cm) return LS_ERR_INVALID_ARG;
  const int64_t W = (int64_t)region->tile_cm + 2 * (int64_t)params->pad_cm;
  if (W > kInterpMaxWindow) return LS_ERR_UNSUPPORTED;
  if (W % res) return LS_ERR_INVALID_ARG;
  if (out->triangles && out->tri_cap <= 0) return LS_ERR_INVALID_ARG;
  if (n_out == 0) return LS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Rec* recs = static_cast<Rec*>(workspace(kWsInterpRecs, (size_t)(samples->n > 0 ? samples->n : 1) * sizeof(Rec)));
  int32_t* queue = static_cast<int32_t*>(workspace(kWsInterpQueue, (size_t)3 * (n_out + 1) * sizeof(int32_t)));
  if (!recs || !queue) return LS_ERR_NO_MEMORY;
  if (samples->n > 0)
    k_pack<<<grid_cap((T + 7) / 8, kSmCount * 16), 256, 0, s>>>(*samples, T, region->x0_cm, region->y0_cm,
                                                                 region->tile_cm, region->tiles_x, recs);
  LS_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int32_t), s));
  LS_CUDA_TRY(cudaMemsetAsync(queue + n_out + 1, 0, sizeof(int32_t), s));
  LS_CUDA_TRY(cudaMemsetAsync(queue + 2 * (n_out + 1), 0, sizeof(int32_t), s));
  InterpArgs a;
  a.toff = samples->tile_offsets;
  a.recs = recs;
  a.tile_ids = tile_ids;
  a.n_out = n_out;
  a.n_samples = samples->n;
  a.tiles_x = region->tiles_x;
  a.tiles_y = region->tiles_y;
  a.tile_cm = region->tile_cm;
  a.res = res;
  a.cell_cm = (int32_t)(W / res);
  a.pad_cm = params->pad_cm;
  a.W = (int32_t)W;
  a.z_scale = region->z_scale;
  a.z_offset = region->z_offset;
  a.zs_f = (float)region->z_scale;
  a.zo_f = (float)region->z_offset;
  a.out = *out;
  a.queue = queue;
  const size_t small_smem = sizeof(InterpWarp<kInterpSmallCap>) * kInterpSmallWarps;
  const size_t mid1_smem = sizeof(InterpWarp<kInterpMid1Cap>);
  const size_t mid_smem = sizeof(InterpWarp<kInterpMidCap>);
  const size_t big_smem = sizeof(InterpWarp<kInterpBigCap>);
  // kernel attributes and resident CTAs per SM of the tiers, once per device
  static DeviceOnce once;
  static int small_per_sm[kMaxDevicesOnce] = {}, mid1_per_sm[kMaxDevicesOnce] = {}, mid_per_sm[kMaxDevicesOnce] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ERR_CUDA;
  const bool known = dev >= 0 && dev < kMaxDevicesOnce;
  const bool ok = device_once(once, dev, [&] {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(k_interp<kInterpSmallCap, 0>, attr, (int)small_smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_interp<kInterpMid1Cap, 1>, attr, (int)mid1_smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_interp<kInterpMidCap, 2>, attr, (int)mid_smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_interp<kInterpBigCap, 3>, attr, (int)big_smem) != cudaSuccess)
      return false;
    int b = 0, c1 = 0, c = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_interp<kInterpSmallCap, 0>, 32 * kInterpSmallWarps,
                                                      small_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c1, k_interp<kInterpMid1Cap, 1>, 32, mid1_smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_interp<kInterpMidCap, 2>, 32, mid_smem) != cudaSuccess)
      return false;
    if (known) {
      small_per_sm[dev] = b > 0 ? b : 1;
      mid1_per_sm[dev] = c1 > 0 ? c1 : 1;
      mid_per_sm[dev] = c > 0 ? c : 1;
    }
    return true;
  });
  if (!ok) return LS_ERR_CUDA;
  const int per_sm = known ? small_per_sm[dev] : 1, mid_sm = known ? mid_per_sm[dev] : 1;
  const int mid1_sm = known ? mid1_per_sm[dev] : 1;
  k_interp<kInterpSmallCap, 0>
      <<<grid_cap((n_out + kInterpSmallWarps - 1) / kInterpSmallWarps, (int64_t)kSmCount * per_sm),
         32 * kInterpSmallWarps, small_smem, s>>>(a);
  k_interp<kInterpMid1Cap, 1><<<grid_cap(n_out, (int64_t)kSmCount * mid1_sm), 32, mid1_smem, s>>>(a);
  k_interp<kInterpMidCap, 2><<<grid_cap(n_out, (int64_t)kSmCount * mid_sm), 32, mid_smem, s>>>(a);
  k_interp<kInterpBigCap, 3><<<grid_cap(n_out, kSmCount), 32, big_smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
