// Software rasterizers into a headless framebuffer (Sec. 3.5, rendering): points and
// heightmap triangles drawn with a 64-bit atomicMin of (depth bits << 32 | colour) per
// pixel, and the resolve that extracts the colours into an RGBA8 image.
//
// Design (B300):
//  * points: grid-stride over the point arrays (coalesced 4- and 2-byte loads); a
//    fragment reads the pixel's word first, loads its colour only when its depth is
//    not behind that word, and issues the atomicMin only when its word is smaller
//    (words only decrease, so the skipped ones could never win).  A 1080p framebuffer
//    (16.6 MB) stays in L2, where the atomics resolve;
//  * heightmaps: the mesh is implicit (two triangles per quad of adjacent texel
//    centres), so there is no triangle list in memory.  Persistent CTAs of 128 threads
//    take 128 quads at a time; a thread projects its quad's four vertices and draws
//    each triangle whose candidate pixels number at most 1024 itself; larger ones go
//    to a shared-memory queue that the whole CTA then draws, pixel-parallel;
//  * every float operation goes through IEEE round-to-nearest PTX (no fused
//    multiply-add, denormals kept) in the order the C ABI fixes, so the framebuffer
//    is bit-exact against a float32 reference whatever the order of the fragments.
#include "ls_internal.cuh"

namespace ls {
namespace {

constexpr int kRenderThreads = 256;
constexpr int kMeshThreads = 128;
constexpr int kLargeTri = 1024;  // candidate pixels above which a CTA draws the triangle

__device__ __forceinline__ float f_add(float a, float b) {
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f_sub(float a, float b) {
  float r;
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f_mul(float a, float b) {
  float r;
  asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f_div(float a, float b) {
  float r;
  asm("div.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f_of(long long v) {
  // the 32-bit conversion when the value fits (the same rounded value, a cheaper
  // instruction than the 64-bit one)
  float r;
  if (v == (long long)(int)v) {
    asm("cvt.rn.f32.s32 %0, %1;" : "=f"(r) : "r"((int)v));
  } else {
    asm("cvt.rn.f32.s64 %0, %1;" : "=f"(r) : "l"(v));
  }
  return r;
}
__device__ __forceinline__ bool finite_f(float v) { return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u; }

struct Cam {
  long long ox, oy, oz;
  float M[16];
  int W, H;
};

struct Vtx {
  float x, y, d;
  bool kept;
};

// Camera frame (cm) to screen: clip rows ((M0 qx + M1 qy) + M2 qz) + M3, perspective
// division (IEEE quotients c / c_w), viewport; kept when c_w > 0 and 0 <= d <= 1.
__device__ __forceinline__ Vtx project(const Cam& c, float qx, float qy, float qz) {
  float cl[4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    cl[r] = f_add(f_add(f_add(f_mul(c.M[4 * r], qx), f_mul(c.M[4 * r + 1], qy)), f_mul(c.M[4 * r + 2], qz)),
                  c.M[4 * r + 3]);
  Vtx v;
  v.kept = cl[3] > 0.f;
  const float nx = f_div(cl[0], cl[3]), ny = f_div(cl[1], cl[3]), nz = f_div(cl[2], cl[3]);
  v.x = f_mul(f_add(f_mul(nx, 0.5f), 0.5f), (float)c.W);
  v.y = f_mul(f_add(f_mul(ny, 0.5f), 0.5f), (float)c.H);
  v.d = f_add(f_mul(nz, 0.5f), 0.5f);
  v.kept = v.kept && v.d >= 0.f && v.d <= 1.f && finite_f(v.x) && finite_f(v.y);
  return v;
}

__device__ __forceinline__ uint32_t to8(uint32_t c16) {
  const uint32_t v = (c16 + 128u) >> 8;
  return v > 255u ? 255u : v;
}

__device__ __forceinline__ void frag(unsigned long long* fb, size_t p, unsigned long long w) {
  if (w < *reinterpret_cast<volatile unsigned long long*>(fb + p)) atomicMin(fb + p, w);
}

// Screen pixel and depth bits of a point with LAS integers (x, y, z); false when it is
// not drawn.  Every coordinate difference to the origin fits int32 (checked on the host
// for the origin; a point farther than 2^31 - 1 cm on an axis is outside the camera's
// range), so it is one 32-bit subtraction and conversion.  floor(s) in [0, W) is tested
// as s in [0, W), which also rejects non-finite coordinates.
__device__ __forceinline__ bool point_pixel(const Cam& c, int x, int y, int z, uint32_t& p, uint32_t& dbits) {
  const float qx = (float)(int)((uint32_t)x - (uint32_t)c.ox);
  const float qy = (float)(int)((uint32_t)y - (uint32_t)c.oy);
  const float qz = (float)(int)((uint32_t)z - (uint32_t)c.oz);
  float cl[4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    cl[r] = f_add(f_add(f_add(f_mul(c.M[4 * r], qx), f_mul(c.M[4 * r + 1], qy)), f_mul(c.M[4 * r + 2], qz)),
                  c.M[4 * r + 3]);
  const float W = (float)c.W, H = (float)c.H;
  const float sx = f_mul(f_add(f_mul(f_div(cl[0], cl[3]), 0.5f), 0.5f), W);
  const float sy = f_mul(f_add(f_mul(f_div(cl[1], cl[3]), 0.5f), 0.5f), H);
  const float d = f_add(f_mul(f_div(cl[2], cl[3]), 0.5f), 0.5f);
  p = (uint32_t)(int)fmaxf(0.f, fminf(sy, H - 1.f)) * (uint32_t)c.W + (uint32_t)(int)fmaxf(0.f, fminf(sx, W - 1.f));
  dbits = __float_as_uint(d);
  return cl[3] > 0.f && d >= 0.f && d <= 1.f && sx >= 0.f && sx < W && sy >= 0.f && sy < H;
}

// The fragment of point i after its pixel's word `cur` was read: a fragment strictly
// behind that word cannot win (words only decrease) and never loads its colour.
template <typename Index>
__device__ __forceinline__ void point_fragment(const ls_points& pts, unsigned long long* fb, Index i, uint32_t p,
                                               uint32_t dbits, unsigned long long cur) {
  if (dbits > (uint32_t)(cur >> 32)) return;
  const uint32_t col = to8(pts.r[i]) | (to8(pts.g[i]) << 8) | (to8(pts.b[i]) << 16) | (255u << 24);
  const unsigned long long w = ((unsigned long long)dbits << 32) | col;
  if (w < cur) atomicMin(fb + p, w);
}

// Four consecutive points per thread: their coordinates come with one 16-byte load per
// array (the arrays are 16-byte aligned: VEC), the four pixel reads are issued together,
// then the fragments; the tail (and unaligned arrays) go point by point.
template <typename Index, bool VEC>
__global__ void __launch_bounds__(kRenderThreads) k_render_points(ls_points pts, Cam c, unsigned long long* fb) {
  const Index n = (Index)pts.n, tid = (Index)blockIdx.x * blockDim.x + threadIdx.x;
  const Index threads = (Index)gridDim.x * blockDim.x;
  const volatile unsigned long long* vfb = fb;
  Index done = 0;
  if (VEC) {
    const Index groups = n / 4;
    for (Index g = tid; g < groups; g += threads) {
      const int4 x = __ldcs(reinterpret_cast<const int4*>(pts.x) + g);
      const int4 y = __ldcs(reinterpret_cast<const int4*>(pts.y) + g);
      const int4 z = __ldcs(reinterpret_cast<const int4*>(pts.z) + g);
      const int xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w}, zs[4] = {z.x, z.y, z.z, z.w};
      uint32_t p[4], db[4];
      bool on[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) on[k] = point_pixel(c, xs[k], ys[k], zs[k], p[k], db[k]);
      unsigned long long cur[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cur[k] = on[k] ? vfb[p[k]] : 0ull;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (on[k]) point_fragment(pts, fb, 4 * g + k, p[k], db[k], cur[k]);
    }
    done = groups * 4;
  }
  for (Index i = done + tid; i < n; i += threads) {
    uint32_t p, db;
    if (point_pixel(c, pts.x[i], pts.y[i], pts.z[i], p, db)) point_fragment(pts, fb, i, p, db, vfb[p]);
  }
}

// One triangle: screen vertices and 8-bit colours.
struct Tri {
  float x[3], y[3], d[3];
  float r[3], g[3], b[3];
};

struct TriSetup {
  float A;        // |signed area|, > 0
  float sign;     // the sign that makes the edge functions non-negative inside
  int ixa, ixb, iya, iyb;
  bool ok;
};

__device__ __forceinline__ TriSetup tri_setup(const Tri& t, int W, int H) {
  TriSetup s;
  const float A = f_sub(f_mul(f_sub(t.x[1], t.x[0]), f_sub(t.y[2], t.y[0])),
                        f_mul(f_sub(t.y[1], t.y[0]), f_sub(t.x[2], t.x[0])));
  s.ok = finite_f(A) && A != 0.f;
  s.sign = A < 0.f ? -1.f : 1.f;
  s.A = fabsf(A);
  // candidate pixels floor(min) .. floor(max), clamped to the framebuffer (the
  // coordinates of kept vertices are finite)
  const float xmin = fminf(t.x[0], fminf(t.x[1], t.x[2])), xmax = fmaxf(t.x[0], fmaxf(t.x[1], t.x[2]));
  const float ymin = fminf(t.y[0], fminf(t.y[1], t.y[2])), ymax = fmaxf(t.y[0], fmaxf(t.y[1], t.y[2]));
  s.ixa = (int)fmaxf(0.f, floorf(fminf(xmin, (float)W)));
  s.ixb = (int)fminf((float)(W - 1), floorf(fmaxf(xmax, -1.f)));
  s.iya = (int)fmaxf(0.f, floorf(fminf(ymin, (float)H)));
  s.iyb = (int)fminf((float)(H - 1), floorf(fmaxf(ymax, -1.f)));
  s.ok = s.ok && s.ixa <= s.ixb && s.iya <= s.iyb;
  return s;
}

__device__ __forceinline__ void tri_pixel(const Tri& t, const TriSetup& s, int ix, int iy, int W,
                                          unsigned long long* fb) {
  const float px = f_add((float)ix, 0.5f), py = f_add((float)iy, 0.5f);
  float e0 = f_sub(f_mul(f_sub(t.x[2], t.x[1]), f_sub(py, t.y[1])), f_mul(f_sub(t.y[2], t.y[1]), f_sub(px, t.x[1])));
  float e1 = f_sub(f_mul(f_sub(t.x[0], t.x[2]), f_sub(py, t.y[2])), f_mul(f_sub(t.y[0], t.y[2]), f_sub(px, t.x[2])));
  float e2 = f_sub(f_mul(f_sub(t.x[1], t.x[0]), f_sub(py, t.y[0])), f_mul(f_sub(t.y[1], t.y[0]), f_sub(px, t.x[0])));
  e0 *= s.sign;
  e1 *= s.sign;
  e2 *= s.sign;
  if (!(e0 >= 0.f && e1 >= 0.f && e2 >= 0.f)) return;
  const float l0 = f_div(e0, s.A), l1 = f_div(e1, s.A), l2 = f_div(e2, s.A);
  const float d = f_add(f_add(f_mul(l0, t.d[0]), f_mul(l1, t.d[1])), f_mul(l2, t.d[2]));
  const float* cs[3] = {t.r, t.g, t.b};
  uint32_t col = 255u << 24;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float v = floorf(f_add(f_add(f_add(f_mul(l0, cs[k][0]), f_mul(l1, cs[k][1])), f_mul(l2, cs[k][2])), 0.5f));
    col |= (uint32_t)fminf(255.f, fmaxf(0.f, v)) << (8 * k);
  }
  frag(fb, (size_t)iy * W + ix, ((unsigned long long)__float_as_uint(d) << 32) | col);
}

struct MeshArgs {
  const float* __restrict__ height;
  const uint8_t* __restrict__ rgb;
  const int32_t* __restrict__ tile_ids;
  int64_t n, quads;  // heightmaps; quads in all of them
  int res, cell, tile_cm, tiles_x, tiles_y;
  // quad index -> heightmap and texel by 32-bit division by invariants when every quad
  // index fits 32 bits (a 64-bit division is a long routine, partly on the FP64 pipe)
  int q32;
  FastDiv div_qsq, div_qs;
  long long x0, y0;
  float zo, izs, ozf;
  Cam c;
  unsigned long long* fb;
};

// Vertex (texel centre) i, j of heightmap o.
__device__ __forceinline__ Vtx mesh_vertex(const MeshArgs& a, int64_t o, int tx, int ty, int i, int j, float& r,
                                           float& g, float& b) {
  const size_t e = (size_t)o * a.res * a.res + (size_t)i * a.res + j;
  const long long xc = a.x0 + (long long)tx * a.tile_cm + (long long)a.cell * j + a.cell / 2;
  const long long yc = a.y0 + (long long)ty * a.tile_cm + (long long)a.cell * i + a.cell / 2;
  const float qz = f_sub(f_mul(f_sub(a.height[e], a.zo), a.izs), a.ozf);
  r = (float)a.rgb[3 * e];
  g = (float)a.rgb[3 * e + 1];
  b = (float)a.rgb[3 * e + 2];
  return project(a.c, f_of(xc - a.c.ox), f_of(yc - a.c.oy), qz);
}

// Quad q: its heightmap, tile and texel (i, j); false (with the status set) for a bad
// tile id.
__device__ __forceinline__ bool mesh_quad_at(const MeshArgs& a, int64_t q, int64_t& o, int& tx, int& ty, int& i,
                                             int& j) {
  const int qs = a.res - 1;
  int rem;
  if (a.q32) {
    const uint32_t oq = fdiv((uint32_t)q, a.div_qsq);
    rem = (int)((uint32_t)q - oq * (uint32_t)(qs * qs));
    o = oq;
    i = (int)fdiv((uint32_t)rem, a.div_qs);
  } else {
    o = q / ((int64_t)qs * qs);
    rem = (int)(q - o * qs * qs);
    i = rem / qs;
  }
  j = rem - i * qs;
  const int tile = a.tile_ids ? a.tile_ids[o] : (int)o;
  if (tile < 0 || tile >= a.tiles_x * a.tiles_y) {
    set_status(LS_ERR_INVALID_ARG);
    return false;
  }
  tx = tile % a.tiles_x;
  ty = tile / a.tiles_x;
  return true;
}

// Corners c = 0..3 of a quad in the order v00, v01, v11, v10 (row offset c >> 1,
// column offset 1 for c = 1, 2); triangle `half` (0: v00 v01 v11, 1: v00 v11 v10)
// takes the corners 0, 1 + half, 2 + half.
__device__ __forceinline__ int corner_di(int c) { return c >> 1; }
__device__ __forceinline__ int corner_dj(int c) { return ((c + 1) >> 1) & 1; }
__device__ __forceinline__ int tri_corner(int half, int k) { return k == 0 ? 0 : k + half; }

// The four projected corners of quad q (each vertex projected once for both triangles).
struct Quad {
  Vtx v[4];
  float r[4], g[4], b[4];
};

__device__ __forceinline__ bool mesh_quad(const MeshArgs& a, int64_t q, Quad& Q) {
  int64_t o;
  int tx, ty, i, j;
  if (!mesh_quad_at(a, q, o, tx, ty, i, j)) return false;
#pragma unroll
  for (int k = 0; k < 4; ++k) Q.v[k] = mesh_vertex(a, o, tx, ty, i + corner_di(k), j + corner_dj(k), Q.r[k], Q.g[k], Q.b[k]);
  return true;
}

// Triangle `half` of a projected quad; false when a vertex is not kept.  The corners
// are chosen with selects, so the quad stays in registers.
__device__ __forceinline__ void quad_corner(const Quad& Q, int c, Tri& t, int k, bool& ok) {
  t.x[k] = Q.v[c].x;
  t.y[k] = Q.v[c].y;
  t.d[k] = Q.v[c].d;
  t.r[k] = Q.r[c];
  t.g[k] = Q.g[c];
  t.b[k] = Q.b[c];
  ok = ok && Q.v[c].kept;
}

__device__ __forceinline__ bool quad_tri(const Quad& Q, int half, Tri& t) {
  bool ok = true;
  quad_corner(Q, 0, t, 0, ok);
  if (half) {
    quad_corner(Q, 2, t, 1, ok);
    quad_corner(Q, 3, t, 2, ok);
  } else {
    quad_corner(Q, 1, t, 1, ok);
    quad_corner(Q, 2, t, 2, ok);
  }
  return ok;
}

// Triangle `half` of quad q, projected on its own (the CTA-wide path of large
// triangles).
__device__ __forceinline__ bool mesh_tri(const MeshArgs& a, int64_t q, int half, Tri& t) {
  int64_t o;
  int tx, ty, i, j;
  if (!mesh_quad_at(a, q, o, tx, ty, i, j)) return false;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = tri_corner(half, k);
    const Vtx v = mesh_vertex(a, o, tx, ty, i + corner_di(c), j + corner_dj(c), t.r[k], t.g[k], t.b[k]);
    t.x[k] = v.x;
    t.y[k] = v.y;
    t.d[k] = v.d;
    ok = ok && v.kept;
  }
  return ok;
}

__global__ void __launch_bounds__(kMeshThreads) k_render_mesh(MeshArgs a) {
  __shared__ unsigned long long queue[2 * kMeshThreads];  // (quad << 1) | half
  __shared__ int qn;
  const int64_t total = a.quads;
  for (int64_t base = (int64_t)blockIdx.x * kMeshThreads; base < total; base += (int64_t)gridDim.x * kMeshThreads) {
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    const int64_t q = base + threadIdx.x;
    Quad Q;
    if (q < total && mesh_quad(a, q, Q)) {
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        Tri t;
        if (!quad_tri(Q, half, t)) continue;
        const TriSetup s = tri_setup(t, a.c.W, a.c.H);
        if (!s.ok) continue;
        const long long cand = (long long)(s.ixb - s.ixa + 1) * (s.iyb - s.iya + 1);
        if (cand > kLargeTri) {
          queue[atomicAdd(&qn, 1)] = ((unsigned long long)q << 1) | (unsigned)half;
          continue;
        }
        for (int iy = s.iya; iy <= s.iyb; ++iy)
          for (int ix = s.ixa; ix <= s.ixb; ++ix) tri_pixel(t, s, ix, iy, a.c.W, a.fb);
      }
    }
    __syncthreads();
    // large triangles: the whole CTA, one after the other
    const int nq = qn;
    for (int k = 0; k < nq; ++k) {
      const unsigned long long e = queue[k];
      Tri t;
      if (!mesh_tri(a, (int64_t)(e >> 1), (int)(e & 1u), t)) continue;  // uniform: same entry
      const TriSetup s = tri_setup(t, a.c.W, a.c.H);
      const int bw = s.ixb - s.ixa + 1;
      const long long cand = (long long)bw * (s.iyb - s.iya + 1);
      for (long long p = threadIdx.x; p < cand; p += kMeshThreads)
        tri_pixel(t, s, s.ixa + (int)(p % bw), s.iya + (int)(p / bw), a.c.W, a.fb);
    }
    __syncthreads();
  }
}

__global__ void k_render_resolve(const unsigned long long* __restrict__ fb, int64_t n, uint32_t background,
                          uint32_t* __restrict__ rgba) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long w = fb[p];
    rgba[p] = w == ~0ull ? background : (uint32_t)w;
  }
}

bool make_cam(const ls_camera* cam, Cam& c) {
  if (!cam || cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384) return false;
  c.ox = cam->origin_cm[0];
  c.oy = cam->origin_cm[1];
  c.oz = cam->origin_cm[2];
  for (int k = 0; k < 16; ++k) c.M[k] = cam->view_proj[k];
  c.W = cam->width;
  c.H = cam->height;
  return true;
}

}  // namespace
}  // namespace ls

using namespace ls;

extern "C" ls_status ls_render_clear(uint64_t* fb, int32_t width, int32_t height, ls_stream_t stream) {
  if (!fb || width < 1 || height < 1 || width > 16384 || height > 16384) return LS_ERR_INVALID_ARG;
  LS_CUDA_TRY(cudaMemsetAsync(fb, 0xff, (size_t)width * height * sizeof(uint64_t),
                              reinterpret_cast<cudaStream_t>(stream)));
  return LS_OK;
}

extern "C" ls_status ls_render_points(const ls_points* pts, const ls_camera* camera, uint64_t* fb,
                                      ls_stream_t stream) {
  Cam c;
  if (!pts || !fb || !make_cam(camera, c) || pts->n < 0) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(fb) & 7u) return LS_ERR_INVALID_ARG;
  if (pts->n == 0) return LS_OK;
  if (!pts->x || !pts->y || !pts->z || !pts->r || !pts->g || !pts->b) return LS_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k)
    if (camera->origin_cm[k] < INT32_MIN || camera->origin_cm[k] > INT32_MAX) return LS_ERR_INVALID_ARG;
  const int grid = grid_cap((pts->n / 4 + kRenderThreads - 1) / kRenderThreads, kSmCount * 8);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* f = reinterpret_cast<unsigned long long*>(fb);
  const bool vec = ((reinterpret_cast<uintptr_t>(pts->x) | reinterpret_cast<uintptr_t>(pts->y) |
                     reinterpret_cast<uintptr_t>(pts->z)) & 15u) == 0;
  if (pts->n < (int64_t(1) << 31) - (int64_t)grid * kRenderThreads * 4) {
    if (vec) k_render_points<int, true><<<grid, kRenderThreads, 0, s>>>(*pts, c, f);
    else k_render_points<int, false><<<grid, kRenderThreads, 0, s>>>(*pts, c, f);
  } else {
    if (vec) k_render_points<long long, true><<<grid, kRenderThreads, 0, s>>>(*pts, c, f);
    else k_render_points<long long, false><<<grid, kRenderThreads, 0, s>>>(*pts, c, f);
  }
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_render_heightmaps(const float* height, const uint8_t* rgb, const int32_t* tile_ids,
                                          int64_t n, int32_t res, const ls_region* region,
                                          const ls_camera* camera, uint64_t* fb, ls_stream_t stream) {
  Cam c;
  if (!height || !rgb || !region || !fb || !make_cam(camera, c) || n < 0) return LS_ERR_INVALID_ARG;
  if (res < 2 || res > 1024 || region->tile_cm <= 0 || region->tile_cm % res) return LS_ERR_INVALID_ARG;
  if (region->tiles_x <= 0 || region->tiles_y <= 0 || !(region->z_scale != 0.0)) return LS_ERR_INVALID_ARG;
  if (!tile_ids && n > (int64_t)region->tiles_x * region->tiles_y) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(fb) & 7u) return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  MeshArgs a;
  a.height = height;
  a.rgb = rgb;
  a.tile_ids = tile_ids;
  a.n = n;
  a.quads = n * (int64_t)(res - 1) * (res - 1);
  a.q32 = a.quads + kMeshThreads < (int64_t(1) << 32);
  a.div_qsq = make_fastdiv((uint32_t)((res - 1) * (res - 1)));
  a.div_qs = make_fastdiv((uint32_t)(res - 1));
  a.res = res;
  a.cell = region->tile_cm / res;
  a.tile_cm = region->tile_cm;
  a.tiles_x = region->tiles_x;
  a.tiles_y = region->tiles_y;
  a.x0 = region->x0_cm;
  a.y0 = region->y0_cm;
  a.zo = (float)region->z_offset;
  a.izs = (float)(1.0 / region->z_scale);
  a.ozf = (float)camera->origin_cm[2];
  a.c = c;
  a.fb = reinterpret_cast<unsigned long long*>(fb);
  k_render_mesh<<<grid_cap((a.quads + kMeshThreads - 1) / kMeshThreads, kSmCount * 12), kMeshThreads, 0,
           reinterpret_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_render_resolve(const uint64_t* fb, int32_t width, int32_t height, uint32_t background,
                                       uint8_t* rgba, ls_stream_t stream) {
  if (!fb || !rgba || width < 1 || height < 1 || width > 16384 || height > 16384) return LS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(fb) & 7u) || (reinterpret_cast<uintptr_t>(rgba) & 3u)) return LS_ERR_INVALID_ARG;
  const int64_t n = (int64_t)width * height;
  k_render_resolve<<<grid_cap((n + 255) / 256, kSmCount * 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const unsigned long long*>(fb), n, background, reinterpret_cast<uint32_t*>(rgba));
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
