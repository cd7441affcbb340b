// Seeded synthetic point generator on the GPU: the same integer definition as the
// numpy generator in synth/__init__.py (SplitMix64 counter hash, value-noise fBm
// terrain, 8 m strip stream order, height-ramp RGB with Irwin-Hall noise), so both
// produce bit-identical points.  Input generation only: no arithmetic of the
// heightmap method lives here.  Built as its own shared library (libsynth.so).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kC1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kC2 = 0x94D049BB133111EBull;
constexpr uint64_t kSaltTerrain = 0x5445525241494E31ull;
constexpr uint64_t kSaltPoints = 0x504F494E54535F31ull;
constexpr int kStrips = 80;
constexpr int64_t kStripCm = 800;
constexpr int64_t kZBase = 50000;
constexpr int kOctaves = 6;
constexpr int64_t kAmp0 = 8000;
constexpr int64_t kLambda0 = 200000;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += kGolden;
  z = (z ^ (z >> 30)) * kC1;
  z = (z ^ (z >> 27)) * kC2;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t H(uint64_t s, uint64_t v) { return mix64(s + mix64(v)); }

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int64_t fade_q16(int64_t t) { return (t * t * (3 * 65536 - 2 * t)) >> 32; }

__device__ __forceinline__ int64_t lattice(uint64_t seed, int o, int64_t ix, int64_t iy) {
  uint64_t h = H(H(H(seed ^ kSaltTerrain, (uint64_t)o), (uint64_t)ix), (uint64_t)iy);
  return (int64_t)(h >> 48) - 32768;
}

__device__ int64_t terrain_z(uint64_t seed, int64_t x, int64_t y) {
  int64_t z = 0;
#pragma unroll 1
  for (int o = 0; o < kOctaves; ++o) {
    const int64_t lam = kLambda0 >> o;
    const int64_t ix = floor_div(x, lam), iy = floor_div(y, lam);
    const int64_t fx = fade_q16(((x - ix * lam) << 16) / lam);
    const int64_t fy = fade_q16(((y - iy * lam) << 16) / lam);
    const int64_t v00 = lattice(seed, o, ix, iy), v10 = lattice(seed, o, ix + 1, iy);
    const int64_t v01 = lattice(seed, o, ix, iy + 1), v11 = lattice(seed, o, ix + 1, iy + 1);
    const int64_t a = v00 + (((v10 - v00) * fx) >> 16);
    const int64_t b = v01 + (((v11 - v01) * fx) >> 16);
    const int64_t n = a + (((b - a) * fy) >> 16);
    z += ((kAmp0 >> o) * n) >> 15;
  }
  return z;
}

__device__ __forceinline__ int64_t strip_of(int64_t idx, int64_t n_points) {
  const int64_t q = n_points / kStrips, rem = n_points % kStrips;
  if (q == 0) return idx;
  const int64_t big = rem * (q + 1);
  return idx < big ? idx / (q + 1) : rem + (idx - big) / q;
}

__device__ __forceinline__ int64_t irwin_hall(uint64_t base, int lane0) {
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint64_t h = H(base, (uint64_t)(lane0 + k));
#pragma unroll
    for (int j = 0; j < 4; ++j) s += (int64_t)((h >> (16 * j)) & 0xFFFFull);
  }
  return ((s - 393210) * 2000) >> 16;  // floor division by 65536
}

struct Pt { int32_t x, y, z; uint16_t r, g, b; };

__device__ Pt point_at(uint64_t seed, int64_t x0, int64_t y0, int64_t tile_cm, int64_t tiles_x,
                       int64_t tile, int64_t n_points, int64_t idx) {
  const int64_t tx = tile % tiles_x, ty = tile / tiles_x;
  const uint64_t key = H(seed ^ kSaltPoints, (uint64_t)tile);
  const uint64_t base = H(key, (uint64_t)idx);
  const int64_t s = strip_of(idx, n_points);
  const int64_t lx = (int64_t)(H(base, 0) % (uint64_t)tile_cm);
  const int64_t ly = s * kStripCm + (int64_t)(H(base, 1) % (uint64_t)kStripCm);
  const int64_t gx = x0 + tx * tile_cm + lx, gy = y0 + ty * tile_cm + ly;
  const int64_t zn = (int64_t)(H(base, 2) >> 59) - 16;
  const int64_t z = kZBase + terrain_z(seed, gx, gy) + zn;
  int64_t zc = z - 34000;
  zc = zc < 0 ? 0 : (zc > 32000 ? 32000 : zc);
  const int64_t q = zc * 65535 / 32000;
  const int64_t ramp[3] = {q, q / 2 + 16384, 65535 - q};
  uint16_t c[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    int64_t v = ramp[ch] + irwin_hall(base, 3 + 3 * ch);
    v = v < 0 ? 0 : (v > 65535 ? 65535 : v);
    c[ch] = (uint16_t)v;
  }
  return Pt{(int32_t)gx, (int32_t)gy, (int32_t)z, c[0], c[1], c[2]};
}

__device__ __forceinline__ int64_t find_tile(const int64_t* offs, int64_t n_tiles, int64_t i) {
  int64_t lo = 0, hi = n_tiles - 1;  // last t with offs[t] <= i
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_points(uint64_t seed, int64_t x0, int64_t y0, int64_t tile_cm, int64_t tiles_x,
                         const int64_t* __restrict__ offs, int64_t n_tiles, int64_t total,
                         int32_t* __restrict__ x, int32_t* __restrict__ y, int32_t* __restrict__ z,
                         uint16_t* __restrict__ r, uint16_t* __restrict__ g, uint16_t* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = find_tile(offs, n_tiles, i);
    const Pt p = point_at(seed, x0, y0, tile_cm, tiles_x, t, offs[t + 1] - offs[t], i - offs[t]);
    x[i] = p.x; y[i] = p.y; z[i] = p.z; r[i] = p.r; g[i] = p.g; b[i] = p.b;
  }
}

// samples: sample k of tile t = stream point chunk*k; sample_offs is the CSR of samples.
__global__ void k_samples(uint64_t seed, int64_t x0, int64_t y0, int64_t tile_cm, int64_t tiles_x,
                          const int64_t* __restrict__ counts, const int64_t* __restrict__ sample_offs,
                          int64_t n_tiles, int64_t chunk, int64_t total,
                          int32_t* __restrict__ x, int32_t* __restrict__ y, int32_t* __restrict__ z,
                          uint16_t* __restrict__ r, uint16_t* __restrict__ g, uint16_t* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = find_tile(sample_offs, n_tiles, i);
    const int64_t k = i - sample_offs[t];
    const Pt p = point_at(seed, x0, y0, tile_cm, tiles_x, t, counts[t], k * chunk);
    x[i] = p.x; y[i] = p.y; z[i] = p.z; r[i] = p.r; g[i] = p.g; b[i] = p.b;
  }
}

int grid_for(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  if (blocks > 148 * 64) blocks = 148 * 64;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

extern "C" {

// All array pointers are device pointers. tile_offsets: int64[n_tiles+1] (device).
int synth_region_points(uint64_t seed, int64_t x0_cm, int64_t y0_cm, int64_t tile_cm, int64_t tiles_x,
                        const int64_t* tile_offsets, int64_t n_tiles, int64_t total,
                        int32_t* x, int32_t* y, int32_t* z, uint16_t* r, uint16_t* g, uint16_t* b,
                        cudaStream_t stream) {
  if (total <= 0) return 0;
  if (n_tiles <= 0 || tiles_x <= 0 || tile_cm <= 0) return -1;
  k_points<<<grid_for(total), 256, 0, stream>>>(seed, x0_cm, y0_cm, tile_cm, tiles_x, tile_offsets,
                                                 n_tiles, total, x, y, z, r, g, b);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// counts: int64[n_tiles] points per tile (device); sample_offsets: int64[n_tiles+1] (device).
int synth_region_samples(uint64_t seed, int64_t x0_cm, int64_t y0_cm, int64_t tile_cm, int64_t tiles_x,
                         const int64_t* counts, const int64_t* sample_offsets, int64_t n_tiles,
                         int64_t chunk, int64_t total,
                         int32_t* x, int32_t* y, int32_t* z, uint16_t* r, uint16_t* g, uint16_t* b,
                         cudaStream_t stream) {
  if (total <= 0) return 0;
  if (n_tiles <= 0 || tiles_x <= 0 || tile_cm <= 0 || chunk <= 0) return -1;
  k_samples<<<grid_for(total), 256, 0, stream>>>(seed, x0_cm, y0_cm, tile_cm, tiles_x, counts,
                                                  sample_offsets, n_tiles, chunk, total,
                                                  x, y, z, r, g, b);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // extern "C"
