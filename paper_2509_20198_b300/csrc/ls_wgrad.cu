// Weight and bias gradients of a 3x3 convolution on the tensor cores (training of the
// learned filler, Sec. 3.4).  dW^T[k][o] = sum_p X_shift(k)[p] dZ[p][o] with
// k = tap * C_in + c_in: a GEMM with M = 9*C_in (tiles of 128 rows), N = C_out and
// K = pixels.  Both operands are stored pixel-minor (NHWC), so the CUDA-core warps
// transpose them into K-major shared-memory tiles (one 16-byte global load feeds an
// 8-row column of a core matrix); one thread issues tcgen05.mma kind::f16 with the
// FP32 accumulator in TMEM.  Each CTA owns one 128-row tile and one slice of
// pixels; partial sums are added into the FP32 gradient with atomics.
#include <cuda_bf16.h>

#include "ls_tc.cuh"

namespace ls {
namespace {

constexpr int kWgThreads = 160;        // warps 0-3 stage + epilogue, warp 4 issues MMAs
constexpr int kWgStages = 3;
constexpr int kWgPix = 64;             // pixels (K) per stage
constexpr int kWgABytes = 128 * kWgPix * 2;

struct WgArgs {
  const uint16_t* __restrict__ x;   // layer input  [P][cin]
  const uint16_t* __restrict__ dz;  // output grad  [P][cout] (ReLU-masked)
  float* __restrict__ dwt;          // [9*cin][cout] fp32, accumulated
  float* __restrict__ db;           // [cout] fp32, accumulated (m-tile 0 only)
  int32_t n, h, w, cin, cout, rows;  // rows = 9*cin
  int64_t pix_total, pix_per_cta;
  int32_t n_mtiles;
  uint32_t idesc, tmem_cols;
};

__global__ void __launch_bounds__(kWgThreads, 1) k_wgrad(const WgArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ float dbs[256];
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const uint32_t b_bytes = (uint32_t)a.cout * kWgPix * 2;
  const uint32_t stage_bytes = kWgABytes + b_bytes;
  const int mt = blockIdx.x % a.n_mtiles;
  const int64_t slice = blockIdx.x / a.n_mtiles;
  const int64_t p_begin = slice * a.pix_per_cta;
  const int64_t p_end = min(p_begin + a.pix_per_cta, a.pix_total);
  const int n_steps = (int)((p_end - p_begin + kWgPix - 1) / kWgPix);
  const int m0 = mt * 128;

  if (tid == 0) {
    for (int i = 0; i < kWgStages; ++i) {
      tc::mbar_init(&full[i], 128);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (tid < 256) dbs[tid] = 0.f;
  if (warp == 4) tc::tmem_alloc(&tmem_base, a.tmem_cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;

  if (warp < 4) {
    // ---------------- staging (128 threads)
    const int og_n = a.cout / 8;
    const int og = tid % og_n;           // fixed output-channel group: bias partials in registers
    float dbp[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = 0; s < n_steps && !abort_flag; ++s) {
      const int slot = s % kWgStages;
      const uint32_t ph = (uint32_t)(s / kWgStages) & 1u;
      if (!tc::mbar_wait(&empty[slot], ph ^ 1u)) { abort_flag = 1; break; }
      uint8_t* A = smem + (size_t)slot * stage_bytes;
      uint8_t* B = A + kWgABytes;
      const int64_t p0 = p_begin + (int64_t)s * kWgPix;
      // A: 16 row groups x 64 pixels; element (k_l, p_l) at
      //    (k_l/8)*128 + (p_l/8)*2048 + (k_l%8)*16 + (p_l%8)*2
      for (int e = tid; e < 16 * kWgPix; e += 128) {
        const int g = e / kWgPix, pl = e - g * kWgPix;
        const int64_t p = p0 + pl;
        const int k = m0 + g * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p < p_end && k < a.rows) {
          const int tap = k / a.cin, ci = k - tap * a.cin;
          const int ky = tap / 3, kx = tap - ky * 3;
          const int64_t hw = (int64_t)a.h * a.w;
          const int64_t nn = p / hw;
          const int rem = (int)(p - nn * hw);
          const int yy = rem / a.w + ky - 1, xx = rem % a.w + kx - 1;
          if (yy >= 0 && yy < a.h && xx >= 0 && xx < a.w)
            v = *reinterpret_cast<const uint4*>(a.x + ((nn * a.h + yy) * a.w + xx) * a.cin + ci);
        }
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
        uint16_t* base = reinterpret_cast<uint16_t*>(A + g * 128 + (pl >> 3) * 2048) + (pl & 7);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          base[(2 * j) * 8] = (uint16_t)(vv[j] & 0xffffu);
          base[(2 * j + 1) * 8] = (uint16_t)(vv[j] >> 16);
        }
      }
      // B: C_out/8 row groups x 64 pixels; element (o, p_l) at
      //    (o/8)*128 + (p_l/8)*(C_out*16) + (o%8)*16 + (p_l%8)*2
      for (int e = tid; e < og_n * kWgPix; e += 128) {
        const int pl = e / og_n;  // og == e % og_n == tid % og_n (128 is a multiple of og_n)
        const int64_t p = p0 + pl;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p < p_end) v = *reinterpret_cast<const uint4*>(a.dz + p * a.cout + og * 8);
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
        uint16_t* base = reinterpret_cast<uint16_t*>(B + og * 128 + (pl >> 3) * (a.cout * 16)) + (pl & 7);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint16_t lo = (uint16_t)(vv[j] & 0xffffu), hi = (uint16_t)(vv[j] >> 16);
          base[(2 * j) * 8] = lo;
          base[(2 * j + 1) * 8] = hi;
          dbp[2 * j] += __uint_as_float((uint32_t)lo << 16);
          dbp[2 * j + 1] += __uint_as_float((uint32_t)hi << 16);
        }
      }
      // generic-proxy writes must be visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_arrive(&full[slot]);
    }
    if (mt == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) atomicAdd(&dbs[og * 8 + j], dbp[j]);
    }
    // ---------------- epilogue: TMEM row (k) per thread, atomics into dW^T
    if (n_steps > 0 && !abort_flag && tc::mbar_wait(&done, 0)) {
      tc::fence_after();
      const int row = (warp & 3) * 32 + lane;
      const int k = m0 + row;
      for (int c0 = 0; c0 < a.cout; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
        if (k < a.rows) {
#pragma unroll
          for (int i = 0; i < 16; ++i) atomicAdd(&a.dwt[(int64_t)k * a.cout + c0 + i], v[i]);
        }
      }
    }
  } else if (warp == 4 && lane == 0) {
    // ---------------- MMA issuer
    for (int s = 0; s < n_steps && !abort_flag; ++s) {
      const int slot = s % kWgStages;
      const uint32_t ph = (uint32_t)(s / kWgStages) & 1u;
      if (!tc::mbar_wait(&full[slot], ph)) { abort_flag = 1; break; }
      tc::fence_after();
      const uint32_t A = tc::saddr(smem + (size_t)slot * stage_bytes);
      const uint32_t B = A + kWgABytes;
#pragma unroll
      for (int j = 0; j < kWgPix / 16; ++j) {
        const uint64_t ad = tc::sdesc(A + j * 2 * 2048, 2048, 128);
        const uint64_t bd = tc::sdesc(B + j * 2 * (a.cout * 16), a.cout * 16, 128);
        tc::mma_bf16(taddr, ad, bd, a.idesc, (s > 0 || j > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[slot]);
    }
    if (n_steps > 0) tc::mma_commit(&done);
  }
  tc::fence_before();
  __syncthreads();
  if (mt == 0 && tid < a.cout && a.db) atomicAdd(&a.db[tid], dbs[tid]);
  if (warp == 4) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, a.tmem_cols);
  }
}

}  // namespace

// Accumulates into dwt ([9*cin][cout], fp32) and db ([cout], may be NULL).
ls_status wgrad_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cin, int cout, float* dwt,
                       float* db, cudaStream_t stream) {
  if (!x || !dz || !dwt || n <= 0) return LS_ERR_INVALID_ARG;
  if (cin % 8 || cout < 16 || cout > 128 || cout % 16) return LS_ERR_UNSUPPORTED;
  WgArgs a = {};
  a.x = x; a.dz = dz; a.dwt = dwt; a.db = db;
  a.n = n; a.h = h; a.w = w; a.cin = cin; a.cout = cout; a.rows = 9 * cin;
  a.pix_total = (int64_t)n * h * w;
  a.n_mtiles = (a.rows + 127) / 128;
  // about 2 waves of CTAs over the SMs, slices a multiple of the stage
  int64_t slices = (2 * kSmCount + a.n_mtiles - 1) / a.n_mtiles;
  int64_t per = (a.pix_total + slices - 1) / slices;
  per = (per + kWgPix - 1) / kWgPix * kWgPix;
  if (per < 1024) per = 1024;
  a.pix_per_cta = per;
  slices = (a.pix_total + per - 1) / per;
  a.idesc = tc::idesc_bf16(128, cout);
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < cout) a.tmem_cols <<= 1;
  const size_t smem = (size_t)kWgStages * (kWgABytes + cout * kWgPix * 2);
  static bool attr_set[64] = {};
  int dev = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    LS_CUDA_TRY(cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kWgStages * (kWgABytes + 128 * kWgPix * 2)));
    attr_set[dev] = true;
  }
  k_wgrad<<<(unsigned)(slices * a.n_mtiles), kWgThreads, smem, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace ls

extern "C" ls_status ls_conv3x3_wgrad(const uint16_t* x, const uint16_t* dz, const ls_conv_shape* shape, float* dw,
                                      float* db, ls_stream_t stream) {
  if (!shape) return LS_ERR_INVALID_ARG;
  return ls::wgrad_launch(x, dz, shape->n, shape->h, shape->w, shape->cin, shape->cout, dw, db,
                          reinterpret_cast<cudaStream_t>(stream));
}
