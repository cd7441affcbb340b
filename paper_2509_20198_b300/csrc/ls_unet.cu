// The learned heightmap filler: a U-Net (the paper's network, Sec. 3.4, is
// "inspired by the U-Net"; this one has L levels of two 3x3 conv + ReLU each, 2x2
// max pooling, 2x nearest upsampling, skip concatenation [upsampled, skip] and a
// 1x1 head with 5 outputs).  Native runtime: layer table, packed tensor-core weights,
// activations for the largest batch, forward, backward (dgrad through the tcgen05
// conv with transposed/flipped weights, wgrad through the tcgen05 weight-gradient
// GEMM), the masked and clipped MSE loss and AdamW of Sec. 3.4.
//
// Flat parameter layout (fp32, caller-owned): layers in the order e1a, e1b, ...,
// eLa, eLb, d(L-1)a, d(L-1)b, ..., d1a, d1b, head; each as W[c_out][k][k][c_in]
// followed by b[c_out].  The network input has 5 channels stored padded to 8.
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <vector>

#include "ls_tc.cuh"

namespace ls {

ls_status conv3x3_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, const uint16_t* mask, int relu,
                         int n, int h, int w, int cin, int cout, uint16_t* y, cudaStream_t stream);
ls_status wgrad_launch(const uint16_t* x, const uint16_t* dz, int n, int h, int w, int cin, int cout, float* dwt,
                       float* db, cudaStream_t stream);
ls_status conv3x3_up2_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, int n, int h, int w, int cin,
                             int cout, uint16_t* y_up, cudaStream_t stream);
ls_status conv3x3_head_launch(const uint16_t* x, const uint16_t* wpk, const float* bias, int n, int h, int w, int cin,
                              int cout, uint16_t* y, const float* head, float* head_y, int head_out, int store_y,
                              cudaStream_t stream);

namespace {

constexpr int kInPad = 8;   // network input channels stored (5 used)
constexpr int kOut = 5;     // head outputs

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ void unpack8(const uint4& v, float (&f)[8]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) w[i] = (uint32_t)f2bf(f[2 * i]) | ((uint32_t)f2bf(f[2 * i + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---- 2x2 max pooling (NHWC, 8 channels per thread) --------------------------------
__global__ void k_maxpool(const uint16_t* __restrict__ x, int n, int h, int w, int c, uint16_t* __restrict__ y) {
  const int ho = h / 2, wo = w / 2, g = c / 8;
  const int64_t total = (int64_t)n * ho * wo * g;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(e % g);
    const int64_t op = e / g;
    const int xo = (int)(op % wo), yo = (int)((op / wo) % ho);
    const int64_t nn = op / ((int64_t)wo * ho);
    float m[8], v[8];
    for (int k = 0; k < 4; ++k) {
      const int64_t ip = (nn * h + 2 * yo + (k >> 1)) * w + 2 * xo + (k & 1);
      unpack8(*reinterpret_cast<const uint4*>(x + ip * c + gi * 8), v);
#pragma unroll
      for (int i = 0; i < 8; ++i) m[i] = k == 0 ? v[i] : fmaxf(m[i], v[i]);
    }
    *reinterpret_cast<uint4*>(y + op * c + gi * 8) = pack8(m);
  }
}

// ---- backward of max pooling: route to the first maximum (row-major window order),
// add the skip gradient, apply the ReLU derivative of the pooled activation ---------
__global__ void k_maxpool_bwd(const uint16_t* __restrict__ x, const uint16_t* __restrict__ dpool,
                              const uint16_t* __restrict__ dskip, int skip_stride, int skip_off, int n, int h, int w,
                              int c, uint16_t* __restrict__ dx) {
  const int ho = h / 2, wo = w / 2, g = c / 8;
  const int64_t total = (int64_t)n * ho * wo * g;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(e % g);
    const int64_t op = e / g;
    const int xo = (int)(op % wo), yo = (int)((op / wo) % ho);
    const int64_t nn = op / ((int64_t)wo * ho);
    float v[4][8], dp[8], m[8];
    int arg[8];
    unpack8(*reinterpret_cast<const uint4*>(dpool + op * c + gi * 8), dp);
    for (int k = 0; k < 4; ++k) {
      const int64_t ip = (nn * h + 2 * yo + (k >> 1)) * w + 2 * xo + (k & 1);
      unpack8(*reinterpret_cast<const uint4*>(x + ip * c + gi * 8), v[k]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (k == 0 || v[k][i] > m[i]) { m[i] = v[k][i]; arg[i] = k; }
      }
    }
    for (int k = 0; k < 4; ++k) {
      const int64_t ip = (nn * h + 2 * yo + (k >> 1)) * w + 2 * xo + (k & 1);
      float s[8], o[8];
      unpack8(*reinterpret_cast<const uint4*>(dskip + ip * skip_stride + skip_off + gi * 8), s);
#pragma unroll
      for (int i = 0; i < 8; ++i) o[i] = v[k][i] > 0.f ? s[i] + (arg[i] == k ? dp[i] : 0.f) : 0.f;
      *reinterpret_cast<uint4*>(dx + ip * c + gi * 8) = pack8(o);
    }
  }
}

// ---- 2x nearest upsampling of `up` concatenated with `skip` along channels --------
// One output row per CTA iteration; its 16-byte groups (8 channels) are spread over the
// threads in order, so loads and stores are coalesced.  The group index e of a row
// splits into pixel e / g and group e % g with a float reciprocal: e < w * g <= 2^15
// and (e + 0.5) / g lies at least 0.5 / g from an integer, far beyond the float error.
__global__ void k_upcat(const uint16_t* __restrict__ up, int cu, const uint16_t* __restrict__ skip, int cs, int n,
                        int h, int w, uint16_t* __restrict__ y) {  // h, w: output (full) size
  const int c = cu + cs, g = c / 8;
  const int row_groups = w * g;
  const int rows = n * h;
  const float inv_g = 1.f / (float)g;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int nn = r / h, yy = r - nn * h;
    const uint16_t* uprow = up + ((int64_t)nn * (h / 2) + yy / 2) * (w / 2) * cu;
    const uint16_t* skrow = skip ? skip + (int64_t)r * w * cs : nullptr;
    uint4* yrow = reinterpret_cast<uint4*>(y + (int64_t)r * w * c);
    for (int e = threadIdx.x; e < row_groups; e += blockDim.x) {
      const int xx = (int)(((float)e + 0.5f) * inv_g);
      const int gi = e - xx * g;
      uint4 v;
      if (gi * 8 < cu)
        v = *reinterpret_cast<const uint4*>(uprow + (xx / 2) * cu + gi * 8);
      else
        v = *reinterpret_cast<const uint4*>(skrow + xx * cs + gi * 8 - cu);
      yrow[e] = v;
    }
  }
}

// ---- backward of the upsampling: sum each 2x2 block of the first cu channels -------
__global__ void k_up_bwd(const uint16_t* __restrict__ dc, int c, int cu, int n, int h, int w,
                         uint16_t* __restrict__ dup) {  // h, w: low-res size
  const int g = cu / 8;
  const int64_t total = (int64_t)n * h * w * g;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(e % g);
    const int64_t p = e / g;
    const int xx = (int)(p % w), yy = (int)((p / w) % h);
    const int64_t nn = p / ((int64_t)w * h);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, v[8];
    for (int k = 0; k < 4; ++k) {
      const int64_t ip = (nn * 2 * h + 2 * yy + (k >> 1)) * (2 * w) + 2 * xx + (k & 1);
      unpack8(*reinterpret_cast<const uint4*>(dc + ip * c + gi * 8), v);
#pragma unroll
      for (int i = 0; i < 8; ++i) s[i] += v[i];
    }
    *reinterpret_cast<uint4*>(dup + p * cu + gi * 8) = pack8(s);
  }
}

// ---- 1x1 head: y[p][o] = b[o] + sum_c top[p][c] W[o][c], fp32 out -----------------
__global__ void k_head_fwd(const uint16_t* __restrict__ top, int c, const float* __restrict__ wb, int64_t P,
                           float* __restrict__ y) {
  extern __shared__ float sw[];  // [kOut*c + kOut]
  for (int i = threadIdx.x; i < kOut * c + kOut; i += blockDim.x) sw[i] = wb[i];
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float acc[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) acc[o] = sw[kOut * c + o];
    for (int g = 0; g < c / 8; ++g) {
      float v[8];
      unpack8(*reinterpret_cast<const uint4*>(top + p * c + g * 8), v);
#pragma unroll
      for (int o = 0; o < kOut; ++o)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[o] = fmaf(v[i], sw[o * c + g * 8 + i], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) y[p * kOut + o] = acc[o];
  }
}

// ---- head backward: dtop = (dy W) masked by top > 0 (bf16); this block's dW, db into
// part[block] (warps combined in a fixed order; k_head_sum adds the blocks in order) --
constexpr int kHeadThreads = 256;
__global__ void __launch_bounds__(kHeadThreads) k_head_bwd(const uint16_t* __restrict__ top, int c,
                                                           const float* __restrict__ wb, const float* __restrict__ dy,
                                                           int64_t P, uint16_t* __restrict__ dtop,
                                                           float* __restrict__ part /* [blocks][kOut*c + kOut] */) {
  extern __shared__ float sh[];  // weights [kOut*c], per-warp partial grads [warps][kOut*c + kOut]
  const int ng = kOut * c + kOut, nw = blockDim.x / 32, warp = threadIdx.x >> 5;
  float* sw = sh;
  float* sg = sh + kOut * c + warp * ng;
  for (int i = threadIdx.x; i < kOut * c; i += blockDim.x) sw[i] = wb[i];
  __syncthreads();
  float gacc[kOut * 8];
  for (int i = 0; i < kOut * 8; ++i) gacc[i] = 0.f;
  for (int g = 0; g < c / 8; ++g) {
    for (int i = 0; i < kOut * 8; ++i) gacc[i] = 0.f;
    float gb[kOut] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
      float d[kOut], v[8], o[8];
#pragma unroll
      for (int k = 0; k < kOut; ++k) d[k] = dy[p * kOut + k];
      unpack8(*reinterpret_cast<const uint4*>(top + p * c + g * 8), v);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kOut; ++k) {
          s = fmaf(d[k], sw[k * c + g * 8 + i], s);
          gacc[k * 8 + i] = fmaf(d[k], v[i], gacc[k * 8 + i]);
        }
        o[i] = v[i] > 0.f ? s : 0.f;
      }
      *reinterpret_cast<uint4*>(dtop + p * c + g * 8) = pack8(o);
      if (g == 0) {
#pragma unroll
        for (int k = 0; k < kOut; ++k) gb[k] += d[k];
      }
    }
    for (int k = 0; k < kOut; ++k)
      for (int i = 0; i < 8; ++i) {
        float s = gacc[k * 8 + i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sg[k * c + g * 8 + i] = s;
      }
    if (g == 0)
      for (int k = 0; k < kOut; ++k) {
        float s = gb[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sg[kOut * c + k] = s;
      }
  }
  __syncthreads();
  const float* all = sh + kOut * c;
  for (int i = threadIdx.x; i < ng; i += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += all[w * ng + i];
    part[(size_t)blockIdx.x * ng + i] = s;
  }
}

// The same in one pass over the pixels when the c / 8 channel groups are a power of two
// up to 32: G = c / 8 neighbouring threads take the groups of one pixel (a warp reads
// 32 / G whole pixels: contiguous 16-byte loads and stores), dy is read once, and each
// thread keeps the kOut x 8 weight-gradient terms of its group.  The lanes of a group
// are combined with xor shuffles, the warps in order in shared memory: a fixed order.
__global__ void __launch_bounds__(kHeadThreads) k_head_bwd_g(const uint16_t* __restrict__ top, int c,
                                                             const float* __restrict__ wb,
                                                             const float* __restrict__ dy, int64_t P,
                                                             uint16_t* __restrict__ dtop,
                                                             float* __restrict__ part /* [blocks][kOut*c + kOut] */) {
  extern __shared__ float sh[];  // weights [kOut*c], per-warp partial grads [warps][kOut*c + kOut]
  const int ng = kOut * c + kOut, nw = blockDim.x / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = c / 8, g = threadIdx.x & (G - 1);
  float* sw = sh;
  float* sg = sh + kOut * c + warp * ng;
  for (int i = threadIdx.x; i < kOut * c; i += blockDim.x) sw[i] = wb[i];
  __syncthreads();
  float gacc[kOut * 8], gb[kOut];
#pragma unroll
  for (int i = 0; i < kOut * 8; ++i) gacc[i] = 0.f;
#pragma unroll
  for (int k = 0; k < kOut; ++k) gb[k] = 0.f;
  const int64_t per_iter = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t p = blockIdx.x * (int64_t)(blockDim.x / G) + threadIdx.x / G; p < P; p += per_iter) {
    float d[kOut], v[8], o[8];
#pragma unroll
    for (int k = 0; k < kOut; ++k) d[k] = dy[p * kOut + k];
    unpack8(*reinterpret_cast<const uint4*>(top + p * c + g * 8), v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kOut; ++k) {
        s = fmaf(d[k], sw[k * c + g * 8 + i], s);
        gacc[k * 8 + i] = fmaf(d[k], v[i], gacc[k * 8 + i]);
      }
      o[i] = v[i] > 0.f ? s : 0.f;
    }
    *reinterpret_cast<uint4*>(dtop + p * c + g * 8) = pack8(o);
    if (g == 0) {
#pragma unroll
      for (int k = 0; k < kOut; ++k) gb[k] += d[k];
    }
  }
  // lanes with the same group: lane = g + G * j; xor over G, 2G, ..., 16
#pragma unroll
  for (int i = 0; i < kOut * 8; ++i) {
    float s = gacc[i];
    for (int off = 16; off >= G; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    gacc[i] = s;
  }
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    float s = gb[k];  // only the g == 0 lanes hold nonzero terms
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    gb[k] = s;
  }
  if (lane < G) {
#pragma unroll
    for (int k = 0; k < kOut; ++k)
#pragma unroll
      for (int i = 0; i < 8; ++i) sg[k * c + g * 8 + i] = gacc[k * 8 + i];
  }
  if (lane == 0)
    for (int k = 0; k < kOut; ++k) sg[kOut * c + k] = gb[k];
  __syncthreads();
  const float* all = sh + kOut * c;
  for (int i = threadIdx.x; i < ng; i += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += all[w * ng + i];
    part[(size_t)blockIdx.x * ng + i] = s;
  }
}

// grads of the head += its per-block partials: one block per element, thread t sums
// blocks t, t + 256, ... in order, then a fixed-shape tree over the threads
__global__ void __launch_bounds__(256) k_head_sum(const float* __restrict__ part, int blocks, int ng,
                                                  float* __restrict__ gw) {
  __shared__ float red[256];
  const int i = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) s += part[(size_t)b * ng + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) gw[i] += red[0];
}

// ---- dW^T [9*cin_pad][cout] (+ db) into the flat fp32 gradient ---------------------
__global__ void k_dwt_to_grad(const float* __restrict__ dwt, const float* __restrict__ db, int cin_pad, int cin,
                              int cout, float* __restrict__ gw, float* __restrict__ gb) {
  const int total = cout * 9 * cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int ci = e % cin, tap = (e / cin) % 9, o = e / (9 * cin);
    gw[e] = dwt[(tap * cin_pad + ci) * cout + o];
  }
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < cout; o += gridDim.x * blockDim.x) gb[o] = db[o];
}

// pack the network's first-layer weights (c_in = 5) into an 8-channel fp32 copy
__global__ void k_pad_in(const float* __restrict__ w, int cout, int cin, int cin_pad, float* __restrict__ out) {
  const int total = cout * 9 * cin_pad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int ci = e % cin_pad, r = e / cin_pad;
    out[e] = ci < cin ? w[r * cin + ci] : 0.f;
  }
}

// ---- loss (Sec. 3.4): masked MSE of height and colour, each squared error clipped to
// 1, height and colour terms averaged; plus the squared error of the bound channel
// against the detached absolute height error ---------------------------------------
// y [P][5]; base [P][4] (normalised fill height, colour 0..1); target [P][4]; mask [P]
// Detached target of the bound channel: |e|, or the excess max(|e| - |e_base|, 0) of
// the learned height's error over the base fill's error (e_base = base - target).
__device__ __forceinline__ float bound_target(float eh, float base_h, float t_h, int excess) {
  const float a = fabsf(eh);
  return excess ? fmaxf(a - fabsf(base_h - t_h), 0.f) : a;
}

__global__ void k_loss_sums(const float* __restrict__ y, const float* __restrict__ base,
                            const float* __restrict__ target, const uint8_t* __restrict__ mask, int64_t P,
                            int excess, double* __restrict__ part /* [gridDim.x][4]: count, sh, sc, sb */) {
  __shared__ double ws[8][4];  // per warp (256 threads)
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[p]) continue;
    const float eh = base[p * 4] + y[p * kOut] - target[p * 4];
    s[0] += 1.0;
    s[1] += fminf(eh * eh, 1.f);
    for (int k = 1; k < 4; ++k) {
      const float ec = base[p * 4 + k] + y[p * kOut + k] - target[p * 4 + k];
      s[2] += fminf(ec * ec, 1.f);
    }
    const float db = y[p * kOut + 4] - bound_target(eh, base[p * 4], target[p * 4], excess);
    s[3] += db * db;
  }
  // fixed-order sums: warp tree, then the block's warps in order; the blocks' partials are
  // added in order by k_loss_reduce (no contended atomics, the same sums every run)
  const int warp = threadIdx.x >> 5;
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) ws[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += ws[w][threadIdx.x];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
  }
}

// One warp: sums[k] = the blocks' partials k in a fixed order (lane-strided, then a tree)
__global__ void k_loss_reduce(const double* __restrict__ part, int nb, double* __restrict__ sums) {
  for (int k = 0; k < 4; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) v += part[(size_t)b * 4 + k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) sums[k] = v;
  }
}

__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ base,
                            const float* __restrict__ target, const uint8_t* __restrict__ mask, int64_t P,
                            const double* __restrict__ sums, float bound_weight, int excess, float* __restrict__ dy,
                            float* __restrict__ loss /* [4] total, height, colour, bound */) {
  const double cnt = sums[0] > 1.0 ? sums[0] : 1.0;
  const float inv = (float)(1.0 / cnt), inv3 = (float)(1.0 / (3.0 * cnt));
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    const double lh = sums[1] / cnt, lc = sums[2] / (3.0 * cnt), lb = sums[3] / cnt;
    loss[0] = (float)(0.5 * (lh + lc) + bound_weight * lb);
    loss[1] = (float)lh; loss[2] = (float)lc; loss[3] = (float)lb;
  }
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float g[kOut] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (mask[p]) {
      const float eh = base[p * 4] + y[p * kOut] - target[p * 4];
      g[0] = eh * eh < 1.f ? eh * inv : 0.f;  // 0.5 * 2 * e / cnt
      for (int k = 1; k < 4; ++k) {
        const float ec = base[p * 4 + k] + y[p * kOut + k] - target[p * 4 + k];
        g[k] = ec * ec < 1.f ? ec * inv3 : 0.f;
      }
      const float db = y[p * kOut + 4] - bound_target(eh, base[p * 4], target[p * 4], excess);
      g[4] = bound_weight * 2.f * db * inv;
    }
#pragma unroll
    for (int k = 0; k < kOut; ++k) dy[p * kOut + k] = g[k];
  }
}

// ---- AdamW (decoupled weight decay), Sec. 3.4 hyper-parameters by default ---------
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd,
                        float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float pi = p[i] * (1.f - lr * wd);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[i] = pi - lr * mh / (sqrtf(vh) + eps);
  }
}

struct LayerDesc {
  int cin, cout, k, cin_pad, level, h;  // h: spatial size (square)
  int64_t w_off, b_off;
  uint16_t* wpk = nullptr;   // forward operand
  uint16_t* wpk_t = nullptr; // input-gradient operand
};

}  // namespace
}  // namespace ls

struct ls_model {
  int levels = 0;
  int widths[4] = {0, 0, 0, 0};
  int res = 0;
  int max_batch = 0;
  int64_t n_params = 0;
  std::vector<ls::LayerDesc> layers;
  // device memory owned by the model
  void* arena = nullptr;
  uint16_t* act[32] = {};     // forward activations (bf16 NHWC), see slot map in code
  uint16_t* gbuf[3] = {};     // gradient ping-pong buffers (bf16), largest activation size
  uint16_t* gskip[4] = {};    // d(concat) per decoder level
  float* dwt = nullptr;       // [max 9*cin*cout]
  float* dbs = nullptr;       // [max cout]
  float* head = nullptr;      // head weights + bias (fp32, from the last load)
  float* w0pad = nullptr;     // first layer weights padded to 8 input channels
  const uint16_t* x = nullptr;  // input of the last forward
  int last_n = 0;
  int recompute = 0;           // e{l}a and d{l}a share one buffer; backward recomputes them
  size_t device_bytes = 0;     // size of the arena
};

namespace ls {
namespace {

// activation slot ids: e{l}a -> 4*(l-1), e{l}b -> 4*(l-1)+1, p{l} -> 4*(l-1)+2,
// c{l} -> 4*(l-1)+3 (l < levels), d{l}a -> 16 + 2*(l-1), d{l}b -> 16 + 2*(l-1)+1
int slot_ea(int l) { return 4 * (l - 1); }
int slot_eb(int l) { return 4 * (l - 1) + 1; }
int slot_p(int l) { return 4 * (l - 1) + 2; }
int slot_c(int l) { return 4 * (l - 1) + 3; }
int slot_da(int l) { return 16 + 2 * (l - 1); }
int slot_db(int l) { return 16 + 2 * (l - 1) + 1; }

int grid_for(int64_t work, int threads) { return grid_cap((work + threads - 1) / threads, kSmCount * 16); }

}  // namespace
}  // namespace ls

using namespace ls;

extern "C" ls_status ls_model_create_opts(int32_t levels, const int32_t* widths, int32_t res, int32_t max_batch,
                                          int32_t flags, ls_model** out) {
  if (!out || !widths || levels < 2 || levels > 4 || max_batch <= 0 || res <= 0) return LS_ERR_INVALID_ARG;
  if (flags & ~LS_MODEL_RECOMPUTE) return LS_ERR_INVALID_ARG;
  if (res % (1 << (levels - 1))) return LS_ERR_INVALID_ARG;
  for (int l = 0; l < levels; ++l)
    if (widths[l] < 16 || widths[l] > 128 || widths[l] % 16) return LS_ERR_UNSUPPORTED;
  ls_model* m = new (std::nothrow) ls_model();
  if (!m) return LS_ERR_NO_MEMORY;
  m->levels = levels;
  m->res = res;
  m->max_batch = max_batch;
  m->recompute = (flags & LS_MODEL_RECOMPUTE) ? 1 : 0;
  for (int l = 0; l < levels; ++l) m->widths[l] = widths[l];
  int64_t off = 0;
  auto add = [&](int cin, int cout, int k, int level, int h) {
    LayerDesc d;
    d.cin = cin; d.cout = cout; d.k = k; d.level = level; d.h = h;
    d.cin_pad = cin < 8 ? 8 : cin;
    d.w_off = off; off += (int64_t)cout * k * k * cin;
    d.b_off = off; off += cout;
    m->layers.push_back(d);
  };
  int cin = 5;
  for (int l = 1; l <= levels; ++l) {
    const int h = res >> (l - 1);
    add(cin, widths[l - 1], 3, l, h);
    add(widths[l - 1], widths[l - 1], 3, l, h);
    cin = widths[l - 1];
  }
  int up = widths[levels - 1];
  for (int l = levels - 1; l >= 1; --l) {
    const int h = res >> (l - 1);
    add(up + widths[l - 1], widths[l - 1], 3, l, h);
    add(widths[l - 1], widths[l - 1], 3, l, h);
    up = widths[l - 1];
  }
  add(widths[0], 5, 1, 1, res);
  m->n_params = off;
  // ---- device memory: one arena
  const int64_t B = max_batch;
  std::vector<std::pair<int, int64_t>> acts;  // slot, elements
  int64_t max_act = 0;
  for (int l = 1; l <= levels; ++l) {
    const int64_t hw = (int64_t)(res >> (l - 1)) * (res >> (l - 1));
    acts.push_back({slot_ea(l), B * hw * widths[l - 1]});
    acts.push_back({slot_eb(l), B * hw * widths[l - 1]});
    if (l < levels) {
      acts.push_back({slot_p(l), B * (hw / 4) * widths[l - 1]});
      const int cu = (l + 1 == levels) ? widths[levels - 1] : widths[l];
      acts.push_back({slot_c(l), B * hw * (cu + widths[l - 1])});
      acts.push_back({slot_da(l), B * hw * widths[l - 1]});
      acts.push_back({slot_db(l), B * hw * widths[l - 1]});
    }
  }
  for (auto& a : acts) max_act = a.second > max_act ? a.second : max_act;
  int64_t max_wk = 0, max_pk = 0;
  for (auto& d : m->layers) {
    if (d.k != 3) continue;
    max_wk = std::max<int64_t>(max_wk, (int64_t)9 * d.cin_pad * d.cout);
    max_pk = std::max<int64_t>(max_pk, ls_conv3x3_packed_elems(d.cin_pad, d.cout));
    if (d.cin >= 16) max_pk = std::max<int64_t>(max_pk, ls_conv3x3_packed_elems(d.cout, d.cin));
  }
  size_t bytes = 0;
  auto take = [&](size_t nbytes) { size_t o = bytes; bytes += (nbytes + 255) / 256 * 256; return o; };
  std::vector<size_t> act_off;
  // with recomputation the first conv output of every level (e{l}a, d{l}a) lives in one
  // shared buffer: the forward consumes it at once, the backward recomputes it
  int64_t max_first = 0;
  for (int l = 1; l <= levels; ++l) {
    const int64_t hw = (int64_t)(res >> (l - 1)) * (res >> (l - 1));
    max_first = std::max<int64_t>(max_first, B * hw * widths[l - 1]);
  }
  const size_t first_off = m->recompute ? take((size_t)max_first * 2) : 0;
  auto shared_first = [&](int slot) {
    if (!m->recompute) return false;
    for (int l = 1; l <= levels; ++l)
      if (slot == slot_ea(l) || (l < levels && slot == slot_da(l))) return true;
    return false;
  };
  for (auto& a : acts) act_off.push_back(shared_first(a.first) ? first_off : take((size_t)a.second * 2));
  size_t g_off[3];
  for (int i = 0; i < 3; ++i) g_off[i] = take((size_t)max_act * 2);
  size_t gs_off[4] = {0, 0, 0, 0};
  for (int l = 1; l < levels; ++l) {
    const int64_t hw = (int64_t)(res >> (l - 1)) * (res >> (l - 1));
    const int cu = (l + 1 == levels) ? widths[levels - 1] : widths[l];
    gs_off[l - 1] = take((size_t)B * hw * (cu + widths[l - 1]) * 2);
  }
  std::vector<std::pair<size_t, size_t>> pk_off;
  for (auto& d : m->layers) {
    if (d.k != 3) { pk_off.push_back({0, 0}); continue; }
    const size_t a = take((size_t)ls_conv3x3_packed_elems(d.cin_pad, d.cout) * 2);
    const size_t b = d.cin >= 16 ? take((size_t)ls_conv3x3_packed_elems(d.cout, d.cin) * 2) : 0;
    pk_off.push_back({a, b});
  }
  const size_t dwt_off = take((size_t)max_wk * 4);
  const size_t dbs_off = take(256 * 4);
  const size_t head_off = take((size_t)(5 * widths[0] + 5) * 4);
  const size_t w0_off = take((size_t)9 * 8 * widths[0] * 4);
  if (cudaMalloc(&m->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return LS_ERR_NO_MEMORY;
  }
  char* base = static_cast<char*>(m->arena);
  m->device_bytes = bytes;
  for (size_t i = 0; i < acts.size(); ++i) m->act[acts[i].first] = reinterpret_cast<uint16_t*>(base + act_off[i]);
  for (int i = 0; i < 3; ++i) m->gbuf[i] = reinterpret_cast<uint16_t*>(base + g_off[i]);
  for (int l = 1; l < levels; ++l) m->gskip[l - 1] = reinterpret_cast<uint16_t*>(base + gs_off[l - 1]);
  for (size_t i = 0; i < m->layers.size(); ++i) {
    if (m->layers[i].k != 3) continue;
    m->layers[i].wpk = reinterpret_cast<uint16_t*>(base + pk_off[i].first);
    if (m->layers[i].cin >= 16) m->layers[i].wpk_t = reinterpret_cast<uint16_t*>(base + pk_off[i].second);
  }
  m->dwt = reinterpret_cast<float*>(base + dwt_off);
  m->dbs = reinterpret_cast<float*>(base + dbs_off);
  m->head = reinterpret_cast<float*>(base + head_off);
  m->w0pad = reinterpret_cast<float*>(base + w0_off);
  *out = m;
  return LS_OK;
}

extern "C" ls_status ls_model_create(int32_t levels, const int32_t* widths, int32_t res, int32_t max_batch,
                                     ls_model** out) {
  return ls_model_create_opts(levels, widths, res, max_batch, 0, out);
}

extern "C" size_t ls_model_device_bytes(const ls_model* m) { return m ? m->device_bytes : 0; }

extern "C" void ls_model_destroy(ls_model* m) {
  if (!m) return;
  if (m->arena) cudaFree(m->arena);
  delete m;
}

extern "C" int64_t ls_model_param_count(const ls_model* m) { return m ? m->n_params : -1; }
extern "C" int32_t ls_model_layer_count(const ls_model* m) { return m ? (int32_t)m->layers.size() : -1; }

extern "C" ls_status ls_model_layer_info(const ls_model* m, int32_t i, int32_t* cin, int32_t* cout, int32_t* ksize,
                                         int64_t* w_offset, int64_t* b_offset) {
  if (!m || i < 0 || i >= (int)m->layers.size()) return LS_ERR_INVALID_ARG;
  const LayerDesc& d = m->layers[i];
  if (cin) *cin = d.cin;
  if (cout) *cout = d.cout;
  if (ksize) *ksize = d.k;
  if (w_offset) *w_offset = d.w_off;
  if (b_offset) *b_offset = d.b_off;
  return LS_OK;
}

extern "C" ls_status ls_model_load(ls_model* m, const float* params, ls_stream_t stream) {
  if (!m || !params) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every layer's packs (and the transposed packs of the input gradients) in one launch,
  // after the first layer's input channels are padded
  std::vector<PackJob> jobs;
  for (auto& d : m->layers) {
    if (d.k == 1) {
      LS_CUDA_TRY(cudaMemcpyAsync(m->head, params + d.w_off, (size_t)(d.cout * d.cin + d.cout) * 4,
                                  cudaMemcpyDeviceToDevice, s));
      continue;
    }
    const float* w = params + d.w_off;
    if (d.cin != d.cin_pad) {
      const int total = d.cout * 9 * d.cin_pad;
      k_pad_in<<<grid_for(total, 256), 256, 0, s>>>(w, d.cout, d.cin, d.cin_pad, m->w0pad);
      w = m->w0pad;
    }
    jobs.push_back({w, d.wpk, d.cin_pad, d.cout, 0});
    if (d.wpk_t) jobs.push_back({params + d.w_off, d.wpk_t, d.cout, d.cin, 1});
  }
  const ls_status st = conv3x3_pack_batch(jobs.data(), (int)jobs.size(), s);
  if (st != LS_OK) return st;
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// Forward pass.  keep_top = false (inference): the 1x1 head is fused into the last
// convolution where the shape has a halo form and that convolution's output is not
// stored (no backward can follow: last_n is cleared).
ls_status filler_forward(ls_model* m, const float* params, const uint16_t* x, int32_t n, float* y, cudaStream_t s,
                         bool keep_top) {
  if (!m || !params || !x || !y || n <= 0 || n > m->max_batch) return LS_ERR_INVALID_ARG;
  const int L = m->levels, R = m->res;
  auto conv = [&](int li, const uint16_t* in, int h, uint16_t* out) {
    const LayerDesc& d = m->layers[li];
    return conv3x3_launch(in, d.wpk, params + d.b_off, nullptr, 1, n, h, h, d.cin_pad, d.cout, out, s);
  };
  int li = 0;
  const uint16_t* h_in = x;
  ls_status st;
  bool up_ready = false;  // the next decoder level's upsampled input is already stored
  for (int l = 1; l <= L; ++l) {
    const int h = R >> (l - 1);
    if (l > 1) {
      const int c = m->widths[l - 2];
      const int64_t work = (int64_t)n * (h * h) * (c / 8);
      k_maxpool<<<grid_for(work, 256), 256, 0, s>>>(m->act[slot_eb(l - 1)], n, 2 * h, 2 * h, c, m->act[slot_p(l - 1)]);
      h_in = m->act[slot_p(l - 1)];
    }
    if ((st = conv(li++, h_in, h, m->act[slot_ea(l)])) != LS_OK) return st;
    if (!keep_top && l == L && L > 1) {
      // inference: the bottleneck's output feeds only the first decoder level's
      // upsampling, so it is stored upsampled there
      const LayerDesc& d = m->layers[li];
      st = d.cout == m->widths[L - 1]
               ? conv3x3_up2_launch(m->act[slot_ea(l)], d.wpk, params + d.b_off, n, h, h, d.cin_pad, d.cout,
                                    m->act[slot_c(L - 1)], s)
               : LS_ERR_UNSUPPORTED;
      if (st == LS_OK) {
        ++li;
        up_ready = true;
        continue;
      }
      if (st != LS_ERR_UNSUPPORTED) return st;
    }
    if ((st = conv(li++, m->act[slot_ea(l)], h, m->act[slot_eb(l)])) != LS_OK) return st;
    h_in = m->act[slot_eb(l)];
  }
  for (int l = L - 1; l >= 1; --l) {
    const int h = R >> (l - 1);
    const int cu = (l + 1 == L) ? m->widths[L - 1] : m->widths[l];
    const int cs = m->widths[l - 1];
    if (keep_top) {
      k_upcat<<<grid_cap((int64_t)n * h, kSmCount * 16), 256, 0, s>>>(h_in, cu, m->act[slot_eb(l)], cs, n, h, h,
                                                                       m->act[slot_c(l)]);
      if ((st = conv(li++, m->act[slot_c(l)], h, m->act[slot_da(l)])) != LS_OK) return st;
    } else {
      // inference: only the upsampled channels are written (unless the level below
      // already stored its output upsampled); the convolution reads the skip
      // connection's channels from the encoder output directly
      if (!up_ready)
        k_upcat<<<grid_cap((int64_t)n * h, kSmCount * 16), 256, 0, s>>>(h_in, cu, nullptr, 0, n, h, h,
                                                                         m->act[slot_c(l)]);
      up_ready = false;
      const LayerDesc& d = m->layers[li++];
      if ((st = conv3x3_launch_groups(m->act[slot_c(l)], d.wpk, params + d.b_off, nullptr, 1, n, h, h, d.cin_pad,
                                      d.cout, m->act[slot_da(l)], d.cout, 0, s, m->act[slot_eb(l)], cu)) != LS_OK)
        return st;
    }
    if (l == 1 && L > 1) {
      // the last convolution with the head in its epilogue
      const LayerDesc& d = m->layers[li];
      const LayerDesc& hd = m->layers[li + 1];
      st = conv3x3_head_launch(m->act[slot_da(l)], d.wpk, params + d.b_off, n, h, h, d.cin_pad, d.cout,
                               m->act[slot_db(l)], params + hd.w_off, y, kOut, keep_top ? 1 : 0, s);
      if (st == LS_OK) {
        m->x = keep_top ? x : nullptr;
        m->last_n = keep_top ? n : 0;
        return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
      }
      if (st != LS_ERR_UNSUPPORTED) return st;
    }
    if (!keep_top && l >= 2) {
      // inference: this output feeds only the next level's upsampling, so the
      // convolution stores it upsampled, where that level reads it
      const LayerDesc& d = m->layers[li];
      const int cu_next = m->widths[l - 1];
      st = d.cout == cu_next ? conv3x3_up2_launch(m->act[slot_da(l)], d.wpk, params + d.b_off, n, h, h, d.cin_pad,
                                                  d.cout, m->act[slot_c(l - 1)], s)
                             : LS_ERR_UNSUPPORTED;
      if (st == LS_OK) {
        ++li;
        up_ready = true;
        continue;
      }
      if (st != LS_ERR_UNSUPPORTED) return st;
    }
    if ((st = conv(li++, m->act[slot_da(l)], h, m->act[slot_db(l)])) != LS_OK) return st;
    h_in = m->act[slot_db(l)];
  }
  const LayerDesc& hd = m->layers[li];
  const int64_t P = (int64_t)n * R * R;
  k_head_fwd<<<grid_for(P, 256), 256, (size_t)(kOut * hd.cin + kOut) * 4, s>>>(h_in, hd.cin, params + hd.w_off, P, y);
  m->x = x;
  m->last_n = n;
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_filler_forward(ls_model* m, const float* params, const uint16_t* x, int32_t n, float* y,
                                       ls_stream_t stream) {
  return filler_forward(m, params, x, n, y, reinterpret_cast<cudaStream_t>(stream), true);
}

extern "C" ls_status ls_filler_backward(ls_model* m, const float* params, const float* dy, int32_t n, float* grads,
                                        ls_stream_t stream) {
  if (!m || !params || !dy || !grads || n != m->last_n || !m->x) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int L = m->levels, R = m->res;
  const int64_t P = (int64_t)n * R * R;
  LS_CUDA_TRY(cudaMemsetAsync(grads, 0, (size_t)m->n_params * 4, s));
  const int nl = (int)m->layers.size();
  const LayerDesc& hd = m->layers[nl - 1];
  // input of every conv layer, in layer order
  std::vector<const uint16_t*> lin(nl, nullptr);
  {
    int li = 0;
    for (int l = 1; l <= L; ++l) {
      lin[li++] = l == 1 ? m->x : m->act[slot_p(l - 1)];
      lin[li++] = m->act[slot_ea(l)];
    }
    for (int l = L - 1; l >= 1; --l) {
      lin[li++] = m->act[slot_c(l)];
      lin[li++] = m->act[slot_da(l)];
    }
  }
  auto out_of = [&](int li) -> const uint16_t* {  // post-ReLU output of conv layer li
    int k = 0;
    for (int l = 1; l <= L; ++l) {
      if (k++ == li) return m->act[slot_ea(l)];
      if (k++ == li) return m->act[slot_eb(l)];
    }
    for (int l = L - 1; l >= 1; --l) {
      if (k++ == li) return m->act[slot_da(l)];
      if (k++ == li) return m->act[slot_db(l)];
    }
    return nullptr;
  };
  auto wgrad = [&](int li, const uint16_t* dz) -> ls_status {
    const LayerDesc& d = m->layers[li];
    const int h = d.h;
    if (cudaMemsetAsync(m->dwt, 0, (size_t)9 * d.cin_pad * d.cout * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    if (cudaMemsetAsync(m->dbs, 0, (size_t)d.cout * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    ls_status st = wgrad_launch(lin[li], dz, n, h, h, d.cin_pad, d.cout, m->dwt, m->dbs, s);
    if (st != LS_OK) return st;
    const int total = d.cout * 9 * d.cin;
    k_dwt_to_grad<<<grid_for(total, 256), 256, 0, s>>>(m->dwt, m->dbs, d.cin_pad, d.cin, d.cout, grads + d.w_off,
                                                        grads + d.b_off);
    return LS_OK;
  };
  auto dgrad = [&](int li, const uint16_t* dz, const uint16_t* mask, uint16_t* dx) -> ls_status {
    const LayerDesc& d = m->layers[li];
    return conv3x3_launch(dz, d.wpk_t, nullptr, mask, 0, n, d.h, d.h, d.cout, d.cin, dx, s);
  };
  // recomputation: the first conv (layer li) of a level again, from its stored input,
  // into the shared buffer; the kernel is deterministic, so the activation and every
  // gradient equal those of a model that kept it
  auto recompute = [&](int li) -> ls_status {
    if (!m->recompute) return LS_OK;
    const LayerDesc& d = m->layers[li];
    return conv3x3_launch(lin[li], d.wpk, params + d.b_off, nullptr, 1, n, d.h, d.h, d.cin_pad, d.cout,
                          const_cast<uint16_t*>(lin[li + 1]), s);
  };
  ls_status st;
  // head
  uint16_t* gz = m->gbuf[0];
  {
    const int blocks = grid_cap((P + kHeadThreads - 1) / kHeadThreads, kSmCount * 4);
    const int ng = kOut * hd.cin + kOut;
    float* part = static_cast<float*>(workspace(kWsHeadPart, (size_t)blocks * ng * 4));
    if (!part) return LS_ERR_NO_MEMORY;
    const size_t smem = (size_t)(kOut * hd.cin + (kHeadThreads / 32) * ng) * 4;
    const int G = hd.cin / 8;
    if (hd.cin % 8 == 0 && G <= 32 && (G & (G - 1)) == 0)
      k_head_bwd_g<<<blocks, kHeadThreads, smem, s>>>(out_of(nl - 2), hd.cin, params + hd.w_off, dy, P, gz, part);
    else
      k_head_bwd<<<blocks, kHeadThreads, smem, s>>>(out_of(nl - 2), hd.cin, params + hd.w_off, dy, P, gz, part);
    k_head_sum<<<ng, 256, 0, s>>>(part, blocks, ng, grads + hd.w_off);
  }
  int li = nl - 2;  // d1b
  int gi = 0;
  // decoder levels 1 .. L-1 (reverse of the forward order)
  for (int l = 1; l < L; ++l, li -= 2) {
    const int h = R >> (l - 1);
    // layer li = d{l}b, li-1 = d{l}a
    if ((st = recompute(li - 1)) != LS_OK) return st;
    if ((st = wgrad(li, gz)) != LS_OK) return st;
    uint16_t* gz2 = m->gbuf[(gi + 1) % 3];
    if ((st = dgrad(li, gz, lin[li], gz2)) != LS_OK) return st;  // masked by d{l}a > 0
    if ((st = wgrad(li - 1, gz2)) != LS_OK) return st;
    uint16_t* dc = m->gskip[l - 1];
    if ((st = dgrad(li - 1, gz2, lin[li - 1], dc)) != LS_OK) return st;  // masked by concat > 0
    const int cu = (l + 1 == L) ? m->widths[L - 1] : m->widths[l];
    const int cs = m->widths[l - 1];
    gi = (gi + 2) % 3;
    gz = m->gbuf[gi];
    const int64_t work = (int64_t)n * (h / 2) * (h / 2) * (cu / 8);
    k_up_bwd<<<grid_for(work, 256), 256, 0, s>>>(dc, cu + cs, cu, n, h / 2, h / 2, gz);
  }
  // encoder levels L .. 1; li now points at e{L}b
  for (int l = L; l >= 1; --l, li -= 2) {
    const int h = R >> (l - 1);
    if (l < L) {
      // gz holds d(pooled) from the dgrad of e{l+1}a; combine with the skip gradient
      const int c = m->widths[l - 1];
      const int cu = (l + 1 == L) ? m->widths[L - 1] : m->widths[l];
      uint16_t* dz = m->gbuf[(gi + 1) % 3];
      const int64_t work = (int64_t)n * (h / 2) * (h / 2) * (c / 8);
      k_maxpool_bwd<<<grid_for(work, 256), 256, 0, s>>>(m->act[slot_eb(l)], gz, m->gskip[l - 1], cu + c, cu, n, h, h,
                                                         c, dz);
      gi = (gi + 1) % 3;
      gz = dz;
    }
    if ((st = recompute(li - 1)) != LS_OK) return st;
    if ((st = wgrad(li, gz)) != LS_OK) return st;
    uint16_t* gz2 = m->gbuf[(gi + 1) % 3];
    if ((st = dgrad(li, gz, lin[li], gz2)) != LS_OK) return st;  // masked by e{l}a > 0
    if ((st = wgrad(li - 1, gz2)) != LS_OK) return st;
    if (l > 1) {
      uint16_t* gp = m->gbuf[(gi + 2) % 3];
      if ((st = dgrad(li - 1, gz2, nullptr, gp)) != LS_OK) return st;  // d(pooled), raw
      gi = (gi + 2) % 3;
      gz = gp;
    }
  }
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_filler_loss(const float* y, const float* base, const float* target, const uint8_t* mask,
                                    int64_t n_px, float bound_weight, int32_t bound_excess, double* sums,
                                    float* loss, float* dy, ls_stream_t stream) {
  if (!y || !base || !target || !mask || !sums || !dy || n_px <= 0) return LS_ERR_INVALID_ARG;
  if (bound_excess != 0 && bound_excess != 1) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nb = grid_cap((n_px + 255) / 256, kSmCount * 8);
  double* part = static_cast<double*>(workspace(kWsLossPart, (size_t)nb * 4 * sizeof(double)));
  if (!part) return LS_ERR_NO_MEMORY;
  k_loss_sums<<<nb, 256, 0, s>>>(y, base, target, mask, n_px, bound_excess, part);
  k_loss_reduce<<<1, 32, 0, s>>>(part, nb, sums);
  k_loss_grad<<<grid_cap((n_px + 255) / 256, kSmCount * 8), 256, 0, s>>>(y, base, target, mask, n_px, sums,
                                                                         bound_weight, bound_excess, dy, loss);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_adamw_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1,
                                   float beta2, float eps, float wd, int32_t step, ls_stream_t stream) {
  if (!p || !g || !m || !v || n <= 0 || step < 1) return LS_ERR_INVALID_ARG;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, step));
  k_adamw<<<grid_cap((n + 255) / 256, kSmCount * 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      p, g, m, v, n, lr, beta1, beta2, eps, wd, bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
