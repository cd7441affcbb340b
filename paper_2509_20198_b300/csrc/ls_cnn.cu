// The paper's own network variant (Sec. 3.4): the NN and linear heightmaps and
// textures of Alg. 1 on a res x res patch are encoded independently (four encoders),
// merged by fully connected layers in two steps, decoded by separate height and
// texture CNNs, concatenated with the original inputs (the one skip connection),
// reduced by a final CNN and cropped to the centre.  The text fixes no sizes; the
// readings (the layer table below) give 2,481,733 parameters at res 128, the paper's
// 2.5M.
//
// Native runtime on this library's kernels: every 3x3 convolution, forward, input
// gradient and weight gradient, runs on the tcgen05 kernels of ls_conv.cu and
// ls_wgrad.cu; pooling, upsampling and the 1x1 head reuse the U-Net's kernels.  The
// fully connected layers (0.4 % of the network's FLOPs) run in a small fp32 tiled
// GEMM with a fixed summation order, so training stays bit-reproducible.
//
// Flat parameter layout (fp32, caller-owned): the layers in table order, each as its
// weights followed by its bias; 3x3 conv weights [C_out][3][3][C_in], fully connected
// [out][in], head [5][16].
//  e{k}.0 .. e{k}.4   encoder k = 0..3 (lin height, NN height, lin RGB, NN RGB):
//                     C_in -> 16, 32, 64, 64 (each + ReLU + 2x2 max pool), -> 16 + ReLU
//  fc1.{k}            16 (res/16)^2 -> 256 + ReLU
//  fc2                1024 -> 16 (res/16)^2 + ReLU, reshaped [res/16][res/16][16]
//  d{h,t}.0 .. .4     16 -> 64, 32, 32, 16 (each + ReLU + 2x upsampling), -> 16 + ReLU
//  f.0, f.1           concat [input 8, height 16, texture 16] = 40 -> 32, -> 16 (+ ReLU)
//  head               1x1, 16 -> 5 (height, R, G, B, error bound); centre res/2 crop
#include <vector>

namespace ls {
namespace {

constexpr int kCnnIn = 8;
constexpr int kCatUsed = 40;  // channels of the skip concat
constexpr int kCatPad = 48;   // stored with 8 zero channels: its input gradient has 48
constexpr int kCnnEncW[4] = {16, 32, 64, 64};
constexpr int kCnnEncOut = 16;
constexpr int kCnnFc1 = 256;
constexpr int kCnnDecW[5] = {64, 32, 32, 16, 16};
constexpr int kCnnEncC0[4] = {0, 1, 2, 5};
constexpr int kCnnEncCk[4] = {1, 1, 3, 3};
// the four encoders' first layers read the same 8-channel input: the forward runs them
// as one convolution with 4 x 16 output channels, written to the four encoders' buffers
constexpr int kCnnE0Fused = 4 * 16;

enum CnnKind { kCnnConv = 0, kCnnFc = 1, kCnnHead = 2 };

struct CnnLayer {
  int kind, cin, cout;
  int cin_pad;  // channels of the stored input operand (8: encoders' first layers, 48: f.0)
  int c0;       // first operand channel of the layer's own inputs (encoders' first layers)
  int h;        // spatial size (conv)
  int64_t w_off, b_off;
  uint16_t* wpk = nullptr;    // forward operand
  uint16_t* wpk_t = nullptr;  // input-gradient operand
};

// ---- fp32 tiled GEMM: C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n]) * [mask(m,n) > 0]
// with A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn]; one thread per 4 x 4 block
// of C, k in increasing order (deterministic).  With split-K (gridDim.z > 1) the CTAs
// of slice z sum k in [z kc, (z + 1) kc) into part[z][M][N] (no bias, activation or
// mask), and k_gemm_reduce adds the slices in increasing z: still one fixed order.
constexpr int kGt = 64, kGk = 16;
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int64_t sam,
                                              int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbn,
                                              float* __restrict__ C, int64_t ldc, const float* __restrict__ bias,
                                              int relu, const float* __restrict__ mask, int64_t ldm, int kc,
                                              float* __restrict__ part) {
  __shared__ float As[kGk][kGt + 1], Bs[kGk][kGt + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kGt, n0 = blockIdx.x * kGt;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kGk) {
    for (int e = threadIdx.x; e < kGt * kGk; e += blockDim.x) {
      const int mm = e / kGk, ka = e % kGk, kb2 = e / kGt, nn = e % kGt;
      const int gm = m0 + mm, gka = k0 + ka, gkb = k0 + kb2, gn = n0 + nn;
      As[ka][mm] = (gm < M && gka < ke) ? A[gm * sam + gka * sak] : 0.f;
      Bs[kb2][nn] = (gkb < ke && gn < N) ? B[gkb * sbk + gn * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGk; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty + 16 * i];
        b[i] = Bs[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      if (part) {
        part[((int64_t)blockIdx.z * M + m) * N + n] = acc[i][j];
        continue;
      }
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      if (mask && !(mask[m * ldm + n] > 0.f)) v = 0.f;
      C[m * ldc + n] = v;
    }
}

// C[m][n] = act(sum over z in increasing order of part[z][m][n] + bias[n]) * mask
__global__ void k_gemm_reduce(int M, int N, int splits, const float* __restrict__ part, float* __restrict__ C,
                              int64_t ldc, const float* __restrict__ bias, int relu, const float* __restrict__ mask,
                              int64_t ldm) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += part[(int64_t)z * total + e];
    v += bias ? bias[n] : 0.f;
    if (relu) v = fmaxf(v, 0.f);
    if (mask && !(mask[m * ldm + n] > 0.f)) v = 0.f;
    C[m * ldc + n] = v;
  }
}

// column sums of a [rows][cols] block (leading dimension lda), rows in order
__global__ void k_colsum_rows(const float* __restrict__ a, int rows, int cols, int64_t lda, float* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += a[r * lda + c];
    out[c] = s;
  }
}

__global__ void k_bf16_to_f32(const uint16_t* __restrict__ a, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = bf2f(a[i]);
}

// out = a where mask > 0 (mask: bf16, or none), as bf16
__global__ void k_f32_to_bf16_masked(const float* __restrict__ a, const uint16_t* __restrict__ mask, int64_t n,
                                     uint16_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (!mask || bf2f(mask[i]) > 0.f) ? f2bf(a[i]) : (uint16_t)0;
}

__global__ void k_add_bf16_f32(const uint16_t* __restrict__ a, const uint16_t* __restrict__ b, int64_t n,
                               float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = bf2f(a[i]) + bf2f(b[i]);
}

// skip concat [x 8 | height decoder 16 | texture decoder 16 | zeros 8] per pixel
__global__ void k_cnn_concat(const uint16_t* __restrict__ x, const uint16_t* __restrict__ dh,
                             const uint16_t* __restrict__ dt, int64_t P, uint16_t* __restrict__ cat) {
  const int g = kCatPad / 8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * g; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / g;
    const int gi = (int)(e - p * g);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gi == 0) v = reinterpret_cast<const uint4*>(x)[p];
    else if (gi <= 2) v = reinterpret_cast<const uint4*>(dh)[p * 2 + gi - 1];
    else if (gi <= 4) v = reinterpret_cast<const uint4*>(dt)[p * 2 + gi - 3];
    reinterpret_cast<uint4*>(cat)[p * g + gi] = v;
  }
}

// channels [off, off + 16) of the [P][48] concat gradient
__global__ void k_cnn_slice16(const uint16_t* __restrict__ cat, int off, int64_t P, uint16_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * 2; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / 2;
    reinterpret_cast<uint4*>(out)[e] = reinterpret_cast<const uint4*>(cat + p * kCatPad + off)[e - p * 2];
  }
}

// centre crop (and its zero-padded adjoint) of [n][R][R][5] outputs
__global__ void k_cnn_crop(const float* __restrict__ yf, int n, int R, float* __restrict__ y) {
  const int C = R / 2, o = R / 4;
  const int64_t total = (int64_t)n * C * C * 5;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e % 5);
    const int64_t p = e / 5;
    const int j = (int)(p % C), i = (int)((p / C) % C);
    const int64_t nn = p / ((int64_t)C * C);
    y[e] = yf[(((nn * R) + o + i) * R + o + j) * 5 + ch];
  }
}
__global__ void k_cnn_uncrop(const float* __restrict__ dy, int n, int R, float* __restrict__ dyf) {
  const int C = R / 2, o = R / 4;
  const int64_t total = (int64_t)n * R * R * 5;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e % 5);
    const int64_t p = e / 5;
    const int j = (int)(p % R) - o, i = (int)((p / R) % R) - o;
    const int64_t nn = p / ((int64_t)R * R);
    dyf[e] = (i >= 0 && i < C && j >= 0 && j < C) ? dy[(((nn * C) + i) * C + j) * 5 + ch] : 0.f;
  }
}

// backward of 2x2 max pooling without a skip: route each pooled gradient to the first
// maximum (row-major window order), times the ReLU derivative of the pooled input
// dx: c channels of every pixel at dx[pixel * dx_ld + dx_off] (dense: dx_ld = c, dx_off = 0)
__global__ void k_maxpool_bwd_relu(const uint16_t* __restrict__ x, const uint16_t* __restrict__ dpool, int n, int h,
                                   int w, int c, uint16_t* __restrict__ dx, int dx_ld, int dx_off) {
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
      for (int i = 0; i < 8; ++i)
        if (k == 0 || v[k][i] > m[i]) { m[i] = v[k][i]; arg[i] = k; }
    }
    for (int k = 0; k < 4; ++k) {
      const int64_t ip = (nn * h + 2 * yo + (k >> 1)) * w + 2 * xo + (k & 1);
      float o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) o[i] = (v[k][i] > 0.f && arg[i] == k) ? dp[i] : 0.f;
      *reinterpret_cast<uint4*>(dx + ip * dx_ld + dx_off + gi * 8) = pack8(o);
    }
  }
}

// weights [cout][3][3][cin] placed at operand channels [c0, c0 + cin) of cin_pad
__global__ void k_cnn_pad_w(const float* __restrict__ w, int cout, int cin, int cin_pad, int c0,
                            float* __restrict__ out) {
  const int total = cout * 9 * cin_pad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int ci = e % cin_pad - c0, r = e / cin_pad;
    out[e] = (ci >= 0 && ci < cin) ? w[r * cin + ci] : 0.f;
  }
}

// dW^T [9*cin_pad][cout] (+ db), the layer's channels [c0, c0 + cin), into the gradient
// (dW^T rows of ld columns, the layer's outputs at columns [o0, o0 + cout))
__global__ void k_cnn_dwt_to_grad(const float* __restrict__ dwt, const float* __restrict__ db, int cin_pad, int cin,
                                  int c0, int cout, int ld, int o0, float* __restrict__ gw, float* __restrict__ gb) {
  const int total = cout * 9 * cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int ci = e % cin, tap = (e / cin) % 9, o = e / (9 * cin);
    gw[e] = dwt[(tap * cin_pad + c0 + ci) * ld + o0 + o];
  }
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < cout; o += gridDim.x * blockDim.x) gb[o] = db[o0 + o];
}

// network input from the Alg. 1 maps: (h - c_z) / r for both heights (c_z the mean of
// the linear map's 4 central texels), colours / 255; NaN heights become 0
__global__ void k_cnn_inputs(const float* __restrict__ lin_h, const float* __restrict__ nn_h,
                             const uint8_t* __restrict__ lin_rgb, const uint8_t* __restrict__ nn_rgb, int R,
                             float r_m, uint16_t* __restrict__ x, float* __restrict__ cz) {
  const int64_t o = blockIdx.x;
  const float* lh = lin_h + o * R * R;
  const int m = R / 2;
  const float c = 0.25f * (lh[(m - 1) * R + m - 1] + lh[(m - 1) * R + m] + lh[m * R + m - 1] + lh[m * R + m]);
  if (threadIdx.x == 0) cz[o] = c;
  const float inv = 1.f / r_m;
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
    const int64_t e = o * R * R + p;
    float f[8];
    const float a = (lin_h[e] - c) * inv, b = (nn_h[e] - c) * inv;
    f[0] = a == a ? a : 0.f;
    f[1] = b == b ? b : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f[2 + k] = (float)lin_rgb[e * 3 + k] * (1.f / 255.f);
      f[5 + k] = (float)nn_rgb[e * 3 + k] * (1.f / 255.f);
    }
    reinterpret_cast<uint4*>(x)[e] = pack8(f);
  }
}

int cnn_grid(int64_t work) { return grid_cap((work + 255) / 256, kSmCount * 16); }

// the tensor-core convolutions at the res/16 bottleneck take 128 / (res/16)^2 patches
// per 128-pixel tile, so batches are multiples of that
int cnn_batch_multiple(int res) {
  const int bb = (res / 16) * (res / 16);
  return bb >= 128 ? 1 : 128 / bb;
}

}  // namespace
}  // namespace ls

struct ls_cnn {
  int res = 0, max_batch = 0, training = 0;
  int64_t n_params = 0;
  std::vector<ls::CnnLayer> layers;
  void* arena = nullptr;
  // forward activations (bf16 NHWC unless noted)
  uint16_t* ez[4][5] = {};  // encoder conv outputs
  uint16_t* ep[4][4] = {};  // encoder pool outputs
  float* f1in[4] = {};      // flattened encoder outputs (fp32)
  float* zc = nullptr;      // fc1 outputs concatenated [B][1024] (fp32)
  float* g = nullptr;       // fc2 output [B][16 b^2] (fp32)
  uint16_t* gb = nullptr;   // fc2 output as the decoders' input [B][b][b][16]
  uint16_t* dz[2][5] = {};  // decoder conv outputs
  uint16_t* du[2][4] = {};  // decoder upsampled outputs
  uint16_t* cat = nullptr;  // [B][R][R][48]
  uint16_t* fz[2] = {};     // final CNN outputs
  float* yfull = nullptr;   // head output [B][R][R][5]
  // backward scratch
  uint16_t* gbuf[3] = {};
  uint16_t* dgd[2] = {};    // decoder input gradients [B][b][b][16]
  float* dyfull = nullptr, *dg = nullptr, *dzc = nullptr, *dh = nullptr, *df = nullptr;
  float* dwt = nullptr, *dbs = nullptr, *wpad = nullptr;
  // fused first encoder layers: packed operand, bias, padded fp32 weights [64][3][3][8]
  uint16_t* wpk_e0 = nullptr;
  float* bias_e0 = nullptr, *wpad_e0 = nullptr;
  int64_t e0_plane = 0;  // elements between ez[k][0] and ez[k + 1][0]
  uint16_t* dz_e0 = nullptr;  // training: their output gradients interleaved [B][R][R][64]
  const uint16_t* x = nullptr;  // input of the last forward
  int last_n = 0;
};

using namespace ls;

extern "C" ls_status ls_cnn_create(int32_t res, int32_t max_batch, int32_t training, ls_cnn** out) {
  if (!out || max_batch <= 0) return LS_ERR_INVALID_ARG;
  if (res != 32 && res != 64 && res != 128) return LS_ERR_UNSUPPORTED;
  const int b = res / 16;
  if (max_batch % cnn_batch_multiple(res)) return LS_ERR_UNSUPPORTED;
  ls_cnn* m = new (std::nothrow) ls_cnn();
  if (!m) return LS_ERR_NO_MEMORY;
  m->res = res;
  m->max_batch = max_batch;
  m->training = training ? 1 : 0;
  int64_t off = 0;
  auto add = [&](int kind, int cin, int cout, int cin_pad, int c0, int h) {
    CnnLayer d;
    d.kind = kind; d.cin = cin; d.cout = cout; d.cin_pad = cin_pad; d.c0 = c0; d.h = h;
    d.w_off = off;
    off += (int64_t)cout * cin * (kind == kCnnConv ? 9 : 1);
    d.b_off = off;
    off += cout;
    m->layers.push_back(d);
  };
  for (int k = 0; k < 4; ++k) {
    int cin = kCnnEncCk[k];
    for (int l = 0; l < 4; ++l) {
      add(kCnnConv, cin, kCnnEncW[l], l == 0 ? kCnnIn : cin, l == 0 ? kCnnEncC0[k] : 0, res >> l);
      cin = kCnnEncW[l];
    }
    add(kCnnConv, cin, kCnnEncOut, cin, 0, b);
  }
  const int flat = kCnnEncOut * b * b;
  for (int k = 0; k < 4; ++k) add(kCnnFc, flat, kCnnFc1, flat, 0, 0);
  add(kCnnFc, 4 * kCnnFc1, flat, 4 * kCnnFc1, 0, 0);
  for (int j = 0; j < 2; ++j) {
    int cin = kCnnEncOut;
    for (int l = 0; l < 5; ++l) {
      add(kCnnConv, cin, kCnnDecW[l], cin, 0, b << l);
      cin = kCnnDecW[l];
    }
  }
  add(kCnnConv, kCatUsed, 32, kCatPad, 0, res);
  add(kCnnConv, 32, 16, 32, 0, res);
  add(kCnnHead, 16, 5, 16, 0, res);
  m->n_params = off;
  // ---- one arena
  const int64_t B = max_batch, R = res;
  size_t bytes = 0;
  auto take = [&](size_t nbytes) { size_t o = bytes; bytes += (nbytes + 255) / 256 * 256; return o; };
  size_t o_ez[4][5], o_ep[4][4], o_f1[4], o_dz[2][5], o_du[2][4];
  // the four encoders' first-layer outputs back to back (the fused layer's output groups)
  const int64_t e0_plane = B * R * R * kCnnEncW[0];
  const size_t o_e0 = take((size_t)4 * e0_plane * 2);
  for (int k = 0; k < 4; ++k) {
    for (int l = 0; l < 4; ++l) {
      o_ez[k][l] = l == 0 ? o_e0 + (size_t)k * e0_plane * 2 : take((size_t)B * (R >> l) * (R >> l) * kCnnEncW[l] * 2);
      o_ep[k][l] = take((size_t)B * (R >> (l + 1)) * (R >> (l + 1)) * kCnnEncW[l] * 2);
    }
    o_ez[k][4] = take((size_t)B * flat * 2);
    o_f1[k] = take((size_t)B * flat * 4);
  }
  const size_t o_zc = take((size_t)B * 4 * kCnnFc1 * 4), o_g = take((size_t)B * flat * 4);
  const size_t o_gb = take((size_t)B * flat * 2);
  for (int j = 0; j < 2; ++j)
    for (int l = 0; l < 5; ++l) {
      const int64_t h = (int64_t)b << l;
      o_dz[j][l] = take((size_t)B * h * h * kCnnDecW[l] * 2);
      if (l < 4) o_du[j][l] = take((size_t)B * 4 * h * h * kCnnDecW[l] * 2);
    }
  const size_t o_cat = take((size_t)B * R * R * kCatPad * 2);
  const size_t o_f0 = take((size_t)B * R * R * 32 * 2), o_f1x = take((size_t)B * R * R * 16 * 2);
  const size_t o_y = take((size_t)B * R * R * 5 * 4);
  std::vector<size_t> o_pk, o_pkt;
  std::vector<bool> has_t;
  for (auto& d : m->layers) {
    const bool conv = d.kind == kCnnConv;
    // the input-gradient operand, for training, except for the encoders' first layers
    // (the network input needs no gradient)
    const bool need_t = conv && training && d.cin >= 8;
    o_pk.push_back(conv ? take((size_t)ls_conv3x3_packed_elems(d.cin_pad, d.cout) * 2) : 0);
    o_pkt.push_back(need_t ? take((size_t)ls_conv3x3_packed_elems(d.cout, d.cin_pad) * 2) : 0);
    has_t.push_back(need_t);
  }
  size_t o_gbuf[3] = {0, 0, 0}, o_dgd[2] = {0, 0}, o_dyf = 0, o_dg = 0, o_dzc = 0, o_dh = 0, o_df = 0;
  if (training) {
    for (int i = 0; i < 3; ++i) o_gbuf[i] = take((size_t)B * R * R * kCatPad * 2);
    for (int j = 0; j < 2; ++j) o_dgd[j] = take((size_t)B * flat * 2);
    o_dyf = take((size_t)B * R * R * 5 * 4);
    o_dg = take((size_t)B * flat * 4);
    o_dzc = take((size_t)B * 4 * kCnnFc1 * 4);
    o_dh = take((size_t)B * kCnnFc1 * 4);
    o_df = take((size_t)B * flat * 4);
  }
  const size_t o_dz_e0 = training ? take((size_t)B * R * R * kCnnE0Fused * 2) : 0;
  const size_t o_dwt = take((size_t)9 * 64 * 64 * 4), o_dbs = take(256 * 4);
  const size_t o_wpad = take((size_t)9 * kCatPad * 32 * 4);
  const size_t o_wpk_e0 = take((size_t)ls_conv3x3_packed_elems(kCnnIn, kCnnE0Fused) * 2);
  const size_t o_bias_e0 = take((size_t)kCnnE0Fused * 4), o_wpad_e0 = take((size_t)kCnnE0Fused * 9 * kCnnIn * 4);
  if (cudaMalloc(&m->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return LS_ERR_NO_MEMORY;
  }
  char* base = static_cast<char*>(m->arena);
  auto bf = [&](size_t o) { return reinterpret_cast<uint16_t*>(base + o); };
  auto fp = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
  for (int k = 0; k < 4; ++k) {
    for (int l = 0; l < 4; ++l) {
      m->ez[k][l] = bf(o_ez[k][l]);
      m->ep[k][l] = bf(o_ep[k][l]);
    }
    m->ez[k][4] = bf(o_ez[k][4]);
    m->f1in[k] = fp(o_f1[k]);
  }
  m->zc = fp(o_zc);
  m->g = fp(o_g);
  m->gb = bf(o_gb);
  for (int j = 0; j < 2; ++j)
    for (int l = 0; l < 5; ++l) {
      m->dz[j][l] = bf(o_dz[j][l]);
      if (l < 4) m->du[j][l] = bf(o_du[j][l]);
    }
  m->cat = bf(o_cat);
  m->fz[0] = bf(o_f0);
  m->fz[1] = bf(o_f1x);
  m->yfull = fp(o_y);
  for (size_t i = 0; i < m->layers.size(); ++i) {
    if (m->layers[i].kind != kCnnConv) continue;
    m->layers[i].wpk = bf(o_pk[i]);
    if (has_t[i]) m->layers[i].wpk_t = bf(o_pkt[i]);
  }
  if (training) {
    for (int i = 0; i < 3; ++i) m->gbuf[i] = bf(o_gbuf[i]);
    for (int j = 0; j < 2; ++j) m->dgd[j] = bf(o_dgd[j]);
    m->dyfull = fp(o_dyf);
    m->dg = fp(o_dg);
    m->dzc = fp(o_dzc);
    m->dh = fp(o_dh);
    m->df = fp(o_df);
    m->dz_e0 = bf(o_dz_e0);
  }
  m->dwt = fp(o_dwt);
  m->dbs = fp(o_dbs);
  m->wpad = fp(o_wpad);
  m->wpk_e0 = bf(o_wpk_e0);
  m->bias_e0 = fp(o_bias_e0);
  m->wpad_e0 = fp(o_wpad_e0);
  m->e0_plane = e0_plane;
  *out = m;
  return LS_OK;
}

extern "C" void ls_cnn_destroy(ls_cnn* m) {
  if (!m) return;
  if (m->arena) cudaFree(m->arena);
  delete m;
}

extern "C" int64_t ls_cnn_param_count(const ls_cnn* m) { return m ? m->n_params : -1; }
extern "C" int32_t ls_cnn_layer_count(const ls_cnn* m) { return m ? (int32_t)m->layers.size() : -1; }

extern "C" ls_status ls_cnn_layer_info(const ls_cnn* m, int32_t i, int32_t* kind, int32_t* cin, int32_t* cout,
                                       int64_t* w_offset, int64_t* b_offset) {
  if (!m || i < 0 || i >= (int)m->layers.size()) return LS_ERR_INVALID_ARG;
  const CnnLayer& d = m->layers[i];
  if (kind) *kind = d.kind;
  if (cin) *cin = d.cin;
  if (cout) *cout = d.cout;
  if (w_offset) *w_offset = d.w_off;
  if (b_offset) *b_offset = d.b_off;
  return LS_OK;
}

extern "C" ls_status ls_cnn_load(ls_cnn* m, const float* params, ls_stream_t stream) {
  if (!m || !params) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<PackJob> jobs;
  for (size_t li = 0; li < m->layers.size(); ++li) {
    const CnnLayer& d = m->layers[li];
    if (d.kind != kCnnConv) continue;
    const float* w = params + d.w_off;
    if (li < 20 && li % 5 == 0) {
      // first layer of encoder li / 5: its padded weights and bias into the fused layer
      const int k = (int)li / 5;
      k_cnn_pad_w<<<cnn_grid((int64_t)d.cout * 9 * d.cin_pad), 256, 0, s>>>(
          w, d.cout, d.cin, d.cin_pad, d.c0, m->wpad_e0 + (size_t)k * d.cout * 9 * d.cin_pad);
      LS_CUDA_TRY(cudaMemcpyAsync(m->bias_e0 + k * d.cout, params + d.b_off, (size_t)d.cout * 4,
                                  cudaMemcpyDeviceToDevice, s));
      continue;
    }
    // a padded layer packs at once (the padding scratch is reused by the next one); the
    // others join one batched pack launch at the end
    const bool padded = d.cin != d.cin_pad;
    if (padded) {
      k_cnn_pad_w<<<cnn_grid((int64_t)d.cout * 9 * d.cin_pad), 256, 0, s>>>(w, d.cout, d.cin, d.cin_pad, d.c0,
                                                                          m->wpad);
      w = m->wpad;
    }
    PackJob pj[2] = {{w, d.wpk, d.cin_pad, d.cout, 0}, {w, d.wpk_t, d.cout, d.cin_pad, 1}};
    const int np = d.wpk_t ? 2 : 1;  // the input-gradient operand: flipped and transposed
    if (padded) {
      const ls_status st = conv3x3_pack_batch(pj, np, s);
      if (st != LS_OK) return st;
    } else {
      for (int j = 0; j < np; ++j) jobs.push_back(pj[j]);
    }
  }
  jobs.push_back({m->wpad_e0, m->wpk_e0, kCnnIn, kCnnE0Fused, 0});
  const ls_status st = conv3x3_pack_batch(jobs.data(), (int)jobs.size(), s);
  if (st != LS_OK) return st;
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

namespace {

// Few output tiles (batch 256: a 256 x 256 output is 16 CTAs) split K into slices of
// a multiple of 64 so that about two CTAs per SM run; the slices are added in order.
ls_status gemm(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk,
               int64_t sbn, float* C, int64_t ldc, const float* bias, int relu, const float* mask, int64_t ldm,
               cudaStream_t s) {
  const int gx = (N + kGt - 1) / kGt, gy = (M + kGt - 1) / kGt;
  int splits = 1;
  if ((int64_t)gx * gy < 2 * kSmCount && K >= 128) {
    splits = (int)((2 * kSmCount + (int64_t)gx * gy - 1) / ((int64_t)gx * gy));
    splits = std::min(splits, K / 64);
  }
  const int kc = (K + splits * 64 - 1) / (splits * 64) * 64;  // slice length, multiple of 64
  splits = (K + kc - 1) / kc;
  float* part = nullptr;
  if (splits > 1) {
    part = static_cast<float*>(workspace(kWsGemmPart, (size_t)splits * M * N * 4));
    if (!part) return LS_ERR_NO_MEMORY;
  }
  dim3 grid(gx, gy, splits);
  k_gemm<<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu, mask, ldm, kc, part);
  if (splits > 1)
    k_gemm_reduce<<<cnn_grid((int64_t)M * N), 256, 0, s>>>(M, N, splits, part, C, ldc, bias, relu, mask, ldm);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace

extern "C" ls_status ls_cnn_forward(ls_cnn* m, const float* params, const uint16_t* x, int32_t n, float* y,
                                    ls_stream_t stream) {
  if (!m || !params || !x || !y || n <= 0 || n > m->max_batch) return LS_ERR_INVALID_ARG;
  const int R = m->res, b = R / 16, flat = kCnnEncOut * b * b;
  if (n % cnn_batch_multiple(R)) return LS_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto conv = [&](const CnnLayer& d, const uint16_t* in, uint16_t* out) {
    return conv3x3_launch(in, d.wpk, params + d.b_off, nullptr, 1, n, d.h, d.h, d.cin_pad, d.cout, out, s);
  };
  ls_status st;
  // the four encoders' first layers: one convolution, output groups of 16 channels into
  // ez[0..3][0]
  if ((st = conv3x3_launch_groups(x, m->wpk_e0, m->bias_e0, nullptr, 1, n, R, R, kCnnIn, kCnnE0Fused, m->ez[0][0],
                                  kCnnEncW[0], m->e0_plane, s)) != LS_OK)
    return st;
  int li = 0;
  for (int k = 0; k < 4; ++k) {
    const uint16_t* in = x;
    for (int l = 0; l < 4; ++l) {
      const CnnLayer& d = m->layers[li++];
      if (l > 0 && (st = conv(d, in, m->ez[k][l])) != LS_OK) return st;
      const int h = R >> l;
      k_maxpool<<<cnn_grid((int64_t)n * (h / 2) * (h / 2) * (d.cout / 8)), 256, 0, s>>>(m->ez[k][l], n, h, h, d.cout,
                                                                                     m->ep[k][l]);
      in = m->ep[k][l];
    }
    if ((st = conv(m->layers[li++], in, m->ez[k][4])) != LS_OK) return st;
    k_bf16_to_f32<<<cnn_grid((int64_t)n * flat), 256, 0, s>>>(m->ez[k][4], (int64_t)n * flat, m->f1in[k]);
  }
  for (int k = 0; k < 4; ++k) {  // fc1.k into columns [256 k, 256 k + 256) of zc
    const CnnLayer& d = m->layers[li++];
    if ((st = gemm(n, kCnnFc1, flat, m->f1in[k], flat, 1, params + d.w_off, 1, flat, m->zc + kCnnFc1 * k,
                   4 * kCnnFc1, params + d.b_off, 1, nullptr, 0, s)) != LS_OK)
      return st;
  }
  {
    const CnnLayer& d = m->layers[li++];
    if ((st = gemm(n, flat, 4 * kCnnFc1, m->zc, 4 * kCnnFc1, 1, params + d.w_off, 1, 4 * kCnnFc1, m->g, flat,
                   params + d.b_off, 1, nullptr, 0, s)) != LS_OK)
      return st;
    k_f32_to_bf16_masked<<<cnn_grid((int64_t)n * flat), 256, 0, s>>>(m->g, nullptr, (int64_t)n * flat, m->gb);
  }
  for (int j = 0; j < 2; ++j) {
    const uint16_t* in = m->gb;
    for (int l = 0; l < 5; ++l) {
      const CnnLayer& d = m->layers[li++];
      if ((st = conv(d, in, m->dz[j][l])) != LS_OK) return st;
      if (l < 4) {
        const int h2 = 2 * d.h;
        k_upcat<<<cnn_grid((int64_t)n * h2 * h2 * (d.cout / 8)), 256, 0, s>>>(m->dz[j][l], d.cout, nullptr, 0, n, h2,
                                                                             h2, m->du[j][l]);
        in = m->du[j][l];
      }
    }
  }
  const int64_t P = (int64_t)n * R * R;
  k_cnn_concat<<<cnn_grid(P * (kCatPad / 8)), 256, 0, s>>>(x, m->dz[0][4], m->dz[1][4], P, m->cat);
  if ((st = conv(m->layers[li++], m->cat, m->fz[0])) != LS_OK) return st;
  if ((st = conv(m->layers[li++], m->fz[0], m->fz[1])) != LS_OK) return st;
  const CnnLayer& hd = m->layers[li];
  k_head_fwd<<<cnn_grid(P), 256, (size_t)(kOut * hd.cin + kOut) * 4, s>>>(m->fz[1], hd.cin, params + hd.w_off, P,
                                                                         m->yfull);
  k_cnn_crop<<<cnn_grid((int64_t)n * (R / 2) * (R / 2) * 5), 256, 0, s>>>(m->yfull, n, R, y);
  m->x = x;
  m->last_n = n;
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_cnn_backward(ls_cnn* m, const float* params, const float* dy, int32_t n, float* grads,
                                     ls_stream_t stream) {
  if (!m || !params || !dy || !grads || !m->training || n != m->last_n || !m->x) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int R = m->res, b = R / 16, flat = kCnnEncOut * b * b;
  const int64_t P = (int64_t)n * R * R;
  const int nl = (int)m->layers.size();
  LS_CUDA_TRY(cudaMemsetAsync(grads, 0, (size_t)m->n_params * 4, s));
  auto wgrad = [&](const CnnLayer& d, const uint16_t* in, const uint16_t* dz) -> ls_status {
    if (cudaMemsetAsync(m->dwt, 0, (size_t)9 * d.cin_pad * d.cout * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    if (cudaMemsetAsync(m->dbs, 0, (size_t)d.cout * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    ls_status st = wgrad_launch(in, dz, n, d.h, d.h, d.cin_pad, d.cout, m->dwt, m->dbs, s);
    if (st != LS_OK) return st;
    k_cnn_dwt_to_grad<<<cnn_grid((int64_t)d.cout * 9 * d.cin), 256, 0, s>>>(m->dwt, m->dbs, d.cin_pad, d.cin, d.c0,
                                                                          d.cout, d.cout, 0, grads + d.w_off,
                                                                          grads + d.b_off);
    return LS_OK;
  };
  auto dgrad = [&](const CnnLayer& d, const uint16_t* dz, const uint16_t* mask, uint16_t* dx) -> ls_status {
    return conv3x3_launch(dz, d.wpk_t, nullptr, mask, 0, n, d.h, d.h, d.cout, d.cin_pad, dx, s);
  };
  ls_status st;
  // layer indices
  const int l_f0 = nl - 3, l_f1 = nl - 2, l_head = nl - 1;
  const int l_fc1 = 20, l_fc2 = 24, l_dec = 25;  // e*: 0..19, fc1.*: 20..23, fc2: 24, d*: 25..34
  // ---- head and final CNN
  k_cnn_uncrop<<<cnn_grid(P * 5), 256, 0, s>>>(dy, n, R, m->dyfull);
  uint16_t* dfz1 = m->gbuf[0];
  {
    const CnnLayer& hd = m->layers[l_head];
    const int blocks = grid_cap((P + kHeadThreads - 1) / kHeadThreads, kSmCount * 4);
    const int ng = kOut * hd.cin + kOut;
    float* part = static_cast<float*>(workspace(kWsHeadPart, (size_t)blocks * ng * 4));
    if (!part) return LS_ERR_NO_MEMORY;
    const size_t smem = (size_t)(kOut * hd.cin + (kHeadThreads / 32) * ng) * 4;
    k_head_bwd<<<blocks, kHeadThreads, smem, s>>>(m->fz[1], hd.cin, params + hd.w_off, m->dyfull, P, dfz1, part);
    k_head_sum<<<ng, 256, 0, s>>>(part, blocks, ng, grads + hd.w_off);
  }
  if ((st = wgrad(m->layers[l_f1], m->fz[0], dfz1)) != LS_OK) return st;
  uint16_t* dfz0 = m->gbuf[1];
  if ((st = dgrad(m->layers[l_f1], dfz1, m->fz[0], dfz0)) != LS_OK) return st;
  if ((st = wgrad(m->layers[l_f0], m->cat, dfz0)) != LS_OK) return st;
  uint16_t* dcat = m->gbuf[2];
  if ((st = dgrad(m->layers[l_f0], dfz0, m->cat, dcat)) != LS_OK) return st;  // decoder channels: ReLU mask
  // ---- decoders
  for (int j = 0; j < 2; ++j) {
    uint16_t* gz = m->gbuf[0];
    k_cnn_slice16<<<cnn_grid(P * 2), 256, 0, s>>>(dcat, kCnnIn + 16 * j, P, gz);
    for (int l = 4; l >= 0; --l) {
      const CnnLayer& d = m->layers[l_dec + 5 * j + l];
      const uint16_t* in = l == 0 ? m->gb : m->du[j][l - 1];
      if ((st = wgrad(d, in, gz)) != LS_OK) return st;
      uint16_t* gx = l == 0 ? m->dgd[j] : m->gbuf[1];
      if ((st = dgrad(d, gz, in, gx)) != LS_OK) return st;  // masked by the (upsampled) ReLU input > 0
      if (l > 0) {
        const int hl = d.h / 2;  // the previous conv's size
        const int c = m->layers[l_dec + 5 * j + l - 1].cout;
        k_up_bwd<<<cnn_grid((int64_t)n * hl * hl * (c / 8)), 256, 0, s>>>(gx, c, c, n, hl, hl, m->gbuf[0]);
        gz = m->gbuf[0];
      }
    }
  }
  // ---- fc2 and fc1 (fp32); the decoders' input gradients are already ReLU-masked
  k_add_bf16_f32<<<cnn_grid((int64_t)n * flat), 256, 0, s>>>(m->dgd[0], m->dgd[1], (int64_t)n * flat, m->dg);
  {
    const CnnLayer& d = m->layers[l_fc2];
    // dW[out][in] = dg^T zc; db = column sums; dzc = dg W masked by zc > 0
    if ((st = gemm(flat, 4 * kCnnFc1, n, m->dg, 1, flat, m->zc, 4 * kCnnFc1, 1, grads + d.w_off, 4 * kCnnFc1, nullptr,
                   0, nullptr, 0, s)) != LS_OK)
      return st;
    k_colsum_rows<<<cnn_grid(flat), 256, 0, s>>>(m->dg, n, flat, flat, grads + d.b_off);
    if ((st = gemm(n, 4 * kCnnFc1, flat, m->dg, flat, 1, params + d.w_off, 4 * kCnnFc1, 1, m->dzc, 4 * kCnnFc1,
                   nullptr, 0, m->zc, 4 * kCnnFc1, s)) != LS_OK)
      return st;
  }
  for (int k = 0; k < 4; ++k) {
    const CnnLayer& d = m->layers[l_fc1 + k];
    const float* dhk = m->dzc + kCnnFc1 * k;  // [n][256] with row stride 1024
    if ((st = gemm(kCnnFc1, flat, n, dhk, 1, 4 * kCnnFc1, m->f1in[k], flat, 1, grads + d.w_off, flat, nullptr, 0,
                   nullptr, 0, s)) != LS_OK)
      return st;
    k_colsum_rows<<<cnn_grid(kCnnFc1), 256, 0, s>>>(dhk, n, kCnnFc1, 4 * kCnnFc1, grads + d.b_off);
    if ((st = gemm(n, flat, kCnnFc1, dhk, 4 * kCnnFc1, 1, params + d.w_off, flat, 1, m->df, flat, nullptr, 0,
                   m->f1in[k], flat, s)) != LS_OK)
      return st;
    // ---- encoder k, from its last conv back to the first
    uint16_t* gz = m->gbuf[0];
    k_f32_to_bf16_masked<<<cnn_grid((int64_t)n * flat), 256, 0, s>>>(m->df, nullptr, (int64_t)n * flat, gz);
    for (int l = 4; l >= 1; --l) {
      const CnnLayer& d2 = m->layers[5 * k + l];
      const uint16_t* in = m->ep[k][l - 1];
      if ((st = wgrad(d2, in, gz)) != LS_OK) return st;
      uint16_t* gp = m->gbuf[1];
      if ((st = dgrad(d2, gz, nullptr, gp)) != LS_OK) return st;  // d(pooled), raw
      const CnnLayer& prev = m->layers[5 * k + l - 1];
      const int h = prev.h;
      // the first layer's output gradient goes to channels [16 k, 16 k + 16) of dz_e0
      const bool first = l == 1;
      k_maxpool_bwd_relu<<<cnn_grid((int64_t)n * (h / 2) * (h / 2) * (prev.cout / 8)), 256, 0, s>>>(
          m->ez[k][l - 1], gp, n, h, h, prev.cout, first ? m->dz_e0 : m->gbuf[2], first ? kCnnE0Fused : prev.cout,
          first ? prev.cout * k : 0);
      if (first) break;
      gz = m->gbuf[2];
      // keep gz out of the buffers the next layer writes
      uint16_t* t = m->gbuf[0];
      m->gbuf[0] = m->gbuf[2];
      m->gbuf[2] = t;
    }
  }
  // the four encoders' first layers: one weight gradient with 64 output channels, split
  {
    if (cudaMemsetAsync(m->dwt, 0, (size_t)9 * kCnnIn * kCnnE0Fused * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    if (cudaMemsetAsync(m->dbs, 0, (size_t)kCnnE0Fused * 4, s) != cudaSuccess) return LS_ERR_CUDA;
    if ((st = wgrad_launch(m->x, m->dz_e0, n, R, R, kCnnIn, kCnnE0Fused, m->dwt, m->dbs, s)) != LS_OK) return st;
    for (int k = 0; k < 4; ++k) {
      const CnnLayer& d = m->layers[5 * k];
      k_cnn_dwt_to_grad<<<cnn_grid((int64_t)d.cout * 9 * d.cin), 256, 0, s>>>(
          m->dwt, m->dbs, d.cin_pad, d.cin, d.c0, d.cout, kCnnE0Fused, d.cout * k, grads + d.w_off, grads + d.b_off);
    }
  }
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_cnn_inputs(const float* lin_height, const float* nn_height, const uint8_t* lin_rgb,
                                   const uint8_t* nn_rgb, int64_t n, int32_t res, float r_m, uint16_t* x, float* cz,
                                   ls_stream_t stream) {
  if (!lin_height || !nn_height || !lin_rgb || !nn_rgb || !x || !cz || n < 0 || res < 2 || res % 2 || !(r_m > 0.f))
    return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(x) & 15u) return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  k_cnn_inputs<<<(unsigned)n, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(lin_height, nn_height, lin_rgb,
                                                                                  nn_rgb, res, r_m, x, cz);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
