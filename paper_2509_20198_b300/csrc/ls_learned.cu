// Learned heightmap fill around the U-Net of ls_unet.cu:
//  * input raster (5 channels, padded to 8, bf16): height of the tile's own sparse
//    samples, their luma, an occupancy mask, the distance to the nearest sample and
//    the Gaussian-fill height; heights normalised to patch space as (z - c_z) / r
//    with r = half the tile side and c_z the Gaussian-fill height at the tile centre
//    (Sec. 3.3, 3.4: patch-space normalisation with c_z from the patch centre);
//  * training targets: the per-texel mean of the full-resolution points (Sec. 3.4:
//    ground truth is the mean of all points falling onto a texel), masked where a
//    texel has no point (the NaN elements of the paper's ground truth);
//  * finish: de-normalise the residual prediction, estimate the tile's error bound
//    from the fifth output (RMS) and fall back to the Gaussian fill above a limit.
#include "ls_tc.cuh"

namespace ls {

ls_status fill_launch(const ls_points* samples, const ls_region* region, const ls_fill_params* params,
                      const int32_t* tile_ids, int64_t n_out, float* height, uint8_t* rgb, float4* aux_hc,
                      float* aux_d, cudaStream_t s, const void** recs_out);

namespace {

constexpr int kLearnedThreads = 256;

__device__ __forceinline__ uint16_t to_bf16(float f) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&h);
}

__global__ void __launch_bounds__(kLearnedThreads) k_raster(const Rec* __restrict__ recs,
                                                            const int64_t* __restrict__ toff,
                                                            const int32_t* __restrict__ tile_ids, int64_t n,
                                                            int64_t n_tiles, int tiles_x, int tile_cm, int res,
                                                            float radius_cm,
                                                            double z_scale, double z_offset,
                                                            const float4* __restrict__ aux_hc,
                                                            const float* __restrict__ aux_d,
                                                            uint16_t* __restrict__ x, float4* __restrict__ base,
                                                            float* __restrict__ cz_out) {
  extern __shared__ int first[];  // [res*res]
  const int cell = tile_cm / res;
  const float r_m = (float)(0.5 * tile_cm * z_scale);
  for (int64_t o = blockIdx.x; o < n; o += gridDim.x) {
    const int t = tile_ids ? tile_ids[o] : (int)o;
    if (t < 0 || t >= n_tiles) continue;  // reported by the fill kernel; uniform per CTA
    const int tx = t % tiles_x, ty = t / tiles_x;
    const float4* hc = aux_hc + (size_t)o * res * res;
    const int c = res / 2;
    const float cz = 0.25f * (hc[(c - 1) * res + c - 1].x + hc[(c - 1) * res + c].x + hc[c * res + c - 1].x +
                              hc[c * res + c].x);
    for (int e = threadIdx.x; e < res * res; e += blockDim.x) first[e] = INT_MAX;
    __syncthreads();
    const int64_t q0 = toff[t], q1 = toff[t + 1];
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const Rec rc = recs[q];
      const int i = (rc.ly - ty * tile_cm) / cell, j = (rc.lx - tx * tile_cm) / cell;
      if (i >= 0 && i < res && j >= 0 && j < res) atomicMin(&first[i * res + j], (int)q);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < res * res; e += blockDim.x) {
      const float4 f = hc[e];
      float ch[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int q = first[e];
      if (q != INT_MAX) {
        const Rec rc = recs[q];
        const float zm = (float)((double)rc.z * z_scale + z_offset);
        ch[0] = (zm - cz) / r_m;
        ch[1] = (0.299f * (float)(rc.rg & 0xffffu) + 0.587f * (float)(rc.rg >> 16) + 0.114f * (float)rc.b) *
                (1.0f / 65535.0f);
        ch[2] = 1.f;
      }
      ch[3] = fminf(aux_d[(size_t)o * res * res + e], 2.f * radius_cm) / radius_cm;
      ch[4] = (f.x - cz) / r_m;
      uint4 v;
      v.x = (uint32_t)to_bf16(ch[0]) | ((uint32_t)to_bf16(ch[1]) << 16);
      v.y = (uint32_t)to_bf16(ch[2]) | ((uint32_t)to_bf16(ch[3]) << 16);
      v.z = (uint32_t)to_bf16(ch[4]);
      v.w = 0u;
      *reinterpret_cast<uint4*>(x + ((size_t)o * res * res + e) * 8) = v;
      base[(size_t)o * res * res + e] = make_float4(ch[4], f.y, f.z, f.w);
    }
    if (threadIdx.x == 0) cz_out[o] = cz;
    __syncthreads();
  }
}

__global__ void k_targets(ls_bins bins, const int32_t* __restrict__ tile_ids, int64_t n, int64_t n_tiles,
                          double z_scale, double z_offset, float r_m, const float* __restrict__ cz,
                          float4* __restrict__ target, uint8_t* __restrict__ mask) {
  const int64_t cpt = (int64_t)bins.cells * bins.cells;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cpt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e / cpt, c = e - o * cpt;
    const int64_t t = tile_ids ? (int64_t)tile_ids[o] : o;
    if (t < 0 || t >= n_tiles) { set_status(LS_ERR_INVALID_ARG); continue; }
    const int64_t src = t * cpt + c;
    const uint32_t cnt = bins.count[src];
    if (!cnt) {
      mask[e] = 0;
      target[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const double nd = (double)cnt;
    const double zm = (double)bins.zsum[src] / nd * z_scale + z_offset;
    mask[e] = 1;
    target[e] = make_float4((float)((zm - cz[o]) / r_m), (float)((double)bins.rsum[src] / nd / 65535.0),
                            (float)((double)bins.gsum[src] / nd / 65535.0),
                            (float)((double)bins.bsum[src] / nd / 65535.0));
  }
}

__global__ void __launch_bounds__(kLearnedThreads) k_finish(const float* __restrict__ y, const float4* __restrict__ base,
                                                            const float* __restrict__ cz, int64_t n, int res,
                                                            float r_m, float max_err_m,
                                                            const float* fill_h, const uint8_t* fill_c,
                                                            float* height, uint8_t* rgb,  // may alias fill_*
                                                            float* __restrict__ err_bound,
                                                            uint8_t* __restrict__ used_fallback) {
  __shared__ float red[kLearnedThreads / 32];
  __shared__ int fb;
  const int np = res * res;
  for (int64_t o = blockIdx.x; o < n; o += gridDim.x) {
    float s = 0.f;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      const float v = y[((size_t)o * np + e) * 5 + 4];
      const float b = v < 0.f ? 0.f : v;  // max(v, 0) that keeps a NaN (fmaxf would drop it)
      s += b * b;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int k = 0; k < kLearnedThreads / 32; ++k) t += red[k];
      const float bound = sqrtf(t / np) * r_m;
      fb = !(bound <= max_err_m);  // NaN bound also falls back
      if (err_bound) err_bound[o] = bound;
      if (used_fallback) used_fallback[o] = (uint8_t)fb;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      const size_t pe = (size_t)o * np + e;
      if (fb) {
        height[pe] = fill_h[pe];
        rgb[pe * 3] = fill_c[pe * 3]; rgb[pe * 3 + 1] = fill_c[pe * 3 + 1]; rgb[pe * 3 + 2] = fill_c[pe * 3 + 2];
        continue;
      }
      const float4 b = base[pe];
      const float* yp = y + pe * 5;
      height[pe] = (b.x + yp[0]) * r_m + cz[o];
      const float cc[3] = {b.y + yp[1], b.z + yp[2], b.w + yp[3]};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float v = floorf(fminf(fmaxf(cc[k], 0.f), 1.f) * 255.f + 0.5f);
        rgb[pe * 3 + k] = (uint8_t)v;
      }
    }
    __syncthreads();
  }
}

struct LearnedScratch {
  void* mem = nullptr;
  size_t bytes = 0;
};

}  // namespace

ls_status learned_inputs_launch(const ls_points* samples, const ls_region* region, const ls_fill_params* params,
                                const int32_t* tile_ids, int64_t n, uint16_t* x, float4* base, float* cz,
                                float* fill_h, uint8_t* fill_c, float4* aux_hc, float* aux_d, cudaStream_t s) {
  const void* recs = nullptr;
  ls_status st = fill_launch(samples, region, params, tile_ids, n, fill_h, fill_c, aux_hc, aux_d, s, &recs);
  if (st != LS_OK || n == 0) return st;
  const int res = params->res;
  k_raster<<<grid_cap(n, kSmCount * 4), kLearnedThreads, (size_t)res * res * sizeof(int), s>>>(
      static_cast<const Rec*>(recs), samples->tile_offsets, tile_ids, n,
      (int64_t)region->tiles_x * region->tiles_y, region->tiles_x, region->tile_cm, res,
      (float)params->radius_cm, region->z_scale, region->z_offset, aux_hc, aux_d, x, base, cz);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

}  // namespace ls

extern "C" ls_status ls_learned_inputs(const ls_points* samples, const ls_region* region, const ls_fill_params* params,
                                       const int32_t* tile_ids, int64_t n, uint16_t* x, float* base, float* cz,
                                       float* fill_height, uint8_t* fill_rgb, float* aux, ls_stream_t stream) {
  if (!x || !base || !cz || !fill_height || !fill_rgb || !aux || !params) return LS_ERR_INVALID_ARG;
  if (params->res > 128) return LS_ERR_UNSUPPORTED;
  const size_t np = (size_t)n * params->res * params->res;
  return ls::learned_inputs_launch(samples, region, params, tile_ids, n, x, reinterpret_cast<float4*>(base), cz,
                                   fill_height, fill_rgb, reinterpret_cast<float4*>(aux),
                                   aux + 4 * np, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" ls_status ls_learned_targets(const ls_bins* bins, const ls_region* region, const int32_t* tile_ids,
                                        int64_t n, const float* cz, float* target, uint8_t* mask,
                                        ls_stream_t stream) {
  if (!bins || !region || !cz || !target || !mask || n < 0 || !bins->count || bins->cells <= 0) return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  const int64_t T = (int64_t)region->tiles_x * region->tiles_y;
  if (!tile_ids && n > T) return LS_ERR_INVALID_ARG;
  const int64_t total = n * bins->cells * bins->cells;
  const float r_m = (float)(0.5 * region->tile_cm * region->z_scale);
  ls::k_targets<<<ls::grid_cap((total + 255) / 256, ls::kSmCount * 16), 256, 0,
                  reinterpret_cast<cudaStream_t>(stream)>>>(*bins, tile_ids, n, T, region->z_scale, region->z_offset,
                                                            r_m, cz, reinterpret_cast<float4*>(target), mask);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

extern "C" ls_status ls_learned_finish(const float* y, const float* base, const float* cz, int64_t n, int32_t res,
                                       const ls_region* region, float max_err_m, const float* fill_height,
                                       const uint8_t* fill_rgb, float* height, uint8_t* rgb, float* err_bound,
                                       uint8_t* used_fallback, ls_stream_t stream) {
  if (!y || !base || !cz || !region || !fill_height || !fill_rgb || !height || !rgb || n < 0 || res <= 0)
    return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  const float r_m = (float)(0.5 * region->tile_cm * region->z_scale);
  ls::k_finish<<<ls::grid_cap(n, ls::kSmCount * 8), ls::kLearnedThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      y, reinterpret_cast<const float4*>(base), cz, n, res, r_m, max_err_m, fill_height, fill_rgb, height, rgb,
      err_bound, used_fallback);
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

// the filler's forward pass (ls_unet.cu); keep_top = false fuses the head into the last
// convolution and leaves no state for a backward pass
ls_status filler_forward(ls_model* m, const float* params, const uint16_t* x, int32_t n, float* y, cudaStream_t s,
                         bool keep_top);

extern "C" ls_status ls_fill_learned(ls_model* model, const float* params, const ls_points* samples,
                                     const ls_region* region, const ls_fill_params* fp, const int32_t* tile_ids,
                                     int64_t n, float max_err_m, float* height, uint8_t* rgb, float* err_bound,
                                     uint8_t* used_fallback, void* scratch, size_t scratch_bytes,
                                     ls_stream_t stream) {
  if (!model || !params || !samples || !region || !fp || !height || !rgb || n < 0) return LS_ERR_INVALID_ARG;
  if (fp->res != model->res) return LS_ERR_INVALID_ARG;
  const int64_t T = (int64_t)region->tiles_x * region->tiles_y;
  if (!tile_ids && n != T) return LS_ERR_INVALID_ARG;
  const int B = model->max_batch;
  const size_t np = (size_t)B * fp->res * fp->res;
  const size_t need = np * 8 * 2 + np * 16 + (size_t)B * 4 + np * 5 * 4 + np * 20 + 1024;
  if (!scratch || scratch_bytes < need) return LS_ERR_INVALID_ARG;
  char* p = static_cast<char*>(scratch);
  auto take = [&](size_t b) { char* r = p; p += (b + 255) / 256 * 256; return r; };
  uint16_t* x = reinterpret_cast<uint16_t*>(take(np * 16));
  float* base = reinterpret_cast<float*>(take(np * 16));
  float* cz = reinterpret_cast<float*>(take((size_t)B * 4));
  float* y = reinterpret_cast<float*>(take(np * 20));
  float* aux = reinterpret_cast<float*>(take(np * 20));
  for (int64_t o0 = 0; o0 < n; o0 += B) {
    const int64_t nb = n - o0 < B ? n - o0 : B;
    const size_t off = (size_t)o0 * fp->res * fp->res;
    if (!tile_ids && o0 > 0) return LS_ERR_UNSUPPORTED;  // whole-region fills must fit one batch
    const int32_t* tid = tile_ids ? tile_ids + o0 : nullptr;
    ls_status st = ls_learned_inputs(samples, region, fp, tid, nb, x, base, cz, height + off, rgb + off * 3, aux,
                                     stream);
    if (st != LS_OK) return st;
    st = filler_forward(model, params, x, (int32_t)nb, y, reinterpret_cast<cudaStream_t>(stream), false);
    if (st != LS_OK) return st;
    st = ls_learned_finish(y, base, cz, nb, fp->res, region, max_err_m, height + off, rgb + off * 3, height + off,
                           rgb + off * 3, err_bound ? err_bound + o0 : nullptr,
                           used_fallback ? used_fallback + o0 : nullptr, stream);
    if (st != LS_OK) return st;
  }
  return LS_OK;
}

extern "C" size_t ls_fill_learned_scratch_bytes(const ls_model* model) {
  if (!model) return 0;
  const size_t np = (size_t)model->max_batch * model->res * model->res;
  return np * 8 * 2 + np * 16 + (size_t)model->max_batch * 4 + np * 5 * 4 + np * 20 + 1024 + 5 * 256;
}
