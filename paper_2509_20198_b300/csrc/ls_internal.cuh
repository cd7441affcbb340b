// Internal helpers shared by the CUDA translation units of liblidarscout.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lidarscout.h"

namespace ls {

constexpr int kSmCount = 148;  // B300: 148 SMs on two dies

// ---------------------------------------------------------------------------------
// Sticky per-device status word.  Kernels record the first error; the host reads
// and clears it in ls_last_error().  The library is compiled as one translation
// unit (liblidarscout.cu includes every source), so this is the only copy.
// ---------------------------------------------------------------------------------
__device__ int g_status = 0;

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

// Bounded spin limit for every device-side wait (iterations of >= 64 ns each).
constexpr int kSpinLimit = 1 << 22;

// ---------------------------------------------------------------------------------
// Unsigned 32-bit division by a run-time invariant divisor, after Granlund and
// Montgomery, "Division by Invariant Integers using Multiplication" (PLDI 1994),
// Fig. 4.1: with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = mulhi(m, n); exact for all n.
// ---------------------------------------------------------------------------------
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 0 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// ---------------------------------------------------------------------------------
// Library scratch workspace (per device, grown on demand).
// ---------------------------------------------------------------------------------
enum WorkspaceSlot {
  kWsBinRows = 0,
  kWsFillPacked = 1,
  kWsModel = 2,
  kWsGradPart = 3,
  kWsHeadPart = 4,
  kWsInterpRecs = 5,
  kWsInterpQueue = 6,
  kWsGemmPart = 7,
  kWsSlots = 8
};
// Returns a device pointer of at least `bytes` for the given slot (nullptr on failure).
void* workspace(WorkspaceSlot slot, size_t bytes);

// ---------------------------------------------------------------------------------
// Launch shapes and their autotuner (ls_tune.cu).  A call's key groups the arguments
// that decide which shape is fastest; a table (per process) maps keys to the shape
// ls_tune_* measured best or ls_*_shape_set pinned.  Keys without an entry use the
// defaults.  Lookups are host-only and never synchronise (capturable in graphs).
// ---------------------------------------------------------------------------------
using BinShape = ls_bin_shape;
using FillShape = ls_fill_shape;
uint64_t bin_shape_key(int64_t n_points, const ls_bins* levels, int32_t n_levels);
uint64_t fill_shape_key(int64_t n_samples, int64_t n_out, const ls_fill_params* params);
void bin_shape_lookup(uint64_t key, BinShape* out);
void fill_shape_lookup(uint64_t key, int32_t res, int64_t n_out, FillShape* out);
bool bin_shape_valid(const BinShape& s);
bool fill_shape_valid(const FillShape& s, int32_t res);

inline int grid_cap(int64_t blocks, int64_t cap) {
  if (blocks < 1) blocks = 1;
  return (int)(blocks < cap ? blocks : cap);
}

}  // namespace ls

#define LS_CUDA_TRY(expr)                          \
  do {                                             \
    if ((expr) != cudaSuccess) return LS_ERR_CUDA; \
  } while (0)
