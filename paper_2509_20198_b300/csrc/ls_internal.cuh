// Internal helpers shared by the CUDA translation units of liblidarscout.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

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

// Bounded spin limit for every device-side wait, in polls (the binning's row waits
// sleep 64 ns between polls).  A device variable, so that tests of failure detection
// can shorten it (ls_set_spin_limit).  Kernels read it only once a wait's first poll
// has failed, so the fast path of a wait costs no load.
constexpr int kSpinLimitDefault = 1 << 22;
__device__ int g_spin_limit = kSpinLimitDefault;
__device__ __forceinline__ int spin_limit() { return g_spin_limit; }

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

// Numerators below 2^31 need no correction step: with s = ceil(log2 d) - 1 and
// m = ceil(2^(32+s) / d) (below 2^32 because 2^s < d), the error e = m d - 2^(32+s)
// is below d <= 2^(s+1), so n e < 2^(32+s) for every n < 2^31 and
// q = mulhi(m, n) >> s = floor(n / d) (the round-up method of the same paper, Sec. 4).
// d >= 2.
struct FastDiv31 {
  uint32_t m, s;
};

inline FastDiv31 make_fastdiv31(uint32_t d) {
  FastDiv31 f;
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  f.s = l - 1;
  f.m = (uint32_t)(((uint64_t(1) << (32 + f.s)) + d - 1) / d);
  return f;
}

__device__ __forceinline__ uint32_t fdiv31(uint32_t n, const FastDiv31& f) { return __umulhi(f.m, n) >> f.s; }

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
  kWsLossPart = 8,  // per-block partial loss sums
  kWsSlots = 9
};
// One conv weight pack (ls_conv3x3_pack's arguments): w [cout][3][3][cin] FP32 (or the
// transposed, flipped form when tflip), out the packed BF16 operand chunks
struct PackJob {
  const float* w;
  uint16_t* out;
  int32_t cin, cout, tflip;
};
constexpr int kMaxPackJobs = 32;  // packs per launch of the batched pack

// Returns a device pointer of at least `bytes` for the given slot (nullptr on failure).
void* workspace(WorkspaceSlot slot, size_t bytes);
// Forgets the cached device address of the fixed binning scratch of a device, so that
// the next call looks it up again (ls_release_workspace; after a device reset).
void forget_fixed_scratch(int dev);

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

// One-time set-up per device (kernel attributes, occupancy queries).  The first
// caller on a device runs `fn` under a lock; callers from other host threads wait for
// it and then see its effects.  `fn` returns false on failure, and the next call
// tries again.  Devices beyond the table run `fn` on every call.
constexpr int kMaxDevicesOnce = 64;
struct DeviceOnce {
  std::mutex mu;
  bool done[kMaxDevicesOnce] = {};
};
template <class F>
inline bool device_once(DeviceOnce& o, int dev, F&& fn) {
  if (dev < 0 || dev >= kMaxDevicesOnce) return fn();
  std::lock_guard<std::mutex> lock(o.mu);
  if (o.done[dev]) return true;
  if (!fn()) return false;
  o.done[dev] = true;
  return true;
}

inline int grid_cap(int64_t blocks, int64_t cap) {
  if (blocks < 1) blocks = 1;
  return (int)(blocks < cap ? blocks : cap);
}

}  // namespace ls

#define LS_CUDA_TRY(expr)                          \
  do {                                             \
    if ((expr) != cudaSuccess) return LS_ERR_CUDA; \
  } while (0)
