// Launch shapes and their autotuner.  The batched launches of the heightmap build
// (binning of all tiles, the Gaussian fill of all tiles) have shape parameters whose
// best values depend on the workload: how many spans each binning CTA takes (dynamic
// balance against the rows shared at span ends), how far ahead the point stream is
// prefetched into L2, how many CTAs share one tile's fill and how many CTAs per SM the
// persistent fill grid assumes.  The paper batches tiles because batching pays off
// (Sec. 4.2); this file picks the shapes of those batches by measurement.
//
// A key groups the arguments that decide the best shape (level sizes and the order of
// magnitude of the point count for binning; resolution, radius and the orders of
// magnitude of the tile and sample counts for the fill).  A per-process table maps
// keys to shapes; ls_tune_* time every candidate on the caller's own data and store
// the fastest, ls_*_shape_set pins one.  Keys without an entry get the defaults.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ls_internal.cuh"

namespace ls {
namespace {

enum TuneKind { kTuneBin = 1, kTuneFill = 2 };

struct TuneEntry {
  int kind;
  uint64_t key;
  int32_t v0, v1;
};

constexpr size_t kTuneEntries = 256;  // oldest entries are replaced beyond this
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

bool tune_get(int kind, uint64_t key, int32_t* v0, int32_t* v1) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const TuneEntry& e : g_tune)
    if (e.kind == kind && e.key == key) {
      *v0 = e.v0;
      *v1 = e.v1;
      return true;
    }
  return false;
}

void tune_put(int kind, uint64_t key, int32_t v0, int32_t v1) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (TuneEntry& e : g_tune)
    if (e.kind == kind && e.key == key) {
      e.v0 = v0;
      e.v1 = v1;
      return;
    }
  if (g_tune.size() >= kTuneEntries) g_tune.erase(g_tune.begin());
  g_tune.push_back(TuneEntry{kind, key, v0, v1});
}

void tune_erase(int kind, uint64_t key) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (size_t i = 0; i < g_tune.size(); ++i)
    if (g_tune[i].kind == kind && g_tune[i].key == key) {
      g_tune.erase(g_tune.begin() + (long)i);
      return;
    }
}

uint64_t log2_bucket(int64_t n) {
  uint64_t b = 0;
  while (n > 1) {
    n >>= 1;
    ++b;
  }
  return b;
}

const BinShape kBinDefault = {16, 2};
const int32_t kBinSpans[] = {8, 16, 32};
const int32_t kBinPrefetch[] = {1, 2, 3};
const int32_t kFillSplits[] = {1, 2, 4};
const int32_t kFillCtas[] = {1, 2, 3, 4};

// the grid is sized for at most as many CTAs as fit on an SM with the launch's stage
FillShape fill_default(int32_t res, int64_t n_out) {
  return FillShape{(n_out < 4 * kSmCount && res % 64 == 0) ? 4 : 1, 4};
}

// Timer of a sequence of library calls on one stream (CUDA events; synchronises).
struct CallTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = false;
  CallTimer() { ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess; }
  ~CallTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Runs `call` `calls` times between two events: ms per call, or a negative status.
template <class F>
ls_status time_calls(CallTimer& t, cudaStream_t s, int32_t calls, F call, float* ms) {
  if (cudaEventRecord(t.e0, s) != cudaSuccess) return LS_ERR_CUDA;
  for (int32_t r = 0; r < calls; ++r) {
    const ls_status st = call();
    if (st != LS_OK) return st;
  }
  if (cudaEventRecord(t.e1, s) != cudaSuccess || cudaEventSynchronize(t.e1) != cudaSuccess) return LS_ERR_CUDA;
  float total = 0.f;
  if (cudaEventElapsedTime(&total, t.e0, t.e1) != cudaSuccess) return LS_ERR_CUDA;
  *ms = total / (float)calls;
  return LS_OK;
}

// The measurement shared by the tuners.  Candidates are timed round-robin, `rounds`
// rounds of two calls each after one untimed call per candidate, so that a drift of
// the clocks or of the cache state during tuning affects all of them alike; each
// candidate's score is its median over the rounds.  A candidate replaces the default
// (candidate 0) only when its median is at least 1 % lower: shapes within the noise
// of each other keep the default.  `use(i)` makes candidate i the table entry.
template <class Use, class Call>
ls_status tune_candidates(cudaStream_t s, int n_cand, int32_t rounds, Use use, Call call, int* win, float* win_ms) {
  CallTimer timer;
  if (!timer.ok) return LS_ERR_CUDA;
  std::vector<std::vector<float>> t((size_t)n_cand);
  for (int i = 0; i < n_cand; ++i) {
    use(i);
    const ls_status st = call();
    if (st != LS_OK) return st;
  }
  for (int32_t r = 0; r < rounds; ++r)
    for (int i = 0; i < n_cand; ++i) {
      use(i);
      float ms = 0.f;
      const ls_status st = time_calls(timer, s, 2, call, &ms);
      if (st != LS_OK) return st;
      t[(size_t)i].push_back(ms);
    }
  std::vector<float> med((size_t)n_cand);
  for (int i = 0; i < n_cand; ++i) {
    std::vector<float>& v = t[(size_t)i];
    std::sort(v.begin(), v.end());
    med[(size_t)i] = v[v.size() / 2];
  }
  int best = 0;
  for (int i = 1; i < n_cand; ++i)
    if (med[(size_t)i] < med[(size_t)best]) best = i;
  if (best != 0 && med[(size_t)best] > 0.99f * med[0]) best = 0;
  *win = best;
  *win_ms = med[(size_t)best];
  return LS_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

}  // namespace

uint64_t bin_shape_key(int64_t n_points, const ls_bins* levels, int32_t n_levels) {
  const uint64_t c0 = (n_levels >= 1 && levels) ? (uint64_t)(levels[0].cells & 0x1fff) : 0;
  const uint64_t c1 = (n_levels >= 2 && levels) ? (uint64_t)(levels[1].cells & 0x1fff) : 0;
  return (uint64_t)(n_levels & 3) | (c0 << 2) | (c1 << 15) | (log2_bucket(n_points) << 28);
}

uint64_t fill_shape_key(int64_t n_samples, int64_t n_out, const ls_fill_params* p) {
  return (uint64_t)(p->res & 0x7ff) | ((uint64_t)(p->radius_cm & 0xfffff) << 11) |
         (log2_bucket(n_out) << 31) | (log2_bucket(n_samples) << 37);
}

bool bin_shape_valid(const BinShape& s) {
  return s.spans_per_cta >= 1 && s.spans_per_cta <= 256 && s.prefetch_batches >= 1 && s.prefetch_batches <= 4;
}

bool fill_shape_valid(const FillShape& s, int32_t res) {
  if (s.ctas_per_sm < 1 || s.ctas_per_sm > 4) return false;
  if (s.split == 1) return true;
  // a band of res / split rows is made of whole 8-row texel blocks and starts its output
  // rows at 16-byte boundaries
  return (s.split == 2 || s.split == 4) && res % (16 * s.split) == 0;
}

void bin_shape_lookup(uint64_t key, BinShape* out) {
  int32_t v0, v1;
  if (tune_get(kTuneBin, key, &v0, &v1)) {
    *out = BinShape{v0, v1};
    return;
  }
  *out = kBinDefault;
}

void fill_shape_lookup(uint64_t key, int32_t res, int64_t n_out, FillShape* out) {
  int32_t v0, v1;
  if (tune_get(kTuneFill, key, &v0, &v1) && fill_shape_valid(FillShape{v0, v1}, res)) {
    *out = FillShape{v0, v1};
    return;
  }
  *out = fill_default(res, n_out);
}

}  // namespace ls

extern "C" ls_status ls_bin_shape_get(const ls_points* pts, const ls_bins* levels, int32_t n_levels,
                                      ls_bin_shape* out) {
  if (!pts || !levels || !out || n_levels < 1 || n_levels > 2) return LS_ERR_INVALID_ARG;
  ls::bin_shape_lookup(ls::bin_shape_key(pts->n, levels, n_levels), out);
  return LS_OK;
}

extern "C" ls_status ls_bin_shape_set(const ls_points* pts, const ls_bins* levels, int32_t n_levels,
                                      const ls_bin_shape* shape) {
  if (!pts || !levels || n_levels < 1 || n_levels > 2) return LS_ERR_INVALID_ARG;
  const uint64_t key = ls::bin_shape_key(pts->n, levels, n_levels);
  if (!shape) {
    ls::tune_erase(ls::kTuneBin, key);
    return LS_OK;
  }
  if (!ls::bin_shape_valid(*shape)) return LS_ERR_INVALID_ARG;
  ls::tune_put(ls::kTuneBin, key, shape->spans_per_cta, shape->prefetch_batches);
  return LS_OK;
}

extern "C" ls_status ls_fill_shape_get(const ls_points* samples, const ls_fill_params* params, int64_t n_out,
                                       ls_fill_shape* out) {
  if (!samples || !params || !out || n_out < 0) return LS_ERR_INVALID_ARG;
  ls::fill_shape_lookup(ls::fill_shape_key(samples->n, n_out, params), params->res, n_out, out);
  return LS_OK;
}

extern "C" ls_status ls_fill_shape_set(const ls_points* samples, const ls_fill_params* params, int64_t n_out,
                                       const ls_fill_shape* shape) {
  if (!samples || !params || n_out < 0) return LS_ERR_INVALID_ARG;
  const uint64_t key = ls::fill_shape_key(samples->n, n_out, params);
  if (!shape) {
    ls::tune_erase(ls::kTuneFill, key);
    return LS_OK;
  }
  if (!ls::fill_shape_valid(*shape, params->res)) return LS_ERR_INVALID_ARG;
  ls::tune_put(ls::kTuneFill, key, shape->split, shape->ctas_per_sm);
  return LS_OK;
}

extern "C" ls_status ls_tune_clear(void) {
  std::lock_guard<std::mutex> lock(ls::g_tune_mu);
  ls::g_tune.clear();
  return LS_OK;
}

extern "C" ls_status ls_tune_bin_points(const ls_points* pts, const ls_region* region, const ls_bins* levels,
                                        int32_t n_levels, uint64_t* dropped, int32_t reps, ls_stream_t stream,
                                        ls_bin_shape* best, float* best_ms) {
  if (!pts || !levels || n_levels < 1 || n_levels > 2 || reps < 1 || reps > 1000) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (ls::capturing(s)) return LS_ERR_INVALID_ARG;  // tuning synchronises
  const uint64_t key = ls::bin_shape_key(pts->n, levels, n_levels);
  std::vector<ls_bin_shape> cand{ls::kBinDefault};
  for (int32_t sp : ls::kBinSpans)
    for (int32_t pf : ls::kBinPrefetch)
      if (sp != ls::kBinDefault.spans_per_cta || pf != ls::kBinDefault.prefetch_batches) cand.push_back({sp, pf});
  int wi = 0;
  float win_ms = 0.f;
  const ls_status tst = ls::tune_candidates(
      s, (int)cand.size(), reps,
      [&](int i) { ls::tune_put(ls::kTuneBin, key, cand[(size_t)i].spans_per_cta, cand[(size_t)i].prefetch_batches); },
      [&] { return ls_bin_points(pts, region, levels, n_levels, dropped, stream); }, &wi, &win_ms);
  if (tst != LS_OK) {
    ls::tune_erase(ls::kTuneBin, key);
    return tst;
  }
  const ls_bin_shape win = cand[(size_t)wi];
  ls::tune_put(ls::kTuneBin, key, win.spans_per_cta, win.prefetch_batches);
  // leave the outputs as the chosen shape computes them (every candidate gives the same)
  const ls_status st = ls_bin_points(pts, region, levels, n_levels, dropped, stream);
  if (st != LS_OK) return st;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return LS_OK;
}

extern "C" ls_status ls_tune_fill_sparse(const ls_points* samples, const ls_region* region,
                                         const ls_fill_params* params, const int32_t* tile_ids, int64_t n_out,
                                         float* height, uint8_t* rgb, int32_t reps, ls_stream_t stream,
                                         ls_fill_shape* best, float* best_ms) {
  if (!samples || !params || n_out < 0 || reps < 1 || reps > 1000) return LS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (ls::capturing(s)) return LS_ERR_INVALID_ARG;
  const uint64_t key = ls::fill_shape_key(samples->n, n_out, params);
  const ls_fill_shape def = ls::fill_default(params->res, n_out);
  std::vector<ls_fill_shape> cand{def};
  for (int32_t sp : ls::kFillSplits)
    for (int32_t c : ls::kFillCtas)
      if ((sp != def.split || c != def.ctas_per_sm) && ls::fill_shape_valid(ls_fill_shape{sp, c}, params->res))
        cand.push_back({sp, c});
  int wi = 0;
  float win_ms = 0.f;
  const ls_status tst = ls::tune_candidates(
      s, (int)cand.size(), reps,
      [&](int i) { ls::tune_put(ls::kTuneFill, key, cand[(size_t)i].split, cand[(size_t)i].ctas_per_sm); },
      [&] { return ls_fill_sparse(samples, region, params, tile_ids, n_out, height, rgb, stream); }, &wi,
      &win_ms);
  if (tst != LS_OK) {
    ls::tune_erase(ls::kTuneFill, key);
    return tst;
  }
  const ls_fill_shape win = cand[(size_t)wi];
  ls::tune_put(ls::kTuneFill, key, win.split, win.ctas_per_sm);
  const ls_status st = ls_fill_sparse(samples, region, params, tile_ids, n_out, height, rgb, stream);
  if (st != LS_OK) return st;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return LS_OK;
}
