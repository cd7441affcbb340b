// Runtime pieces of liblidarscout.so: sticky device status, scratch workspace,
// status strings.
#include <mutex>

#include "ls_internal.cuh"

namespace ls {

namespace {
constexpr int kMaxDevices = 64;
struct Ws {
  void* ptr[kWsSlots] = {};
  size_t size[kWsSlots] = {};
};
Ws g_ws[kMaxDevices];
std::mutex g_ws_mu;
}  // namespace

void* workspace(WorkspaceSlot slot, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_ws_mu);
  Ws& w = g_ws[dev];
  if (bytes == 0) bytes = 256;
  if (w.size[slot] >= bytes) return w.ptr[slot];
  if (w.ptr[slot]) {
    // the old buffer may still be in use by queued work on any stream
    if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
    cudaFree(w.ptr[slot]);
    w.ptr[slot] = nullptr;
    w.size[slot] = 0;
  }
  size_t grow = bytes + bytes / 4;
  void* p = nullptr;
  if (cudaMalloc(&p, grow) != cudaSuccess) {
    cudaGetLastError();  // clear the runtime error of the failed allocation
    return nullptr;
  }
  w.ptr[slot] = p;
  w.size[slot] = grow;
  return p;
}

}  // namespace ls

extern "C" {

const char* ls_status_string(ls_status s) {
  switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_INVALID_ARG: return "invalid argument";
    case LS_ERR_CUDA: return "CUDA runtime error";
    case LS_ERR_OUT_OF_RANGE: return "output capacity exceeded";
    case LS_ERR_TIMEOUT: return "bounded device wait ran out";
    case LS_ERR_NO_MEMORY: return "workspace allocation failed";
    case LS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

ls_status ls_last_error(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) return LS_ERR_CUDA;
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, ls::g_status, sizeof(int)) != cudaSuccess) return LS_ERR_CUDA;
  if (cudaMemcpyToSymbol(ls::g_status, &zero, sizeof(int)) != cudaSuccess) return LS_ERR_CUDA;
  return v;
}

ls_status ls_release_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return LS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(ls::g_ws_mu);
  if (dev < 0 || dev >= ls::kMaxDevices) return LS_ERR_INVALID_ARG;
  for (int s = 0; s < ls::kWsSlots; ++s) {
    if (ls::g_ws[dev].ptr[s]) cudaFree(ls::g_ws[dev].ptr[s]);
    ls::g_ws[dev].ptr[s] = nullptr;
    ls::g_ws[dev].size[s] = 0;
  }
  ls::forget_fixed_scratch(dev);
  return LS_OK;
}

ls_status ls_set_spin_limit(int32_t polls) {
  const int v = polls > 0 ? polls : ls::kSpinLimitDefault;
  if (cudaDeviceSynchronize() != cudaSuccess) return LS_ERR_CUDA;
  return cudaMemcpyToSymbol(ls::g_spin_limit, &v, sizeof(int)) == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}

int32_t ls_version(void) { return 100; }

}  // extern "C"
