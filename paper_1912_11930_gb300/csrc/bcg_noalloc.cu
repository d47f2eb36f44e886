// bcg_bdot_noalloc: the BDOT kernel for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph capture that must not
// allocate, plug-ins of hosts that own every device allocation through their own pool, or real-time paths
// where an allocation may block or fail. This entry point computes the same block product as bcg_bdot but
// needs no handle (creating one allocates) and no workspace: its per-CTA partial sums live in one
// file-scope device array of fixed size, kNoAllocScratchDoubles doubles (2 MiB), which every GPU that loads
// the library holds until the process exits. The paper has no counterpart; it is a deployment variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>

#include "../../include/bcg.h"
#include "bcg_launch.h"

void bcg_internal_set_error(const char *msg);   // bcg_capi.cu

namespace {

constexpr int kNoAllocScratchDoubles = 1 << 18;   // 2 MiB of FP64 partial sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device with that device current.
std::atomic<double *> g_scratch_addr[kMaxDevices];

bcg_status noalloc_fail(bcg_status s, const char *msg, cudaError_t e = cudaSuccess) {
  char buf[384];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "bcg_bdot_noalloc: %s: %s", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "bcg_bdot_noalloc: %s", msg);
  bcg_internal_set_error(buf);
  return s;
}

bool device_pointer(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" bcg_status bcg_bdot_noalloc(int64_t n, int32_t k, int32_t p, int32_t sub, const double *X,
                                       const double *Y, double *gamma, void *cuda_stream) {
  using namespace bcgk;
  if (n < 1) return noalloc_fail(BCG_ERR_INVALID_ARG, "n must be >= 1");
  if (k < 1 || k > kNT) return noalloc_fail(BCG_ERR_INVALID_ARG, "k must lie in 1..256");
  int global = 0;
  switch (sub) {
    case BCG_SUB_HYBRID: break;
    case BCG_SUB_GLOBAL: global = 1; break;
    case BCG_SUB_PARALLEL: p = 1; break;
    case BCG_SUB_CLASSICAL: p = k; break;
    default: return noalloc_fail(BCG_ERR_INVALID_ARG, "unknown subalgebra");
  }
  if (p < 1 || k % p != 0) return noalloc_fail(BCG_ERR_INVALID_ARG, "p must divide k");
  if (p > kMaxP) return noalloc_fail(BCG_ERR_INVALID_ARG, "p > 32 is not supported");
  const int64_t per_cta = (int64_t)k * p;   // doubles of one CTA's partial
  if (per_cta > kNoAllocScratchDoubles)
    return noalloc_fail(BCG_ERR_INVALID_ARG, "k*p exceeds the static scratch (262144 doubles)");
  if (!device_pointer(X) || !device_pointer(Y) || !device_pointer(gamma))
    return noalloc_fail(BCG_ERR_INVALID_ARG, "X, Y and gamma must be device pointers");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(BCG_ERR_INVALID_ARG, "device ordinal out of range");
  // Set-up on the first call on this device: in host code g_noalloc_scratch names a host-side shadow, so the
  // kernel must be given the device address, looked up here with this device current.
  double *scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (scratch == nullptr) {
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || addr == nullptr) return noalloc_fail(BCG_ERR_CUDA, "cudaGetSymbolAddress", e);
    scratch = static_cast<double *>(addr);
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "cudaDeviceGetAttribute", e);
  // every CTA overwrites its whole partial row, so nothing in the scratch has to start at zero
  const int grid = (int)std::min<int64_t>(bdot_grid<double>(n, k, p, nsm), kNoAllocScratchDoubles / per_cta);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  e = launch_bdot<double>(X, Y, n, k, p, scratch, grid, s);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "BDOT launch", e);
  e = launch_finish_gram(scratch, grid, k, p, global, gamma, nullptr, s);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "reduction launch", e);
  return BCG_OK;
}
