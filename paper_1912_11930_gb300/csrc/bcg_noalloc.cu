// bcg_bdot_noalloc: the BDOT kernel for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph capture that must not
// allocate, plug-ins of hosts that own every device allocation through their own pool, or real-time paths
// where an allocation may block or fail. This entry point computes the same block product as bcg_bdot but
// needs no handle (creating one allocates) and no workspace: its column maxima, exponent shifts and per-CTA
// partial sums live in one file-scope device array of fixed size, kNoAllocScratchDoubles doubles (2 MiB), which
// every GPU that loads the library holds until the process exits. The paper has no counterpart; it is a
// deployment variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>

#include "../../include/bcg.h"
#include "bcg_launch.h"

void bcg_internal_set_error(const char *msg);   // bcg_capi.cu

namespace {

constexpr int kNoAllocScratchDoubles = 1 << 18;   // 2 MiB
// layout: [0, 2k) column maxima of X and of Y, then 2k int shifts; the partial sums start at kPartOff
// (k <= 256 keeps the head below 1024 doubles, and the partials 256-byte aligned)
constexpr int kPartOff = 1024;
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

// 1: device (or managed) memory of device dev; 0: not device memory; -1: device memory of another device
int device_pointer(const void *p, int dev) {
  if (p == nullptr) return 0;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type != cudaMemoryTypeDevice) return 0;
  return at.device == dev ? 1 : -1;
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
  if (per_cta > kNoAllocScratchDoubles - kPartOff)
    return noalloc_fail(BCG_ERR_INVALID_ARG, "k*p exceeds the static scratch (261120 doubles)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(BCG_ERR_INVALID_ARG, "device ordinal out of range");
  const int kx = device_pointer(X, dev), ky = device_pointer(Y, dev), kg = device_pointer(gamma, dev);
  if (kx == 0 || ky == 0 || kg == 0)
    return noalloc_fail(BCG_ERR_INVALID_ARG, "X, Y and gamma must be device pointers");
  if (kx < 0 || ky < 0 || kg < 0)
    return noalloc_fail(BCG_ERR_INVALID_ARG,
                        "X, Y and gamma must live on the current device (the scratch used is this device's)");
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
  // Every CTA overwrites its whole partial row, so the partials need no clearing; the column maxima are cleared
  // by launch_col_shifts (a memset of the array, which allocates nothing).
  const int grid = (int)std::min<int64_t>(bdot_grid<double>(n, k, p, nsm), (kNoAllocScratchDoubles - kPartOff) / per_cta);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *cmax = scratch;
  int *sh = reinterpret_cast<int *>(scratch + 2 * k);
  double *part = scratch + kPartOff;
  e = launch_col_shifts(X, n, k, cmax, sh, nsm, s);
  if (e == cudaSuccess) e = launch_col_shifts(Y, n, k, cmax + k, sh + k, nsm, s);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "column maxima launch", e);
  e = launch_bdot<double>(X, Y, n, k, p, part, grid, s, sh, sh + k);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "BDOT launch", e);
  e = launch_finish_gram(part, grid, k, p, global, gamma, nullptr, s);
  if (e != cudaSuccess) return noalloc_fail(BCG_ERR_CUDA, "reduction launch", e);
  return BCG_OK;
}
