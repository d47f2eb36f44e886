#include <algorithm>
#include <type_traits>
#define BCG_T double
#include "bcg_stream.inc"
#include "bcg_kernels_tc.cuh"

namespace bcgk {
bool tc_ok(int k, int p) { return tc_layout_ok(k, p); }
size_t tc_workspace_bytes(int nblkC, int p) { return tc_cmat_bytes(nblkC, p); }

cudaError_t launch_tc_slice(const double *C, int nblkC, int p, uint16_t *Cs, int *Cexp, cudaStream_t s) {
  const int nthr = nblkC * p;
  kt_slice_cmat<<<(nthr + 127) / 128, 128, 0, s>>>(C, nblkC, p, Cs, Cexp);
  return cudaGetLastError();
}

cudaError_t launch_tc_gram(const double *X, const double *Y, const double *xscale, int64_t n, int k, int p,
                           int global, const int *active, double *part, int chunks, int *ecol, DevStatus *st,
                           cudaStream_t s, int nsm) {
  if (!tc_layout_ok(k, p)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ecol, 0, 2 * sizeof(int) * (size_t)k, s);
  if (e != cudaSuccess) return e;
  const int ge = (int)std::min<int64_t>((n * k + kNT - 1) / kNT, (int64_t)nsm * 8);
  kt_col_exp<<<ge, kNT, 0, s>>>(X, xscale, n, k, ecol);
  kt_col_exp<<<ge, kNT, 0, s>>>(Y, nullptr, n, k, ecol + k);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kt_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem)) != cudaSuccess)
    return e;
  const int tiles = (k / p) * ((p + kTcRows - 1) / kTcRows) * (p / kTcCols);
  dim3 grid((unsigned)tiles, (unsigned)chunks);
  kt_gram<<<grid, kTcThreads, kTcSmem, s>>>(X, Y, xscale, n, k, p, global, active, part, ecol, ecol + k, st);
  return cudaGetLastError();
}

cudaError_t launch_tc_baxpy(double *OUT, const double *BASE, const double *Y, const uint16_t *Cs, const int *Cexp,
                            int64_t n, int k, int p, int global, double sign, const int *active, DevStatus *st,
                            int bump, cudaStream_t s, const double *bscale, int nsm) {
  if (!tc_layout_ok(k, p)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kt_baxpy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = ((n + kTcRows - 1) / kTcRows) * (k / kTcCols);
  const int grid = (int)std::min<int64_t>(ntiles, nsm);
  kt_baxpy<<<grid, kTcThreads, kTcSmem, s>>>(OUT, BASE, Y, Cs, Cexp, n, k, p, global, sign, active, st, bump, bscale);
  return cudaGetLastError();
}

cudaError_t launch_inv_diag(const OpDesc &A, int64_t n, double *dinv, double *opmax, int nsm, cudaStream_t s) {
  if (opmax) {
    cudaError_t e = cudaMemsetAsync(opmax, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  return with_op(A.kind, [&](auto ok) -> cudaError_t {
    constexpr int OPK = decltype(ok)::value;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)nsm * 8);
    k_inv_diag<double, OPK><<<grid, 256, 0, s>>>(A, n, dinv, reinterpret_cast<unsigned long long *>(opmax));
    return cudaGetLastError();
  });
}
}  // namespace bcgk
