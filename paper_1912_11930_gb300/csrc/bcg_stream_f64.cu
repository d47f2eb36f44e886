#include <algorithm>
#include <type_traits>
#define BCG_T double
#include "bcg_stream.inc"

namespace bcgk {
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
