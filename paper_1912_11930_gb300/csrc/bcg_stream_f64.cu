#include <algorithm>
#include <type_traits>
#define BCG_T double
#include "bcg_stream.inc"
#include "bcg_kernels_tc.cuh"

namespace bcgk {
bool tc_ok(int k, int p) { return tc_layout_ok(k, p); }
// blocks of 16 fit the kernels too, but measured slower than their fused FMA path: K1 must then form the recomputed
// rho (K3 does at p <= 16), and rho and the norms need passes of their own (160^3, k = 64: 44.7 s against 40.3 s)
bool tc_pair_ok(int k, int p) { return p == 32 && tc_pair_layout_ok(k, p); }
// blocks of 32 in 32-column tiles (k a multiple of 32 that 64 does not divide)
bool tc_b32_ok(int k, int p) { return p == 32 && k % 32 == 0 && k <= 256 && k % 64 != 0; }

cudaError_t launch_tc_pair_cmat(const double *C, int k, int p, int global, double *out, cudaStream_t s) {
  if (!tc_pair_layout_ok(k, p)) return cudaErrorInvalidValue;
  const int nout = global ? 1 : k / 64;
  kt_pair_cmat<<<(nout * 4096 + 255) / 256, 256, 0, s>>>(C, nout, p, global, out);
  return cudaGetLastError();
}
size_t tc_workspace_bytes(int nblkC, int p) { return tc_cmat_bytes(nblkC, p); }

cudaError_t launch_tc_slice(const double *C, int nblkC, int p, uint16_t *Cs, int *Cexp, cudaStream_t s) {
  const int nthr = nblkC * p;
  if (p % 64 == 0) kt_slice_cmat<64><<<(nthr + 127) / 128, 128, 0, s>>>(C, nblkC, p, Cs, Cexp);
  else if (p == 32) kt_slice_cmat<32><<<(nthr + 127) / 128, 128, 0, s>>>(C, nblkC, p, Cs, Cexp);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

size_t tc_row_image_size(int64_t n, int k) { return tc_row_image_bytes(n, k); }
size_t tc_col_image_size(int64_t n, int k) { return tc_col_image_bytes(n, k); }

template <typename T>
cudaError_t launch_tc_col_exp(const T *X, const T *xscale, int64_t n, int k, int *ecol, int nsm, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ecol, 0, sizeof(int) * (size_t)k, s);
  if (e != cudaSuccess) return e;
  const int ge = (int)std::min<int64_t>((n * k + kNT - 1) / kNT, (int64_t)nsm * 8);
  kt_col_exp<T><<<ge, kNT, 0, s>>>(X, xscale, n, k, ecol);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tc_cut_cols(const T *X, const T *xscale, int64_t n, int k, const int *ecol, unsigned char *img,
                               int nsm, cudaStream_t s) {
  if (k % kTcCols) return cudaErrorInvalidValue;
  const int64_t nrc = (n + kTcK - 1) / kTcK;
  const int cts = k / kTcCols;
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(nrc, ((int64_t)nsm * 8 + cts - 1) / cts));
  kt_cut_cols<T><<<dim3((unsigned)cts, (unsigned)gy), kTcThreads, 0, s>>>(X, xscale, n, k, ecol, img);
  return cudaGetLastError();
}
template cudaError_t launch_tc_col_exp<double>(const double *, const double *, int64_t, int, int *, int, cudaStream_t);
template cudaError_t launch_tc_col_exp<float>(const float *, const float *, int64_t, int, int *, int, cudaStream_t);
template cudaError_t launch_tc_cut_cols<double>(const double *, const double *, int64_t, int, const int *,
                                                unsigned char *, int, cudaStream_t);
template cudaError_t launch_tc_cut_cols<float>(const float *, const float *, int64_t, int, const int *,
                                               unsigned char *, int, cudaStream_t);

template <typename T>
cudaError_t launch_tc_cut_rows(const T *Y, int64_t n, int k, int p, unsigned char *img, int *erow, cudaStream_t s) {
  if (!tc_layout_ok(k, p) && !tc_pair_layout_ok(k, p) && !tc_b32_ok(k, p)) return cudaErrorInvalidValue;
  const int64_t nrt = (n + kTcRows - 1) / kTcRows;
  kt_cut_rows<T><<<dim3((unsigned)nrt, (unsigned)(k / p)), kTcThreads, 0, s>>>(Y, n, k, p, img, erow);
  return cudaGetLastError();
}
template cudaError_t launch_tc_cut_rows<double>(const double *, int64_t, int, int, unsigned char *, int *,
                                                cudaStream_t);
template cudaError_t launch_tc_cut_rows<float>(const float *, int64_t, int, int, unsigned char *, int *,
                                               cudaStream_t);

cudaError_t launch_tc_gram_img(const unsigned char *imgX, const unsigned char *imgY, int64_t n, int k, int p,
                               int global, const int *active, double *part, int chunks, const int *ecx,
                               const int *ecy, DevStatus *st, cudaStream_t s) {
  if (!tc_layout_ok(k, p)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kt_gram_img, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const int tiles = (k / p) * ((p + kTcRows - 1) / kTcRows) * (p / kTcCols);
  kt_gram_img<<<dim3((unsigned)tiles, (unsigned)chunks), kTcThreads, kTcSmem, s>>>(imgX, imgY, n, k, p, global,
                                                                                   active, part, ecx, ecy, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tc_baxpy_img(T *OUT, const typename TcId<T>::type *BASE, const unsigned char *imgY,
                                const int *erow, const uint16_t *Cs, const int *Cexp, int64_t n, int k, int p,
                                int global, double sign, const int *active, DevStatus *st, int bump, cudaStream_t s,
                                const typename TcId<T>::type *bscale, int nsm, int pe) {
  if (pe == 0) pe = p;
  const bool b32 = tc_b32_ok(k, p) && pe == p;   // 32-column tiles
  if (!b32 && (!tc_layout_ok(k, p) || !(pe == p || (p == 64 && tc_pair_layout_ok(k, pe)))))
    return cudaErrorInvalidValue;
  auto kern = b32 ? kt_baxpy_img<T, 32> : kt_baxpy_img<T, 64>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = ((n + kTcRows - 1) / kTcRows) * (k / (b32 ? 32 : 64));
  const int grid = (int)std::min<int64_t>(ntiles, nsm);
  kern<<<grid, kTcBaxThreads, kTcSmem, s>>>(OUT, BASE, imgY, erow, Cs, Cexp, n, k, p, global, sign, active, st, bump,
                                            bscale, pe);
  return cudaGetLastError();
}
template cudaError_t launch_tc_baxpy_img<double>(double *, const double *, const unsigned char *, const int *,
                                                 const uint16_t *, const int *, int64_t, int, int, int, double,
                                                 const int *, DevStatus *, int, cudaStream_t, const double *, int,
                                                 int);
template cudaError_t launch_tc_baxpy_img<float>(float *, const float *, const unsigned char *, const int *,
                                                const uint16_t *, const int *, int64_t, int, int, int, double,
                                                const int *, DevStatus *, int, cudaStream_t, const float *, int,
                                                int);

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
