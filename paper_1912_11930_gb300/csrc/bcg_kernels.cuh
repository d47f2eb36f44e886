// Device kernels of the block CG iteration (Algorithm 1 of Section 3, M = I) for sm_103a.
//
// Data layout: block vectors are row-major n x k (element (i, c) at i*k + c), so the k values of a row
// are contiguous and each stored matrix entry is read once per product for all k columns. A CTA of NT
// threads covers rpp = NT / k rows per pass; thread t owns row slot g = t / k and column c = t % k.
// Column c lies in block j = c / p at position b = c % p (Section 2: block j = columns [jp, (j+1)p)).
//
// Every block product <<X, Y>>_S entry (a, b) of block j is accumulated by the thread that owns column
// jp + b, with X's row values broadcast through shared memory; a CTA reduces its row slots in a fixed
// order and writes one partial per CTA, and the small-solve kernels sum the partials in CTA order, so
// results are bitwise repeatable run to run. Gram accumulators are FP64 on both precisions.
//
// Partial layout (per CTA, k*p doubles): entry (a, b) of block j at j*p*p + b*p + a.
// Solve-result layout (lambda, beta, rho_rec; per distinct block p*p doubles): entry (a, b) at a*p + b.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bcgk {

enum OpKind { OP_CSR = 0, OP_ST5 = 1, OP_ST7 = 2, OP_ST7VC = 3 };

// Device status word shared by all kernels of one solve.
struct DevStatus {
  int flags;           // ST_* bits; any nonzero value makes every later kernel of the solve a no-op
  int iter;            // highest iteration whose convergence test ran
  int breakdown_iter;  // iteration of the first breakdown (0 if none)
  int n_active;        // distinct blocks still iterating
  int cur;             // number of the iteration in progress (1-based), advanced by K3
};
enum { ST_DONE = 1, ST_BREAKDOWN = 2, ST_NUMERIC = 4 };

// Operator description; vals/faces point to T (double or float) copies.
struct OpDesc {
  int kind;
  int64_t n;
  const int64_t *rowptr;
  const int32_t *colind;
  const void *vals;
  int nx, ny, nz;
  double scale;
  const void *faces;
};

constexpr int kNT = 256;   // threads per CTA of the streaming kernels (k <= 256)

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
// dynamic shared memory layouts (bytes), shared by kernels and launchers
__host__ __device__ constexpr size_t op_gram_smem(int p) { return kNT * sizeof(double) + (size_t)kNT * p * sizeof(double); }
__host__ __device__ constexpr size_t update_xr_red_offset(int k, int p, int global, size_t tsize) {
  return align16((2 * kNT + (size_t)(global ? 1 : k / p) * p * p) * tsize);
}
__host__ __device__ constexpr size_t update_xr_smem(int k, int p, int global, size_t tsize) {
  return update_xr_red_offset(k, p, global, tsize) + (size_t)kNT * p * sizeof(double);
}
__host__ __device__ constexpr size_t update_p_smem(int k, int p, int global, size_t tsize) {
  return (kNT + (size_t)(global ? 1 : k / p) * p * p) * tsize;
}
__host__ __device__ constexpr size_t residual_smem() { return kNT * sizeof(double); }

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// One row of BOP: (A X)_{r,c}.
template <typename T, int OPK>
__device__ __forceinline__ T apply_row(const OpDesc &A, const T *__restrict__ X, int64_t r, int k, int c) {
  if constexpr (OPK == OP_CSR) {
    const T *__restrict__ v = static_cast<const T *>(A.vals);
    const int64_t e0 = __ldg(A.rowptr + r), e1 = __ldg(A.rowptr + r + 1);
    T s = T(0);
    for (int64_t e = e0; e < e1; ++e)
      s = fma_t(__ldg(v + e), __ldg(X + (int64_t)__ldg(A.colind + e) * k + c), s);
    return s;
  } else if constexpr (OPK == OP_ST5) {
    const int nx = A.nx, ny = A.ny;
    const int ix = (int)(r % nx), iy = (int)(r / nx);
    const int64_t o = r * k + c;
    T s = T(4) * X[o];
    if (ix > 0) s -= X[o - k];
    if (ix < nx - 1) s -= X[o + k];
    if (iy > 0) s -= X[o - (int64_t)nx * k];
    if (iy < ny - 1) s -= X[o + (int64_t)nx * k];
    return T(A.scale) * s;
  } else if constexpr (OPK == OP_ST7) {
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int64_t pl = (int64_t)nx * ny;
    const int ix = (int)(r % nx), iy = (int)((r / nx) % ny), iz = (int)(r / pl);
    const int64_t o = r * k + c;
    T s = T(6) * X[o];
    if (ix > 0) s -= X[o - k];
    if (ix < nx - 1) s -= X[o + k];
    if (iy > 0) s -= X[o - (int64_t)nx * k];
    if (iy < ny - 1) s -= X[o + (int64_t)nx * k];
    if (iz > 0) s -= X[o - pl * k];
    if (iz < nz - 1) s -= X[o + pl * k];
    return T(A.scale) * s;
  } else {  // OP_ST7VC: face coefficients, x-faces [nz][ny][nx+1], y-faces [nz][ny+1][nx], z-faces [nz+1][ny][nx]
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int64_t pl = (int64_t)nx * ny;
    const int ix = (int)(r % nx), iy = (int)((r / nx) % ny), iz = (int)(r / pl);
    const T *__restrict__ f = static_cast<const T *>(A.faces);
    const int64_t nfx = (int64_t)nz * ny * (nx + 1), nfy = (int64_t)nz * (ny + 1) * nx;
    const T *fx = f, *fy = f + nfx, *fz = f + nfx + nfy;
    const int64_t bx = ((int64_t)iz * ny + iy) * (nx + 1) + ix;
    const int64_t by = ((int64_t)iz * (ny + 1) + iy) * nx + ix;
    const int64_t bz = ((int64_t)iz * ny + iy) * nx + ix;
    const T wxm = __ldg(fx + bx), wxp = __ldg(fx + bx + 1);
    const T wym = __ldg(fy + by), wyp = __ldg(fy + by + nx);
    const T wzm = __ldg(fz + bz), wzp = __ldg(fz + bz + pl);
    const int64_t o = r * k + c;
    const T d = ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
    T s = d * X[o];
    if (ix > 0) s = fma_t(-wxm, X[o - k], s);
    if (ix < nx - 1) s = fma_t(-wxp, X[o + k], s);
    if (iy > 0) s = fma_t(-wym, X[o - (int64_t)nx * k], s);
    if (iy < ny - 1) s = fma_t(-wyp, X[o + (int64_t)nx * k], s);
    if (iz > 0) s = fma_t(-wzm, X[o - pl * k], s);
    if (iz < nz - 1) s = fma_t(-wzp, X[o + pl * k], s);
    return T(A.scale) * s;
  }
}

// Reduce per-thread accumulators acc[0..p) over the CTA's row slots into this CTA's partial.
// red: shared scratch of kNT * p doubles. Fixed order (row slot 0, 1, ...).
template <int PM>
__device__ __forceinline__ void cta_reduce_partial(const double (&acc)[PM], double *red, int k, int p,
                                                   int g, int c, int rpp, double *__restrict__ out) {
  if (g < rpp) {
    double *dst = red + ((int64_t)g * k + c) * p;
#pragma unroll
    for (int a = 0; a < PM; ++a)
      if (a < p) dst[a] = acc[a];
  }
  __syncthreads();
  const int E = k * p;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double s = 0.0;
    for (int gg = 0; gg < rpp; ++gg) s += red[(int64_t)gg * E + e];
    out[e] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool block_active(const int *__restrict__ active, int global, int j) {
  return active == nullptr || active[global ? 0 : j] != 0;
}

// ---------------------------------------------------------------------------------------------------
// K1: Q = A P (BOP), alpha = <<P, Q>>_S, and the recomputed rho^{i-1} = <<P, R^{i-1}>>_S (BDOT x 2),
// one pass over the rows.
template <typename T, int OPK, int PM>
__global__ void __launch_bounds__(kNT) k_op_gram(OpDesc A, const T *__restrict__ P, const T *__restrict__ R,
                                                 T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                 const int *__restrict__ active, double *__restrict__ partA,
                                                 double *__restrict__ partR, const DevStatus *__restrict__ st) {
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  double *red = reinterpret_cast<double *>(smem + kNT * sizeof(double));
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p, b = c - j * p;
  const bool act = slot && block_active(active, global, j);
  double accA[PM], accR[PM];
#pragma unroll
  for (int a = 0; a < PM; ++a) { accA[a] = 0.0; accR[a] = 0.0; }
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    T pv = T(0), qv = T(0), rv = T(0);
    if (act && r < n) {
      const int64_t o = r * k + c;
      qv = apply_row<T, OPK>(A, P, r, k, c);
      pv = P[o];
      rv = R[o];
      Q[o] = qv;
    }
    if (slot) sP[g * k + c] = pv;
    __syncthreads();
    if (act) {
      const T *prow = sP + g * k + j * p;
#pragma unroll
      for (int a = 0; a < PM; ++a) {
        if (a < p) {
          const double pa = (double)prow[a];
          accA[a] = fma(pa, (double)qv, accA[a]);
          accR[a] = fma(pa, (double)rv, accR[a]);
        }
      }
    }
    __syncthreads();
  }
  (void)b;
  const int64_t E = (int64_t)k * p;
  cta_reduce_partial<PM>(accA, red, k, p, g, c, rpp, partA + blockIdx.x * E);
  cta_reduce_partial<PM>(accR, red, k, p, g, c, rpp, partR + blockIdx.x * E);
}

// ---------------------------------------------------------------------------------------------------
// K2: X += P lambda, R -= Q lambda (BAXPY x 2), then rho^i = <<R, R>>_S and the per-column ||R_c||^2.
template <typename T, int PM>
__global__ void __launch_bounds__(kNT) k_update_xr(T *__restrict__ X, T *__restrict__ R, const T *__restrict__ P,
                                                   const T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                   const double *__restrict__ lam, const int *__restrict__ active,
                                                   double *__restrict__ partRho, double *__restrict__ partN,
                                                   const DevStatus *__restrict__ st) {
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sQ = sP + kNT;
  T *sL = sQ + kNT;                       // lambda in T, [nblk][p][p]
  const int nblk = global ? 1 : k / p;
  double *red = reinterpret_cast<double *>(smem + update_xr_red_offset(k, p, global, sizeof(T)));
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sL[e] = (T)lam[e];
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p, b = c - j * p;
  const bool act = slot && block_active(active, global, j);
  const T *lj = sL + (global ? 0 : j) * p * p + b;   // lj[a*p] = lambda_j(a, b)
  double accRho[PM];
  double accN = 0.0;
#pragma unroll
  for (int a = 0; a < PM; ++a) accRho[a] = 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    const bool live = act && r < n;
    const int64_t o = r * k + c;
    T xv = T(0), rv = T(0), pv = T(0), qv = T(0);
    if (live) { xv = X[o]; rv = R[o]; pv = P[o]; qv = Q[o]; }
    if (slot) { sP[g * k + c] = pv; sQ[g * k + c] = qv; }
    __syncthreads();
    if (live) {
      const T *prow = sP + g * k + j * p;
      const T *qrow = sQ + g * k + j * p;
#pragma unroll
      for (int a = 0; a < PM; ++a) {
        if (a < p) {
          const T l = lj[a * p];
          xv = fma_t(prow[a], l, xv);
          rv = fma_t(-qrow[a], l, rv);
        }
      }
      X[o] = xv;
      R[o] = rv;
    }
    __syncthreads();
    if (slot) sP[g * k + c] = live ? rv : T(0);
    __syncthreads();
    if (live) {
      const T *rrow = sP + g * k + j * p;
      const double rd = (double)rv;
#pragma unroll
      for (int a = 0; a < PM; ++a)
        if (a < p) accRho[a] = fma((double)rrow[a], rd, accRho[a]);
      accN = fma(rd, rd, accN);
    }
    __syncthreads();
  }
  const int64_t E = (int64_t)k * p;
  cta_reduce_partial<PM>(accRho, red, k, p, g, c, rpp, partRho + blockIdx.x * E);
  double an[1] = {accN};
  cta_reduce_partial<1>(an, red, k, 1, g, c, rpp, partN + (int64_t)blockIdx.x * k);
}

// ---------------------------------------------------------------------------------------------------
// K3: P = R + P beta (BAXPY with the direction-update sign read as "+").
template <typename T, int PM>
__global__ void __launch_bounds__(kNT) k_update_p(T *__restrict__ P, const T *__restrict__ R, int64_t n, int k,
                                                  int p, int global, const double *__restrict__ beta,
                                                  const int *__restrict__ active, DevStatus *__restrict__ st) {
  if (st->flags != 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->cur += 1;   // no other kernel of this launch reads it
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sB = sP + kNT;
  const int nblk = global ? 1 : k / p;
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sB[e] = (T)beta[e];
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p, b = c - j * p;
  const bool act = slot && block_active(active, global, j);
  const T *bj = sB + (global ? 0 : j) * p * p + b;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    const bool live = act && r < n;
    const int64_t o = r * k + c;
    T pv = T(0), rv = T(0);
    if (live) { pv = P[o]; rv = R[o]; }
    if (slot) sP[g * k + c] = pv;
    __syncthreads();
    if (live) {
      const T *prow = sP + g * k + j * p;
      T s = rv;
#pragma unroll
      for (int a = 0; a < PM; ++a)
        if (a < p) s = fma_t(prow[a], bj[a * p], s);
      P[o] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------------
// K0: R = B - A X (and optionally P = R), per-column ||R_c||^2 partials. T is the precision of X, B, R;
// R32/P32 (optional) receive a float copy of R (the mixed-precision inner right-hand side).
template <typename T, int OPK>
__global__ void __launch_bounds__(kNT) k_residual(OpDesc A, const T *__restrict__ X, const T *__restrict__ B,
                                                  T *__restrict__ R, T *__restrict__ P, float *__restrict__ R32,
                                                  float *__restrict__ P32, int64_t n, int k,
                                                  double *__restrict__ partN) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *red = reinterpret_cast<double *>(smem);
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  double accN = 0.0;
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    if (slot && r < n) {
      const int64_t o = r * k + c;
      const T rv = B[o] - apply_row<T, OPK>(A, X, r, k, c);
      if (R) R[o] = rv;
      if (P) P[o] = rv;
      if (R32) { R32[o] = (float)rv; }
      if (P32) { P32[o] = (float)rv; }
      const double rd = (double)rv;
      accN = fma(rd, rd, accN);
    }
  }
  double an[1] = {accN};
  cta_reduce_partial<1>(an, red, k, 1, g, c, rpp, partN + (int64_t)blockIdx.x * k);
}

// BDOT alone: per-CTA partials of gamma = <<X, Y>>_S (entry (a, b) of block j = sum_rows X[jp+a] Y[jp+b]).
template <typename T, int PM>
__global__ void __launch_bounds__(kNT) k_bdot(const T *__restrict__ X, const T *__restrict__ Y, int64_t n, int k,
                                              int p, double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *sX = reinterpret_cast<T *>(smem);
  double *red = reinterpret_cast<double *>(smem + kNT * sizeof(double));
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p;
  double acc[PM];
#pragma unroll
  for (int a = 0; a < PM; ++a) acc[a] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    T xv = T(0), yv = T(0);
    if (slot && r < n) { xv = X[r * k + c]; yv = Y[r * k + c]; }
    if (slot) sX[g * k + c] = xv;
    __syncthreads();
    if (slot) {
      const T *xrow = sX + g * k + j * p;
#pragma unroll
      for (int a = 0; a < PM; ++a)
        if (a < p) acc[a] = fma((double)xrow[a], (double)yv, acc[a]);
    }
    __syncthreads();
  }
  cta_reduce_partial<PM>(acc, red, k, p, g, c, rpp, part + (int64_t)blockIdx.x * k * p);
}

// BOP alone: Y = A X.
template <typename T, int OPK>
__global__ void __launch_bounds__(kNT) k_bop(OpDesc A, const T *__restrict__ X, T *__restrict__ Y, int64_t n, int k) {
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  if (g >= rpp) return;
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t r = (int64_t)blockIdx.x * rpp + g; r < n; r += stride) Y[r * k + c] = apply_row<T, OPK>(A, X, r, k, c);
}

}  // namespace bcgk
