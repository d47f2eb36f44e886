// BSOLVE kernels (Section 3, "solve a block system in the *-subalgebra"), the stopping test and the
// status bookkeeping. One CTA per distinct block of the subalgebra (q for hybrid, 1 for global), FP64.
//
// Each CTA first sums the per-CTA partials of its block in CTA order (deterministic), then factors:
//   lambda = alpha^{-1} rho_rec  by Cholesky of alpha (SPD), reading alpha's lower triangle;
//   beta   = rho_rec^{-1} rho    by LU with partial pivoting of the recomputed rho (not symmetric in
//                                floating point).
// A pivot <= 64 eps max|diag| or a non-finite value is a breakdown: the method has no deflation, so
// the solve stops and reports it.
#include <cfloat>
#include <cmath>
#include <math_constants.h>

#include "bcg_launch.h"

namespace bcgk {

constexpr int kSmallNT = 512;
constexpr double kPivotFactor = 64.0;
constexpr size_t kSmallSmemMax = 200 * 1024;   // larger p x p workspaces live in global memory

// per-block workspace (doubles): 3 p x p matrices + reduction scratch, or the column-norm scratch of K4b
__host__ __device__ inline size_t small_ws_doubles_dev(int p) {
  const size_t pp = (size_t)p * p;
  const size_t solve = 3 * pp + (pp > (size_t)kSmallNT ? pp : (size_t)kSmallNT);
  const size_t norms = (size_t)kNT + kSmallNT;
  return solve > norms ? solve : norms;
}

// Deterministic reduction out[e] = sum over pi < nparts of load(pi, e), e < E: each entry's sum is split
// over S = blockDim/E thread subsets (pi = sub, sub + S, ...) with 4 independent accumulators per thread
// (several loads in flight), then the subsets are added in a fixed order. scratch: >= max(E, blockDim)
// doubles. The order is fixed by (E, nparts, blockDim), so results repeat bitwise.
template <typename F>
__device__ void det_reduce(int E, int nparts, F load, double *out, double *scratch) {
  const int NT = blockDim.x;
  const int S = E >= NT ? 1 : NT / E;
  for (int t = threadIdx.x; t < E * S; t += NT) {
    const int el = t % E, sub = t / E;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int pi = sub;
    for (; pi + 3 * S < nparts; pi += 4 * S) {
      a0 += load(pi, el);
      a1 += load(pi + S, el);
      a2 += load(pi + 2 * S, el);
      a3 += load(pi + 3 * S, el);
    }
    for (; pi < nparts; pi += S) a0 += load(pi, el);
    scratch[t] = (a0 + a1) + (a2 + a3);
  }
  __syncthreads();
  for (int el = threadIdx.x; el < E; el += NT) {
    double v = 0.0;
    for (int sub = 0; sub < S; ++sub) v += scratch[sub * E + el];
    out[el] = v;
  }
  __syncthreads();
}

// Sum the partials of distinct block jb into dst[b*p + a] (the partial layout).
__device__ void reduce_block(const double *__restrict__ part, int nparts, int k, int p, int global, int jb,
                             double *dst, double *scratch) {
  const int Eb = p * p;
  const int64_t E = (int64_t)k * p;
  const int q = k / p;
  if (!global) {
    const double *base = part + (int64_t)jb * Eb;
    det_reduce(Eb, nparts, [&](int pi, int el) { return base[pi * E + el]; }, dst, scratch);
  } else {
    det_reduce(Eb, nparts, [&](int pi, int el) {
      double v = 0.0;
      for (int j = 0; j < q; ++j) v += part[pi * E + (int64_t)j * Eb + el];
      return v;
    }, dst, scratch);
  }
}

// dst[a*p + b] = src[b*p + a]
__device__ void transpose_into(const double *src, double *dst, int p) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int b = e / p, a = e - b * p;
    dst[a * p + b] = src[e];
  }
  __syncthreads();
}

// Symmetric product stored by circulant diagonals (p a power of two): src[b*p + d] = entry ((b + d) mod p, b)
// for d < p/2, and for d = p/2 when b < p/2. dst[a*p + b] receives the full symmetric matrix.
__device__ void unpack_circulant(const double *src, double *dst, int p) {
  const int h = p / 2;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int a = e / p, b = e - a * p;
    const int d = (a - b) & (p - 1);
    double v;
    if (p == 1) v = src[0];
    else if (d < h || (d == h && b < h)) v = src[b * p + d];
    else v = src[a * p + ((b - a) & (p - 1))];
    dst[e] = v;
  }
  __syncthreads();
}

// Block-wide max of |diag| (every thread passes its partial) -- result valid in all threads.
__device__ double block_max(double v) {
  __shared__ double wmax[kSmallNT / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
  __syncthreads();
  return m;
}

// Partial-pivot choice: the row i in [a, p) with the largest |M[i][a]|, the smallest i on ties. Valid in all
// threads.
__device__ void block_argmax_col(const double *M, int p, int a, double *best_v, int *best_i) {
  __shared__ double wv[kSmallNT / 32];
  __shared__ int wi[kSmallNT / 32];
  double v = -1.0;
  int idx = p;
  for (int i = a + threadIdx.x; i < p; i += blockDim.x) {
    const double x = fabs(M[(int64_t)i * p + a]);
    if (x > v || (x == v && i < idx) || !(x == x)) { v = (x == x) ? x : INFINITY; idx = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { wv[threadIdx.x >> 5] = v; wi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  double bv = -1.0;
  int bi = p;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
    if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
  __syncthreads();
  *best_v = bv;
  *best_i = bi;
}

__device__ void flag_breakdown(DevStatus *st) {
  atomicOr(&st->flags, ST_BREAKDOWN);
  atomicCAS(&st->breakdown_iter, 0, st->cur);
}

// K4a: lambda_j = alpha_j^{-1} rho_rec_j; also stores rho_rec_j (row-major a*p + b) for K4b.
__global__ void __launch_bounds__(kSmallNT) k_solve_lambda(const double *__restrict__ partA,
                                                           const double *__restrict__ partR, int nparts, int k,
                                                           int p, int global, const int *__restrict__ active,
                                                           double *__restrict__ lam, double *__restrict__ rho_rec,
                                                           DevStatus *st, double *gws, int alpha_circ,
                                                           int nparts_r) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  const int pp = p * p;
  double *lj = lam + (int64_t)jb * pp;
  if (!active[jb]) {
    for (int e = threadIdx.x; e < pp; e += blockDim.x) lj[e] = 0.0;
    return;
  }
  extern __shared__ __align__(16) double sm_dyn[];
  double *sm = gws ? gws + (int64_t)jb * small_ws_doubles_dev(p) : sm_dyn;
  double *sA = sm;            // alpha, row-major, factored in place into L (lower)
  double *sR = sA + pp;       // rho_rec, row-major; overwritten by Y then lambda
  double *tmp = sR + pp;      // p*p
  double *scr = tmp + pp;     // max(NT, p*p)
  __shared__ int bad;
  __shared__ double thresh;
  reduce_block(partA, nparts, k, p, global, jb, tmp, scr);
  if (alpha_circ) unpack_circulant(tmp, sA, p);
  else transpose_into(tmp, sA, p);
  reduce_block(partR, nparts_r, k, p, global, jb, tmp, scr);
  transpose_into(tmp, sR, p);
  for (int e = threadIdx.x; e < pp; e += blockDim.x) rho_rec[(int64_t)jb * pp + e] = sR[e];
  {
    double m = 0.0;
    for (int a = threadIdx.x; a < p; a += blockDim.x) m = fmax(m, fabs(sA[a * p + a]));
    m = block_max(m);
    if (threadIdx.x == 0) {
      thresh = kPivotFactor * DBL_EPSILON * m;
      bad = 0;
    }
  }
  __syncthreads();
  // right-looking Cholesky on the lower triangle
  for (int a = 0; a < p; ++a) {
    if (threadIdx.x == 0) {
      const double d = sA[a * p + a];
      if (!(isfinite(d) && d > thresh)) bad = 1;
      else sA[a * p + a] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const double la = sA[a * p + a];
    for (int i = a + 1 + threadIdx.x; i < p; i += blockDim.x) sA[i * p + a] /= la;
    __syncthreads();
    const int m = p - a - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = a + 1 + e / m, jj = a + 1 + e % m;
      if (jj <= i) sA[i * p + jj] -= sA[i * p + a] * sA[jj * p + a];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  // L Y = rho_rec, then L^T lambda = Y; one thread per right-hand-side column b
  for (int b = threadIdx.x; b < p; b += blockDim.x) {
    for (int a = 0; a < p; ++a) {
      double s = sR[a * p + b];
      for (int m2 = 0; m2 < a; ++m2) s -= sA[a * p + m2] * sR[m2 * p + b];
      sR[a * p + b] = s / sA[a * p + a];
    }
    for (int a = p - 1; a >= 0; --a) {
      double s = sR[a * p + b];
      for (int m2 = a + 1; m2 < p; ++m2) s -= sA[m2 * p + a] * sR[m2 * p + b];
      sR[a * p + b] = s / sA[a * p + a];
    }
  }
  __syncthreads();
  bool finite = true;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    lj[e] = sR[e];
    if (!isfinite(sR[e])) finite = false;
  }
  if (!__syncthreads_and(finite) && threadIdx.x == 0) flag_breakdown(st);
}

// K4b: per-column norms, stopping test, beta_j = rho_rec_j^{-1} rho_j by LU with partial pivoting.
__global__ void __launch_bounds__(kSmallNT) k_solve_beta(const double *__restrict__ partRho,
                                                         const double *__restrict__ partN, int nparts, int k, int p,
                                                         int global, const double *__restrict__ tol2p,
                                                         const double *__restrict__ r0n2,
                                                         double *__restrict__ rn2, int *__restrict__ active,
                                                         int *__restrict__ block_iters,
                                                         const double *__restrict__ rho_rec,
                                                         double *__restrict__ beta, DevStatus *st, double *gws,
                                                         int rho_circ, int nparts_n, int split, ShiftCtl sc) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  const int pp = p * p;
  const int it = st->cur;
  const double tol2 = *tol2p;   // squared tolerance in device memory: a captured graph serves every tolerance
  const int c0 = global ? 0 : jb * p, c1 = global ? k : c0 + p;
  extern __shared__ __align__(16) double sm_dyn[];
  double *sm = gws ? gws + (int64_t)jb * small_ws_doubles_dev(p) : sm_dyn;
  {
    double *ncol = sm, *nscr = sm + kNT;   // column norms of this block, scratch
    det_reduce(c1 - c0, nparts_n, [&](int pi, int c) { return partN[(int64_t)pi * k + c0 + c]; }, ncol, nscr);
  }
  bool conv = true, finite = true;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const double s = sm[c - c0];
    rn2[c] = s;
    write_shifts(sc, k, c, s);   // Gram shifts of the next products follow the new norms
    if (!isfinite(s)) finite = false;
    if (!(s <= tol2 * r0n2[c])) conv = false;
  }
  finite = __syncthreads_and(finite);
  conv = __syncthreads_and(conv);
  double *bj = beta + (int64_t)jb * pp;
  if (!finite) {
    if (threadIdx.x == 0) atomicOr(&st->flags, ST_NUMERIC);
    return;
  }
  if (conv) {
    for (int e = threadIdx.x; e < pp; e += blockDim.x) bj[e] = 0.0;
    if (threadIdx.x == 0) {
      active[jb] = 0;
      block_iters[jb] = it;
      atomicMax(&st->iter, it);
      if (atomicSub(&st->n_active, 1) == 1) atomicOr(&st->flags, ST_DONE);
    }
    return;
  }
  if (split) return;        // wide blocks: k_bs_gather, the blocked LU and k_trsm_cols follow
  double *sM = sm;          // rho_rec (row-major), LU-factored in place
  double *sB = sM + pp;     // right-hand sides rho (row-major), become beta
  double *tmp = sB + pp;    // reduction output
  double *scr = tmp + pp;
  __shared__ int bad, piv;
  __shared__ double thresh;
  reduce_block(partRho, nparts, k, p, global, jb, tmp, scr);
  if (rho_circ) unpack_circulant(tmp, sB, p);
  else transpose_into(tmp, sB, p);
  for (int e = threadIdx.x; e < pp; e += blockDim.x) sM[e] = rho_rec[(int64_t)jb * pp + e];
  __syncthreads();
  {
    double m = 0.0;
    bool fin = true;
    for (int a = threadIdx.x; a < p; a += blockDim.x) m = fmax(m, fabs(sM[a * p + a]));
    for (int e = threadIdx.x; e < pp; e += blockDim.x) fin = fin && isfinite(sM[e]);
    m = block_max(m);
    fin = __syncthreads_and(fin);
    if (threadIdx.x == 0) {
      thresh = kPivotFactor * DBL_EPSILON * m;
      bad = fin ? 0 : 1;
    }
  }
  __syncthreads();
  for (int a = 0; a < p && !bad; ++a) {
    double bv;
    int best;
    if (p > 64) {   // wide blocks: all threads search the pivot column
      block_argmax_col(sM, p, a, &bv, &best);
    } else if (threadIdx.x == 0) {   // narrow blocks: one thread is faster than a block reduction
      best = a;
      bv = fabs(sM[a * p + a]);
      for (int i = a + 1; i < p; ++i) {
        const double v = fabs(sM[i * p + a]);
        if (v > bv) { bv = v; best = i; }
      }
    }
    if (threadIdx.x == 0) {
      piv = best;
      if (!(bv > thresh)) bad = 1;
    }
    __syncthreads();
    if (bad) break;
    if (piv != a) {
      for (int col = threadIdx.x; col < p; col += blockDim.x) {
        double t = sM[a * p + col]; sM[a * p + col] = sM[piv * p + col]; sM[piv * p + col] = t;
        t = sB[a * p + col]; sB[a * p + col] = sB[piv * p + col]; sB[piv * p + col] = t;
      }
    }
    __syncthreads();
    const double ua = sM[a * p + a];
    for (int i = a + 1 + threadIdx.x; i < p; i += blockDim.x) sM[i * p + a] /= ua;   // multipliers
    __syncthreads();
    const int m = p - a - 1;
    const int w = m + p;
    for (int e = threadIdx.x; e < m * w; e += blockDim.x) {
      const int i = a + 1 + e / w, col = e % w;
      const double l = sM[i * p + a];
      if (col < m) sM[i * p + a + 1 + col] -= l * sM[a * p + a + 1 + col];
      else sB[i * p + (col - m)] -= l * sB[a * p + (col - m)];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  for (int b = threadIdx.x; b < p; b += blockDim.x) {
    for (int a = p - 1; a >= 0; --a) {
      double s = sB[a * p + b];
      for (int m2 = a + 1; m2 < p; ++m2) s -= sM[a * p + m2] * sB[m2 * p + b];
      sB[a * p + b] = s / sM[a * p + a];
    }
  }
  __syncthreads();
  bool fin = true;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    bj[e] = sB[e];
    if (!isfinite(sB[e])) fin = false;
  }
  if (!__syncthreads_and(fin)) {
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  if (threadIdx.x == 0) atomicMax(&st->iter, it);
}

// Triangular solves of the large-block BSOLVEs (chol = 2: the backward solve with L^T alone), spread over the
// right-hand-side columns: CTA (jb, g) solves columns [2g, 2g + 2) of block jb, one column per warp. The factors
// come from the blocked factorizations (k_chol_* / k_lu_*) in the block's global workspace
// ws = gws + jb * small_ws_doubles(p): M = ws (p x p row-major), B = ws + p*p (right-hand sides, row-major),
// pivots (LU) as ints at ws + 2*p*p.
//   chol = 1: M holds L (lower) of alpha = L L^T; out = L^{-T} L^{-1} B  (lambda)
//   chol = 0: M holds P rho_rec = L U (unit L below the diagonal, U on and above it) with the row
//             interchanges `pivots`; out = U^{-1} L^{-1} P B  (beta)
// Each substitution is column oriented (B[i] -= M[i][a] B[a] once B[a] is final). A warp keeps its column in
// registers (lane l: rows l, l + 32, ..., p <= 256), so a step is a shuffle of the final B[a] and one FMA per row
// the lane holds, with no block barrier. The factor is staged in shared memory 32 columns (or rows) at a time,
// double-buffered: the asynchronous copies of the next panel run while the warps work on this one. A diagonal
// entry d enters as a product with 1 / d (as LAPACK's unblocked LU scales by a reciprocal), by division only
// where 1 / d would overflow.
constexpr int kTrsmCols = 2;
constexpr int kTrsmPanel = 32;
constexpr int kTrsmLd = kTrsmPanel + 1;
constexpr int kTrsmSlots = 8;   // rows per lane: p <= 256
__host__ __device__ inline size_t trsm_smem(int p) {
  return 2 * (size_t)p * kTrsmLd * sizeof(double) + 2 * (size_t)p * sizeof(int);
}

__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Copies of panel `s0` into pan: forward, rows a0 .. p-1 of columns a0 .. a0+31 (pan[r ld + j] = M[a0 + r][a0 + j]);
// backward, rows 0 .. a0+31 of the upper factor's columns a0 .. a0+31 (pan[i ld + j] = U[i][a0 + j], with
// U = L^T for chol: M[a0 + j][i]).
__device__ __forceinline__ void trsm_issue(double *pan, const double *M, int p, int s0, bool fwd, bool lt) {
  const int a0 = s0 * kTrsmPanel, NT = blockDim.x;
  if (fwd) {
    const int n = (p - a0) * kTrsmPanel;
    for (int e = threadIdx.x; e < n; e += NT)
      cp_async8(pan + (e >> 5) * kTrsmLd + (e & 31), M + (int64_t)(a0 + (e >> 5)) * p + a0 + (e & 31));
  } else if (lt) {
    const int a1 = a0 + kTrsmPanel;
    for (int e = threadIdx.x; e < kTrsmPanel * a1; e += NT) {
      const int j = e / a1, i = e - j * a1;
      cp_async8(pan + i * kTrsmLd + j, M + (int64_t)(a0 + j) * p + i);
    }
  } else {
    const int n = (a0 + kTrsmPanel) * kTrsmPanel;
    for (int e = threadIdx.x; e < n; e += NT)
      cp_async8(pan + (e >> 5) * kTrsmLd + (e & 31), M + (int64_t)(e >> 5) * p + a0 + (e & 31));
  }
}

// The 32 steps of panel S0 on this warp's column b (forward: rows a0 + jl final in order jl = 0..31, rows below
// updated; backward: jl = 31..0, rows above updated). unit: the forward factor has a unit diagonal (LU).
template <int S0>
__device__ __forceinline__ void trsm_steps(double (&b)[kTrsmSlots], const double *pan, int ns, bool fwd, bool unit,
                                           int lane) {
  constexpr unsigned kAll = 0xffffffffu;
  // this lane's diagonal entry of the panel (row a0 + lane, column a0 + lane)
  const double d = fwd ? pan[lane * kTrsmLd + lane] : pan[(S0 * kTrsmPanel + lane) * kTrsmLd + lane];
  const bool scale = !(fwd && unit);
  const double rd = 1.0 / d;
  const bool rec = fabs(d) >= DBL_MIN;
  if (fwd) {
    for (int jl = 0; jl < kTrsmPanel; ++jl) {
      const double own = scale ? (rec ? b[S0] * rd : b[S0] / d) : b[S0];
      const double x = __shfl_sync(kAll, own, jl);
      if (lane == jl) b[S0] = x;
      else if (lane > jl) b[S0] = fma(-pan[lane * kTrsmLd + jl], x, b[S0]);
#pragma unroll
      for (int s = S0 + 1; s < kTrsmSlots; ++s)
        if (s < ns) b[s] = fma(-pan[((s - S0) * kTrsmPanel + lane) * kTrsmLd + jl], x, b[s]);
    }
  } else {
    for (int jl = kTrsmPanel - 1; jl >= 0; --jl) {
      const double own = rec ? b[S0] * rd : b[S0] / d;
      const double x = __shfl_sync(kAll, own, jl);
      if (lane == jl) b[S0] = x;
      else if (lane < jl) b[S0] = fma(-pan[(S0 * kTrsmPanel + lane) * kTrsmLd + jl], x, b[S0]);
#pragma unroll
      for (int s = 0; s < S0; ++s) b[s] = fma(-pan[(s * kTrsmPanel + lane) * kTrsmLd + jl], x, b[s]);
    }
  }
}

__global__ void __launch_bounds__(kTrsmCols * 32) k_trsm_cols(int p, int chol, const double *__restrict__ gws,
                                                              const int *__restrict__ active,
                                                              double *__restrict__ out, DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;   // frozen block: its lambda / beta were zeroed by the factorization kernel
  const int pp = p * p;
  const double *M = gws + (int64_t)jb * small_ws_doubles_dev(p);
  const double *Bg = M + pp;
  const int *pivots = reinterpret_cast<const int *>(M + 2 * pp);
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.y * kTrsmCols + (threadIdx.x >> 5);   // this warp's column
  const int ns = p / kTrsmPanel;
  extern __shared__ __align__(16) double sm_dyn[];
  double *pan0 = sm_dyn, *pan1 = sm_dyn + (size_t)p * kTrsmLd;
  int *perm = reinterpret_cast<int *>(pan1 + (size_t)p * kTrsmLd);
  // panel sequence: forward panels 0 .. ns-1 (not for chol = 2), then backward panels ns-1 .. 0
  const int nfwd = chol == 2 ? 0 : ns, npan = nfwd + ns;
  auto panel_of = [&](int t) { return t < nfwd ? t : nfwd + ns - 1 - t; };
  trsm_issue(pan0, M, p, panel_of(0), nfwd > 0, chol != 0);
  cp_async_commit();
  // LU: row i of P B is row perm[i] of B (the interchanges applied in factorization order)
  if (!chol) {
    int *pv = perm + p;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      perm[i] = i;
      pv[i] = pivots[i];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int a = 0; a < p; ++a) {
        const int r = pv[a];
        if (r != a) {
          const int t = perm[a];
          perm[a] = perm[r];
          perm[r] = t;
        }
      }
    __syncthreads();
  }
  double b[kTrsmSlots];
#pragma unroll
  for (int s = 0; s < kTrsmSlots; ++s) {
    const int i = s * kTrsmPanel + lane;
    b[s] = s < ns ? Bg[(int64_t)(chol ? i : perm[i]) * p + c] : 0.0;
  }
  for (int t = 0; t < npan; ++t) {
    const double *cur = (t & 1) ? pan1 : pan0;
    if (t + 1 < npan) trsm_issue((t & 1) ? pan0 : pan1, M, p, panel_of(t + 1), t + 1 < nfwd, chol != 0);
    cp_async_commit();
    cp_async_wait1();   // this thread's copies of panel t are in
    __syncthreads();    // and everyone's
    const bool fwd = t < nfwd, unit = chol == 0;
    switch (panel_of(t)) {
      case 0: trsm_steps<0>(b, cur, ns, fwd, unit, lane); break;
      case 1: trsm_steps<1>(b, cur, ns, fwd, unit, lane); break;
      case 2: trsm_steps<2>(b, cur, ns, fwd, unit, lane); break;
      case 3: trsm_steps<3>(b, cur, ns, fwd, unit, lane); break;
      case 4: trsm_steps<4>(b, cur, ns, fwd, unit, lane); break;
      case 5: trsm_steps<5>(b, cur, ns, fwd, unit, lane); break;
      case 6: trsm_steps<6>(b, cur, ns, fwd, unit, lane); break;
      default: trsm_steps<7>(b, cur, ns, fwd, unit, lane); break;
    }
    __syncthreads();    // panel t's buffer is refilled in step t + 1
  }
  bool fin = true;
  double *oj = out + (int64_t)jb * pp;
#pragma unroll
  for (int s = 0; s < kTrsmSlots; ++s)
    if (s < ns) {
      oj[(int64_t)(s * kTrsmPanel + lane) * p + c] = b[s];
      fin = fin && isfinite(b[s]);
    }
  if (!__syncthreads_and(fin) && threadIdx.x == 0) flag_breakdown(st);
}

// ---- Blocked factorizations of the large-block BSOLVEs (p > 32, a multiple of 32) -------------------------
// A p x p factorization on one CTA is a sequence of p barrier-separated rank-1 steps on one SM's share of the
// FP64 pipe (at p = 256: 4.2 ms for Cholesky, 6.6 ms for LU). Here the partial sums, the panel solves and the
// trailing updates are spread over many CTAs in separate launches, panel by panel (width 32, right-looking as in
// LAPACK's blocked xPOTRF / xGETRF): only the 32-column panel factorization runs on one CTA per block.
// Block jb's workspace ws = gws + jb * small_ws_doubles(p): M (p x p row-major, factored in place), B (p x p
// row-major right-hand sides), the LU pivots (p ints) at ws + 2 p^2 and the pivot threshold at ws + 3 p^2.
constexpr int kPB = 32;   // panel width

__device__ __forceinline__ double *blk_ws(double *gws, int jb, int p) {
  return gws + (int64_t)jb * small_ws_doubles_dev(p);
}

// Sum the partial rows of two products of block jb, entry (a, b) of each (partial layout b*p + a): M[a][b] =
// the first (swapM: stored transposed, M[b][a]), B[a][b] = the second; copyB (optional) receives B row-major,
// zeroOut (optional) is zeroed for a frozen block. Each thread one entry, partials added in partial-row order.
__global__ void __launch_bounds__(256) k_bs_gather(const double *__restrict__ partM, int npM,
                                                   const double *__restrict__ partB, int npB, int k, int p,
                                                   int global, const int *__restrict__ active, double *gws,
                                                   double *__restrict__ copyB, double *__restrict__ zeroOut,
                                                   const double *__restrict__ srcM, const DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x, pp = p * p;
  const int e = blockIdx.y * blockDim.x + threadIdx.x;   // source index b*p + a
  if (e >= pp) return;
  if (!active[jb]) {
    if (zeroOut) zeroOut[(int64_t)jb * pp + e] = 0.0;
    return;
  }
  const int b = e / p, a = e - b * p;
  const int64_t E = (int64_t)k * p;
  const int q = global ? k / p : 1;
  const int64_t base = global ? 0 : (int64_t)jb * pp;
  auto sum = [&](const double *part, int np) {
    double v = 0.0;
    for (int pi = 0; pi < np; ++pi)
      for (int j = 0; j < q; ++j) v += part[pi * E + base + (int64_t)j * pp + e];
    return v;
  };
  double *ws = blk_ws(gws, jb, p);
  if (srcM) ws[e] = srcM[(int64_t)jb * pp + e];           // already row-major (the recomputed rho)
  else ws[a * p + b] = sum(partM, npM);
  const double vb = sum(partB, npB);
  ws[pp + a * p + b] = vb;
  if (copyB) copyB[(int64_t)jb * pp + a * p + b] = vb;
}

// Cholesky of the diagonal 32 x 32 block at a0 (lower triangle), after the trailing updates of the earlier
// panels. At a0 = 0 the pivot threshold 64 eps max|diag| of the unfactored matrix is set first.
// colrel: the pivot test of the retooled form (each pivot against 64 eps times its own original diagonal entry,
// kept at ws + 3 p^2 + 8 .. + p), else Algorithm 1's (against 64 eps max|diag|).
__global__ void __launch_bounds__(256) k_chol_diag(double *gws, int p, int a0, const int *__restrict__ active,
                                                   DevStatus *st, int colrel) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  double *thr = M + 3 * (int64_t)p * p;
  double *dg = thr + 8;
  __shared__ double L[kPB][kPB + 1];
  __shared__ int bad;
  if (a0 == 0) {
    double m = 0.0;
    for (int a = threadIdx.x; a < p; a += blockDim.x) {
      const double d = M[(int64_t)a * p + a];
      m = fmax(m, fabs(d));
      if (colrel) dg[a] = d;
    }
    m = block_max(m);
    if (threadIdx.x == 0) thr[0] = kPivotFactor * DBL_EPSILON * m;
  }
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    L[i][j] = M[(int64_t)(a0 + i) * p + a0 + j];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int a = 0; a < kPB; ++a) {
    if (threadIdx.x == 0) {
      const double d = L[a][a];
      const double thresh = colrel ? kPivotFactor * DBL_EPSILON * dg[a0 + a] : thr[0];
      if (!(isfinite(d) && d > thresh)) bad = 1;
      else L[a][a] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    for (int i = a + 1 + threadIdx.x; i < kPB; i += blockDim.x) L[i][a] /= L[a][a];
    __syncthreads();
    const int m = kPB - a - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = a + 1 + e / m, j = a + 1 + e % m;
      if (j <= i) L[i][j] -= L[i][a] * L[j][a];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    if (j <= i) M[(int64_t)(a0 + i) * p + a0 + j] = L[i][j];
  }
}

// The panel below the diagonal block: L21 = A21 L11^{-T}, one row per thread.
__global__ void __launch_bounds__(128) k_chol_panel(double *gws, int p, int a0, const int *__restrict__ active,
                                                    DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  __shared__ double L[kPB][kPB + 1];
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    L[i][j] = j <= i ? M[(int64_t)(a0 + i) * p + a0 + j] : 0.0;
  }
  __syncthreads();
  const int r = a0 + kPB + blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= p) return;
  double *row = M + (int64_t)r * p + a0;
  double x[kPB];
#pragma unroll
  for (int j = 0; j < kPB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < kPB; ++j) {
    double v = x[j];
#pragma unroll
    for (int m = 0; m < j; ++m) v -= x[m] * L[j][m];
    x[j] = v / L[j][j];
  }
#pragma unroll
  for (int j = 0; j < kPB; ++j) row[j] = x[j];
}

// Trailing update of the lower triangle, A22 -= L21 L21^T, one 32 x 32 tile (ti >= tj) per CTA.
__global__ void __launch_bounds__(256) k_chol_update(double *gws, int p, int a0, const int *__restrict__ active,
                                                     DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  const int y = blockIdx.y;
  int ti = (int)((sqrt(8.0 * y + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= y) ++ti;
  while (ti * (ti + 1) / 2 > y) --ti;
  const int tj = y - ti * (ti + 1) / 2;
  const int r0 = a0 + kPB + ti * kPB, c0 = a0 + kPB + tj * kPB;
  __shared__ double Li[kPB][kPB + 1], Lj[kPB][kPB + 1];
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, m = e % kPB;
    Li[i][m] = M[(int64_t)(r0 + i) * p + a0 + m];
    Lj[i][m] = M[(int64_t)(c0 + i) * p + a0 + m];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    double acc = 0.0;
#pragma unroll 8
    for (int m = 0; m < kPB; ++m) acc = fma(Li[i][m], Lj[j][m], acc);
    M[(int64_t)(r0 + i) * p + c0 + j] -= acc;
  }
}

// LU with partial pivoting of the panel of columns [a0, a0 + 32), rows a0..p-1, in shared memory; the row
// interchanges are recorded (global row numbers, factorization order) and applied to the rest of each row. At
// a0 = 0 the threshold 64 eps max|diag| and the finiteness of the matrix are checked first. After the last panel
// the iteration counter is raised as the one-CTA factorization does.
__global__ void __launch_bounds__(256) k_lu_panel(double *gws, int p, int a0, const int *__restrict__ active,
                                                  DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  const int64_t pp = (int64_t)p * p;
  int *piv = reinterpret_cast<int *>(M + 2 * pp);
  double *thr = M + 3 * pp;
  const int rows = p - a0;
  extern __shared__ __align__(16) double sm_dyn[];
  double *Pn = sm_dyn;   // Pn[r * 33 + c] = M[a0 + r][a0 + c]
  constexpr int LD = kPB + 1;
  __shared__ int bad, best;
  __shared__ double srec;
  if (a0 == 0) {
    double m = 0.0;
    bool fin = true;
    for (int a = threadIdx.x; a < p; a += blockDim.x) m = fmax(m, fabs(M[(int64_t)a * p + a]));
    for (int64_t e = threadIdx.x; e < pp; e += blockDim.x) fin = fin && isfinite(M[e]);
    m = block_max(m);
    fin = __syncthreads_and(fin);
    if (threadIdx.x == 0) thr[0] = fin ? kPivotFactor * DBL_EPSILON * m : NAN;
  }
  for (int e = threadIdx.x; e < rows * kPB; e += blockDim.x) {
    const int r = e / kPB, c = e % kPB;
    Pn[r * LD + c] = M[(int64_t)(a0 + r) * p + a0 + c];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const double thresh = thr[0];
  if (!(thresh >= 0.0)) {   // a non-finite entry
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  __shared__ double wv[8];
  __shared__ int wi[8];
  for (int a = 0; a < kPB; ++a) {
    // pivot: the largest |Pn[r][a]|, r >= a, smallest r on ties (NaN counts as infinite)
    double v = -1.0;
    int idx = rows;
    for (int r = a + threadIdx.x; r < rows; r += blockDim.x) {
      const double x = fabs(Pn[r * LD + a]);
      const double xv = (x == x) ? x : INFINITY;
      if (xv > v) { v = xv; idx = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { wv[threadIdx.x >> 5] = v; wi[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bv = -1.0;
      int bi = rows;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
      best = bi;
      piv[a0 + a] = a0 + bi;
      if (!(bv > thresh)) bad = 1;
      else srec = 1.0 / Pn[bi * LD + a];   // the pivot's reciprocal, used while it stays finite
    }
    __syncthreads();
    if (bad) break;
    const int bi = best;
    if (bi != a && threadIdx.x < kPB) {
      const double t = Pn[a * LD + threadIdx.x];
      Pn[a * LD + threadIdx.x] = Pn[bi * LD + threadIdx.x];
      Pn[bi * LD + threadIdx.x] = t;
    }
    __syncthreads();
    const double ua = Pn[a * LD + a], ru = srec;
    const bool rec = fabs(ua) >= DBL_MIN;
    for (int r = a + 1 + threadIdx.x; r < rows; r += blockDim.x)
      Pn[r * LD + a] = rec ? Pn[r * LD + a] * ru : Pn[r * LD + a] / ua;
    __syncthreads();
    // rank-1 update of the entries (r, c), r, c > a, taken in row-major order e = (r - a - 1) w + (c - a - 1);
    // thread t takes e = t, t + T, ... with (r, c) advanced incrementally (one division per step)
    const int w = kPB - a - 1;
    if (w > 0) {
      const int T = blockDim.x, dq = T / w, dr = T - dq * w;
      int rr = threadIdx.x / w, cc = threadIdx.x - rr * w;
      for (int r = a + 1 + rr; r < rows;) {
        const int c = a + 1 + cc;
        Pn[r * LD + c] -= Pn[r * LD + a] * Pn[a * LD + c];
        r += dq;
        cc += dr;
        if (cc >= w) {
          cc -= w;
          ++r;
        }
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) flag_breakdown(st);
    return;
  }
  for (int e = threadIdx.x; e < rows * kPB; e += blockDim.x) {
    const int r = e / kPB, c = e % kPB;
    M[(int64_t)(a0 + r) * p + a0 + c] = Pn[r * LD + c];
  }
  // the panel's interchanges on the columns outside it: composed into "row dst[q] receives row src[q]" (at most
  // 2 x 32 rows move), then each column reads all its moving entries before writing any (one column per thread)
  __shared__ int mv_dst[2 * kPB], mv_src[2 * kPB], nmv;
  int *rowmap = reinterpret_cast<int *>(Pn);   // the panel is in M again: its buffer holds the row map of rows a0..
  __syncthreads();
  for (int i = threadIdx.x; i < rows; i += blockDim.x) rowmap[i] = a0 + i;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int a = 0; a < kPB; ++a) {
      const int r = piv[a0 + a] - a0;
      if (r != a) {
        const int t = rowmap[a];
        rowmap[a] = rowmap[r];
        rowmap[r] = t;
      }
    }
    int m = 0;
    for (int i = 0; i < rows; ++i)
      if (rowmap[i] != a0 + i) {
        mv_dst[m] = a0 + i;
        mv_src[m] = rowmap[i];
        ++m;
      }
    nmv = m;
  }
  __syncthreads();
  const int nm = nmv;
  for (int c = threadIdx.x; c < p - kPB; c += blockDim.x) {
    const int col = c < a0 ? c : c + kPB;
    double v[2 * kPB];
#pragma unroll
    for (int q = 0; q < 2 * kPB; ++q)
      if (q < nm) v[q] = M[(int64_t)mv_src[q] * p + col];
#pragma unroll
    for (int q = 0; q < 2 * kPB; ++q)
      if (q < nm) M[(int64_t)mv_dst[q] * p + col] = v[q];
  }
  if (a0 + kPB == p && threadIdx.x == 0) atomicMax(&st->iter, st->cur);
}

// U12 = L11^{-1} A12 (L11 unit lower) for 32 columns right of the panel, one column per thread.
__global__ void __launch_bounds__(32) k_lu_u12(double *gws, int p, int a0, const int *__restrict__ active,
                                               DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  __shared__ double L[kPB][kPB + 1];
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    L[i][j] = M[(int64_t)(a0 + i) * p + a0 + j];
  }
  __syncthreads();
  const int c = a0 + kPB + blockIdx.y * kPB + threadIdx.x;
  if (c >= p) return;
  double x[kPB];
#pragma unroll
  for (int j = 0; j < kPB; ++j) x[j] = M[(int64_t)(a0 + j) * p + c];
#pragma unroll
  for (int j = 1; j < kPB; ++j) {
    double v = x[j];
#pragma unroll
    for (int m = 0; m < j; ++m) v -= L[j][m] * x[m];
    x[j] = v;
  }
#pragma unroll
  for (int j = 0; j < kPB; ++j) M[(int64_t)(a0 + j) * p + c] = x[j];
}

// Trailing update A22 -= L21 U12, one 32 x 32 tile per CTA.
__global__ void __launch_bounds__(256) k_lu_update(double *gws, int p, int a0, const int *__restrict__ active,
                                                   DevStatus *st) {
  if (st->flags != 0) return;
  const int jb = blockIdx.x;
  if (!active[jb]) return;
  double *M = blk_ws(gws, jb, p);
  const int t = (p - a0 - kPB) / kPB;
  const int ti = blockIdx.y / t, tj = blockIdx.y % t;
  const int r0 = a0 + kPB + ti * kPB, c0 = a0 + kPB + tj * kPB;
  __shared__ double Ls[kPB][kPB + 1], Us[kPB][kPB + 1];
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, m = e % kPB;
    Ls[i][m] = M[(int64_t)(r0 + i) * p + a0 + m];
    Us[i][m] = M[(int64_t)(a0 + i) * p + c0 + m];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kPB * kPB; e += blockDim.x) {
    const int i = e / kPB, j = e % kPB;
    double acc = 0.0;
#pragma unroll 8
    for (int m = 0; m < kPB; ++m) acc = fma(Ls[i][m], Us[m][j], acc);
    M[(int64_t)(r0 + i) * p + c0 + j] -= acc;
  }
}

// Start of a solve: reduce the initial residual norms, mark zero columns converged, reset the status.
__global__ void k_init_status(const double *__restrict__ partN, int nparts, int k, int p, int global,
                              double *__restrict__ r0n2, double *__restrict__ rn2, int *__restrict__ active,
                              int *__restrict__ block_iters, double *__restrict__ lam, double *__restrict__ beta,
                              DevStatus *st, ShiftCtl sc) {
  const int nblk = global ? 1 : k / p;
  __shared__ int nact, nonfinite;
  if (threadIdx.x == 0) { nact = 0; nonfinite = 0; }
  __syncthreads();
  __shared__ double ncol[kNT], nscr[kSmallNT > kNT ? kSmallNT : kNT];
  det_reduce(k, nparts, [&](int pi, int c) { return partN[(int64_t)pi * k + c]; }, ncol, nscr);
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double s = ncol[c];
    r0n2[c] = s;
    rn2[c] = s;
    write_shifts(sc, k, c, s);
    if (!isfinite(s)) atomicOr(&nonfinite, 1);
  }
  __syncthreads();
  for (int jb = threadIdx.x; jb < nblk; jb += blockDim.x) {
    const int c0 = global ? 0 : jb * p, c1 = global ? k : c0 + p;
    bool all_zero = true;   // ||R_c^0|| <= tol ||R_c^0|| holds for tol < 1 only when R_c^0 = 0
    for (int c = c0; c < c1; ++c) all_zero = all_zero && (r0n2[c] == 0.0);
    active[jb] = all_zero ? 0 : 1;
    block_iters[jb] = 0;
    if (!all_zero) atomicAdd(&nact, 1);
  }
  const int pp = p * p;
  for (int e = threadIdx.x; e < nblk * pp; e += blockDim.x) { lam[e] = 0.0; beta[e] = 0.0; }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->n_active = nact;
    st->iter = 0;
    st->cur = 1;
    st->breakdown_iter = 0;
    st->flags = nonfinite ? ST_NUMERIC : (nact == 0 ? ST_DONE : 0);
  }
}

// Residual replacement found columns whose true residual is not yet below the tolerance although every
// block had stopped on its recursive residual: reopen those blocks (their P is kept) and clear the
// "done" flag so that the iterations resume.
__global__ void k_reactivate(const double *__restrict__ rtn2, const double *__restrict__ r0n2, double tol2, int k,
                             int p, int global, int *__restrict__ active, DevStatus *st) {
  const int nblk = global ? 1 : k / p;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int jb = threadIdx.x; jb < nblk; jb += blockDim.x) {
    const int c0 = global ? 0 : jb * p, c1 = global ? k : c0 + p;
    bool need = false;
    for (int c = c0; c < c1; ++c) need = need || !(rtn2[c] <= tol2 * r0n2[c]);
    active[jb] = need ? 1 : 0;
    if (need) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && st->flags == ST_DONE) {
    st->n_active = cnt;
    st->flags = cnt > 0 ? 0 : ST_DONE;
  }
}

// Sum BDOT partials in CTA order into gamma (per distinct block p*p, row-major a*p + b).
__global__ void __launch_bounds__(kSmallNT) k_finish_gram(const double *__restrict__ part, int nparts, int k, int p,
                                                          int global, double *__restrict__ gamma, double *gws) {
  extern __shared__ __align__(16) double sm_dyn[];
  double *sm = gws ? gws + (int64_t)blockIdx.x * small_ws_doubles_dev(p) : sm_dyn;
  const int pp = p * p;
  double *tmp = sm, *scr = sm + pp;
  const int jb = blockIdx.x;
  reduce_block(part, nparts, k, p, global, jb, tmp, scr);
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    const int b = e / p, a = e - b * p;
    gamma[(int64_t)jb * pp + a * p + b] = tmp[e];
  }
}

// Gram shifts from the squared norms n2 (NULL: every column taken at the squared norm 2^(2 kGramCenter), whose
// base shift is 0, so that only the role offsets remain).
__global__ void k_fill_shifts(const double *__restrict__ n2, int k, ShiftCtl sc) {
  const double unit2 = (double)(1 << kGramCenter) * (double)(1 << kGramCenter);
  for (int c = threadIdx.x; c < k; c += blockDim.x) write_shifts(sc, k, c, n2 ? n2[c] : unit2);
}

__global__ void k_reduce_norms(const double *__restrict__ partN, int nparts, int k, double *__restrict__ out) {
  __shared__ double ncol[kNT], nscr[kSmallNT > kNT ? kSmallNT : kNT];
  det_reduce(k, nparts, [&](int pi, int c) { return partN[(int64_t)pi * k + c]; }, ncol, nscr);
  for (int c = threadIdx.x; c < k; c += blockDim.x) out[c] = ncol[c];
}

// out[e] = sum over pi < nparts of part[pi * E + e], in partial order (one thread per entry): the per-CTA
// partials of one product collapsed into a single partial row, ready for a sum over ranks.
__global__ void k_sum_partials(const double *__restrict__ part, int nparts, int64_t E, double *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int pi = 0;
    for (; pi + 1 < nparts; pi += 2) {
      a0 += part[(int64_t)pi * E + e];
      a1 += part[(int64_t)(pi + 1) * E + e];
    }
    if (pi < nparts) a0 += part[(int64_t)pi * E + e];
    out[e] = a0 + a1;
  }
}

// buf[i * k + c] = P[rows[i] * k + c]: the rows of P another rank needs (halo exchange of the row-sharded solve)
__global__ void k_gather_rows(const double *__restrict__ P, const int32_t *__restrict__ rows, int64_t nrows, int k,
                              double *__restrict__ buf) {
  const int64_t total = nrows * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    buf[e] = P[(int64_t)rows[i] * k + (e - i * k)];
  }
}

// Row permutation of an n x k block vector: gather dst[s] = src[perm[s]], or scatter dst[perm[s]] = src[s].
__global__ void k_permute_rows(const double *__restrict__ src, const int32_t *__restrict__ perm, int64_t n, int k,
                               double *__restrict__ dst, int scatter) {
  const int64_t total = n * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / k, c = e - s * k;
    const int64_t r = perm[s];
    if (scatter) dst[r * k + c] = src[e];
    else dst[e] = src[r * k + c];
  }
}

// X64 += D32 (the refinement update of the mixed-precision form)
// X += D 2^sigma_c (sig: the FP32 process's scale exponent per column, NULL: 0), len = n k
__global__ void k_add_correction(double *__restrict__ X, const float *__restrict__ D, int64_t len, int k,
                                 const int *__restrict__ sig) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    X[i] += sig ? (double)D[i] * pow2d(sig[i % k]) : (double)D[i];
}

// Column maxima for the shifts of a standalone BDOT: out[c] = max_r |X[r][c]| as the bit pattern of a
// non-negative double (ordered like the integers; the caller zeroes out first). Thread (g, c) of a CTA covers
// rows g, g + rows per CTA pass, ... of column c. (The maximum itself, not its square: the square of an entry
// above 1e154 would overflow.)
__global__ void __launch_bounds__(kNT) k_col_maxabs(const double *__restrict__ X, int64_t n, int k,
                                                    unsigned long long *__restrict__ out) {
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  if (g >= rpp) return;
  double m = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpp + g; r < n; r += (int64_t)gridDim.x * rpp) m = fmax(m, fabs(X[r * k + c]));
  atomicMax(out + c, (unsigned long long)__double_as_longlong(m));
}

// sh[c] = floor(log2 cmax[c]) - kGramCenter: the column's largest entry scaled into [2^10, 2^11) (a zero or
// subnormal maximum: the shift of 1.0; one row, no role offsets)
__global__ void k_shift_from_max(const double *__restrict__ cmax, int k, int *__restrict__ sh) {
  for (int c = threadIdx.x; c < k; c += blockDim.x) sh[c] = clamp_shift(exponent_of(cmax[c]) - kGramCenter);
}

// Mixed form: the FP32 process of block j runs on R_j 2^-sigma_j, an exact scaling, so that FP32 holds its values
// whatever the scale of the FP64 residual (FP32 alone covers about 1e-38 .. 3e38). sigma_j = floor(log2 of the
// largest column norm of the block) (global: of all columns; 0 for a zero or non-finite block), stored for every
// column of the block. cur_s = cur 2^(-2 sigma), ref_s = ref 2^(-2 sigma) (squared norms in the process's scale).
__global__ void k_mixed_scale(const double *__restrict__ cur, const double *__restrict__ ref, int k, int p,
                              int global, int *__restrict__ sig, double *__restrict__ cur_s,
                              double *__restrict__ ref_s) {
  const int nblk = global ? 1 : k / p;
  for (int jb = threadIdx.x; jb < nblk; jb += blockDim.x) {
    const int c0 = global ? 0 : jb * p, c1 = global ? k : c0 + p;
    double m = 0.0;
    for (int c = c0; c < c1; ++c) m = fmax(m, cur[c]);
    const int sg = exponent_of(m) >> 1;
    const double f = pow2d(-2 * sg);
    for (int c = c0; c < c1; ++c) {
      sig[c] = sg;
      if (cur_s) cur_s[c] = cur[c] * f;
      if (ref_s) ref_s[c] = ref[c] * f;
    }
  }
}

// R32 = fl(R 2^-sigma_c), P32 = fl(M^{-1} R 2^-sigma_c) (dinv NULL: M = I), n x k row-major
__global__ void k_cast_scaled(const double *__restrict__ R, const double *__restrict__ dinv,
                              const int *__restrict__ sig, int64_t n, int k, float *__restrict__ R32,
                              float *__restrict__ P32) {
  const int64_t len = n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = R[i] * pow2d(-sig[i % k]);
    R32[i] = (float)v;
    if (P32) P32[i] = (float)(dinv ? v * dinv[i / k] : v);
  }
}

__global__ void k_cast_to_float(const double *__restrict__ src, float *__restrict__ dst, int64_t len) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Gradient with respect to the stored CSR values: grad[e] = -Lambda_row(e) . X_col(e).
__global__ void k_grad_values(const int32_t *__restrict__ rowidx, const int32_t *__restrict__ colind,
                              const double *__restrict__ Lam, const double *__restrict__ X, int64_t nnz, int k,
                              double *__restrict__ grad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const double *l = Lam + (int64_t)rowidx[e] * k;
    const double *x = X + (int64_t)colind[e] * k;
    double s = 0.0;
    for (int c = 0; c < k; ++c) s = fma(l[c], x[c], s);
    grad[e] = -s;
  }
}

__global__ void k_row_index(const int64_t *__restrict__ rowptr, int64_t n, int32_t *__restrict__ rowidx) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) rowidx[e] = (int32_t)r;
}

// ---------------------------------------------------------------------------------------------------
// host launchers

size_t small_ws_doubles(int p) { return small_ws_doubles_dev(p); }

// Row chunks (= partial rows) of the tiled large-block products: about 8 CTAs per SM over all tiles.
int lp_chunks(int64_t n, int k, int p, int nsm) {
  const int tiles = (k / p) * (p / 32) * (p / 32);
  int64_t ch = ((int64_t)nsm * 8 + tiles - 1) / tiles;
  const int64_t max_ch = (n + 31) / 32;
  if (ch > max_ch) ch = max_ch;
  return (int)(ch < 1 ? 1 : ch);
}
// Large blocks keep the p x p matrices in global memory (the column-parallel triangular solves read them
// there); smaller ones in shared memory unless they do not fit.
bool small_needs_gws(int p) { return p > kMaxP || small_ws_doubles_dev(p) * sizeof(double) > kSmallSmemMax; }
static size_t small_smem(int p) { return small_needs_gws(p) ? 0 : small_ws_doubles_dev(p) * sizeof(double); }
static bool small_split(int p) { return p > kMaxP; }
// Threads of a p x p solve CTA: its time is the partial-sum reduction when there are many partial rows and
// the serial factorization steps (each a barrier) when there are few; 128 threads measured faster below
// 8192 partial entries per block (64^2 Poisson, k = 8: 9.4 -> 7.9 ms per solve), 512 above (128^3, k = 32).
static int small_threads(int nparts, int p) { return (int64_t)nparts * p * p < 8192 ? 128 : kSmallNT; }

static size_t lu_panel_smem(int p, int a0) { return (size_t)(p - a0) * (kPB + 1) * sizeof(double); }

cudaError_t small_prepare(int p) {
  const size_t sm = small_smem(p);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_solve_lambda, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_solve_beta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (small_split(p)) {
    if (lu_panel_smem(p, 0) > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)lu_panel_smem(p, 0));
      if (e != cudaSuccess) return e;
    }
    if (trsm_smem(p) > 48 * 1024)
      return cudaFuncSetAttribute(k_trsm_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem(p));
  }
  return cudaSuccess;
}

static cudaError_t launch_trsm(int p, int nblk, int chol, const double *gws, const int *active, double *out,
                               DevStatus *st, cudaStream_t s) {
  dim3 grid((unsigned)nblk, (unsigned)(p / kTrsmCols));
  k_trsm_cols<<<grid, kTrsmCols * 32, trsm_smem(p), s>>>(p, chol, gws, active, out, st);
  return cudaGetLastError();
}

// Wide blocks: the partial sums (k_bs_gather), the blocked factorization panel by panel, then the
// column-parallel triangular solves.
static cudaError_t launch_blocked_chol(int p, int nblk, double *gws, const int *active, DevStatus *st,
                                       cudaStream_t s, int colrel = 0) {
  for (int a0 = 0; a0 < p; a0 += kPB) {
    k_chol_diag<<<nblk, 256, 0, s>>>(gws, p, a0, active, st, colrel);
    const int rows = p - a0 - kPB;
    if (rows > 0) {
      k_chol_panel<<<dim3((unsigned)nblk, (unsigned)((rows + 127) / 128)), 128, 0, s>>>(gws, p, a0, active, st);
      const int t = rows / kPB;
      k_chol_update<<<dim3((unsigned)nblk, (unsigned)(t * (t + 1) / 2)), 256, 0, s>>>(gws, p, a0, active, st);
    }
  }
  return cudaGetLastError();
}

static cudaError_t launch_blocked_lu(int p, int nblk, double *gws, const int *active, DevStatus *st,
                                     cudaStream_t s) {
  for (int a0 = 0; a0 < p; a0 += kPB) {
    k_lu_panel<<<nblk, 256, lu_panel_smem(p, a0), s>>>(gws, p, a0, active, st);
    const int rows = p - a0 - kPB;
    if (rows > 0) {
      const int t = rows / kPB;
      k_lu_u12<<<dim3((unsigned)nblk, (unsigned)t), kPB, 0, s>>>(gws, p, a0, active, st);
      k_lu_update<<<dim3((unsigned)nblk, (unsigned)(t * t)), 256, 0, s>>>(gws, p, a0, active, st);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_solve_lambda(const double *partA, const double *partR, int nparts, int nparts_r, int k, int p,
                                int global, const int *active, double *lam, double *rho_rec, DevStatus *st,
                                double *gws, int alpha_circ, cudaStream_t s) {
  const int nblk = global ? 1 : k / p;
  if (small_needs_gws(p) && gws == nullptr) return cudaErrorInvalidValue;
  if (!small_split(p)) {
    k_solve_lambda<<<nblk, small_threads(std::max(nparts, nparts_r), p), small_smem(p), s>>>(
        partA, partR, nparts, k, p, global, active, lam, rho_rec, st, small_needs_gws(p) ? gws : nullptr,
        alpha_circ, nparts_r);
    return cudaGetLastError();
  }
  const int pp = p * p;
  k_bs_gather<<<dim3((unsigned)nblk, (unsigned)((pp + 255) / 256)), 256, 0, s>>>(
      partA, nparts, partR, nparts_r, k, p, global, active, gws, rho_rec, lam, nullptr, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_blocked_chol(p, nblk, gws, active, st, s)) != cudaSuccess) return e;
  return launch_trsm(p, nblk, 1, gws, active, lam, st, s);
}

cudaError_t launch_solve_beta(const double *partRho, const double *partN, int nparts, int nparts_n, int k, int p,
                              int global, const double *tol2, const double *r0n2, double *rn2, int *active,
                              int *block_iters,
                              const double *rho_rec, double *beta, DevStatus *st, double *gws, int rho_circ,
                              cudaStream_t s, const ShiftCtl &sc) {
  const int nblk = global ? 1 : k / p;
  if (small_needs_gws(p) && gws == nullptr) return cudaErrorInvalidValue;
  const int split = small_split(p) ? 1 : 0;
  // the column norms, the stopping test and the shifts (wide blocks: only these; the solve follows)
  k_solve_beta<<<nblk, small_threads(nparts, p), small_smem(p), s>>>(
      partRho, partN, nparts, k, p, global, tol2, r0n2, rn2, active, block_iters, rho_rec, beta, st,
      small_needs_gws(p) ? gws : nullptr, rho_circ, nparts_n, split, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !split) return e;
  const int pp = p * p;
  k_bs_gather<<<dim3((unsigned)nblk, (unsigned)((pp + 255) / 256)), 256, 0, s>>>(
      nullptr, 0, partRho, nparts, k, p, global, active, gws, nullptr, nullptr, rho_rec, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_blocked_lu(p, nblk, gws, active, st, s)) != cudaSuccess) return e;
  return launch_trsm(p, nblk, 0, gws, active, beta, st, s);
}

cudaError_t launch_init_status(const double *partN, int nparts, int k, int p, int global, double *r0n2, double *rn2,
                               int *active, int *block_iters, double *lam, double *beta, DevStatus *st,
                               cudaStream_t s, const ShiftCtl &sc) {
  k_init_status<<<1, kSmallNT, 0, s>>>(partN, nparts, k, p, global, r0n2, rn2, active, block_iters, lam, beta, st,
                                       sc);
  return cudaGetLastError();
}

cudaError_t launch_fill_shifts(const double *n2, int k, const ShiftCtl &sc, cudaStream_t s) {
  if (sc.sh == nullptr) return cudaSuccess;
  k_fill_shifts<<<1, 256, 0, s>>>(n2, k, sc);
  return cudaGetLastError();
}

cudaError_t launch_finish_gram(const double *part, int nparts, int k, int p, int global, double *gamma, double *gws,
                               cudaStream_t s) {
  const int nblk = global ? 1 : k / p;
  const bool g = small_needs_gws(p);
  if (g && gws == nullptr) return cudaErrorInvalidValue;
  const size_t sm = g ? 0 : small_ws_doubles_dev(p) * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_finish_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_finish_gram<<<nblk, kSmallNT, sm, s>>>(part, nparts, k, p, global, gamma, g ? gws : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_reactivate(const double *rtn2, const double *r0n2, double tol2, int k, int p, int global,
                              int *active, DevStatus *st, cudaStream_t s) {
  k_reactivate<<<1, kSmallNT, 0, s>>>(rtn2, r0n2, tol2, k, p, global, active, st);
  return cudaGetLastError();
}

cudaError_t launch_reduce_norms(const double *partN, int nparts, int k, double *out, cudaStream_t s) {
  k_reduce_norms<<<1, kSmallNT, 0, s>>>(partN, nparts, k, out);
  return cudaGetLastError();
}

static int stream_grid(int64_t len, int nsm) {
  int64_t g = (len + 255) / 256;
  const int64_t cap = (int64_t)nsm * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

cudaError_t launch_sum_partials(const double *part, int nparts, int64_t E, double *out, int nsm, cudaStream_t s) {
  k_sum_partials<<<stream_grid(E, nsm), 256, 0, s>>>(part, nparts, E, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double *P, const int32_t *rows, int64_t nrows, int k, double *buf, int nsm,
                               cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  k_gather_rows<<<stream_grid(nrows * k, nsm), 256, 0, s>>>(P, rows, nrows, k, buf);
  return cudaGetLastError();
}

cudaError_t launch_permute_rows(const double *src, const int32_t *perm, int64_t n, int k, double *dst, int scatter,
                                int nsm, cudaStream_t s) {
  k_permute_rows<<<stream_grid(n * k, nsm), 256, 0, s>>>(src, perm, n, k, dst, scatter);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(double *X, const float *D, int64_t len, int k, const int *sig, int nsm,
                                  cudaStream_t s) {
  k_add_correction<<<stream_grid(len, nsm), 256, 0, s>>>(X, D, len, k, sig);
  return cudaGetLastError();
}

cudaError_t launch_col_shifts(const double *X, int64_t n, int k, double *cmax, int *sh, int nsm, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(double) * k, s);
  if (e != cudaSuccess) return e;
  k_col_maxabs<<<stream_grid(n * k, nsm), kNT, 0, s>>>(X, n, k, reinterpret_cast<unsigned long long *>(cmax));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_shift_from_max<<<1, 256, 0, s>>>(cmax, k, sh);
  return cudaGetLastError();
}

cudaError_t launch_mixed_scale(const double *cur, const double *ref, int k, int p, int global, int *sig,
                               double *cur_s, double *ref_s, cudaStream_t s) {
  k_mixed_scale<<<1, 256, 0, s>>>(cur, ref, k, p, global, sig, cur_s, ref_s);
  return cudaGetLastError();
}

cudaError_t launch_cast_scaled(const double *R, const double *dinv, const int *sig, int64_t n, int k, float *R32,
                               float *P32, int nsm, cudaStream_t s) {
  k_cast_scaled<<<stream_grid(n * k, nsm), 256, 0, s>>>(R, dinv, sig, n, k, R32, P32);
  return cudaGetLastError();
}

cudaError_t launch_cast_to_float(const double *src, float *dst, int64_t len, int nsm, cudaStream_t s) {
  k_cast_to_float<<<stream_grid(len, nsm), 256, 0, s>>>(src, dst, len);
  return cudaGetLastError();
}

cudaError_t launch_grad_values(const int32_t *rowidx, const int32_t *colind, const double *Lam, const double *X,
                               int64_t nnz, int k, double *grad, int nsm, cudaStream_t s) {
  k_grad_values<<<stream_grid(nnz, nsm), 256, 0, s>>>(rowidx, colind, Lam, X, nnz, k, grad);
  return cudaGetLastError();
}

cudaError_t launch_row_index(const int64_t *rowptr, int64_t n, int32_t *rowidx, int nsm, cudaStream_t s) {
  k_row_index<<<stream_grid(n, nsm), 256, 0, s>>>(rowptr, n, rowidx);
  return cudaGetLastError();
}

#include "bcg_retooled.inc"

}  // namespace bcgk
