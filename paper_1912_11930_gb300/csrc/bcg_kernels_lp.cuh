// Large-block kernels (32 < p <= 256, p a multiple of 32): the block products and block updates become
// tall-skinny matrix products (n x p times p x p per block), so they are tiled like small GEMMs instead of
// keeping a whole p-wide accumulator row per thread.
//   kl_bop      Q = A P (16-byte vector gathers), status-aware
//   kl_gram     per-chunk partials of <<X, Y>>_S by 32 x 32 output tiles (Dot2 accumulation, Section 2)
//   kl_baxpy    OUT_j = BASE_j + sign * Y_j C_j by (64 rows x 32 columns) output tiles, C staged by 32 x 32
//   kl_colnorm  per-column ||R_c||^2 partials
#pragma once

#include "bcg_kernels_wc.cuh"

namespace bcgk {

constexpr int kLT = 32;      // tile edge

__host__ __device__ constexpr bool lp_layout_ok(int k, int p) {
  return p > 32 && p <= kNT && p % kLT == 0 && k % p == 0 && k <= kNT;
}

// Q = A P, each thread V columns of one row.
template <typename T, int OPK, int V>
__global__ void __launch_bounds__(kNT) kl_bop(OpDesc A, const T *__restrict__ P, T *__restrict__ Q, int64_t n, int k,
                                              const DevStatus *__restrict__ st) {
  using VT = typename VecOf<T, V>::type;
  if (st != nullptr && st->flags != 0) return;
  const int kv = k / V;
  const int64_t total = n * kv;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kv;
    const int cv = (int)(i - r * kv);
    const VecU<T, V> q = apply_row_vec<T, OPK, V>(A, P, r, k, cv * V);
    reinterpret_cast<VT *>(Q)[i] = q.v;
  }
}

// d += (s + c) 2^(sx + sy) (FP64 operands were shifted before their split; FP32 ones were not)
template <typename T>
__device__ __forceinline__ void lp_flush(double &d, float &s, float &c, int sx, int sy) {
  if constexpr (Gram<T>::kShifted) {
    const double fx = pow2d(sx), fy = pow2d(sy);
    d += ((double)s * fx) * fy;
    d += ((double)c * fx) * fy;
  } else {
    d += (double)s;
    d += (double)c;
  }
  s = c = 0.0f;
}

// Partials of gamma = <<X, Y>>_S: grid.x = 32 x 32 tiles (block j, a-tile, b-tile), grid.y = row chunks.
// Partial row blockIdx.y holds entry (a, b) of block j at j*p*p + b*p + a (the layout of the small path).
// xscale (optional): X's row r is multiplied by xscale[r] (forms Z = M^{-1} R on the fly).
template <typename T>
__global__ void __launch_bounds__(kNT) kl_gram(const T *__restrict__ X, const T *__restrict__ Y, int64_t n, int k,
                                               int p, int global, const int *__restrict__ active,
                                               double *__restrict__ part, const DevStatus *__restrict__ st,
                                               const T *__restrict__ xscale, const int *__restrict__ shX,
                                               const int *__restrict__ shY) {
  using G = Gram<T>;
  using BT = typename G::B;
  if (st != nullptr && st->flags != 0) return;
  __shared__ BT Xs[kLT][kLT + 1], Ys[kLT][kLT + 1];
  __shared__ int sxs[kLT], sys[kLT];   // exponent shifts of this tile's X and Y columns
  const int ta_n = p / kLT;
  const int tile = blockIdx.x;
  const int j = tile / (ta_n * ta_n);
  const int ta = (tile / ta_n) % ta_n, tb = tile % ta_n;
  const int a0 = ta * kLT, b0 = tb * kLT;
  if (threadIdx.x < kLT) {
    sxs[threadIdx.x] = G::kShifted ? shift_at(shX, j * p + a0 + threadIdx.x) : 0;
    sys[threadIdx.x] = G::kShifted ? shift_at(shY, j * p + b0 + threadIdx.x) : 0;
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;   // this thread: a = a0+2ty+{0,1}, b = b0+2tx+{0,1}
  double *out = part + (int64_t)blockIdx.y * k * p + (int64_t)j * p * p;
  const bool act = block_active(active, global, j);
  const int64_t chunk = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r_begin = (int64_t)blockIdx.y * chunk, r_end = r_begin + chunk < n ? r_begin + chunk : n;
  float s[2][2], c[2][2];
  double d[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) { s[u][v] = c[u][v] = 0.0f; d[u][v] = 0.0; }
  if (act) {
    int rows_since_flush = 0;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kLT) {
      // stage 32 rows x 32 columns of X (a-range) and Y (b-range)
      for (int e = threadIdx.x; e < kLT * kLT; e += kNT) {
        const int rr = e / kLT, cc = e % kLT;
        const int64_t r = r0 + rr;
        BT xb = G::zero(), yb = G::zero();
        if (r < r_end) {
          const T xv = X[r * k + (int64_t)j * p + a0 + cc];
          xb = G::conv(xscale ? xv * xscale[r] : xv, sxs[cc]);
          yb = G::conv(Y[r * k + (int64_t)j * p + b0 + cc], sys[cc]);
        }
        Xs[rr][cc] = xb;
        Ys[rr][cc] = yb;
      }
      __syncthreads();
#pragma unroll 4
      for (int rr = 0; rr < kLT; ++rr) {
        const BT x0 = Xs[rr][2 * ty], x1 = Xs[rr][2 * ty + 1];
        const BT y0 = Ys[rr][2 * tx], y1 = Ys[rr][2 * tx + 1];
        G::add(s[0][0], c[0][0], x0, y0);
        G::add(s[0][1], c[0][1], x0, y1);
        G::add(s[1][0], c[1][0], x1, y0);
        G::add(s[1][1], c[1][1], x1, y1);
      }
      __syncthreads();
      rows_since_flush += kLT;
      if (rows_since_flush >= kFlushPasses) {
        rows_since_flush = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) lp_flush<T>(d[u][v], s[u][v], c[u][v], sxs[2 * ty + u], sys[2 * tx + v]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      lp_flush<T>(d[u][v], s[u][v], c[u][v], sxs[2 * ty + u], sys[2 * tx + v]);
      const int a = a0 + 2 * ty + u, b = b0 + 2 * tx + v;
      out[(int64_t)b * p + a] = d[u][v];
    }
}

// OUT_j = BASE_j + sign * Y_j C_j (C_j row-major p x p per distinct block, FP64 in memory). grid.x = column
// tiles (k/32), grid.y = row tiles of kLRows. OUT may equal BASE; Y must not alias OUT. bump != 0: CTA (0,0)
// advances the iteration counter (this launch then plays the role of K3).
// bscale (optional): BASE's row r is multiplied by bscale[r] (P = M^{-1} R + P beta).
// Register tiling: thread (ty4, tx4) owns rows 4 ty4 .. 4 ty4 + 3 and columns 4 tx4 .. 4 tx4 + 3 of the
// 128 x 32 output tile; per step of the contraction it reads 4 Y values and 4 C values (two 16-byte shared
// loads for FP32) for 16 FMAs. Y is staged transposed (Yt[a][row]) so that those loads are vectors.
constexpr int kLRows = 128;   // rows of a BAXPY output tile
constexpr int kLYs = kLRows + 4;   // padded row length of the transposed Y tile (16-byte aligned rows)
template <typename T>
__global__ void __launch_bounds__(kNT) kl_baxpy(T *OUT, const T *BASE, const T *__restrict__ Y,
                                                const double *__restrict__ C, int64_t n, int k, int p, int global,
                                                T sign, const int *__restrict__ active, DevStatus *__restrict__ st,
                                                int bump, const T *__restrict__ bscale) {
  if (st->flags != 0) return;
  if (bump && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) st->cur += 1;
  __shared__ __align__(16) T Yt[kLT][kLYs];
  __shared__ __align__(16) T Cs[kLT][kLT + 4];
  const int c0 = blockIdx.x * kLT;
  const int j = c0 / p, b0 = c0 - j * p;
  const int tx4 = threadIdx.x % 8, ty4 = threadIdx.x / 8;   // columns 4 tx4 + v, rows 4 ty4 + u
  const int64_t r0 = (int64_t)blockIdx.y * kLRows;
  const double *Cj = C + (int64_t)(global ? 0 : j) * p * p;
  const bool act = block_active(active, global, j);
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + 4 * ty4 + u;
    const T s = (r < n && bscale) ? bscale[r] : T(1);
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = r < n ? BASE[r * k + c0 + 4 * tx4 + v] * s : T(0);
  }
  if (act) {
    for (int a0 = 0; a0 < p; a0 += kLT) {
      for (int e = threadIdx.x; e < kLRows * kLT; e += kNT) {   // coalesced rows of Y, stored transposed
        const int rr = e / kLT, aa = e % kLT;
        const int64_t r = r0 + rr;
        Yt[aa][rr] = r < n ? Y[r * k + (int64_t)j * p + a0 + aa] : T(0);
      }
      for (int e = threadIdx.x; e < kLT * kLT; e += kNT) {
        const int aa = e / kLT, bb = e % kLT;
        Cs[aa][bb] = sign * (T)Cj[(int64_t)(a0 + aa) * p + b0 + bb];
      }
      __syncthreads();
#pragma unroll 4
      for (int aa = 0; aa < kLT; ++aa) {
        T yv[4], cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) yv[u] = Yt[aa][4 * ty4 + u];
#pragma unroll
        for (int v = 0; v < 4; ++v) cv[v] = Cs[aa][4 * tx4 + v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma_t(yv[u], cv[v], acc[u][v]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + 4 * ty4 + u;
    if (r < n)
#pragma unroll
      for (int v = 0; v < 4; ++v) OUT[r * k + c0 + 4 * tx4 + v] = acc[u][v];
  }
}

// Per-column ||R_c||^2 partials (Dot2), one partial row of k entries per CTA.
template <typename T>
__global__ void __launch_bounds__(kNT) kl_colnorm(const T *__restrict__ R, int64_t n, int k,
                                                  double *__restrict__ partN, const DevStatus *__restrict__ st,
                                                  const int *__restrict__ shR) {
  using G = Gram<T>;
  using BT = typename G::B;
  if (st != nullptr && st->flags != 0) return;
  __shared__ double red[kNT];
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int sR = G::kShifted ? shift_at(shR, c) : 0;
  float s = 0.0f, cc = 0.0f;
  double d = 0.0;
  int pass = 0;
  if (slot) {
    // rows r, r + stride, ... in order; 8 loads in flight per thread (the flushes fall every kFlushPasses rows
    // as in a one-row loop, a multiple of 8)
    static_assert(kFlushPasses % 8 == 0, "flush cadence");
    const int64_t stride = (int64_t)gridDim.x * rpp;
    int64_t r = (int64_t)blockIdx.x * rpp + g;
    for (; r + 7 * stride < n; r += 8 * stride) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = R[(r + u * stride) * k + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const BT b = G::conv(v[u], sR);
        G::add(s, cc, b, b);
      }
      pass += 8;
      if (pass == kFlushPasses) {
        pass = 0;
        norm_flush<T>(d, s, cc, sR);
      }
    }
    for (; r < n; r += stride) {
      const BT b = G::conv(R[r * k + c], sR);
      G::add(s, cc, b, b);
      if (++pass == kFlushPasses) {
        pass = 0;
        norm_flush<T>(d, s, cc, sR);
      }
    }
  }
  norm_flush<T>(d, s, cc, sR);
  red[threadIdx.x] = slot ? d : 0.0;
  cta_sum_slots(red, k, rpp, partN + (int64_t)blockIdx.x * k);
}

}  // namespace bcgk
