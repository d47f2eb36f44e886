// Warp-chunk variants of the three streaming kernels (K1 op+Gram, K2 X/R update + Gram, K3 P update).
//
// Each warp owns chunks of 32*V block-vector elements (V = 16 bytes / element size: float4 or double2
// accesses) and works on them alone:
//   memory phase   lane l moves V consecutive elements of one row with 16-byte loads/stores (and, in K1,
//                  computes their BOP values with V-wide gathers) between HBM and a warp-private
//                  shared-memory tile;
//   compute phase  the same 32*V elements are processed in V sub-passes of 32, lane l always owning one
//                  column, so the block-product accumulators stay one column wide.
// Only __syncwarp orders the two phases, so warps never wait for each other inside the row loop. K1 and K2
// are register heavy; up to p = 16 they are compiled for at least 3 resident CTAs per SM, which measured
// faster than the 2 their unconstrained register counts allow. The
// layout needs V | k, and k | 32 or 32 | k (with k/32 dividing the 8 warps of a CTA), and every block of p
// columns inside one warp's 32 columns (p | 32); other shapes use the per-element kernels of bcg_kernels.cuh.
//
// Chunk geometry: k >= 32 -- a chunk is V rows x 32 columns of column group cg = warp % (k/32) (fixed per
// warp); sub-pass s is row R0 + s. k < 32 -- a chunk is 32*V/k whole rows; sub-pass s covers 32/k rows.
#pragma once

#include "bcg_kernels.cuh"

namespace bcgk {

constexpr int kWarps = kNT / 32;

template <typename T, int V>
struct VecOf;
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<double, 1> { using type = double; };
template <> struct VecOf<double, 2> { using type = double2; };

template <typename T, int V>
union VecU {
  typename VecOf<T, V>::type v;
  T e[V];
};

// One vector width per precision: 16-byte accesses (float4, double2).
template <typename T>
__host__ __device__ constexpr int wc_vec() { return 16 / (int)sizeof(T); }
// k | 32, or 32 | k with the k/32 column groups dividing the 8 warps of a CTA (so each warp keeps one column
// group); blocks of p columns must not straddle a warp; k must be a multiple of the vector width.
template <typename T>
__host__ __device__ constexpr bool wc_layout_ok(int k, int p) {
  return k >= 1 && k <= kNT && k % wc_vec<T>() == 0 &&
         ((32 % k == 0) || (k % 32 == 0 && kWarps % (k / 32) == 0 && 32 % p == 0));
}

struct WcGeom {
  int k, ng, gr, rc, cg, lane, warp;
  int64_t rb0, rbs, nrb;
  // compute-phase identity of this lane: column and row offset inside a sub-pass
  int col, ro;
  // memory-phase identity: sub-pass group and element offset within its 32 elements
  int sm, om;
  __device__ void init(int64_t n, int k_, int V) {
    k = k_;
    lane = threadIdx.x & 31;
    warp = threadIdx.x >> 5;
    ng = k >= 32 ? k / 32 : 1;
    gr = k >= 32 ? 1 : 32 / k;      // rows per sub-pass
    rc = V * gr;                    // rows per chunk
    const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
    cg = (int)(gw % ng);
    rb0 = gw / ng;
    rbs = (int64_t)gridDim.x * kWarps / ng;
    nrb = (n + rc - 1) / rc;
    col = k >= 32 ? cg * 32 + lane : lane % k;
    ro = k >= 32 ? 0 : lane / k;
    const int lpg = 32 / V;         // memory lanes per sub-pass group
    sm = lane / lpg;
    om = (lane % lpg) * V;
  }
  // memory-phase element: row and column of the first of this lane's V elements in chunk R0
  __device__ __forceinline__ void mem_pos(int64_t R0, int64_t &row, int &c) const {
    if (k >= 32) { row = R0 + sm; c = cg * 32 + om; }
    else { row = R0 + (int64_t)sm * gr + om / k; c = om % k; }
  }
};

// V columns of one row of BOP: (A X)_{r, c..c+V-1}
template <typename T, int OPK, int V>
__device__ __forceinline__ VecU<T, V> apply_row_vec(const OpDesc &A, const T *__restrict__ X, int64_t r, int k,
                                                   int c) {
  using VT = typename VecOf<T, V>::type;
  VecU<T, V> s;
#pragma unroll
  for (int v = 0; v < V; ++v) s.e[v] = T(0);
  const VT *__restrict__ Xv = reinterpret_cast<const VT *>(X);
  const int kv = k / V, cv = c / V;
  if constexpr (OPK == OP_CSR) {
    const T *__restrict__ vals = static_cast<const T *>(A.vals);
    const int64_t e0 = __ldg(A.rowptr + r), e1 = __ldg(A.rowptr + r + 1);
    for (int64_t e = e0; e < e1; e += 8) {
      int colj[8];
      T w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = e + u < e1;
        colj[u] = in ? __ldg(A.colind + e + u) : 0;
        w[u] = in ? __ldg(vals + e + u) : T(0);
      }
      VecU<T, V> xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (e + u < e1) xv[u].v = __ldg(Xv + (int64_t)colj[u] * kv + cv);
        else {
#pragma unroll
          for (int v = 0; v < V; ++v) xv[u].e[v] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < e1) {   // warp-uniform for the lanes of one row: no wasted FMAs on short rows
#pragma unroll
          for (int v = 0; v < V; ++v) s.e[v] = fma_t(w[u], xv[u].e[v], s.e[v]);
        }
    }
    return s;
  } else if constexpr (OPK == OP_SELL) {
    const T *__restrict__ vals = static_cast<const T *>(A.vals);
    const int64_t base = __ldg(A.rowptr + r / kSellC) + r % kSellC;
    const int len = __ldg(A.rowlen + r);
    for (int j = 0; j < len; j += 8) {
      int colj[8];
      T w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = j + u < len;
        const int64_t e = base + (int64_t)(j + u) * kSellC;
        colj[u] = in ? __ldg(A.colind + e) : 0;
        w[u] = in ? __ldg(vals + e) : T(0);
      }
      VecU<T, V> xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (j + u < len) xv[u].v = __ldg(Xv + (int64_t)colj[u] * kv + cv);
        else {
#pragma unroll
          for (int v = 0; v < V; ++v) xv[u].e[v] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j + u < len) {
#pragma unroll
          for (int v = 0; v < V; ++v) s.e[v] = fma_t(w[u], xv[u].e[v], s.e[v]);
        }
    }
    return s;
  } else {
    const int nx = A.nx, ny = A.ny, nz = (OPK == OP_ST5) ? 1 : A.nz;
    const int64_t pl = (int64_t)nx * ny;
    const int ix = (int)(r % nx), iy = (int)((r / nx) % ny), iz = (int)(r / pl);
    const int64_t o = r * kv + cv;
    VecU<T, V> t;
    auto add = [&](int64_t off, T w) {
      t.v = __ldg(Xv + off);
#pragma unroll
      for (int v = 0; v < V; ++v) s.e[v] = fma_t(w, t.e[v], s.e[v]);
    };
    if constexpr (OPK == OP_ST7VC) {
      const T *__restrict__ f = static_cast<const T *>(A.faces);
      const int64_t nfx = (int64_t)nz * ny * (nx + 1), nfy = (int64_t)nz * (ny + 1) * nx;
      const T *fx = f, *fy = f + nfx, *fz = f + nfx + nfy;
      const int64_t bx = ((int64_t)iz * ny + iy) * (nx + 1) + ix;
      const int64_t by = ((int64_t)iz * (ny + 1) + iy) * nx + ix;
      const int64_t bz = ((int64_t)iz * ny + iy) * nx + ix;
      const T wxm = __ldg(fx + bx), wxp = __ldg(fx + bx + 1);
      const T wym = __ldg(fy + by), wyp = __ldg(fy + by + nx);
      const T wzm = __ldg(fz + bz), wzp = __ldg(fz + bz + pl);
      add(o, ((wxm + wxp) + (wym + wyp)) + (wzm + wzp));
      if (ix > 0) add(o - kv, -wxm);
      if (ix < nx - 1) add(o + kv, -wxp);
      if (iy > 0) add(o - (int64_t)nx * kv, -wym);
      if (iy < ny - 1) add(o + (int64_t)nx * kv, -wyp);
      if (iz > 0) add(o - pl * kv, -wzm);
      if (iz < nz - 1) add(o + pl * kv, -wzp);
    } else {
      add(o, OPK == OP_ST5 ? T(4) : T(6));
      if (ix > 0) add(o - kv, T(-1));
      if (ix < nx - 1) add(o + kv, T(-1));
      if (iy > 0) add(o - (int64_t)nx * kv, T(-1));
      if (iy < ny - 1) add(o + (int64_t)nx * kv, T(-1));
      if constexpr (OPK == OP_ST7) {
        if (iz > 0) add(o - pl * kv, T(-1));
        if (iz < nz - 1) add(o + pl * kv, T(-1));
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) s.e[v] *= T(A.scale);
    return s;
  }
}

// CTA reduction of the per-thread FP64 slots red[t*p + a] into out[c*p + a], summing, in a fixed order,
// the threads whose compute column is c.
__device__ __forceinline__ void wc_cta_reduce(const double *red, int k, int p, double *__restrict__ out) {
  __syncthreads();
  const int ng = k >= 32 ? k / 32 : 1;
  const int E = k * p;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const int c = e / p, a = e - c * p;
    double v = 0.0;
    if (k >= 32) {
      const int lane = c & 31, cgc = c >> 5;
      for (int w = cgc; w < kWarps; w += ng) v += red[(w * 32 + lane) * p + a];
    } else {
      for (int w = 0; w < kWarps; ++w)
        for (int l = c; l < 32; l += k) v += red[(w * 32 + l) * p + a];
    }
    out[e] = v;
  }
  __syncthreads();
}

template <typename T>
__host__ __device__ constexpr size_t wc_tile_bytes(int V) { return (size_t)32 * V * sizeof(T); }
// Per-warp tiles: K1 3 broadcast tiles (P, Q, R as Dot2 operands); K2 4 T tiles (X, R, P, Q) + 1 broadcast
// tile; K3 3 T tiles. A broadcast element is a float for FP32 data and a float pair for FP64 data.
template <typename T>
__host__ __device__ constexpr size_t wc_bt_size() { return sizeof(T) == 4 ? 4 : 8; }
template <typename T>
__host__ __device__ constexpr size_t wc_op_warp_bytes(int V) { return (size_t)3 * 32 * V * wc_bt_size<T>(); }
template <typename T>
__host__ __device__ constexpr size_t wc_upd_warp_bytes(int V) {
  return (size_t)32 * V * (4 * sizeof(T) + wc_bt_size<T>());
}
template <typename T>
__host__ __device__ constexpr size_t wc_op_smem(int p, int V) {
  return (size_t)kWarps * wc_op_warp_bytes<T>(V) + 2 * (size_t)kNT * p * sizeof(double);
}
template <typename T>
__host__ __device__ constexpr size_t wc_upd_smem(int k, int p, int global, int V) {
  return align16((size_t)kWarps * wc_upd_warp_bytes<T>(V) + (size_t)(global ? 1 : k / p) * p * p * sizeof(T)) +
         (size_t)kNT * (p + 1) * sizeof(double);
}
// K3: 3 T tiles (P, Z, P_new) per warp, plus (RR) P_new and R as Dot2 operands and the FP64 slots of rho
template <typename T>
__host__ __device__ constexpr size_t wc_pup_warp_bytes(int V, bool rr) {
  return (size_t)32 * V * (3 * sizeof(T) + (rr ? 2 * wc_bt_size<T>() : 0));
}
template <typename T>
__host__ __device__ constexpr size_t wc_pup_smem(int k, int p, int global, int V, bool rr) {
  return align16((size_t)kWarps * wc_pup_warp_bytes<T>(V, rr) + (size_t)(global ? 1 : k / p) * p * p * sizeof(T)) +
         (rr ? (size_t)kNT * p * sizeof(double) : 0);
}

// ---------------------------------------------------------------------------------------------------
// K1 (warp-chunk): Q = A P, alpha = <<P, Q>>_S, and (RR) the recomputed rho = <<P, R>>_S; without RR the
// previous iteration's K3 has formed the recomputed rho and K1 does not read R.
// at least 3 CTAs per SM up to p = 16; p = 32 needs its registers (64 accumulator pairs per thread)
template <int PM>
constexpr int wc_min_ctas() { return PM <= 16 ? 3 : 1; }
// the FP32 CSR K1 up to p = 8 runs faster at 4 CTAs per SM despite a few spilled registers (0.73 -> 0.67 ms,
// 128^3, k = 32); the FP64 CSR K1 fits 4 CTAs without spills once the recomputed rho has moved to K3 (with it,
// 4 CTAs spilled and measured slower); the stencil instantiations stay at 3
template <typename T, int OPK, int PM, bool RR>
constexpr int wc_min_ctas_op() {
  return (OPK == OP_CSR && PM <= 8 && (sizeof(T) == 4 || !RR)) ? 4 : wc_min_ctas<PM>();
}

template <typename T, int OPK, int PM, int V, bool RR>
__global__ void __launch_bounds__(kNT, wc_min_ctas_op<T, OPK, PM, RR>()) kw_op_gram(OpDesc A, const T *__restrict__ P, const T *__restrict__ R,
                                                  T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                  const int *__restrict__ active, double *__restrict__ partA,
                                                  double *__restrict__ partR, const DevStatus *__restrict__ st,
                                                  const int *__restrict__ shP, const int *__restrict__ shQ,
                                                  const int *__restrict__ shR) {
  using G = Gram<T>;
  using BT = typename G::B;
  using VT = typename VecOf<T, V>::type;
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  WcGeom geo;
  geo.init(n, k, V);
  static_assert(sizeof(BT) == wc_bt_size<T>(), "broadcast tile element");
  // the memory-phase columns of a lane are the same in every chunk: their exponent shifts stay in registers
  int mshP[V], mshQ[V], mshR[V];
  {
    int64_t row0;
    int mc0;
    geo.mem_pos(0, row0, mc0);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      mshP[v] = G::kShifted ? shift_at(shP, mc0 + v) : 0;
      mshQ[v] = G::kShifted ? shift_at(shQ, mc0 + v) : 0;
      mshR[v] = (G::kShifted && RR) ? shift_at(shR, mc0 + v) : 0;
    }
  }
  BT *tile = reinterpret_cast<BT *>(smem + (size_t)geo.warp * wc_op_warp_bytes<T>(V));
  BT *sP = tile, *sQ = tile + 32 * V, *sR = tile + 64 * V;
  double *redA = reinterpret_cast<double *>(smem + (size_t)kWarps * wc_op_warp_bytes<T>(V));
  double *redR = redA + kNT * p;
  const int c = geo.col, j = c / p, b = c - j * p;
  const bool act = block_active(active, global, j);
  double *slotA = redA + threadIdx.x * p, *slotR = redR + threadIdx.x * p;
  for (int a = 0; a < p; ++a) { slotA[a] = 0.0; if (RR) slotR[a] = 0.0; }
  // alpha is symmetric: lane b accumulates only its circulant diagonals d = 0..p/2, entry ((b + d) mod p, b)
  // (d = p/2 only for b < p/2); the recomputed rho stays a full product. p == PM here (p divides 32).
  constexpr int PMH = PM == 1 ? 1 : PM / 2 + 1;
  // flush scales: accumulator d of alpha holds entry ((b + d) mod p, b); accR entry a holds (a, b)
  auto sxA = [&](int d) { return shift_at(shP, j * p + ((b + d) & (PM - 1))); };
  auto sxR = [&](int a) { return shift_at(shP, j * p + a); };
  const int syQ = G::kShifted ? shift_at(shQ, c) : 0;
  const int syR = (G::kShifted && RR) ? shift_at(shR, c) : 0;
  GramAcc<PMH> accA;
  GramAcc<RR ? PM : 1> accR;
  accA.zero();
  accR.zero();
  int pass = 0;
  const int kv = k / V;
  for (int64_t rb = geo.rb0; rb < geo.nrb; rb += geo.rbs) {
    const int64_t R0 = rb * geo.rc;
    int64_t row;
    int mc;
    geo.mem_pos(R0, row, mc);
    VecU<T, V> pv, rv, qv;
    if (row < n) {
      const int64_t o = row * kv + mc / V;
      pv.v = reinterpret_cast<const VT *>(P)[o];
      if constexpr (RR) rv.v = reinterpret_cast<const VT *>(R)[o];
      qv = apply_row_vec<T, OPK, V>(A, P, row, k, mc);
      reinterpret_cast<VT *>(Q)[o] = qv.v;
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) pv.e[v] = rv.e[v] = qv.e[v] = T(0);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = 32 * geo.sm + geo.om + v;
      sP[t] = G::conv(pv.e[v], mshP[v]);
      sQ[t] = G::conv(qv.e[v], mshQ[v]);
      if constexpr (RR) sR[t] = G::conv(rv.e[v], mshR[v]);
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int s = 0; s < V; ++s) {
        const int t = 32 * s + geo.lane;
        const BT qb = sQ[t];
        const BT *rowp = sP + t - b;
        if constexpr (RR) {
          const BT rb2 = sR[t];
          BT prow[PM];
          load_row<BT, PM>(rowp, prow, p);
#pragma unroll
          for (int a = 0; a < PM; ++a) G::add(accR.s[a], accR.c[a], prow[a], rb2);
        }
#pragma unroll
        for (int d = 0; d < PMH; ++d)
          if (PM == 1 || d < PM / 2 || b < PM / 2) G::add(accA.s[d], accA.c[d], rowp[(b + d) & (PM - 1)], qb);
      }
    }
    __syncwarp();
    if (++pass == kFlushPasses / V) {
      pass = 0;
      gram_flush<T>(accA, slotA, PMH, sxA, syQ);
      if constexpr (RR) gram_flush<T>(accR, slotR, p, sxR, syR);
    }
  }
  gram_flush<T>(accA, slotA, PMH, sxA, syQ);
  if constexpr (RR) gram_flush<T>(accR, slotR, p, sxR, syR);
  const int E = k * p;
  wc_cta_reduce(redA, k, p, partA + (int64_t)blockIdx.x * E);
  if constexpr (RR) wc_cta_reduce(redR, k, p, partR + (int64_t)blockIdx.x * E);
}

// ---------------------------------------------------------------------------------------------------
// K2 (warp-chunk): X += P lambda, R -= Q lambda, rho = <<Z, R>>_S, column norms (ZS: Z = M^{-1} R).
// K2 keeps fewer live values than K1: its unpreconditioned FP32 instantiations up to p = 8 fit 64 registers
// (4 CTAs per SM); the FP64 one at p = 16 runs better at 2 CTAs without spills than at 3 with them
// (3.61 / 3.71 ms, 128^3, k = 32)
// The double-float instantiations are bound by instruction issue, not by the FP64 pipe: 2 CTAs per SM without
// spills rather than 3 with them.
template <typename T, int PM, bool ZS, bool DF = false>
constexpr int wc_min_ctas_upd() {
  return DF ? 2 : (sizeof(T) == 4 && PM <= 8 && !ZS) ? 4 : ((sizeof(T) == 8 && PM == 16) ? 2 : wc_min_ctas<PM>());
}

// DF (FP64, p >= 2): the two BAXPYs split between the two pipes. X += P lambda keeps its p FP64 FMAs, and
// R -= Q lambda is summed in double-float arithmetic (bcg_kernels.cuh) on the FP32 pipes and added to R with one
// FP64 addition, so that the narrow FP64 pipe carries p + 1 operations per element instead of 2 p. The Q tile
// then holds float pairs of Q scaled by its columns' Q-role shifts (shQr), and lambda's column is normalised into
// float pairs once per thread.
template <typename T, int PM, int V, bool ZS, bool DF = false>
__global__ void __launch_bounds__(kNT, wc_min_ctas_upd<T, PM, ZS, DF>()) kw_update_xr(T *__restrict__ X, T *__restrict__ R, const T *__restrict__ P,
                                                    const T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                    const double *__restrict__ lam, const int *__restrict__ active,
                                                    double *__restrict__ partRho, double *__restrict__ partN,
                                                    const DevStatus *__restrict__ st, const T *__restrict__ dinv,
                                                    const int *__restrict__ shZ, const int *__restrict__ shR,
                                                    const int *__restrict__ shQr) {
  static_assert(!DF || sizeof(T) == 8, "double-float updates replace FP64 arithmetic");
  using G = Gram<T>;
  using BT = typename G::B;
  using VT = typename VecOf<T, V>::type;
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  WcGeom geo;
  geo.init(n, k, V);
  static_assert(sizeof(BT) == wc_bt_size<T>(), "broadcast tile element");
  unsigned char *wbase = smem + (size_t)geo.warp * wc_upd_warp_bytes<T>(V);
  T *sX = reinterpret_cast<T *>(wbase);
  T *sR = sX + 32 * V, *sP = sR + 32 * V, *sQ = sP + 32 * V;
  BT *sRb = reinterpret_cast<BT *>(wbase + 4 * 32 * V * sizeof(T));
  const int nblk = global ? 1 : k / p;
  T *sL = reinterpret_cast<T *>(smem + (size_t)kWarps * wc_upd_warp_bytes<T>(V));
  double *red = reinterpret_cast<double *>(smem + align16((size_t)kWarps * wc_upd_warp_bytes<T>(V) +
                                                          (size_t)nblk * p * p * sizeof(T)));
  double *nred = red + kNT * p;
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sL[e] = (T)lam[e];
  const int c = geo.col, j = c / p, b = c - j * p;
  const bool act = block_active(active, global, j);
  double *slotRho = red + threadIdx.x * p;
  double *slotN = nred + threadIdx.x;
  for (int a = 0; a < p; ++a) slotRho[a] = 0.0;
  *slotN = 0.0;
  __syncthreads();
  constexpr int PMH = PM == 1 ? 1 : PM / 2 + 1;   // rho = R^T R is symmetric: circulant diagonals only
  // compute-phase shifts: this lane's column for R, and the broadcast Z columns at flush time
  // without a preconditioner Z = R, and the P role's shift equals the R role's
  const int cshR = G::kShifted ? shift_at(shR, c) : 0;
  const int cshZ = (G::kShifted && ZS) ? shift_at(shZ, c) : cshR;
  auto sxZ = [&](int d) { return shift_at(shZ, j * p + ((b + d) & (PM - 1))); };
  T lcol[PM];
  const T *lj = sL + (global ? 0 : j) * p * p + b;
#pragma unroll
  for (int a = 0; a < PM; ++a) lcol[a] = a < p ? lj[a * p] : T(0);
  // DF at p = 16: the FP64 column of lambda is re-read from shared memory (conflict-free: the lanes read
  // consecutive entries of one row) so that it and the float-pair column fit the 128 registers of 2 CTAs per SM
  constexpr bool kLamSmem = DF && PM > 8;
  // DF: lambda's column as float pairs for Q's shifts, the Q shifts of this lane's memory-phase columns (tile
  // writes) and the output exponent of its compute-phase column (R -= 2^tr (s + c))
  float2 lpair[DF ? PM : 1];
  int dfSQm[DF ? V : 1], dfTr = 0;
  if constexpr (DF) {
    int64_t row0;
    int mc0;
    geo.mem_pos(0, row0, mc0);
#pragma unroll
    for (int v = 0; v < V; ++v) dfSQm[v] = shift_at(shQr, mc0 + v);
    dfTr = df_matrix_col<PM>(lcol, p, shQr, j, lpair, 0);
  }
  float2 *sQf = reinterpret_cast<float2 *>(sQ);
  GramAcc<PMH> acc;
  acc.zero();
  float ns = 0.0f, nc = 0.0f;
  int pass = 0;
  const int kv = k / V;
  for (int64_t rb = geo.rb0; rb < geo.nrb; rb += geo.rbs) {
    const int64_t R0 = rb * geo.rc;
    int64_t row;
    int mc;
    geo.mem_pos(R0, row, mc);
    const int64_t o = row * kv + mc / V;
    VecU<T, V> xv, rv, pv, qv;
    if (row < n) {
      xv.v = reinterpret_cast<const VT *>(X)[o];
      rv.v = reinterpret_cast<const VT *>(R)[o];
      pv.v = reinterpret_cast<const VT *>(P)[o];
      qv.v = reinterpret_cast<const VT *>(Q)[o];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) xv.e[v] = rv.e[v] = pv.e[v] = qv.e[v] = T(0);
    }
    const int tm = 32 * geo.sm + geo.om;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sX[tm + v] = xv.e[v];
      sR[tm + v] = rv.e[v];
      sP[tm + v] = pv.e[v];
      if constexpr (DF) sQf[tm + v] = split_f64_ftz(qv.e[v], dfSQm[v]);
      else sQ[tm + v] = qv.e[v];
    }
    __syncwarp();
    // BAXPY x 2 for each sub-pass; the new residual is written as its broadcast representation
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int t = 32 * s + geo.lane;
      T x = sX[t], r = sR[t];
      if constexpr (DF) {
        if (act) {
          constexpr int C = PM > 8 ? 8 : PM;   // rows read in chunks of 8 terms (register pressure at p = 16)
          float rs = 0.0f, rc = 0.0f;
#pragma unroll
          for (int h = 0; h < PM; h += C) {
            T prow[C];
            float2 qrow[C];
            load_row<T, C>(sP + t - b + h, prow, min(p - h, C));
            load_row<float2, C>(sQf + t - b + h, qrow, min(p - h, C));
#pragma unroll
            for (int a = 0; a < C; ++a)
              if (h + a < p) {
                x = fma_t(prow[a], kLamSmem ? lj[(h + a) * p] : lcol[h + a], x);
                Gram<double>::add(rs, rc, qrow[a], lpair[h + a]);
              }
          }
          r = r - df_pair_to_double(rs, rc, dfTr);
        }
      } else if (act) {
        T prow[PM], qrow[PM];
        load_row<T, PM>(sP + t - b, prow, p);
        load_row<T, PM>(sQ + t - b, qrow, p);
#pragma unroll
        for (int a = 0; a < PM; ++a)
          if (a < p) {
            x = fma_t(prow[a], lcol[a], x);
            r = fma_t(-qrow[a], lcol[a], r);
          }
      }
      sX[t] = x;
      sR[t] = r;
      // broadcast Z = M^{-1} R (R without a preconditioner); the own operand R is re-read from sR below
      if constexpr (ZS) {
        const int64_t rw = R0 + (int64_t)s * geo.gr + geo.ro;
        sRb[t] = G::conv(rw < n ? r * dinv[rw] : T(0), cshZ);
      } else {
        sRb[t] = G::conv(r, cshZ);
      }
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int s = 0; s < V; ++s) {
        const int t = 32 * s + geo.lane;
        const BT rb2 = ZS ? G::conv(sR[t], cshR) : sRb[t];   // own operand: R
        const BT *rowr = sRb + t - b;                      // broadcast: Z
#pragma unroll
        for (int d = 0; d < PMH; ++d)
          if (PM == 1 || d < PM / 2 || b < PM / 2) G::add(acc.s[d], acc.c[d], rowr[(b + d) & (PM - 1)], rb2);
        G::add(ns, nc, rb2, rb2);   // ||R_c||^2 for the stopping test
      }
    }
    if (row < n) {
      VecU<T, V> xo, ro2;
#pragma unroll
      for (int v = 0; v < V; ++v) { xo.e[v] = sX[tm + v]; ro2.e[v] = sR[tm + v]; }
      reinterpret_cast<VT *>(X)[o] = xo.v;
      reinterpret_cast<VT *>(R)[o] = ro2.v;
    }
    __syncwarp();
    if (++pass == kFlushPasses / V) {
      pass = 0;
      gram_flush<T>(acc, slotRho, PMH, sxZ, cshR);
      norm_flush<T>(*slotN, ns, nc, cshR);
    }
  }
  gram_flush<T>(acc, slotRho, PMH, sxZ, cshR);
  norm_flush<T>(*slotN, ns, nc, cshR);
  const int E = k * p;
  wc_cta_reduce(red, k, p, partRho + (int64_t)blockIdx.x * E);
  wc_cta_reduce(nred, k, 1, partN + (int64_t)blockIdx.x * k);
}

// ---------------------------------------------------------------------------------------------------
// K3 (warp-chunk): P = Z + P beta (ZS: Z = M^{-1} R, else Z = R).
// RR: also the recomputed rho of the next iteration, <<P_new, R>>_S (Algorithm 1 recomputes
// rho^{i-1} = <<P^i, R^{i-1}>>_S; both operands are in this kernel's registers, and its FP32 pipes are idle
// while it waits on the FP64 pipe or on HBM). Partials as in K1, entry (a, b) of block j at j*p*p + b*p + a.
template <typename T, int PM, int V, bool ZS, bool RR>
__global__ void __launch_bounds__(kNT) kw_update_p(T *__restrict__ P, const T *__restrict__ R, int64_t n, int k,
                                                   int p, int global, const double *__restrict__ beta,
                                                   const int *__restrict__ active, DevStatus *__restrict__ st,
                                                   const T *__restrict__ dinv, double *__restrict__ partR,
                                                   const int *__restrict__ shP, const int *__restrict__ shR) {
  using G = Gram<T>;
  using BT = typename G::B;
  using VT = typename VecOf<T, V>::type;
  if (st->flags != 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->cur += 1;   // no other kernel of this launch reads it
  extern __shared__ __align__(16) unsigned char smem[];
  WcGeom geo;
  geo.init(n, k, V);
  unsigned char *wbase = smem + (size_t)geo.warp * wc_pup_warp_bytes<T>(V, RR);
  T *sP = reinterpret_cast<T *>(wbase);
  T *sR = sP + 32 * V, *sN = sR + 32 * V;
  BT *sNb = reinterpret_cast<BT *>(sN + 32 * V);   // RR: P_new (broadcast) and R (own) as Dot2 operands
  BT *sRb = sNb + 32 * V;
  const int nblk = global ? 1 : k / p;
  T *sB = reinterpret_cast<T *>(smem + (size_t)kWarps * wc_pup_warp_bytes<T>(V, RR));
  double *red = reinterpret_cast<double *>(smem + align16((size_t)kWarps * wc_pup_warp_bytes<T>(V, RR) +
                                                          (size_t)nblk * p * p * sizeof(T)));
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sB[e] = (T)beta[e];
  const int c = geo.col, j = c / p, b = c - j * p;
  const bool act = block_active(active, global, j);
  double *slotR = red + threadIdx.x * p;
  if constexpr (RR)
    for (int a = 0; a < p; ++a) slotR[a] = 0.0;
  __syncthreads();
  T bcol[PM];
  {
    const T *bj = sB + (global ? 0 : j) * p * p + b;
#pragma unroll
    for (int a = 0; a < PM; ++a) bcol[a] = a < p ? bj[a * p] : T(0);
  }
  GramAcc<RR ? PM : 1> acc;
  acc.zero();
  // RR shifts: P_new and R in the compute phase (this lane's column); with the Jacobi scaling R is converted in
  // the memory phase (the tile then holds Z), by the shift table s_shR
  __shared__ int s_shR[kNT];
  if (G::kShifted && RR && ZS) {
    for (int cc = threadIdx.x; cc < k; cc += blockDim.x) s_shR[cc] = shift_at(shR, cc);
    __syncthreads();
  }
  const int sPn = (G::kShifted && RR) ? shift_at(shP, c) : 0;
  const int syR = (G::kShifted && RR) ? shift_at(shR, c) : 0;
  auto sxP = [&](int a) { return shift_at(shP, j * p + a); };
  int pass = 0;
  const int kv = k / V;
  for (int64_t rb = geo.rb0; rb < geo.nrb; rb += geo.rbs) {
    const int64_t R0 = rb * geo.rc;
    int64_t row;
    int mc;
    geo.mem_pos(R0, row, mc);
    const int64_t o = row * kv + mc / V;
    VecU<T, V> pv, rv, zv;
    if (row < n) {
      pv.v = reinterpret_cast<const VT *>(P)[o];
      rv.v = reinterpret_cast<const VT *>(R)[o];
      zv = rv;
      if constexpr (ZS) {   // Z = M^{-1} R
        const T di = dinv[row];
#pragma unroll
        for (int v = 0; v < V; ++v) zv.e[v] *= di;
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) pv.e[v] = rv.e[v] = zv.e[v] = T(0);
    }
    const int tm = 32 * geo.sm + geo.om;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sP[tm + v] = pv.e[v];
      sR[tm + v] = zv.e[v];
      if constexpr (RR && ZS) sRb[tm + v] = G::conv(rv.e[v], G::kShifted ? s_shR[mc + v] : 0);
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int t = 32 * s + geo.lane;
      T out = sP[t];
      if (act) {
        T prow[PM];
        load_row<T, PM>(sP + t - b, prow, p);
        out = sR[t];
#pragma unroll
        for (int a = 0; a < PM; ++a)
          if (a < p) out = fma_t(prow[a], bcol[a], out);
      }
      sN[t] = out;
      if constexpr (RR) sNb[t] = G::conv(out, sPn);
    }
    __syncwarp();
    if constexpr (RR) {
      if (act) {
#pragma unroll
        for (int s = 0; s < V; ++s) {
          const int t = 32 * s + geo.lane;
          BT nrow[PM];
          load_row<BT, PM>(sNb + t - b, nrow, p);
          const BT rb2 = ZS ? sRb[t] : G::conv(sR[t], syR);   // own operand R (the tile holds Z = R)
#pragma unroll
          for (int a = 0; a < PM; ++a)
            if (a < p) G::add(acc.s[a], acc.c[a], nrow[a], rb2);
        }
      }
      if (++pass == kFlushPasses / V) {
        pass = 0;
        gram_flush<T>(acc, slotR, p, sxP, syR);
      }
    }
    if (row < n) {
      VecU<T, V> po;
#pragma unroll
      for (int v = 0; v < V; ++v) po.e[v] = sN[tm + v];
      reinterpret_cast<VT *>(P)[o] = po.v;
    }
    __syncwarp();
  }
  if constexpr (RR) {
    gram_flush<T>(acc, slotR, p, sxP, syR);
    wc_cta_reduce(red, k, p, partR + (int64_t)blockIdx.x * k * p);
  }
}

}  // namespace bcgk
