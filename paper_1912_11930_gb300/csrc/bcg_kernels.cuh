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
#include <cstring>
#include <cuda_runtime.h>

namespace bcgk {

enum OpKind { OP_CSR = 0, OP_ST5 = 1, OP_ST7 = 2, OP_ST7VC = 3, OP_SELL = 4 };

// SELL-C-sigma (Kreutzer et al., SIAM J. Sci. Comput. 36(5), 2014, the format Section 4 suggests for BOP):
// rows in chunks of kSellC; entry j of row r is stored at rowptr[r / kSellC] + j * kSellC + r % kSellC
// (column-major inside a chunk, so lanes holding consecutive rows read consecutive words); rowlen[r] entries
// per row, the chunk padded to its longest row. The sigma-sorting of rows is a permutation applied outside
// the operator (the handle iterates on the permuted system).
constexpr int kSellC = 32;

// Device status word shared by all kernels of one solve.
struct DevStatus {
  int flags;           // ST_* bits; any nonzero value makes every later kernel of the solve a no-op
  int iter;            // highest iteration whose convergence test ran
  int breakdown_iter;  // iteration of the first breakdown (0 if none)
  int n_active;        // distinct blocks still iterating
  int cur;             // number of the iteration in progress (1-based), advanced by K3
};
// ST_TIMEOUT: a bounded device-side wait (the tensor-core kernels' completion barriers) gave up
enum { ST_DONE = 1, ST_BREAKDOWN = 2, ST_NUMERIC = 4, ST_TIMEOUT = 8 };

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
  const int32_t *rowlen;   // SELL: entries per row (rowptr then holds the chunk offsets)
};

constexpr int kNT = 256;   // threads per CTA of the streaming kernels (k <= 256)

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
// dynamic shared memory layouts (bytes), shared by kernels and launchers
// Rows per thread per pass: every load of a pass is issued before its arithmetic, so RPT rows' worth of
// memory requests are in flight per thread (the row loops are otherwise latency-bound on GB300).
// (measured on GB300: FP64 kernels are bound by the FP64 pipe and lose occupancy with RPT > 1; the FP32
// updates gain a little from RPT = 4; K1 is register heavy and keeps RPT = 1)
template <typename T>
__host__ __device__ constexpr int rpt_stream() { return sizeof(T) == 4 ? 4 : 1; }   // K2, K3
template <typename T>
__host__ __device__ constexpr int rpt_op() { return 1; }                              // K1

// K1: broadcast tile (RPT rows per slot) + FP64 slot sums of alpha and of the recomputed rho
__host__ __device__ constexpr size_t op_gram_smem(int p, int rpt) {
  return (size_t)rpt * kNT * sizeof(double) + 2 * (size_t)kNT * p * sizeof(double);
}
__host__ __device__ constexpr size_t bdot_smem(int p) { return kNT * sizeof(double) + (size_t)kNT * p * sizeof(double); }
__host__ __device__ constexpr size_t update_xr_red_offset(int k, int p, int global, size_t tsize, int rpt) {
  return align16((2 * (size_t)rpt * kNT + (size_t)(global ? 1 : k / p) * p * p) * tsize);
}
// K2: P, Q tiles, lambda, then FP64 slot sums of rho and of the column norms
__host__ __device__ constexpr size_t update_xr_smem(int k, int p, int global, size_t tsize, int rpt) {
  return update_xr_red_offset(k, p, global, tsize, rpt) + (size_t)kNT * (p + 1) * sizeof(double);
}
__host__ __device__ constexpr size_t update_p_smem(int k, int p, int global, size_t tsize, int rpt) {
  return ((size_t)rpt * kNT + (size_t)(global ? 1 : k / p) * p * p) * tsize;
}
__host__ __device__ constexpr size_t residual_smem() { return kNT * sizeof(double); }

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// ---- Gram accumulation off the FP64 pipe ----------------------------------------------------------------
// GB300 executes FP64 at 1/61 of its FP32 rate, so block-product entries are accumulated as unevaluated float
// pairs (s, c) with error-free transformations -- TwoProd by FMA and TwoSum, i.e. algorithm Dot2 of Ogita, Rump
// & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005 -- and added into per-thread FP64
// sums in shared memory every kFlushPasses rows (which bounds the pair's own error growth). FP64 inputs are
// first split into hi + lo floats (48 significant bits) with integer operations only. The per-CTA and grid
// reductions stay in FP64.
constexpr int kFlushPasses = 128;

__device__ __forceinline__ void two_sum_acc(float &s, float &c, float p, float e) {
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // s + p = t + err exactly
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// ---- Exponent shifts of FP64 Gram operands ----------------------------------------------------------------
// The float pairs cover FP32's exponent range only, while the block products of the method are defined on FP64
// values (Section 2). So every FP64 operand column c is scaled by an exact power of two 2^-s_c before it is
// split, and each flushed partial sum of entry (a, b) is scaled back by 2^(s_a + s_b) in FP64. Scaling by a power
// of two commutes with rounding, so for values whose scaled products stay inside FP32's range the sums are
// bitwise those of the unshifted arithmetic; the shift only moves the window.
//
// Shifts are chosen from FP64 column norms the solver already holds (the latest ||R_c||^2 of every column), so
// that a scaled column has 2-norm about 2^kGramCenter. An operand of another scale than R adds a uniform offset
// (M^{-1} R: the exponent of max|diag(A)^{-1}|; A P: that of A's largest absolute row sum besides). A shift array
// holds one int per column (NULL: no shift). Without flushes in between, a scaled product loses accuracy below
// about 2^-102 (error terms turn subnormal) and overflows at 2^121 (128 rows summed): with a column norm of 2^10
// that leaves a factor of about 2^49 of shrinking and 2^50 of growth of a column between two norm updates.
constexpr int kGramCenter = 10;
constexpr int kGramShiftMax = 1000;

__host__ __device__ __forceinline__ int clamp_shift(int s) {
  return s < -kGramShiftMax ? -kGramShiftMax : (s > kGramShiftMax ? kGramShiftMax : s);
}
// floor(log2(sqrt(v))) - kGramCenter for a squared norm v (zero or subnormal v: the smallest normal exponent;
// non-finite v: no shift)
__host__ __device__ __forceinline__ int shift_from_norm2(double v) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long u;
  memcpy(&u, &v, sizeof u);
#endif
  int e = (int)((u >> 52) & 0x7FF);
  if (e == 0x7FF) return 0;
  if (e == 0) e = 1;
  return ((e - 1023) >> 1) - kGramCenter;
}
// floor(log2 v) for a finite v > 0 (normal), else 0: the uniform offset taken from one of the operator maxima
__host__ __device__ __forceinline__ int exponent_of(double v) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long u;
  memcpy(&u, &v, sizeof u);
#endif
  const int e = (int)((u >> 52) & 0x7FF);
  return (e == 0 || e == 0x7FF || (u >> 63)) ? 0 : e - 1023;
}

// Where a solve's shift array lives and how its three rows are offset (see the roles in bcg_launch.h).
struct ShiftCtl {
  int *sh = nullptr;                  // 3 k ints, rewritten with the column norms (NULL: no shifts)
  const double *opmax = nullptr;      // [max row sum of |A|, max |diag(A)^{-1}|] (NULL: no offsets)
  int precond = 0;                    // 1: directions are M^{-1} R (Jacobi), offset by the second maximum
};
// Shifts of column c (of k) from its squared norm n2.
__device__ __forceinline__ void write_shifts(const ShiftCtl &sc, int k, int c, double n2) {
  if (sc.sh == nullptr) return;
  const int base = shift_from_norm2(n2);
  const int dA = sc.opmax ? exponent_of(sc.opmax[0]) : 0;
  const int dP = (sc.opmax && sc.precond) ? exponent_of(sc.opmax[1]) : 0;
  sc.sh[c] = clamp_shift(base);
  sc.sh[k + c] = clamp_shift(base + dP);
  sc.sh[2 * k + c] = clamp_shift(base + dP + dA);
}

// 2^e for |e| <= kGramShiftMax
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ __forceinline__ int shift_at(const int *__restrict__ sh, int c) { return sh ? __ldg(sh + c) : 0; }

// Tiny, huge or non-finite values (after the shift): plain conversions of x 2^-sh. Kept out of line so that the
// compiler cannot if-convert this branch into every call (its FP64 instructions would then run for every
// element on the narrow pipe).
static __device__ __noinline__ float2 split_f64_rare(double x, int sh) {
  if (!isfinite(x)) return make_float2((float)x, 0.0f);
  const double xs = ldexp(x, -sh);
  const float hi = (float)xs;
  return make_float2(hi, isfinite(hi) ? (float)(xs - (double)hi) : 0.0f);
}

// x 2^-sh = hi + lo with hi = x truncated to 24 significant bits and lo = the remaining 29 bits truncated to
// 24. Both halves are assembled from the bit pattern with integer operations only (no FP64 or conversion
// instruction: on GB300 those share the narrow FP64 pipe) whenever x is a normal double and both halves are
// normal floats.
__device__ __forceinline__ float2 split_f64(double x, int sh) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32);
  const int ef = (int)((hi32 >> 20) & 0x7FFu);
  const int e = ef - sh;   // biased exponent of x 2^-sh
  if ((unsigned)(ef - 1) < 0x7FEu && (unsigned)(e - 949) <= 201u) {
    const unsigned sign = hi32 & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
    // low part: rem * 2^(e - 1075) with rem < 2^29; normalise rem by its leading one
    const unsigned rem = (unsigned)(u & 0x1FFFFFFFu);
    const int msb = 31 - __clz(rem);                       // 0..28 (meaningless if rem == 0)
    const unsigned mant = msb >= 23 ? rem >> (msb - 23) : rem << (23 - msb);
    const unsigned lob = sign | ((unsigned)(msb + e - 948) << 23) | (mant & 0x7FFFFFu);
    return make_float2(hi, rem ? __uint_as_float(lob) : 0.0f);
  }
  if ((u << 1) == 0ull) return make_float2(__uint_as_float(hi32 & 0x80000000u), 0.0f);   // +-0
  return split_f64_rare(x, sh);
}

template <typename T>
struct Gram;
template <>
struct Gram<float> {
  using B = float;   // broadcast / operand representation
  static constexpr bool kShifted = false;   // FP32 operands are accumulated as they are
  __device__ static B conv(float v) { return v; }
  __device__ static B conv(float v, int) { return v; }
  __device__ static B zero() { return 0.0f; }
  __device__ static void add(float &s, float &c, B x, B y) {
    const float p = __fmul_rn(x, y);
    two_sum_acc(s, c, p, __fmaf_rn(x, y, -p));   // x*y = p + e exactly
  }
};
template <>
struct Gram<double> {
  using B = float2;
  static constexpr bool kShifted = true;
  __device__ static B conv(double v) { return split_f64(v, 0); }
  __device__ static B conv(double v, int sh) { return split_f64(v, sh); }
  __device__ static B zero() { return make_float2(0.0f, 0.0f); }
  __device__ static void add(float &s, float &c, B x, B y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);   // exact error of hi*hi
    e = __fmaf_rn(x.x, y.y, e);          // cross terms, relative weight 2^-24
    e = __fmaf_rn(x.y, y.x, e);
    two_sum_acc(s, c, p, e);
  }
};

// ---- Double-float block updates (precision BCG_FP64_DF) ----------------------------------------------------
// A block update out_b = base_b + sum_a y_a l_ab (BAXPY) with part of the p products off the FP64 pipe: for those
// terms y_a and l_ab are split into 48-bit float pairs (after exact power-of-two shifts that put them inside FP32's
// range), the products are accumulated as one float pair (s, c) exactly as the Gram entries are (TwoProd of the
// high parts, the two cross terms, TwoSum), and s 2^t and c 2^t are added to the FP64 value with two FP64
// additions. The error of that part of the increment is about 2^-46 sum_a |y_a l_ab| (FP64 FMAs: about p 2^-53
// of it). The other terms keep their FP64 FMAs, so that both pipes carry a share of the products.

// x 2^-sh as a float pair, branch-free: a normal x whose scaled value lies in [2^-74, 2^128) gives the split of
// split_f64; a scaled value below 2^-74, zero or subnormal gives (0, 0); above the range or non-finite, (+-inf, 0).
// The update operands are scaled by their columns' shifts (about 2^10 times the column norm), so only entries
// more than 2^84 below their column's norm are flushed: far below FP64's own norm-wise update error.
__device__ __forceinline__ float2 split_f64_ftz(double x, int sh) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32);
  const int ef = (int)((hi32 >> 20) & 0x7FFu);
  const int e = ef - sh;
  const unsigned sign = hi32 & 0x80000000u;
  const bool ok = (unsigned)(ef - 1) < 0x7FEu && (unsigned)(e - 949) <= 201u;
  const bool big = ef == 0x7FF || (ef != 0 && e > 1150);
  const unsigned hib = sign | ((unsigned)(e - 896) << 23) | (unsigned)((u >> 29) & 0x7FFFFFu);
  const unsigned rem = (unsigned)(u & 0x1FFFFFFFu);
  const int msb = 31 - __clz(rem);
  const unsigned mant = msb >= 23 ? rem >> (msb - 23) : rem << (23 - msb);
  const unsigned lob = sign | ((unsigned)(msb + e - 948) << 23) | (mant & 0x7FFFFFu);
  const float hi = ok ? __uint_as_float(hib) : (big ? __uint_as_float(sign | 0x7F800000u) : 0.0f);
  return make_float2(hi, (ok && rem != 0u) ? __uint_as_float(lob) : 0.0f);
}

// v 2^t as a double, built from the bit pattern with integer operations and selects only (no conversion
// instruction, which would occupy the FP64 pipe): a non-finite v stays non-finite, an overflow gives +-inf, and
// a zero or subnormal v, or an underflow, gives 0 (the pair being converted is an accumulator of products of
// magnitude 2^-102 and more, so a subnormal part carries nothing).
__device__ __forceinline__ double f2d_scaled(float v, int t) {
  const unsigned u = __float_as_uint(v);
  const int ex = (int)((u >> 23) & 0xFFu);
  int eb = ex + 896 + t;   // biased FP64 exponent of v 2^t
  eb = ex == 0xFF ? 0x7FF : min(eb, 0x7FF);
  const unsigned man = (eb == 0x7FF && ex != 0xFF) ? 0u : (u & 0x7FFFFFu);
  const unsigned hi = (u & 0x80000000u) | ((unsigned)max(eb, 0) << 20) | (man >> 3);
  return (ex == 0 || eb <= 0) ? 0.0 : __hiloint2double((int)hi, (int)(man << 29));
}

// (s + c) 2^t as one double, from the bit patterns of the two floats with integer operations only (so that the
// update needs one FP64 addition, not two): both mantissas are aligned at the larger exponent in a 64-bit fixed-
// point sum, which is normalised and truncated to 53 bits. Bits of the smaller part more than 62 places below the
// larger one's leading bit are dropped, so the result is within 2^-52 of (s + c) 2^t relative to max(|s|, |c|).
// A zero or subnormal part counts as zero (as in f2d_scaled), a non-finite part gives a non-finite result, an
// overflow gives +-inf and an underflow 0.
__device__ __forceinline__ double df_pair_to_double(float s, float c, int t) {
  const unsigned us = __float_as_uint(s), uc = __float_as_uint(c);
  const int es = (int)((us >> 23) & 0xFFu), ec = (int)((uc >> 23) & 0xFFu);
  const int e = max(es, ec);
  // mantissas with their hidden bit at bit 61 (each < 2^62, so the signed sum stays below 2^63)
  const unsigned long long ms = es ? (unsigned long long)((us & 0x7FFFFFu) | 0x800000u) << 38 : 0ull;
  const unsigned long long mc = ec ? (unsigned long long)((uc & 0x7FFFFFu) | 0x800000u) << 38 : 0ull;
  const long long a = (long long)(ms >> min(e - es, 63)), b = (long long)(mc >> min(e - ec, 63));
  const long long m = ((us >> 31) ? -a : a) + ((uc >> 31) ? -b : b);
  const unsigned long long sign = (unsigned long long)m & 0x8000000000000000ull;
  unsigned long long u = m < 0 ? (unsigned long long)(-m) : (unsigned long long)m;
  const int lz = __clzll((long long)u);   // 64 for u == 0
  u <<= (lz & 63);                        // leading bit at 63: value = u 2^(e - 188 - lz)
  const int eb = e + 898 - lz + t;        // biased FP64 exponent of the leading bit
  const double fin = __longlong_as_double((long long)(sign | ((unsigned long long)max(min(eb, 0x7FE), 1) << 52) |
                                                      ((u >> 11) & 0xFFFFFFFFFFFFFull)));
  const double inf = __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  const double r = (lz == 64 || eb <= 0) ? 0.0 : (eb >= 0x7FF ? inf : fin);
  return (es == 0xFF || ec == 0xFF) ? f2d_scaled(es == 0xFF ? s : c, t) : r;
}

// Column b of a p x p update matrix for the float-pair products y_a l_ab (a0 <= a < p), y_a taken at the column
// shifts sh of block j (y~_a = y_a 2^-sh_a): out[a] = the float pair of l_ab 2^(sh_a - t), with t = max_a
// (exponent of l_ab + sh_a), so that every |y~_a l~_ab| <= 2^(kGramCenter + 2) and sum_a y_a l_ab = 2^t sum_a
// y~_a l~_ab; out[a] = 0 for a < a0 (terms summed with FP64 FMAs instead). Returns t.
template <int PM>
__device__ __forceinline__ int df_matrix_col(const double (&l)[PM], int p, const int *__restrict__ sh, int j,
                                             float2 (&out)[PM], int a0) {
  int t = -2 * kGramShiftMax - 2000;
#pragma unroll
  for (int a = 0; a < PM; ++a)
    if (a >= a0 && a < p && l[a] != 0.0) t = max(t, exponent_of(fabs(l[a])) + shift_at(sh, j * p + a));
  if (t < -2 * kGramShiftMax - 1000) t = 0;   // an all-zero column
#pragma unroll
  for (int a = 0; a < PM; ++a)
    out[a] = (a >= a0 && a < p) ? split_f64(l[a], t - shift_at(sh, j * p + a)) : make_float2(0.0f, 0.0f);
  return t;
}

// Read row[a] for a < PM from shared memory, 16 bytes at a time when the row start is aligned.
template <typename E, int PM>
__device__ __forceinline__ void load_row(const E *row, E (&out)[PM], int p) {
  constexpr int V = 16 / sizeof(E);   // elements per 16-byte load
  if (PM >= V && p == PM && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
#pragma unroll
    for (int a = 0; a < PM; a += V) {
      if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(row + a);
        out[a] = t.x; out[a + 1] = t.y; out[a + 2] = t.z; out[a + 3] = t.w;
      } else {   // 8-byte elements (double, or a float2 hi/lo pair)
        const double2 t = *reinterpret_cast<const double2 *>(row + a);
        out[a] = *reinterpret_cast<const E *>(&t.x);
        out[a + 1] = *reinterpret_cast<const E *>(&t.y);
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < PM; ++a) out[a] = a < p ? row[a] : E{};
  }
}

template <int PM>
struct GramAcc {
  float s[PM], c[PM];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int a = 0; a < PM; ++a) { s[a] = 0.0f; c[a] = 0.0f; }
  }
  // move the pairs into the thread's FP64 sums and restart
  __device__ __forceinline__ void flush(double *slot, int p) {
#pragma unroll
    for (int a = 0; a < PM; ++a)
      if (a < p) {
        slot[a] += (double)s[a];
        slot[a] += (double)c[a];
        s[a] = 0.0f;
        c[a] = 0.0f;
      }
  }
  // the same for shifted operands: entry a is scaled back by 2^(sx(a) + sy) (two exact multiplications)
  template <class SX>
  __device__ __forceinline__ void flush_shifted(double *slot, int p, SX sx, int sy) {
    const double fy = pow2d(sy);
#pragma unroll
    for (int a = 0; a < PM; ++a)
      if (a < p) {
        const double fx = pow2d(sx(a));
        slot[a] += ((double)s[a] * fx) * fy;
        slot[a] += ((double)c[a] * fx) * fy;
        s[a] = 0.0f;
        c[a] = 0.0f;
      }
  }
};

// Flush helper for kernels templated on the precision: FP32 operands are not shifted.
template <typename T, int PM, class SX>
__device__ __forceinline__ void gram_flush(GramAcc<PM> &acc, double *slot, int p, SX sx, int sy) {
  if constexpr (Gram<T>::kShifted) acc.flush_shifted(slot, p, sx, sy);
  else acc.flush(slot, p);
}
// A single float pair (a column norm) flushed with shift 2 sy.
template <typename T>
__device__ __forceinline__ void norm_flush(double &slot, float &s, float &c, int sy) {
  if constexpr (Gram<T>::kShifted) {
    const double f = pow2d(sy);
    slot += ((double)s * f) * f;
    slot += ((double)c * f) * f;
  } else {
    slot += (double)s;
    slot += (double)c;
  }
  s = c = 0.0f;
}

// Sum the FP64 slots of all row slots of the CTA in fixed order: out[e] = sum_g red[g*E + e].
__device__ __forceinline__ void cta_sum_slots(const double *red, int E, int rpp, double *__restrict__ out) {
  __syncthreads();
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double v = 0.0;
    for (int gg = 0; gg < rpp; ++gg) v += red[(int64_t)gg * E + e];
    out[e] = v;
  }
  __syncthreads();
}

// One row of BOP: (A X)_{r,c}.
template <typename T, int OPK>
__device__ __forceinline__ T apply_row(const OpDesc &A, const T *__restrict__ X, int64_t r, int k, int c) {
  if constexpr (OPK == OP_CSR) {
    // batches of 8 entries: all column indices and values first, then all gathered X loads, then the FMAs,
    // so a row costs ~2 dependent memory round trips instead of one per entry
    const T *__restrict__ v = static_cast<const T *>(A.vals);
    const int64_t e0 = __ldg(A.rowptr + r), e1 = __ldg(A.rowptr + r + 1);
    T s = T(0);
    for (int64_t e = e0; e < e1; e += 8) {
      int col[8];
      T w[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = e + u < e1;
        col[u] = in ? __ldg(A.colind + e + u) : 0;
        w[u] = in ? __ldg(v + e + u) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = (e + u < e1) ? __ldg(X + (int64_t)col[u] * k + c) : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < e1) s = fma_t(w[u], xv[u], s);
    }
    return s;
  } else if constexpr (OPK == OP_SELL) {
    const T *__restrict__ v = static_cast<const T *>(A.vals);
    const int64_t base = __ldg(A.rowptr + r / kSellC) + r % kSellC;
    const int len = __ldg(A.rowlen + r);
    T s = T(0);
    for (int j = 0; j < len; j += 8) {
      int col[8];
      T w[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = j + u < len;
        const int64_t e = base + (int64_t)(j + u) * kSellC;
        col[u] = in ? __ldg(A.colind + e) : 0;
        w[u] = in ? __ldg(v + e) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = (j + u < len) ? __ldg(X + (int64_t)col[u] * k + c) : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j + u < len) s = fma_t(w[u], xv[u], s);
    }
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

// The shared-memory row tiles are indexed by thread (tile element t = g*k + c). When no block of p columns
// straddles a warp -- k divides 32, or 32 divides k and p divides 32 -- every broadcast read stays inside the
// writing warp, so a warp barrier orders it and the warps of a CTA run their row passes independently
// (better latency hiding than CTA-wide barriers, which make all warps load together and compute together).
__host__ __device__ __forceinline__ bool warp_local_rows(int k, int p) {
  return (32 % k == 0) || (k % 32 == 0 && 32 % p == 0);
}
__device__ __forceinline__ void row_sync(bool warp_local) {
  if (warp_local) __syncwarp();
  else __syncthreads();
}

__device__ __forceinline__ bool block_active(const int *__restrict__ active, int global, int j) {
  return active == nullptr || active[global ? 0 : j] != 0;
}

// ---------------------------------------------------------------------------------------------------
// K1: Q = A P (BOP), alpha = <<P, Q>>_S, and the recomputed rho^{i-1} = <<P, R^{i-1}>>_S (BDOT x 2),
// one pass over the rows. A CTA pass covers RPT * rpp consecutive rows; slot g handles rows
// row0 + u*rpp + g, u < RPT. Without RR the recomputed rho comes from the previous iteration's K3 and R is
// not read.
template <typename T, int OPK, int PM, bool RR>
__global__ void __launch_bounds__(kNT) k_op_gram(OpDesc A, const T *__restrict__ P, const T *__restrict__ R,
                                                 T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                 const int *__restrict__ active, double *__restrict__ partA,
                                                 double *__restrict__ partR, const DevStatus *__restrict__ st,
                                                 const int *__restrict__ shP, const int *__restrict__ shQ,
                                                 const int *__restrict__ shR) {
  using G = Gram<T>;
  using BT = typename G::B;
  constexpr int RPT = rpt_op<T>();
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  BT *sPt = reinterpret_cast<BT *>(smem);   // [RPT][kNT]
  double *redA = reinterpret_cast<double *>(smem + (size_t)RPT * kNT * sizeof(double));
  double *redR = redA + kNT * p;
  const int rpp = kNT / k;
  const bool wl = warp_local_rows(k, p);
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p;
  const bool act = slot && block_active(active, global, j);
  const int sP = shift_at(shP, c), sQ = shift_at(shQ, c), sR = shift_at(shR, c);
  auto sxP = [&](int a) { return shift_at(shP, j * p + a); };
  double *slotA = redA + ((int64_t)g * k + c) * p, *slotR = redR + ((int64_t)g * k + c) * p;
  if (slot)
    for (int a = 0; a < p; ++a) { slotA[a] = 0.0; if (RR) slotR[a] = 0.0; }
  GramAcc<PM> accA;
  GramAcc<RR ? PM : 1> accR;
  accA.zero();
  accR.zero();
  int pass = 0;
  const int64_t span = (int64_t)rpp * RPT;
  const int64_t stride = (int64_t)gridDim.x * span;
  for (int64_t row0 = (int64_t)blockIdx.x * span; row0 < n; row0 += stride) {
    BT qb[RPT], rb[RPT];
    T qv[RPT], pv[RPT], rv[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int64_t r = row0 + u * rpp + g;
      qv[u] = pv[u] = rv[u] = T(0);
      if (act && r < n) {
        const int64_t o = r * k + c;
        pv[u] = P[o];
        if (RR) rv[u] = R[o];
        qv[u] = apply_row<T, OPK>(A, P, r, k, c);
      }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int64_t r = row0 + u * rpp + g;
      if (act && r < n) Q[r * k + c] = qv[u];
      qb[u] = G::conv(qv[u], sQ);
      rb[u] = G::conv(rv[u], sR);
      if (slot) sPt[u * kNT + g * k + c] = G::conv(pv[u], sP);
    }
    row_sync(wl);
    if (act) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        BT prow[PM];
        load_row<BT, PM>(sPt + u * kNT + g * k + j * p, prow, p);
#pragma unroll
        for (int a = 0; a < PM; ++a) {
          if (a < p) {
            G::add(accA.s[a], accA.c[a], prow[a], qb[u]);
            if constexpr (RR) G::add(accR.s[a], accR.c[a], prow[a], rb[u]);
          }
        }
      }
    }
    row_sync(wl);
    if (++pass == kFlushPasses / RPT) {
      pass = 0;
      if (slot) { gram_flush<T>(accA, slotA, p, sxP, sQ); if (RR) gram_flush<T>(accR, slotR, p, sxP, sR); }
    }
  }
  if (slot) { gram_flush<T>(accA, slotA, p, sxP, sQ); if (RR) gram_flush<T>(accR, slotR, p, sxP, sR); }
  const int E = k * p;
  cta_sum_slots(redA, E, rpp, partA + (int64_t)blockIdx.x * E);
  if constexpr (RR) cta_sum_slots(redR, E, rpp, partR + (int64_t)blockIdx.x * E);
}

// ---------------------------------------------------------------------------------------------------
// K2: X += P lambda, R -= Q lambda (BAXPY x 2), then rho^i = <<Z, R>>_S and the per-column ||R_c||^2.
// ZS: Z = M^{-1} R with the Jacobi preconditioner (dinv = 1 / diag(A)); otherwise Z = R and dinv is unused.
// p = 2..8 compiled for 3 CTAs per SM (80 registers): the FP64 instantiation is FP64-pipe bound and
// measured 9 % faster with the extra warps (2.02 -> 1.85 ms, 128^3, k = 32, p = 8)
template <int PM>
constexpr int upd_min_ctas() { return (PM >= 2 && PM <= 8) ? 3 : 1; }

template <typename T, int PM, bool ZS>
__global__ void __launch_bounds__(kNT, upd_min_ctas<PM>()) k_update_xr(T *__restrict__ X, T *__restrict__ R, const T *__restrict__ P,
                                                   const T *__restrict__ Q, int64_t n, int k, int p, int global,
                                                   const double *__restrict__ lam, const int *__restrict__ active,
                                                   double *__restrict__ partRho, double *__restrict__ partN,
                                                   const DevStatus *__restrict__ st, const T *__restrict__ dinv,
                                                   const int *__restrict__ shZ, const int *__restrict__ shR) {
  using G = Gram<T>;
  using BT = typename G::B;
  constexpr int RPT = rpt_stream<T>();
  static_assert(sizeof(BT) <= sizeof(T), "broadcast tile reuses the P tile");
  if (st != nullptr && st->flags != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);     // [RPT][kNT]
  T *sQ = sP + RPT * kNT;                  // [RPT][kNT]
  T *sL = sQ + RPT * kNT;                  // lambda in T, [nblk][p][p]
  BT *sRb = reinterpret_cast<BT *>(smem);  // new residual rows, broadcast (reuses the P tile)
  const int nblk = global ? 1 : k / p;
  double *red = reinterpret_cast<double *>(smem + update_xr_red_offset(k, p, global, sizeof(T), RPT));
  double *nred = red + kNT * p;
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sL[e] = (T)lam[e];
  const int rpp = kNT / k;
  const bool wl = warp_local_rows(k, p);
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p, b = c - j * p;
  const bool act = slot && block_active(active, global, j);
  const int sZ = shift_at(shZ, c), sR = shift_at(shR, c);
  auto sxZ = [&](int a) { return shift_at(shZ, j * p + a); };
  double *slotRho = red + ((int64_t)g * k + c) * p;
  double *slotN = nred + (int64_t)g * k + c;
  if (slot) {
    for (int a = 0; a < p; ++a) slotRho[a] = 0.0;
    *slotN = 0.0;
  }
  GramAcc<PM> acc;
  acc.zero();
  float ns = 0.0f, nc = 0.0f;
  int pass = 0;
  __syncthreads();
  T lcol[PM];   // column b of lambda_j: the same for every row this thread updates
  {
    const T *lj = sL + (global ? 0 : j) * p * p + b;
#pragma unroll
    for (int a = 0; a < PM; ++a) lcol[a] = (slot && a < p) ? lj[a * p] : T(0);
  }
  const int64_t span = (int64_t)rpp * RPT;
  const int64_t stride = (int64_t)gridDim.x * span;
  for (int64_t row0 = (int64_t)blockIdx.x * span; row0 < n; row0 += stride) {
    T xv[RPT], rv[RPT], pv[RPT], qv[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int64_t r = row0 + u * rpp + g;
      xv[u] = rv[u] = pv[u] = qv[u] = T(0);
      if (act && r < n) {
        const int64_t o = r * k + c;
        xv[u] = X[o]; rv[u] = R[o]; pv[u] = P[o]; qv[u] = Q[o];
      }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u)
      if (slot) { sP[u * kNT + g * k + c] = pv[u]; sQ[u * kNT + g * k + c] = qv[u]; }
    row_sync(wl);
    if (act) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        T prow[PM], qrow[PM];
        load_row<T, PM>(sP + u * kNT + g * k + j * p, prow, p);
        load_row<T, PM>(sQ + u * kNT + g * k + j * p, qrow, p);
#pragma unroll
        for (int a = 0; a < PM; ++a) {
          if (a < p) {
            xv[u] = fma_t(prow[a], lcol[a], xv[u]);
            rv[u] = fma_t(-qrow[a], lcol[a], rv[u]);
          }
        }
        const int64_t r = row0 + u * rpp + g;
        if (r < n) {
          X[r * k + c] = xv[u];
          R[r * k + c] = rv[u];
        }
      }
    }
    row_sync(wl);
    BT rb[RPT];   // own operand R; the broadcast row is Z = M^{-1} R (Z = R without a preconditioner)
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int64_t r = row0 + u * rpp + g;
      const bool live = act && r < n;
      rb[u] = live ? G::conv(rv[u], sR) : G::zero();
      if (slot) sRb[u * kNT + g * k + c] = live ? (ZS ? G::conv(rv[u] * dinv[r], sZ) : G::conv(rv[u], sZ)) : G::zero();
    }
    row_sync(wl);
    if (act) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        BT rrow[PM];
        load_row<BT, PM>(sRb + u * kNT + g * k + j * p, rrow, p);
#pragma unroll
        for (int a = 0; a < PM; ++a)
          if (a < p) G::add(acc.s[a], acc.c[a], rrow[a], rb[u]);
        G::add(ns, nc, rb[u], rb[u]);   // ||R_c||^2 for the stopping test
      }
    }
    row_sync(wl);
    if (++pass == kFlushPasses / RPT) {
      pass = 0;
      if (slot) {
        gram_flush<T>(acc, slotRho, p, sxZ, sR);
        norm_flush<T>(*slotN, ns, nc, sR);
      }
    }
  }
  if (slot) {
    gram_flush<T>(acc, slotRho, p, sxZ, sR);
    norm_flush<T>(*slotN, ns, nc, sR);
  }
  const int E = k * p;
  cta_sum_slots(red, E, rpp, partRho + (int64_t)blockIdx.x * E);
  cta_sum_slots(nred, k, rpp, partN + (int64_t)blockIdx.x * k);
}

// ---------------------------------------------------------------------------------------------------
// K3: P = Z + P beta (BAXPY with the direction-update sign read as "+"); ZS as in K2.
template <typename T, int PM, bool ZS>
__global__ void __launch_bounds__(kNT) k_update_p(T *__restrict__ P, const T *__restrict__ R, int64_t n, int k,
                                                  int p, int global, const double *__restrict__ beta,
                                                  const int *__restrict__ active, DevStatus *__restrict__ st,
                                                  const T *__restrict__ dinv) {
  constexpr int RPT = rpt_stream<T>();
  if (st->flags != 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->cur += 1;   // no other kernel of this launch reads it
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);   // [RPT][kNT]
  T *sB = sP + RPT * kNT;
  const int nblk = global ? 1 : k / p;
  for (int e = threadIdx.x; e < nblk * p * p; e += blockDim.x) sB[e] = (T)beta[e];
  const int rpp = kNT / k;
  const bool wl = warp_local_rows(k, p);
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p, b = c - j * p;
  const bool act = slot && block_active(active, global, j);
  __syncthreads();
  T bcol[PM];   // column b of beta_j
  {
    const T *bj = sB + (global ? 0 : j) * p * p + b;
#pragma unroll
    for (int a = 0; a < PM; ++a) bcol[a] = (slot && a < p) ? bj[a * p] : T(0);
  }
  const int64_t span = (int64_t)rpp * RPT;
  const int64_t stride = (int64_t)gridDim.x * span;
  for (int64_t row0 = (int64_t)blockIdx.x * span; row0 < n; row0 += stride) {
    T pv[RPT], rv[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int64_t r = row0 + u * rpp + g;
      pv[u] = rv[u] = T(0);
      if (act && r < n) {
        pv[u] = P[r * k + c];
        rv[u] = ZS ? R[r * k + c] * dinv[r] : R[r * k + c];   // Z = M^{-1} R
      }
      if (slot) sP[u * kNT + g * k + c] = pv[u];
    }
    row_sync(wl);
    if (act) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int64_t r = row0 + u * rpp + g;
        T prow[PM];
        load_row<T, PM>(sP + u * kNT + g * k + j * p, prow, p);
        T s = rv[u];
#pragma unroll
        for (int a = 0; a < PM; ++a)
          if (a < p) s = fma_t(prow[a], bcol[a], s);
        if (r < n) P[r * k + c] = s;
      }
    }
    row_sync(wl);
  }
}

// ---------------------------------------------------------------------------------------------------
// K0: R = B - A X (and optionally P = R), per-column ||R_c||^2 partials. T is the precision of X, B, R;
// R32/P32 (optional) receive a float copy of R and of P (the mixed-precision inner right-hand side), scaled by
// 2^-sig[c] when sig is given. dinv (optional): P = M^{-1} R with the Jacobi preconditioner M = diag(A).
template <typename T, int OPK>
__global__ void __launch_bounds__(kNT) k_residual(OpDesc A, const T *__restrict__ X, const T *__restrict__ B,
                                                  T *__restrict__ R, T *__restrict__ P, float *__restrict__ R32,
                                                  float *__restrict__ P32, int64_t n, int k,
                                                  double *__restrict__ partN, const T *__restrict__ dinv,
                                                  const int *__restrict__ sig) {
  const double fs = sig != nullptr ? pow2d(-sig[threadIdx.x % k]) : 1.0;   // this thread's column is t mod k
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
      const T zv = dinv ? rv * dinv[r] : rv;   // P^1 = M^{-1} R^0
      if (R) R[o] = rv;
      if (P) P[o] = zv;
      if (R32) { R32[o] = (float)((double)rv * fs); }
      if (P32) { P32[o] = (float)((double)zv * fs); }
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
                                              int p, double *__restrict__ part, const int *__restrict__ shX,
                                              const int *__restrict__ shY) {
  using G = Gram<T>;
  using BT = typename G::B;
  extern __shared__ __align__(16) unsigned char smem[];
  BT *sX = reinterpret_cast<BT *>(smem);
  double *red = reinterpret_cast<double *>(smem + kNT * sizeof(double));
  const int rpp = kNT / k;
  const bool wl = warp_local_rows(k, p);
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  const bool slot = g < rpp;
  const int j = c / p;
  const int cshX = shift_at(shX, c), cshY = shift_at(shY, c);
  auto sxX = [&](int a) { return shift_at(shX, j * p + a); };
  double *sl = red + ((int64_t)g * k + c) * p;
  if (slot)
    for (int a = 0; a < p; ++a) sl[a] = 0.0;
  GramAcc<PM> acc;
  acc.zero();
  int pass = 0;
  const int64_t stride = (int64_t)gridDim.x * rpp;
  for (int64_t row0 = (int64_t)blockIdx.x * rpp; row0 < n; row0 += stride) {
    const int64_t r = row0 + g;
    BT xb = G::zero(), yb = G::zero();
    if (slot && r < n) { xb = G::conv(X[r * k + c], cshX); yb = G::conv(Y[r * k + c], cshY); }
    if (slot) sX[g * k + c] = xb;
    row_sync(wl);
    if (slot) {
      BT xrow[PM];
      load_row<BT, PM>(sX + g * k + j * p, xrow, p);
#pragma unroll
      for (int a = 0; a < PM; ++a)
        if (a < p) G::add(acc.s[a], acc.c[a], xrow[a], yb);
    }
    row_sync(wl);
    if (++pass == kFlushPasses) {
      pass = 0;
      if (slot) gram_flush<T>(acc, sl, p, sxX, cshY);
    }
  }
  if (slot) gram_flush<T>(acc, sl, p, sxX, cshY);
  cta_sum_slots(red, k * p, rpp, part + (int64_t)blockIdx.x * k * p);
}

// Inverse diagonal of the operator (Jacobi preconditioner M = diag(A)): one value per row. Also the two maxima
// the exponent shifts of the Gram operands are offset by (as bit patterns of non-negative doubles, which order
// like the integers; the caller zeroes them first): opmax[0] = max over rows of sum_j |A_rj| (a bound of ||A||_2
// for symmetric A), opmax[1] = max |1 / A_rr|.
template <typename T, int OPK>
__global__ void k_inv_diag(OpDesc A, int64_t n, T *__restrict__ dinv, unsigned long long *__restrict__ opmax) {
  double mrow = 0.0, mdinv = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0, rabs = 0.0;
    if constexpr (OPK == OP_CSR) {
      const double *v = static_cast<const double *>(A.vals);
      for (int64_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
        if (A.colind[e] == r) d += v[e];
        rabs += fabs(v[e]);
      }
    } else if constexpr (OPK == OP_SELL) {
      const double *v = static_cast<const double *>(A.vals);
      const int64_t base = A.rowptr[r / kSellC] + r % kSellC;
      for (int j = 0; j < A.rowlen[r]; ++j) {
        if (A.colind[base + (int64_t)j * kSellC] == r) d += v[base + (int64_t)j * kSellC];
        rabs += fabs(v[base + (int64_t)j * kSellC]);
      }
    } else if constexpr (OPK == OP_ST5) {
      d = 4.0 * A.scale;
      rabs = 8.0 * fabs(A.scale);
    } else if constexpr (OPK == OP_ST7) {
      d = 6.0 * A.scale;
      rabs = 12.0 * fabs(A.scale);
    } else {
      const int nx = A.nx, ny = A.ny, nz = A.nz;
      const int64_t pl = (int64_t)nx * ny;
      const int ix = (int)(r % nx), iy = (int)((r / nx) % ny), iz = (int)(r / pl);
      const double *f = static_cast<const double *>(A.faces);
      const int64_t nfx = (int64_t)nz * ny * (nx + 1), nfy = (int64_t)nz * (ny + 1) * nx;
      const double *fx = f, *fy = f + nfx, *fz = f + nfx + nfy;
      const int64_t bx = ((int64_t)iz * ny + iy) * (nx + 1) + ix;
      const int64_t by = ((int64_t)iz * (ny + 1) + iy) * nx + ix;
      const int64_t bz = ((int64_t)iz * ny + iy) * nx + ix;
      d = A.scale * (((fx[bx] + fx[bx + 1]) + (fy[by] + fy[by + nx])) + (fz[bz] + fz[bz + pl]));
      rabs = 2.0 * fabs(d);
    }
    dinv[r] = (T)(1.0 / d);
    mrow = fmax(mrow, rabs);
    mdinv = fmax(mdinv, fabs(1.0 / d));
  }
  if (opmax == nullptr) return;
  unsigned long long b0 = (unsigned long long)__double_as_longlong(mrow);
  unsigned long long b1 = (unsigned long long)__double_as_longlong(mdinv);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t0 = __shfl_xor_sync(0xffffffffu, b0, o), t1 = __shfl_xor_sync(0xffffffffu, b1, o);
    b0 = t0 > b0 ? t0 : b0;
    b1 = t1 > b1 ? t1 : b1;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(opmax, b0);
    atomicMax(opmax + 1, b1);
  }
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
