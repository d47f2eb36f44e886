// Tensor-core (tcgen05) block products and block updates for wide blocks, FP64-accurate:
//   kt_baxpy  OUT_j = BASE_j + sign * Y_j C_j          (Section 3's BAXPY, omega = 2 n p^2 per block)
//   kt_gram   partials of gamma_j = X_j^T Y_j           (Section 2's block product, the BDOT of Section 3)
// for 64 <= p <= 256, p a multiple of 64.
//
// Exact slicing (the Ozaki scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its applications", Numer. Algorithms
// 59, 2012). Every FP64 value is truncated to a 48-bit fixed-point number relative to an exponent shared along the
// contraction and cut into eight 6-bit digits, each held exactly in a bf16 (the tensor cores' kind::f16 inputs):
//   u ~ sgn * sum_i d_i 2^(E - 5 - 6i),  E = floor(log2 max |u|) over the values sharing it,
// so a contraction sum_k u_k v_k with u's exponent E and v's exponent F equals 2^(E + F - 10) sum_s 2^(-6s) acc_s,
// acc_s = sum_k sum_{i+j=s} d_i(u_k) d_j(v_k). Each acc_s (s = 0..7: the 36 digit pairs with i + j <= 7) is summed
// over at most 512 terms of the contraction before it is read out: at most 8 * 512 products below 2^12, an integer
// below 2^24, which the FP32 accumulators of the tensor cores hold exactly whatever their internal order. The
// eight accumulators are combined with error-free float additions (TwoSum) into a float pair. Error: the
// truncations give at most 2^-47 max_k |u_k| sum_k |v_k| (and the same with u and v exchanged; where the values
// sharing an exponent are of one magnitude, about 2^-44 of sum_k |u_k v_k|), the dropped pairs (i + j > 7) about
// 2^-45 of sum_k |u_k v_k|. FP64 FMAs give about K 2^-53 of sum_k |u_k v_k|.
//
//   kt_baxpy: u = Y[r][.] with one exponent per row (over the block's p columns), v = C[.][b] with one per column;
//             output tiles of 128 rows x 64 columns of one block; C is cut once per launch (kt_slice_cmat).
//   kt_gram:  u = X[.][a], v = Y[.][b] with one exponent per column over all rows (kt_col_exp); output tiles of
//             128 x 64 entries of one block (rows of the tile beyond p are zero), partial sums over a range of rows,
//             read out every 512 rows into float pairs.
// Work: one CTA per SM (256 threads, ~200 KB of shared memory, the whole 512-column TMEM: 8 accumulators of 64
// FP32 columns x 128 lanes). The contraction runs in chunks of 32 staged in two shared-memory buffers: while the
// tensor cores multiply one chunk (one thread issues the 2 x 36 MMAs, M = 128, N = 64, K = 16, and commits them to
// the buffer's mbarrier), all threads cut the next chunk into the other buffer's 8 + 8 digit tiles (K-major core
// matrices of 8 rows x 16 bytes, no swizzle). Every wait on an mbarrier is bounded: ST_TIMEOUT if it never
// completes. Accumulators are read back with tcgen05.ld (warp w: TMEM lanes 32 (w mod 4) .. +31, 8 columns at a
// time).
#pragma once

#include <cstdint>

#include "bcg_kernels.cuh"

namespace bcgk {

constexpr int kTcRows = 128;      // M: rows of an output tile (TMEM lanes)
constexpr int kTcCols = 64;       // N: columns of an output tile
constexpr int kTcK = 32;          // contraction chunk of one shared-memory stage
constexpr int kTcSlices = 8;      // 6-bit digits per value (48 bits)
constexpr int kTcDigitBits = 6;
constexpr int kTcThreads = 256;
constexpr int kTcWindow = 512;    // contraction terms an accumulator takes before it is read out (exactness)
constexpr uint32_t kTcSliceBytesA = kTcRows * kTcK * 2;          // 8 KB: one digit slice of an M x K chunk
constexpr uint32_t kTcSliceBytesB = kTcCols * kTcK * 2;          // 4 KB: one digit slice of an N x K chunk
constexpr uint32_t kTcStageBytesA = kTcSlices * kTcSliceBytesA;  // 64 KB
constexpr uint32_t kTcStageBytesB = kTcSlices * kTcSliceBytesB;  // 32 KB: also the pre-sliced image of a C chunk
constexpr uint32_t kTcSbo = (kTcK / 8) * 128;                    // bytes between 8-row core-matrix groups
constexpr size_t kTcSmemOps = 2 * (size_t)(kTcStageBytesA + kTcStageBytesB);   // 192 KB
constexpr size_t kTcSmemMisc = 4096;
constexpr size_t kTcSmem = kTcSmemOps + kTcSmemMisc + 1024;       // + alignment slack
constexpr long long kTcWaitLimit = 1ll << 24;                     // mbarrier polls before ST_TIMEOUT

__host__ __device__ constexpr bool tc_layout_ok(int k, int p) {
  return p >= 64 && p <= 256 && p % 64 == 0 && k % p == 0 && k <= 256;
}
// bf16 digits of the pre-sliced C^T for nblkC distinct blocks: (p / 64) (p / 32) chunk images of 32 KB per block
__host__ __device__ constexpr size_t tc_cmat_bytes(int nblkC, int p) {
  return (size_t)nblkC * (p / kTcCols) * (p / kTcK) * kTcStageBytesB;
}

// ---- PTX wrappers (tcgen05, mbarrier) --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzling: 8-row x 16-byte core matrices,
// lbo = byte distance between core matrices adjacent along K, sbo = between core matrices adjacent along M (N).
// Fields: start address >> 4 (bits 0-13), lbo >> 4 (16-29), sbo >> 4 (32-45), descriptor version 1 (46-47),
// base offset 0, layout "no swizzle" 0 (61-63).
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16 A and B (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// true once the phase with parity `phase` has completed; gives up after kTcWaitLimit polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long i = 0; i < kTcWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// TMEM: 512 columns for the whole CTA (one warp allocates and frees)
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes (one row per thread). The load and its wait form one
// asm statement, so the registers are complete when they leave it (no consumer can be scheduled in between).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- exact slicing -------------------------------------------------------------------------------------------
// floor(|x| 2^(47 - E)) for |x| < 2^(E+1): the 48-bit fixed-point magnitude (zero or subnormal x: 0)
__device__ __forceinline__ unsigned long long tc_fixed48(double x, int E) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sft = 1028 + E - e;   // >= 5 since e - 1023 <= E
  return (e == 0 || e == 0x7FF || sft >= 64) ? 0ull : (m >> (sft < 5 ? 5 : sft));
}
// bf16 bit pattern of sign * d for an integer 0 <= d < 64 (exact: 6 significant bits)
__device__ __forceinline__ uint32_t tc_bf16_digit(uint32_t d, uint32_t sign16) {
  const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | sign16;
}
// digit i (0 = most significant) of a 48-bit fixed-point magnitude
__device__ __forceinline__ uint32_t tc_digit(unsigned long long v, int i) {
  return (uint32_t)(v >> (42 - kTcDigitBits * i)) & 63u;
}

// Digits of 8 values sharing the exponent E (consecutive along the contraction): w[i] = the 16-byte core-matrix
// row of slice i (8 bf16, the first value in the low half of w[i][0]).
__device__ __forceinline__ void tc_pack8(const double (&v)[8], int E, uint32_t (&w)[kTcSlices][4]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const unsigned long long fx = tc_fixed48(v[e], E);
    const uint32_t sg = signbit(v[e]) ? 0x8000u : 0u;
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i) {
      const uint32_t d = tc_bf16_digit(tc_digit(fx, i), sg);
      if (e & 1) w[i][e >> 1] |= d << 16;
      else w[i][e >> 1] = d;
    }
  }
}
// Store the 8 slices of one core-matrix row (row `row` of the M or N dimension, k-group kg of the chunk).
__device__ __forceinline__ void tc_store8(unsigned char *stage, uint32_t slice_bytes, int row, int kg,
                                          const uint32_t (&w)[kTcSlices][4]) {
  const uint32_t off = (uint32_t)(((row >> 3) * (kTcK / 8) + kg) * 128 + (row & 7) * 16);
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i)
    *reinterpret_cast<uint4 *>(stage + i * slice_bytes + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// The 2 x 36 MMAs of one chunk (digit pairs i + j <= 7 into accumulator s = i + j, 64 TMEM columns each).
// fresh: the first chunk since the accumulators were read out (its first MMA into each accumulator overwrites it).
__device__ __forceinline__ void tc_issue_chunk(uint32_t tbase, uint32_t aStage, uint32_t bStage, bool fresh) {
  const uint32_t idesc = tc_idesc_bf16(kTcRows, kTcCols);
#pragma unroll 1
  for (int ks = 0; ks < kTcK / 16; ++ks)
#pragma unroll 1
    for (int sacc = 0; sacc < kTcSlices; ++sacc)
#pragma unroll 1
      for (int i = 0; i <= sacc; ++i) {
        const uint64_t ad = tc_smem_desc(aStage + i * kTcSliceBytesA + ks * 256, 128, kTcSbo);
        const uint64_t bd = tc_smem_desc(bStage + (sacc - i) * kTcSliceBytesB + ks * 256, 128, kTcSbo);
        tc_mma(tbase + (uint32_t)(sacc * kTcCols), ad, bd, idesc, !(fresh && ks == 0 && i == 0));
      }
}

// Read back 8 columns (col .. col + 7) of all 8 accumulators for this warp's 32 lanes and combine them:
// hi[e] + lo[e] = sum_s 2^(-6 s) acc_s (column col + e, this thread's lane), a float pair.
__device__ __forceinline__ void tc_read8(uint32_t tbase, int q, int col, float (&hi)[8], float (&lo)[8]) {
  float acc[kTcSlices][8];
#pragma unroll
  for (int sacc = 0; sacc < kTcSlices; ++sacc)
    tmem_ld8(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(sacc * kTcCols + col), acc[sacc]);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    hi[e] = acc[kTcSlices - 1][e] * 0x1p-42f;
    lo[e] = 0.0f;
#pragma unroll
    for (int sacc = kTcSlices - 2; sacc >= 0; --sacc)
      two_sum_acc(hi[e], lo[e], acc[sacc][e] * __uint_as_float((uint32_t)(127 - kTcDigitBits * sacc) << 23), 0.0f);
  }
}

// Two-stage pipeline state: one mbarrier per shared-memory stage, its phase parity, and whether a commit on it is
// still to be waited for. Every commit is waited for exactly once.
struct TcPipe {
  uint32_t mbar[2];
  uint32_t ph[2];
  int pending[2];
  // Wait for the MMAs that read stage st (if any). Returns false on timeout (the same in every thread).
  __device__ __forceinline__ bool acquire(int st) {
    bool ok = true;
    if (pending[st]) {
      ok = mbar_wait(mbar[st], ph[st]);
      ph[st] ^= 1u;
      pending[st] = 0;
    }
    return !__syncthreads_or(!ok);
  }
  __device__ __forceinline__ bool drain() { return acquire(0) && acquire(1); }
};

// Common start of the tensor-core kernels: 1024-byte aligned shared memory for the two stages, TMEM (512 columns,
// allocated by warp 0), the two mbarriers. Returns the TMEM base address.
__device__ __forceinline__ uint32_t tc_setup(unsigned char *raw, unsigned char *&ops, unsigned char *&misc, TcPipe &pipe) {
  ops = raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
  misc = ops + kTcSmemOps;
  uint64_t *bars = reinterpret_cast<uint64_t *>(misc);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
  if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tslot), 512);
  pipe.mbar[0] = smem_u32(bars);
  pipe.mbar[1] = smem_u32(bars + 1);
  pipe.ph[0] = pipe.ph[1] = 0;
  pipe.pending[0] = pipe.pending[1] = 0;
  if (threadIdx.x == 0) {
    mbar_init(pipe.mbar[0], 1);
    mbar_init(pipe.mbar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *tslot;
}
__device__ __forceinline__ void tc_teardown(uint32_t tbase, bool timeout, DevStatus *st) {
  __syncthreads();
  if (timeout && threadIdx.x == 0 && st != nullptr) atomicOr(&st->flags, ST_TIMEOUT);
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}
// shared-memory stage addresses
__device__ __forceinline__ unsigned char *tc_stage_a(unsigned char *ops, int st) { return ops + st * kTcStageBytesA; }
__device__ __forceinline__ unsigned char *tc_stage_b(unsigned char *ops, int st) {
  return ops + 2 * kTcStageBytesA + st * kTcStageBytesB;
}

// ---- BAXPY ------------------------------------------------------------------------------------------------------
// Pre-slicing of the p x p matrices C_jc (row-major, entry (a, b) at jc p p + a p + b) into the bf16 digit images that
// kt_baxpy copies into a shared-memory B stage: for block jc, N-tile t = b / 64 and chunk c = a / 32, a 32 KB image
// at ((jc (p/64) + t) (p/32) + c) * 32 KB of 8 slices of 4 KB, entry (b, a) at the core-matrix position of tc_store8
// (row b mod 64, k-group (a mod 32) / 8, element a mod 8). Cexp[jc p + b] = F_b. One thread per column (jc, b).
__global__ void kt_slice_cmat(const double *__restrict__ C, int nblkC, int p, uint16_t *__restrict__ Cs,
                              int *__restrict__ Cexp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nblkC * p) return;
  const int jc = idx / p, b = idx - jc * p;
  const double *Cj = C + (size_t)jc * p * p;
  double m = 0.0;
  for (int a = 0; a < p; ++a) m = fmax(m, fabs(Cj[(size_t)a * p + b]));
  const int F = exponent_of(m);
  Cexp[idx] = F;
  const int nt = p / kTcCols, nc = p / kTcK, t = b / kTcCols, bl = b % kTcCols;
  for (int a = 0; a < p; ++a) {
    const double v = Cj[(size_t)a * p + b];
    const unsigned long long fx = tc_fixed48(v, F);
    const uint32_t sg = signbit(v) ? 0x8000u : 0u;
    const int c = a / kTcK, al = a % kTcK;
    const size_t img = ((size_t)(jc * nt + t) * nc + c) * kTcStageBytesB;
    const size_t in_slice = (size_t)((bl >> 3) * (kTcK / 8) + (al >> 3)) * 128 + (bl & 7) * 16 + (al & 7) * 2;
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i)
      Cs[(img + (size_t)i * kTcSliceBytesB + in_slice) / 2] = (uint16_t)tc_bf16_digit(tc_digit(fx, i), sg);
  }
}

// OUT_j = BASE_j (times bscale[r] per row, if given) + sign * Y_j C_j over every block j (global: C_0 for all), with
// C pre-sliced by kt_slice_cmat. OUT may equal BASE; Y must not alias OUT. Frozen blocks (active[j] = 0) get
// OUT = BASE (scaled), as in kl_baxpy. bump: CTA 0 advances the iteration counter (the P update's role).
// Persistent: CTA c takes output tiles c, c + gridDim.x, ...; a row's exponent E_r is the largest exponent field
// of its p values in the block (integer maxima, no FP64 instruction).
__global__ void __launch_bounds__(kTcThreads, 1) kt_baxpy(double *OUT, const double *BASE, const double *__restrict__ Y,
                                                          const uint16_t *__restrict__ Cs, const int *__restrict__ Cexp,
                                                          int64_t n, int k, int p, int global, double sign,
                                                          const int *__restrict__ active, DevStatus *__restrict__ st,
                                                          int bump, const double *__restrict__ bscale) {
  if (st->flags != 0) return;
  if (bump && blockIdx.x == 0 && threadIdx.x == 0) st->cur += 1;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  unsigned char *ops, *misc;
  TcPipe pipe;
  const uint32_t tbase = tc_setup(tc_smem_raw, ops, misc, pipe);
  int *sE = reinterpret_cast<int *>(misc + 64);   // 128 row exponents
  int *sBad = sE + kTcRows;                       // 128 row flags (a non-finite entry)
  int *sF = sBad + kTcRows;                       // 64 column exponents of C
  int *sX = sF + kTcCols;                         // 256 partial maxima of the exponent fields
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = p / kTcCols, nc = p / kTcK;
  const int ntn = k / kTcCols;
  const int64_t ntiles = ((n + kTcRows - 1) / kTcRows) * ntn;
  bool timeout = false;
  for (int64_t tile = blockIdx.x; tile < ntiles && !timeout; tile += gridDim.x) {
    const int tn = (int)(tile % ntn);
    const int64_t r0 = (tile / ntn) * kTcRows;
    const int c0 = tn * kTcCols;            // first output column
    const int j = c0 / p, b0 = c0 - j * p;  // block and column offset inside it
    const int jc = global ? 0 : j;
    if (!block_active(active, global, j)) {   // block-uniform: every thread of the CTA takes this branch
      for (int it = tid; it < kTcRows * (kTcCols / 8); it += kTcThreads) {
        const int rl = it & (kTcRows - 1), cg = it >> 7;
        const int64_t r = r0 + rl;
        if (r >= n) continue;
        const double s = bscale ? bscale[r] : 1.0;
        for (int e = 0; e < 8; ++e) OUT[r * k + c0 + cg * 8 + e] = BASE[r * k + c0 + cg * 8 + e] * s;
      }
      continue;
    }
    {   // row exponents: two threads per row, half of the block's columns each
      const int rl = tid & (kTcRows - 1), half = tid >> 7;
      const int64_t r = r0 + rl;
      int em = 0;
      if (r < n) {
        const int2 *src = reinterpret_cast<const int2 *>(Y + r * k + (int64_t)j * p + half * (p / 2));
#pragma unroll 8
        for (int q = 0; q < p / 2; ++q) em = max(em, (__ldg(src + q).y >> 20) & 0x7FF);
      }
      sX[tid] = em;
      __syncthreads();
      if (tid < kTcRows) {
        const int e2 = max(sX[tid], sX[tid + kTcRows]);
        sE[tid] = e2 > 0 ? e2 - 1023 : -1023;
        sBad[tid] = e2 == 0x7FF;
      }
      if (tid < kTcCols) sF[tid] = Cexp[jc * p + b0 + tid];
      __syncthreads();
    }
    for (int kc = 0; kc < nc; ++kc) {
      const int stg = kc & 1;
      if (!pipe.acquire(stg)) {
        timeout = true;
        break;
      }
      unsigned char *sa = tc_stage_a(ops, stg), *sb = tc_stage_b(ops, stg);
      // cut the chunk of Y: item (row rl, k-group kg), 2 per thread, loads first
      double v[2][8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int it = tid + u * kTcThreads, rl = it & (kTcRows - 1), kg = it >> 7;
        const int64_t r = r0 + rl;
        if (r < n) {
          const double2 *src = reinterpret_cast<const double2 *>(Y + r * k + (int64_t)j * p + kc * kTcK + kg * 8);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const double2 t2 = __ldg(src + q);
            v[u][2 * q] = t2.x;
            v[u][2 * q + 1] = t2.y;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[u][e] = 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int it = tid + u * kTcThreads, rl = it & (kTcRows - 1), kg = it >> 7;
        uint32_t w[kTcSlices][4];
        tc_pack8(v[u], sE[rl], w);
        tc_store8(sa, kTcSliceBytesA, rl, kg, w);
      }
      {   // the pre-sliced chunk of C^T
        const uint4 *src = reinterpret_cast<const uint4 *>(
            reinterpret_cast<const unsigned char *>(Cs) + ((size_t)(jc * nt + b0 / kTcCols) * nc + kc) * kTcStageBytesB);
        uint4 *dst = reinterpret_cast<uint4 *>(sb);
#pragma unroll
        for (int q = 0; q < (int)(kTcStageBytesB / 16 / kTcThreads); ++q) dst[tid + q * kTcThreads] = __ldg(src + tid + q * kTcThreads);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        tc_issue_chunk(tbase, smem_u32(sa), smem_u32(sb), kc == 0);
        tc_commit(pipe.mbar[stg]);
      }
      pipe.pending[stg] = 1;
    }
    if (timeout || !pipe.drain()) {
      timeout = true;
      break;
    }
    tc_fence_after();
    {   // read back: warp w holds rows 32 (w mod 4) .. +31, columns 32 (w / 4) .. +31 of the tile
      const int q = warp & 3, h = warp >> 2;
      const int rl = q * 32 + lane;
      const int64_t r = r0 + rl;
      const int E = sE[rl];
      const bool bad = sBad[rl] != 0;
      const double bs = (r < n && bscale) ? bscale[r] : 1.0;
#pragma unroll 1
      for (int cg = 0; cg < 4; ++cg) {
        float hi[8], lo[8];
        const int cb = h * 32 + cg * 8;
        tc_read8(tbase, q, cb, hi, lo);
        if (r < n) {
          double *o = OUT + r * k + c0 + cb;
          const double *bp = BASE + r * k + c0 + cb;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int t = E + sF[cb + e] - 10;
            const double base = bscale ? bp[e] * bs : bp[e];
            const double res = (base + sign * f2d_scaled(hi[e], t)) + sign * f2d_scaled(lo[e], t);
            o[e] = bad ? __longlong_as_double(0x7FF8000000000000ll) : res;
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  tc_teardown(tbase, timeout, st);
}

// ---- Gram ------------------------------------------------------------------------------------------------------
// Column exponent fields for the Gram slicing: ecol[c] = max over rows of the biased exponent of X[r][c] (times
// xscale[r] if given), by integer maxima (the caller zeroes ecol). Thread (g, c) covers rows g, g + rows per CTA
// pass, ... of column c.
__global__ void __launch_bounds__(kNT) kt_col_exp(const double *__restrict__ X, const double *__restrict__ xscale,
                                                  int64_t n, int k, int *__restrict__ ecol) {
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  if (g >= rpp) return;
  int em = 0;
  for (int64_t r = (int64_t)blockIdx.x * rpp + g; r < n; r += (int64_t)gridDim.x * rpp) {
    const double v = xscale ? X[r * k + c] * xscale[r] : X[r * k + c];
    em = max(em, (__double2hiint(v) >> 20) & 0x7FF);
  }
  atomicMax(ecol + c, em);
}

// Partials of gamma_j = X_j^T Y_j (X's rows times xscale[r] if given): CTA (tile, chunk) takes the 128 x 64 entries
// (a in [128 ta, 128 ta + 128), b in [64 tb, 64 tb + 64)) of block j over the rows of chunk blockIdx.y, and writes them
// into partial row blockIdx.y in the layout of kl_gram (entry (a, b) of block j at j p p + b p + a); rows of the tile
// with a >= p are zero and not written. ecx, ecy: column exponent fields of X and Y (kt_col_exp). Frozen blocks get
// zero partials. The accumulators are read out into float pairs every kTcWindow rows.
__global__ void __launch_bounds__(kTcThreads, 1) kt_gram(const double *__restrict__ X, const double *__restrict__ Y,
                                                         const double *__restrict__ xscale, int64_t n, int k, int p,
                                                         int global, const int *__restrict__ active,
                                                         double *__restrict__ part, const int *__restrict__ ecx,
                                                         const int *__restrict__ ecy, DevStatus *__restrict__ st) {
  if (st != nullptr && st->flags != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ta_n = (p + kTcRows - 1) / kTcRows, tb_n = p / kTcCols;
  const int j = blockIdx.x / (ta_n * tb_n), ta = (blockIdx.x / tb_n) % ta_n, tb = blockIdx.x % tb_n;
  const int a0 = ta * kTcRows, b0 = tb * kTcCols;
  double *out = part + (size_t)blockIdx.y * k * p + (size_t)j * p * p;
  const int q = warp & 3, h = warp >> 2;
  const int al = q * 32 + lane;   // this thread's tile row in the read-out
  if (!block_active(active, global, j)) {
    if (a0 + al < p)
      for (int e = 0; e < 32; ++e) out[(size_t)(b0 + h * 32 + e) * p + a0 + al] = 0.0;
    return;
  }
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  unsigned char *ops, *misc;
  TcPipe pipe;
  const uint32_t tbase = tc_setup(tc_smem_raw, ops, misc, pipe);
  const int64_t chunk = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r_begin = (int64_t)blockIdx.y * chunk, r_end = min(n, r_begin + chunk);
  // cutting items: A (X^T) -- column a = items & 127 of the tile, k-group rg; B (Y) -- column b = tid & 63, k-group
  const int colA[2] = {tid & (kTcRows - 1), tid & (kTcRows - 1)};
  const int rgA[2] = {tid >> 7, (tid + kTcThreads) >> 7};
  const int cA = j * p + a0 + colA[0];
  const bool validA = a0 + colA[0] < p;
  const int EA = validA ? ((ecx[cA] > 0 ? ecx[cA] : 1) - 1023) : 0;
  const int bB = tid & (kTcCols - 1), rgB = tid >> 6;
  const int cB = j * p + b0 + bB;
  const int EB = (ecy[cB] > 0 ? ecy[cB] : 1) - 1023;
  float rs[32], rc[32];   // running float pairs of this thread's 32 read-out entries
#pragma unroll
  for (int e = 0; e < 32; ++e) rs[e] = rc[e] = 0.0f;
  bool timeout = false;
  const int64_t nchunks = (r_end - r_begin + kTcK - 1) / kTcK;
  for (int64_t cc = 0; cc < nchunks && !timeout; ++cc) {
    const int stg = (int)(cc & 1);
    if (!pipe.acquire(stg)) {
      timeout = true;
      break;
    }
    unsigned char *sa = tc_stage_a(ops, stg), *sb = tc_stage_b(ops, stg);
    const int64_t rbase = r_begin + cc * kTcK;
    double va[2][8], vb[8];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t r = rbase + rgA[u] * 8 + e;
        va[u][e] = (validA && r < r_end) ? (xscale ? X[r * k + cA] * xscale[r] : X[r * k + cA]) : 0.0;
      }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t r = rbase + rgB * 8 + e;
      vb[e] = r < r_end ? Y[r * k + cB] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      uint32_t w[kTcSlices][4];
      tc_pack8(va[u], EA, w);
      tc_store8(sa, kTcSliceBytesA, colA[u], rgA[u], w);
    }
    {
      uint32_t w[kTcSlices][4];
      tc_pack8(vb, EB, w);
      tc_store8(sb, kTcSliceBytesB, bB, rgB, w);
    }
    fence_async_smem();
    __syncthreads();
    const bool fresh = (cc % (kTcWindow / kTcK)) == 0;
    if (tid == 0) {
      tc_fence_after();
      tc_issue_chunk(tbase, smem_u32(sa), smem_u32(sb), fresh);
      tc_commit(pipe.mbar[stg]);
    }
    pipe.pending[stg] = 1;
    const bool window_end = ((cc + 1) % (kTcWindow / kTcK)) == 0 || cc + 1 == nchunks;
    if (window_end) {   // read the accumulators out into the running float pairs
      if (!pipe.drain()) {
        timeout = true;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int cg = 0; cg < 4; ++cg) {
        float hi[8], lo[8];
        tc_read8(tbase, q, h * 32 + cg * 8, hi, lo);
#pragma unroll
        for (int e = 0; e < 8; ++e) two_sum_acc(rs[cg * 8 + e], rc[cg * 8 + e], hi[e], lo[e]);
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!timeout && a0 + al < p) {
    const int ca = j * p + a0 + al;
    const int ea = ecx[ca];
#pragma unroll 4
    for (int e = 0; e < 32; ++e) {
      const int cb = j * p + b0 + h * 32 + e;
      const int eb = ecy[cb];
      const int t = ((ea > 0 ? ea : 1) - 1023) + ((eb > 0 ? eb : 1) - 1023) - 10;
      const double v = f2d_scaled(rs[e], t) + f2d_scaled(rc[e], t);
      out[(size_t)(b0 + h * 32 + e) * p + a0 + al] =
          (ea == 0x7FF || eb == 0x7FF) ? __longlong_as_double(0x7FF8000000000000ll) : v;
    }
  }
  tc_teardown(tbase, timeout, st);
}

}  // namespace bcgk
