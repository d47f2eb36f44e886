// Tensor-core (tcgen05) block products and block updates for wide blocks, FP64-accurate:
//   kt_baxpy_img  OUT_j = BASE_j + sign * Y_j C_j          (Section 3's BAXPY, omega = 2 n p^2 per block)
//   kt_gram_img   partials of gamma_j = X_j^T Y_j           (Section 2's block product, the BDOT of Section 3)
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
// The operands are cut once per use into digit images in global memory that are byte for byte the kernels'
// shared-memory stages (kt_cut_rows, kt_cut_cols, kt_slice_cmat; see "Digit images" below):
//   BAXPY: u = Y[r][.] with one exponent per row (over the block's p columns), v = C[.][b] with one per column;
//          output tiles of 128 rows x 64 columns (x 32 for blocks of 32 that 64-column tiles cannot pair).
//   Gram:  u = X[.][a], v = Y[.][b] with one exponent per column over all rows (kt_col_exp); output tiles of
//          128 x 64 entries of one block (rows of the tile beyond p are zero), partial sums over a range of rows,
//          read out every 512 rows into float pairs.
// Work: one CTA per SM (256 threads for the products, 320 for the updates; ~200 KB of shared memory; the whole
// 512-column TMEM: 8 accumulators of 64 FP32 columns x 128 lanes). The contraction runs in chunks of 16 through four
// shared-memory stages: a producer thread fills a stage with bulk copies of the images, an MMA thread issues the
// chunk's 36 MMAs (M = 128, N = 64, K = 16) when the copies are in and commits them to the stage's "empty"
// mbarrier, so the copies of the next three chunks overlap the MMAs of this one (K-major core matrices of 8 rows x
// 16 bytes, no swizzle). Every wait on an mbarrier is bounded: ST_TIMEOUT if it never completes. The accumulators
// are read back with tcgen05.ld (warp w: TMEM lanes 32 (w mod 4) .. +31, 8 columns at a time).
#pragma once

#include <cstdint>

#include "bcg_kernels.cuh"

namespace bcgk {

constexpr int kTcRows = 128;      // M: rows of an output tile (TMEM lanes)
constexpr int kTcCols = 64;       // N: columns of an output tile
constexpr int kTcK = 16;          // contraction chunk of one shared-memory stage (one K step of the MMA)
constexpr int kTcStages = 4;      // shared-memory stages in flight (bulk copies run up to 3 chunks ahead)
constexpr int kTcSlices = 8;      // 6-bit digits per value (48 bits)
constexpr int kTcDigitBits = 6;
constexpr int kTcThreads = 256;
constexpr int kTcWindow = 512;    // contraction terms an accumulator takes before it is read out (exactness)
constexpr uint32_t kTcSliceBytesA = kTcRows * kTcK * 2;          // 4 KB: one digit slice of an M x K chunk
constexpr uint32_t kTcSliceBytesB = kTcCols * kTcK * 2;          // 2 KB: one digit slice of an N x K chunk
constexpr uint32_t kTcStageBytesA = kTcSlices * kTcSliceBytesA;  // 32 KB
constexpr uint32_t kTcStageBytesB = kTcSlices * kTcSliceBytesB;  // 16 KB: also the pre-sliced image of a C chunk
constexpr uint32_t kTcSbo = (kTcK / 8) * 128;                    // bytes between 8-row core-matrix groups
constexpr size_t kTcSmemOps = kTcStages * (size_t)(kTcStageBytesA + kTcStageBytesB);   // 192 KB
constexpr size_t kTcSmemMisc = 4096;
constexpr size_t kTcSmem = kTcSmemOps + kTcSmemMisc + 1024;       // + alignment slack
constexpr long long kTcWaitLimit = 1ll << 24;                     // mbarrier polls before ST_TIMEOUT

__host__ __device__ constexpr bool tc_layout_ok(int k, int p) {
  return p >= 64 && p <= 256 && p % 64 == 0 && k % p == 0 && k <= 256;
}
// blocks of 16 or 32 columns paired into 64-column tiles (block-diagonal C images)
__host__ __device__ constexpr bool tc_pair_layout_ok(int k, int p) {
  return (p == 16 || p == 32) && k % 64 == 0 && k <= 256;
}
// bf16 digits of the pre-sliced C^T for nblkC distinct blocks: 8 digits of 2 bytes per entry (p / NC column tiles
// of p / 16 chunk images of 8 NC K-major rows of 16 entries each)
__host__ __device__ constexpr size_t tc_cmat_bytes(int nblkC, int p) {
  return (size_t)nblkC * p * p * kTcSlices * 2;
}
// digit slice and stage of an N x 16 chunk for output tiles of NC columns (64; 32 for blocks of 32 columns)
template <int NC>
__host__ __device__ constexpr uint32_t tc_slice_b() { return (uint32_t)NC * kTcK * 2; }
template <int NC>
__host__ __device__ constexpr uint32_t tc_stage_b() { return kTcSlices * tc_slice_b<NC>(); }

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
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}
// true once the phase with parity `phase` has completed; gives up after kTcWaitLimit polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long i = 0; i < kTcWaitLimit; ++i)
    if (mbar_try(mbar, phase)) return true;
  return false;
}
// the same, also giving up once *flag is set (another role of the CTA gave up)
__device__ __forceinline__ bool mbar_wait_flag(uint32_t mbar, uint32_t phase, const volatile int *flag) {
  for (long long i = 0; i < kTcWaitLimit; ++i) {
    if (mbar_try(mbar, phase)) return true;
    if ((i & 255) == 255 && *flag != 0) return false;
  }
  return false;
}
// one of the barrier's expected arrivals, without a transaction count
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Bulk copies (global -> this CTA's shared memory) tracked by an mbarrier's transaction count: the issuing thread
// arrives once and announces the bytes; the phase completes when the arrival and all bytes are in.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
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
// the same for an FP32 value (all 24 bits of its mantissa fit the window when its exponent is within 24 of E; zero,
// subnormal or non-finite x: 0)
__device__ __forceinline__ unsigned long long tc_fixed48(float x, int E) {
  const uint32_t u = __float_as_uint(x);
  const int ef = (int)((u >> 23) & 0xFFu);
  const unsigned long long m = (u & 0x7FFFFFu) | 0x800000u;
  const int sft = ef - 103 - E;   // |x| 2^(47 - E) = m 2^sft, below 2^48 since |x| < 2^(E+1)
  if (ef == 0 || ef == 0xFF || sft <= -64) return 0ull;
  return sft >= 0 ? (m << sft) : (m >> -sft);
}
// biased FP64 exponent field of x (a float's normal exponent moved to the FP64 bias; zero or subnormal: 0)
__device__ __forceinline__ int tc_exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }
__device__ __forceinline__ int tc_exp_field(float x) {
  const int ef = (int)((__float_as_uint(x) >> 23) & 0xFFu);
  return ef == 0 ? 0 : (ef == 0xFF ? 0x7FF : ef + 896);
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
template <typename T>
__device__ __forceinline__ void tc_pack8(const T (&v)[8], int E, uint32_t (&w)[kTcSlices][4]) {
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

// The 36 MMAs of one chunk (digit pairs i + j <= 7 into accumulator s = i + j, 64 TMEM columns each), fully
// unrolled: the descriptors of the slices are the stage's descriptor plus constant offsets (the start-address
// field holds address >> 4 in its low bits, and stage addresses stay below 256 KB, so the addition never carries
// into the next field). fresh: the first chunk since the accumulators were read out (its first MMA into each
// accumulator overwrites it).
template <int NC = kTcCols>
__device__ __forceinline__ void tc_issue_chunk(uint32_t tbase, uint32_t aStage, uint32_t bStage, bool fresh) {
  static_assert(kTcK == 16, "one K step of kind::f16 per chunk");
  static_assert(NC == 64 || NC == 32, "N = 64 or 32");
  constexpr uint32_t idesc = tc_idesc_bf16(kTcRows, NC);
  const uint64_t a0 = tc_smem_desc(aStage, 128, kTcSbo), b0 = tc_smem_desc(bStage, 128, kTcSbo);
#pragma unroll
  for (int sacc = 0; sacc < kTcSlices; ++sacc)
#pragma unroll
    for (int i = 0; i <= sacc; ++i)
      tc_mma(tbase + (uint32_t)(sacc * NC), a0 + (uint64_t)((i * kTcSliceBytesA) >> 4),
             b0 + (uint64_t)(((sacc - i) * tc_slice_b<NC>()) >> 4), idesc, i != 0 || !fresh);
}

// Read back 8 columns (col .. col + 7) of all 8 accumulators for this warp's 32 lanes and combine them:
// hi[e] + lo[e] = sum_s 2^(-6 s) acc_s (column col + e, this thread's lane), a float pair.
template <int NC = kTcCols>
__device__ __forceinline__ void tc_read8(uint32_t tbase, int q, int col, float (&hi)[8], float (&lo)[8]) {
  float acc[kTcSlices][8];
#pragma unroll
  for (int sacc = 0; sacc < kTcSlices; ++sacc)
    tmem_ld8(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(sacc * NC + col), acc[sacc]);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    hi[e] = acc[kTcSlices - 1][e] * 0x1p-42f;
    lo[e] = 0.0f;
#pragma unroll
    for (int sacc = kTcSlices - 2; sacc >= 0; --sacc)
      two_sum_acc(hi[e], lo[e], acc[sacc][e] * __uint_as_float((uint32_t)(127 - kTcDigitBits * sacc) << 23), 0.0f);
  }
}

// Common start of the tensor-core kernels: 1024-byte aligned shared memory for the two stages and TMEM (512
// columns, allocated by warp 0). Returns the TMEM base address.
__device__ __forceinline__ uint32_t tc_setup(unsigned char *raw, unsigned char *&ops, unsigned char *&misc) {
  ops = raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
  misc = ops + kTcSmemOps;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(misc);
  if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tslot), 512);
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
  return ops + kTcStages * kTcStageBytesA + st * kTcStageBytesB;
}

// ---- BAXPY ------------------------------------------------------------------------------------------------------
// Pre-slicing of the p x p matrices C_jc (row-major, entry (a, b) at jc p p + a p + b) into the bf16 digit images that
// kt_baxpy copies into a shared-memory B stage: for block jc, N-tile t = b / NC and chunk c = a / 16, an image of
// tc_stage_b<NC>() bytes at ((jc (p/NC) + t) (p/16) + c) of 8 slices, entry (b, a) at the core-matrix position of
// tc_store8 (row b mod NC, k-group (a mod 16) / 8, element a mod 8). Cexp[jc p + b] = F_b. One thread per column
// (jc, b).
template <int NC>
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
  const int nt = p / NC, nc = p / kTcK, t = b / NC, bl = b % NC;
  for (int a = 0; a < p; ++a) {
    const double v = Cj[(size_t)a * p + b];
    const unsigned long long fx = tc_fixed48(v, F);
    const uint32_t sg = signbit(v) ? 0x8000u : 0u;
    const int c = a / kTcK, al = a % kTcK;
    const size_t img = ((size_t)(jc * nt + t) * nc + c) * tc_stage_b<NC>();
    const size_t in_slice = (size_t)((bl >> 3) * (kTcK / 8) + (al >> 3)) * 128 + (bl & 7) * 16 + (al & 7) * 2;
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i)
      Cs[(img + (size_t)i * tc_slice_b<NC>() + in_slice) / 2] = (uint16_t)tc_bf16_digit(tc_digit(fx, i), sg);
  }
}

// Block-diagonal 64 x 64 matrices from p x p blocks (p = 16 or 32): out block o (row-major) holds blocks
// o (64 / p) .. o (64 / p) + 64 / p - 1 of C on its diagonal (global: block 0 of C in every position) and zeros
// elsewhere, so that 64 / p blocks of columns are updated by one 64-column tile. One thread per entry.
__global__ void kt_pair_cmat(const double *__restrict__ C, int nout, int p, int global, double *__restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nout * 64 * 64) return;
  const int o = idx >> 12, a = (idx >> 6) & 63, b = idx & 63;
  const int ba = a / p, bb = b / p;
  double v = 0.0;
  if (ba == bb) {
    const int jc = global ? 0 : o * (64 / p) + ba;
    v = C[(size_t)jc * p * p + (size_t)(a - ba * p) * p + (b - bb * p)];
  }
  out[idx] = v;
}

// ---- Gram ------------------------------------------------------------------------------------------------------
// Column exponent fields for the Gram slicing: ecol[c] = max over rows of the biased exponent of X[r][c] (times
// xscale[r] if given), by integer maxima (the caller zeroes ecol). Thread (g, c) covers rows g, g + rows per CTA
// pass, ... of column c.
// (FP32 data, the mixed form's process: the exponent fields in FP64's bias, so the same images and kernels serve.)
template <typename T>
__global__ void __launch_bounds__(kNT) kt_col_exp(const T *__restrict__ X, const T *__restrict__ xscale,
                                                  int64_t n, int k, int *__restrict__ ecol) {
  const int rpp = kNT / k;
  const int g = threadIdx.x / k, c = threadIdx.x - g * k;
  if (g >= rpp) return;
  int em = 0;
  for (int64_t r = (int64_t)blockIdx.x * rpp + g; r < n; r += (int64_t)gridDim.x * rpp) {
    const T v = xscale ? X[r * k + c] * xscale[r] : X[r * k + c];
    em = max(em, tc_exp_field(v));
  }
  atomicMax(ecol + c, em);
}

// ---- Digit images in global memory ------------------------------------------------------------------------------
// Cutting the operands inside the MMA kernels (one CTA per output tile) would cut an operand feeding several
// output tiles once per tile (4 times for the Gram's X at p = 256), on the integer pipe, while the tensor pipe
// waits. So every operand is cut once per use into HBM images that are byte-for-byte shared-memory stages, and the
// MMA kernels fill their stages with bulk copies (cp.async.bulk, completion counted on an mbarrier).
//   row images (BAXPY's Y, one exponent per row of a block): 32 KB per (128-row tile rt, 16-column chunk kc of
//     k), the A stage of kt_baxpy_img: image (rt, kc) at (rt (k/16) + kc) 32 KB; erow[j * nrows + r] = E_r of
//     block j (kTcBadRow: a non-finite value in the row).
//   column images (the Gram's operands, one exponent per column over all rows): 16 KB per (64-column tile ct,
//     16-row chunk rc), the B stage of kt_gram_img; image (ct, rc) at (ct nrc + rc) 16 KB, nrc = ceil(n / 16). An
//     A stage of 128 columns is the two 64-column images side by side in every 4 KB slice.
constexpr int kTcBadRow = 0x7FFFFFFF;
constexpr uint32_t kTcImgRow = kTcStageBytesA;   // 32 KB
constexpr uint32_t kTcImgCol = kTcStageBytesB;   // 16 KB

__host__ __device__ constexpr size_t tc_row_image_bytes(int64_t n, int k) {
  return (size_t)((n + kTcRows - 1) / kTcRows) * (k / kTcK) * kTcImgRow;
}
__host__ __device__ constexpr size_t tc_col_image_bytes(int64_t n, int k) {
  return (size_t)((n + kTcK - 1) / kTcK) * (k / kTcCols) * kTcImgCol;
}

// 8 consecutive values (16-byte aligned) as T
__device__ __forceinline__ void tc_load8(const double *src, double (&v)[8]) {
  const double2 *q = reinterpret_cast<const double2 *>(src);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 t = __ldg(q + e);
    v[2 * e] = t.x;
    v[2 * e + 1] = t.y;
  }
}
__device__ __forceinline__ void tc_load8(const float *src, float (&v)[8]) {
  const float4 *q = reinterpret_cast<const float4 *>(src);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float4 t = __ldg(q + e);
    v[4 * e] = t.x;
    v[4 * e + 1] = t.y;
    v[4 * e + 2] = t.z;
    v[4 * e + 3] = t.w;
  }
}

// Row images of Y for every block j: CTA (rt, j) computes the 128 row exponents of its rows over the block's p
// columns (integer maxima of the exponent fields) and cuts the p / 16 chunks. T = double, or float (the mixed
// form's FP32 process; its values are exact in the 48-bit window where a row's exponents span at most 24).
template <typename T>
__global__ void __launch_bounds__(kTcThreads) kt_cut_rows(const T *__restrict__ Y, int64_t n, int k, int p,
                                                          unsigned char *__restrict__ img, int *__restrict__ erow) {
  __shared__ int sE[kTcRows];
  const int tid = threadIdx.x;
  const int64_t rt = blockIdx.x;
  const int j = blockIdx.y;
  const int64_t r0 = rt * kTcRows;
  const int64_t nrows = ((n + kTcRows - 1) / kTcRows) * kTcRows;
  {   // row exponents: warp w takes rows w, w + 8, ..., each read whole by the warp (coalesced), max by shuffles
    const int warp = tid >> 5, lane = tid & 31;
    for (int rl = warp; rl < kTcRows; rl += kTcThreads / 32) {
      const int64_t r = r0 + rl;
      int em = 0;
      if (r < n) {
        const T *src = Y + r * k + (int64_t)j * p;
#pragma unroll 8
        for (int q = lane; q < p; q += 32) em = max(em, tc_exp_field(__ldg(src + q)));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
      if (lane == 0) {
        const int E = em > 0 ? em - 1023 : -1023;
        sE[rl] = E;
        erow[(int64_t)j * nrows + r] = em == 0x7FF ? kTcBadRow : E;
      }
    }
    __syncthreads();
  }
  constexpr int kItems = kTcRows * (kTcK / 8);   // (row, 8-value k-group) items of a chunk
  for (int kc = 0; kc < p / kTcK; ++kc) {
    unsigned char *dst = img + ((size_t)rt * (k / kTcK) + (size_t)j * (p / kTcK) + kc) * kTcImgRow;
#pragma unroll
    for (int u = 0; u < (kItems + kTcThreads - 1) / kTcThreads; ++u) {
      const int it = tid + u * kTcThreads, rl = it & (kTcRows - 1), kg = it >> 7;
      if (it >= kItems) break;
      const int64_t r = r0 + rl;
      T v[8];
      if (r < n) {
        tc_load8(Y + r * k + (int64_t)j * p + kc * kTcK + kg * 8, v);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = T(0);
      }
      uint32_t w[kTcSlices][4];
      tc_pack8(v, sE[rl], w);
      tc_store8(dst, kTcSliceBytesA, rl, kg, w);
    }
  }
}

// Column images of X (rows times xscale[r] if given) with the column exponent fields ecol (kt_col_exp): CTA
// (ct, y) cuts the 64 columns of tile ct over the row chunks y, y + gridDim.y, ...
template <typename T>
__global__ void __launch_bounds__(kTcThreads) kt_cut_cols(const T *__restrict__ X, const T *__restrict__ xscale,
                                                          int64_t n, int k, const int *__restrict__ ecol,
                                                          unsigned char *__restrict__ img) {
  const int tid = threadIdx.x;
  const int ct = blockIdx.x;
  constexpr int kItems = kTcCols * (kTcK / 8);   // (column, 8-row k-group) items of a chunk
  constexpr int kPer = kTcThreads / kItems;      // chunks per pass of the CTA
  const int item = tid % kItems, sub = tid / kItems;
  const int col = item & (kTcCols - 1), kg = item >> 6;
  const int c = ct * kTcCols + col;
  const int E = (ecol[c] > 0 ? ecol[c] : 1) - 1023;
  const int64_t nrc = (n + kTcK - 1) / kTcK;
  for (int64_t rc = (int64_t)blockIdx.y * kPer + sub; rc < nrc; rc += (int64_t)gridDim.y * kPer) {
    T v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t r = rc * kTcK + kg * 8 + e;
      v[e] = r < n ? (xscale ? X[r * k + c] * xscale[r] : X[r * k + c]) : T(0);
    }
    uint32_t w[kTcSlices][4];
    tc_pack8(v, E, w);
    tc_store8(img + ((size_t)ct * nrc + rc) * kTcImgCol, kTcSliceBytesB, col, kg, w);
  }
}

// Roles in the image kernels: thread 32 (warp 1, lane 0) is the producer -- it fills the kTcStages shared-memory
// stages with bulk copies of the images; thread 0 issues the MMAs. Chunk g (counted over the whole launch) uses
// stage g mod kTcStages, and its "full" mbarrier (copies in) and "empty" mbarrier (its MMAs complete, by
// tcgen05.commit) complete for the (g / kTcStages)-th time, so the parity of every wait follows from g alone. The
// producer refills a stage once the MMAs of the chunk kTcStages before have completed, so copies run up to
// kTcStages chunks ahead of the tensor cores; a "done" mbarrier (one commit after the last chunk of a tile or
// window) tells thread 0 that the accumulators are complete. Every wait is bounded (kTcWaitLimit polls); a
// timeout sets a flag that ends the kernel for the whole CTA after both roles have waited (bounded) for their own
// copies and MMAs in flight.
constexpr int kTcProducer = 32;

struct TcBars {
  uint32_t full[kTcStages], empty[kTcStages], done;
};
__device__ __forceinline__ TcBars tc_bars_setup(unsigned char *misc) {
  uint64_t *bars = reinterpret_cast<uint64_t *>(misc + 256);
  TcBars b;
  for (int s = 0; s < kTcStages; ++s) {
    b.full[s] = smem_u32(bars + s);
    b.empty[s] = smem_u32(bars + kTcStages + s);
  }
  b.done = smem_u32(bars + 2 * kTcStages);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(b.full[s], 1);
      mbar_init(b.empty[s], 1);
    }
    mbar_init(b.done, 1);
    fence_mbar_init();
  }
  __syncthreads();
  return b;
}
__device__ __forceinline__ uint32_t tc_par(int64_t g) { return (uint32_t)((g / kTcStages) & 1); }

// Roles in kt_baxpy_img: warps 0-7 read the accumulators out (warp w: TMEM lanes 32 (w mod 4) .. +31, the tile's
// rows, and the tile's columns 32 (w / 4) .. +31), lane 0 of warp 8 issues the MMAs, lane 0 of warp 9 issues the
// bulk copies. TMEM holds the 8 accumulators of one tile: the readout warps fold them into float pairs in registers
// and release TMEM (the "free" mbarrier, one arrival per readout warp) before they turn the pairs into doubles, add
// BASE and store, so that this part of the readout overlaps the next tile's MMAs.
constexpr int kTcOutWarps = 8;
constexpr int kTcBaxThreads = (kTcOutWarps + 2) * 32;
constexpr int kTcBaxMma = kTcOutWarps * 32;
constexpr int kTcBaxProducer = kTcBaxMma + 32;

// 16 consecutive values (16-byte aligned) of OUT / BASE, widened to double, and back
__device__ __forceinline__ void tc_load16(const double *src, double (&v)[16]) {
  const double2 *q = reinterpret_cast<const double2 *>(src);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const double2 t = q[e];
    v[2 * e] = t.x;
    v[2 * e + 1] = t.y;
  }
}
__device__ __forceinline__ void tc_load16(const float *src, double (&v)[16]) {
  const float4 *q = reinterpret_cast<const float4 *>(src);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float4 t = q[e];
    v[4 * e] = t.x;
    v[4 * e + 1] = t.y;
    v[4 * e + 2] = t.z;
    v[4 * e + 3] = t.w;
  }
}
__device__ __forceinline__ void tc_store16(double *dst, const double (&v)[16]) {
  double2 *q = reinterpret_cast<double2 *>(dst);
#pragma unroll
  for (int e = 0; e < 8; ++e) q[e] = make_double2(v[2 * e], v[2 * e + 1]);
}
__device__ __forceinline__ void tc_store16(float *dst, const double (&v)[16]) {
  float4 *q = reinterpret_cast<float4 *>(dst);
#pragma unroll
  for (int e = 0; e < 4; ++e)
    q[e] = make_float4((float)v[4 * e], (float)v[4 * e + 1], (float)v[4 * e + 2], (float)v[4 * e + 3]);
}

// OUT_j = BASE_j (times bscale[r] per row, if given; BASE NULL: zero) + sign * Y_j C_j over every block j (global: C_0
// for all), from Y's row images (kt_cut_rows) and C's images (kt_slice_cmat). OUT may equal BASE. T = double, or
// float (the mixed form's FP32 process: the sum is formed in FP64 and rounded once). pe: the width of the column
// blocks that own a row exponent (p; or 16 or 32 where blocks of that width are paired into 64-column tiles with
// block-diagonal C images, kt_pair_cmat: each output column then sums over its own block's digits only). Frozen blocks
// (active[j] = 0) get OUT = BASE (scaled). bump: CTA 0 advances the iteration counter (the P update's role).
// Persistent over 128 x NC output tiles (tile t: row tile t / (k / NC), column tile t mod (k / NC); NC = 64, or 32
// for blocks of 32 columns that are not paired); every role walks the CTA's tiles in the same order, the issuing
// roles skipping frozen blocks.
template <typename T, int NC>
__global__ void __launch_bounds__(kTcBaxThreads, 1) kt_baxpy_img(T *OUT, const T *BASE,
                                                                 const unsigned char *__restrict__ imgY,
                                                                 const int *__restrict__ erow,
                                                                 const uint16_t *__restrict__ Cs,
                                                                 const int *__restrict__ Cexp, int64_t n, int k,
                                                                 int p, int global, double sign,
                                                                 const int *__restrict__ active,
                                                                 DevStatus *__restrict__ st, int bump,
                                                                 const T *__restrict__ bscale, int pe) {
  if (st->flags != 0) return;
  if (bump && blockIdx.x == 0 && threadIdx.x == 0) st->cur += 1;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  unsigned char *ops, *misc;
  const uint32_t tbase = tc_setup(tc_smem_raw, ops, misc);
  const TcBars bars = tc_bars_setup(misc);
  const uint32_t tfree = smem_u32(reinterpret_cast<uint64_t *>(misc + 256) + 2 * kTcStages + 1);
  volatile int *sFlag = reinterpret_cast<volatile int *>(misc + 512);   // [0]: a wait gave up
  long long *sCount = reinterpret_cast<long long *>(misc + 576);       // chunks copied [0] and consumed [1]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int CPT = NC / 2;   // columns per readout thread (two warps per TMEM lane quadrant)
  const int nt = p / NC, nc = p / kTcK;
  const int ntn = k / NC;
  const int64_t nrt = (n + kTcRows - 1) / kTcRows;
  const int64_t nrows = nrt * kTcRows;
  const int64_t ntiles = nrt * ntn;
  if (tid == 0) {
    mbar_init(tfree, kTcOutWarps);
    fence_mbar_init();
    sFlag[0] = 0;
    sCount[0] = sCount[1] = 0;
  }
  __syncthreads();
  auto tile_active = [&](int64_t t) { return block_active(active, global, (int)(t % ntn) * NC / p); };
  auto next_active = [&](int64_t t) {
    while (t < ntiles && !tile_active(t)) t += gridDim.x;
    return t;
  };
  if (tid == kTcBaxProducer) {   // chunk g of the launch into stage g mod kTcStages, once its last MMAs are done
    int64_t g = 0;
    bool ok = true;
    for (int64_t tile = next_active(blockIdx.x); tile < ntiles && ok; tile = next_active(tile + gridDim.x)) {
      const int c0 = (int)(tile % ntn) * NC, j = c0 / p, b0 = c0 - j * p, jc = global ? 0 : j;
      const unsigned char *cimg =
          reinterpret_cast<const unsigned char *>(Cs) + (size_t)(jc * nt + b0 / NC) * nc * tc_stage_b<NC>();
      const unsigned char *yimg = imgY + ((size_t)(tile / ntn) * (k / kTcK) + (size_t)j * nc) * kTcImgRow;
      for (int c = 0; c < nc; ++c, ++g) {
        const int s = (int)(g % kTcStages);
        if (g >= kTcStages && !mbar_wait_flag(bars.empty[s], tc_par(g - kTcStages), sFlag)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(bars.full[s], kTcImgRow + tc_stage_b<NC>());
        bulk_g2s(smem_u32(tc_stage_a(ops, s)), yimg + (size_t)c * kTcImgRow, kTcImgRow, bars.full[s]);
        bulk_g2s(smem_u32(tc_stage_b(ops, s)), cimg + (size_t)c * tc_stage_b<NC>(), tc_stage_b<NC>(), bars.full[s]);
      }
    }
    if (!ok) sFlag[0] = 1;
    sCount[0] = g;
  } else if (tid == kTcBaxMma) {   // a tile's MMAs once the previous tile's accumulators are folded
    int64_t g = 0, i = 0;
    bool ok = true;
    for (int64_t tile = next_active(blockIdx.x); tile < ntiles && ok; tile = next_active(tile + gridDim.x), ++i) {
      if (i > 0 && !mbar_wait_flag(tfree, (uint32_t)((i - 1) & 1), sFlag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int c = 0; c < nc; ++c, ++g) {
        const int s = (int)(g % kTcStages);
        if (!mbar_wait_flag(bars.full[s], tc_par(g), sFlag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        tc_issue_chunk<NC>(tbase, smem_u32(tc_stage_a(ops, s)), smem_u32(tc_stage_b(ops, s)), c == 0);
        tc_commit(bars.empty[s]);
      }
      if (ok) tc_commit(bars.done);
    }
    if (!ok) sFlag[0] = 1;
    sCount[1] = g;
  } else if (warp < kTcOutWarps) {
    const int q = warp & 3, cb0 = (warp >> 2) * CPT;   // TMEM lane quadrant; first of the thread's CPT columns
    const int rl = q * 32 + lane;
    int64_t i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int c0 = (int)(tile % ntn) * NC, j = c0 / p, b0 = c0 - j * p, jc = global ? 0 : j;
      const int64_t r = (tile / ntn) * kTcRows + rl;
      if (!block_active(active, global, j)) {   // frozen block: OUT = BASE (scaled)
        if (r < n) {
          const T s = bscale ? bscale[r] : T(1);
          for (int e = 0; e < CPT; ++e) OUT[r * k + c0 + cb0 + e] = BASE ? BASE[r * k + c0 + cb0 + e] * s : T(0);
        }
        continue;
      }
      // lane 0 waits for the tile's MMAs; the warp follows it (the TMEM loads are warp-collective)
      bool ok = lane == 0 ? mbar_wait_flag(bars.done, (uint32_t)(i & 1), sFlag) : true;
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) sFlag[0] = 1;
        break;
      }
      ++i;
      tc_fence_after();
      float hi[CPT / 8][8], lo[CPT / 8][8];
#pragma unroll
      for (int cg = 0; cg < CPT / 8; ++cg) tc_read8<NC>(tbase, q, cb0 + cg * 8, hi[cg], lo[cg]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tfree);
      if (r >= n) continue;
      // (s + c) 2^t as one double (integer operations), one FP64 addition; 16 columns at a time, their BASE
      // values loaded before any store (OUT may be BASE). Row exponents per pe columns: columns cb0 .. +15 take
      // Eh[0], cb0 + 16 .. +31 (CPT = 32) take Eh[1] (the same value unless pe = 16).
      const int e0 = erow[(int64_t)((c0 + cb0) / pe) * nrows + r];
      const int Eh[2] = {e0, CPT > 16 ? erow[(int64_t)((c0 + cb0 + 16) / pe) * nrows + r] : e0};
      const double bs = bscale ? (double)bscale[r] : 1.0;
      const int4 *F4 = reinterpret_cast<const int4 *>(Cexp + jc * p + b0 + cb0);
#pragma unroll
      for (int half = 0; half < CPT / 16; ++half) {
        const int E = Eh[half];
        const bool bad = E == kTcBadRow;
        double v[16];
        if (BASE) {
          tc_load16(BASE + r * k + c0 + cb0 + half * 16, v);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.0;
        }
#pragma unroll
        for (int cg2 = 0; cg2 < 2; ++cg2) {
          const int cg = half * 2 + cg2;
          const int4 fa = __ldg(F4 + 2 * cg), fb = __ldg(F4 + 2 * cg + 1);
          const int F[8] = {fa.x, fa.y, fa.z, fa.w, fb.x, fb.y, fb.z, fb.w};
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const double base = bscale ? v[cg2 * 8 + e] * bs : v[cg2 * 8 + e];
            const double x = base + sign * df_pair_to_double(hi[cg][e], lo[cg][e], E + F[e] - 10);
            v[cg2 * 8 + e] = bad ? __longlong_as_double(0x7FF8000000000000ll) : x;
          }
        }
        tc_store16(OUT + r * k + c0 + cb0 + half * 16, v);
      }
    }
  }
  __syncthreads();
  const bool timeout = sFlag[0] != 0;
  if (timeout) {   // both issuing roles wait (bounded) for what they started
    if (tid == kTcBaxProducer)
      for (int64_t g = sCount[1]; g < sCount[0]; ++g) (void)mbar_wait(bars.full[g % kTcStages], tc_par(g));
    if (tid == kTcBaxMma && sCount[1] > 0)
      (void)mbar_wait(bars.empty[(sCount[1] - 1) % kTcStages], tc_par(sCount[1] - 1));
  }
  tc_teardown(tbase, timeout, st);
}

// kt_gram with the column images of X and Y (kt_cut_cols; the same image may serve both): CTA (tile, y) covers the
// 128 x 64 entries (a in [128 ta, 128 ta + 128), b in [64 tb, 64 tb + 64)) of block j over the 16-row chunks of
// partial row y, and writes them into partial row y in the layout of kl_gram (entry (a, b) of block j at
// j p p + b p + a); rows of the tile with a >= p are zero and not written. ecx, ecy: the column exponent fields
// the images were cut with. Frozen blocks get zero partials. The accumulators are read out into float pairs every
// kTcWindow rows.
__global__ void __launch_bounds__(kTcThreads, 1) kt_gram_img(const unsigned char *__restrict__ imgX,
                                                             const unsigned char *__restrict__ imgY, int64_t n, int k,
                                                             int p, int global, const int *__restrict__ active,
                                                             double *__restrict__ part, const int *__restrict__ ecx,
                                                             const int *__restrict__ ecy, DevStatus *__restrict__ st) {
  if (st != nullptr && st->flags != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ta_n = (p + kTcRows - 1) / kTcRows, tb_n = p / kTcCols;
  const int j = blockIdx.x / (ta_n * tb_n), ta = (blockIdx.x / tb_n) % ta_n, tb = blockIdx.x % tb_n;
  const int a0 = ta * kTcRows, b0 = tb * kTcCols;
  double *out = part + (size_t)blockIdx.y * k * p + (size_t)j * p * p;
  const int q = warp & 3, h = warp >> 2;
  const int al = q * 32 + lane;
  if (!block_active(active, global, j)) {
    if (a0 + al < p)
      for (int e = 0; e < 32; ++e) out[(size_t)(b0 + h * 32 + e) * p + a0 + al] = 0.0;
    return;
  }
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  unsigned char *ops, *misc;
  const uint32_t tbase = tc_setup(tc_smem_raw, ops, misc);
  const bool two = a0 + kTcCols < p;   // the A stage's second 64 columns exist (else they stay zero)
  if (!two) {   // zero the upper halves of all A stages once; the bulk copies never write them
    for (int s2 = 0; s2 < kTcStages; ++s2)
      for (int i = 0; i < kTcSlices; ++i) {
        uint4 *z = reinterpret_cast<uint4 *>(tc_stage_a(ops, s2) + i * kTcSliceBytesA + kTcSliceBytesB);
        for (int e = tid; e < (int)(kTcSliceBytesB / 16); e += kTcThreads) z[e] = make_uint4(0, 0, 0, 0);
      }
    fence_async_smem();
  }
  const TcBars bars = tc_bars_setup(misc);
  int *sFlag = reinterpret_cast<int *>(misc + 512);
  if (tid == 0) sFlag[0] = 0;
  __syncthreads();
  const int64_t nrc = (n + kTcK - 1) / kTcK;
  const int64_t per = (nrc + gridDim.y - 1) / gridDim.y;
  const int64_t rc_begin = (int64_t)blockIdx.y * per, rc_end = min(nrc, rc_begin + per);
  const int64_t nch = rc_end > rc_begin ? rc_end - rc_begin : 0;
  const int ctA = (j * p + a0) / kTcCols, ctB = (j * p + b0) / kTcCols;
  const uint32_t bytesA = (two ? 2u : 1u) * kTcSlices * kTcSliceBytesB;
  float rs[32], rc[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) rs[e] = rc[e] = 0.0f;
  bool timeout = false;
  constexpr int kWin = kTcWindow / kTcK;   // chunks per accumulator window
  int64_t gprod = 0, gcons = 0, ndone = 0;
  auto produce_until = [&](int64_t upto) -> bool {   // producer: chunks gprod .. upto - 1
    for (; gprod < upto; ++gprod) {
      const int s = (int)(gprod % kTcStages);
      if (gprod >= kTcStages && !mbar_wait(bars.empty[s], tc_par(gprod - kTcStages))) return false;
      const int64_t r = rc_begin + gprod;
      mbar_arrive_expect_tx(bars.full[s], bytesA + kTcImgCol);
      const unsigned char *xa = imgX + ((size_t)ctA * nrc + r) * kTcImgCol;
      const unsigned char *xb = imgX + ((size_t)(ctA + 1) * nrc + r) * kTcImgCol;
      const uint32_t sa = smem_u32(tc_stage_a(ops, s));
#pragma unroll
      for (int i = 0; i < kTcSlices; ++i) {
        bulk_g2s(sa + i * kTcSliceBytesA, xa + i * kTcSliceBytesB, kTcSliceBytesB, bars.full[s]);
        if (two) bulk_g2s(sa + i * kTcSliceBytesA + kTcSliceBytesB, xb + i * kTcSliceBytesB, kTcSliceBytesB, bars.full[s]);
      }
      bulk_g2s(smem_u32(tc_stage_b(ops, s)), imgY + ((size_t)ctB * nrc + r) * kTcImgCol, kTcImgCol, bars.full[s]);
    }
    return true;
  };
  for (int64_t c0 = 0; c0 < nch && !timeout; c0 += kWin) {   // one accumulator window per pass
    const int64_t c1 = min(nch, c0 + kWin);
    // the producer may run kTcStages chunks past the window: those wait only for MMAs of this window
    if (tid == kTcProducer && !sFlag[0] && !produce_until(min(nch, c1 + kTcStages))) sFlag[0] = 1;
    if (tid == 0) {
      bool ok = true;
      for (; gcons < c1 && ok; ++gcons) {
        const int s = (int)(gcons % kTcStages);
        ok = mbar_wait(bars.full[s], tc_par(gcons)) && !*(volatile int *)sFlag;
        if (!ok) break;
        tc_fence_after();
        tc_issue_chunk(tbase, smem_u32(tc_stage_a(ops, s)), smem_u32(tc_stage_b(ops, s)), gcons == c0);
        tc_commit(bars.empty[s]);
      }
      if (ok) {
        tc_commit(bars.done);
        ok = mbar_wait(bars.done, (uint32_t)(ndone & 1));
        ++ndone;
      }
      if (!ok) sFlag[0] = 1;
    }
    __syncthreads();
    if (sFlag[0]) {
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
  if (timeout) {   // both roles wait (bounded) for what they started
    __shared__ long long sCons;
    if (tid == 0) sCons = gcons;
    __syncthreads();
    if (tid == kTcProducer)
      for (int64_t g = sCons; g < gprod; ++g) (void)mbar_wait(bars.full[g % kTcStages], tc_par(g));
    if (tid == 0 && gcons > 0) (void)mbar_wait(bars.empty[(gcons - 1) % kTcStages], tc_par(gcons - 1));
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
