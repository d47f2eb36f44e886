// C ABI of libbcg.so (declared in include/bcg.h) and the host-side iteration driver.
//
// One solve is: K0 (R = B - A X, P = M^{-1} R, ||R^0_c||^2) and a status reset, then iterations of
//   K1  Q = A P, alpha = <<P,Q>>, rho_rec = <<P,R>>        (BOP + 2 BDOT, Algorithm 1)
//   K4a lambda = alpha^{-1} rho_rec                          (BSOLVE, Cholesky)
//   K2  X += P lambda, R -= Q lambda, rho = <<Z,R>>, ||R_c|| (2 BAXPY + BDOT)
//   K4b stopping test, beta = rho_rec^{-1} rho                (BSOLVE, LU with partial pivoting)
//   K3  P = Z + P beta                                        (BAXPY)
// launched in batches of `check_every` iterations (optionally replayed as one CUDA graph) between two
// host reads of the device status word; once the device has flagged completion the remaining kernels
// of a batch return immediately. For FP64 with 2 <= p <= 16 the recomputed rho_rec of the next iteration
// is formed by K3 instead of K1 (and the first one by a BDOT after K0). p > 32 runs tiled kernels with the
// same roles. The mixed form (FP32_REFINE) runs the same iteration in FP32 with FP64 residual replacement
// (solve_replace) or restarted refinement (solve_refine); SELL handles iterate on the permuted system;
// row-sharded handles are driven phase by phase by the caller (bcg_rows_*).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/bcg.h"
#include "bcg_launch.h"

using namespace bcgk;

namespace {

thread_local std::string g_last_error;

bcg_status fail(bcg_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? BCG_ERR_OOM : BCG_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
  } while (0)

#define CKS(expr)                        \
  do {                                   \
    bcg_status s_ = (expr);              \
    if (s_ != BCG_OK) return s_;         \
  } while (0)

bool is_device_ptr(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Lets the other C ABI translation unit (bcg_noalloc.cu) report through bcg_last_error.
void bcg_internal_set_error(const char *msg) { g_last_error = msg; }

namespace {
// Allocation-failure injection for tests (bcg_debug_fail_alloc): the armed count of workspace allocations still
// to succeed before one fails (0: disarmed).
std::atomic<int> g_fail_alloc_in{0};
// Guard bytes after every workspace buffer (checked with option "guards")
constexpr int kGuardBytes = 16;
constexpr unsigned char kGuardByte = 0xA5;

bool injected_alloc_failure() {
  int v = g_fail_alloc_in.load();
  while (v > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(v, v - 1)) return v == 1;
  }
  return false;
}

// NVTX range for the lifetime of a scope (the library's phases and kernel launches; host-side markers that a
// profiler shows on the timeline, free when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct bcg_ctx {
  // problem
  int64_t n = 0, nnz = 0;
  int64_t ncols = 0;                   // operator columns: n, or own + halo rows of a row-sharded handle
  int rows_mode = 0;                   // 1: row-sharded handle (bcg_create_csr_rows), driven by bcg_rows_*
  double *sums1 = nullptr, *sums2 = nullptr;   // row-sharded: caller's buffers of the sums exchanged between ranks
  double *X_rows = nullptr;            // row-sharded: the caller's X of the current solve (borrowed)
  const int32_t *perm = nullptr;       // SELL: row of the original system held by permuted row s (borrowed)
  double *Bp = nullptr, *Xp = nullptr; // SELL: B and X in the permuted row order
  double *tol2_dev = nullptr;          // squared stopping tolerance of the running solve (device, read by K4b)
  double *h_tol2 = nullptr;            // pinned staging for it
  int k = 0, p = 0, global = 0, nblk = 0, prec = BCG_FP64;
  int opkind = OP_CSR;
  OpDesc A64{}, A32{};
  int64_t ncoef = 0;                   // length of vals (CSR) or faces (varcoef), 0 otherwise
  cudaStream_t stream = nullptr;
  int nsm = 0;
  StreamGrids g64{}, g32{};
  int nparts = 0;                      // partial-buffer rows (max CTAs of K0/K1/K2)
  // options
  double inner_tol = 3e-5;             // 2-7 % fewer inner iterations than 1e-5 on the benchmark problems
  int max_outer = 30;
  int check_every = 8;
  int use_graph = 1;
  int profile = 0;
  int precond = 0;                     // 0: M = I; 1: Jacobi, M = diag(A)
  int refine = 1;                      // FP32_REFINE: 1 residual replacement, 0 restarted refinement
  int retooled = 0;                    // FP64: 1 Dubrulle's retooled block CG instead of Algorithm 1's recurrences
  int tensor_cores = 1;                // FP64, p a multiple of 64 or p = 32: tcgen05 kernels
  int guards = 0;                      // 1: check every buffer's guard bytes after each solve
  // live per-kernel timing (profile = 1): CUDA events around every launch of an executed iteration
  // K1 op_gram, K4a solve_lambda, K2 update_xr, K4b solve_beta, K3 update_p, K0 residual, and the tensor-core
  // block products and block updates of wide blocks (kt_gram_img, kt_baxpy_img)
  static constexpr int kKernels = 8;
  double prof_ms[kKernels] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t prof_count[kKernels] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev;         // 2 * 5 * check_every events, reused per batch
  // workspace (owned)
  std::vector<void *> allocs;
  std::vector<size_t> alloc_bytes;     // requested size of each allocation; 16 guard bytes follow it
  double *R = nullptr, *P = nullptr, *Q = nullptr;           // FP64 iteration vectors
  float *R32 = nullptr, *P32 = nullptr, *Q32 = nullptr, *D32 = nullptr;
  void *vals32 = nullptr;              // FP32 copy of CSR values or faces
  double *partA = nullptr, *partR = nullptr, *partRho = nullptr, *partN = nullptr;
  double *lam = nullptr, *beta = nullptr, *rho_rec = nullptr;
  double *r0n2 = nullptr, *rn2 = nullptr, *rtn2 = nullptr, *outer0 = nullptr;
  int *active = nullptr, *block_iters = nullptr;
  int *sh = nullptr;                   // exponent shifts of the FP64 Gram operands, 3 k ints (roles R, P, Q)
  double *opmax = nullptr;             // [max row sum of |A|, max |diag(A)^{-1}|] (offsets of the P and Q shifts)
  double *tmp2k = nullptr;             // 2 k doubles: standalone BDOT column maxima, the mixed form's scaled norms
  int *bdot_sh = nullptr;              // standalone BDOT: their shifts (2 k)
  int *msig = nullptr;                 // mixed form: exponent of the FP32 process's scale per column (k)
  double *gws = nullptr;               // global workspace of the p x p solves when p is large
  uint16_t *tc_cs = nullptr;           // tensor-core block updates: bf16 digit images of lambda or beta
  int *tc_cexp = nullptr;              // their column exponents
  int *tc_ecol = nullptr;              // tensor-core block products: the operands' column exponent fields (2 k)
  unsigned char *tc_img[4] = {nullptr, nullptr, nullptr, nullptr};   // digit images: 2 column, 2 row images
  int *tc_erow = nullptr;              // row exponents of the two row images (2 ceil(n / 128) 128 (k / p))
  int tc_small = 0;                    // FP64 blocks of 32 with their block updates on the tensor cores
  double *tc_pair = nullptr;           // the paired block-diagonal 64 x 64 lambda / beta of those (64 | k)
  double *dinv64 = nullptr;            // 1 / diag(A) (Jacobi preconditioner)
  double *dr_C = nullptr, *dr_xi = nullptr, *dr_psiinv = nullptr, *dr_phi = nullptr;   // retooled form, p x p per block
  float *dinv32 = nullptr;             // its FP32 copy for the mixed form's inner solve
  int32_t *rowidx = nullptr;           // CSR row of each entry (gradient)
  DevStatus *st = nullptr;
  DevStatus *h_st = nullptr;           // pinned
  double *h_vec = nullptr;             // pinned, 3k doubles
  int *h_iters = nullptr;              // pinned, nblk ints
  double *stageB = nullptr, *stageX = nullptr;  // bcg_solve_host staging
  // graph of one batch of inner FP32 iterations (workspace pointers only, so reusable)
  cudaGraphExec_t graph32 = nullptr;
  int graph32_batch = 0;
  std::vector<int> last_block_iters;

  template <typename U>
  bcg_status alloc(U **ptr, size_t count) {
    if (injected_alloc_failure())
      return fail(BCG_ERR_OOM, "cudaMalloc of %zu bytes failed: injected failure (bcg_debug_fail_alloc)",
                  count * sizeof(U));
    void *p_ = nullptr;
    cudaError_t e = cudaMalloc(&p_, count * sizeof(U) + kGuardBytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(BCG_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(U), cudaGetErrorString(e));
    }
    // the guard bytes after the buffer (written before the buffer is first used, on the legacy stream)
    e = cudaMemset(static_cast<unsigned char *>(p_) + count * sizeof(U), kGuardByte, kGuardBytes);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
      cudaFree(p_);
      return fail(BCG_ERR_CUDA, "guard bytes: %s", cudaGetErrorString(e));
    }
    allocs.push_back(p_);
    alloc_bytes.push_back(count * sizeof(U));
    *ptr = static_cast<U *>(p_);
    return BCG_OK;
  }

  ~bcg_ctx() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (graph32) cudaGraphExecDestroy(graph32);
    for (void *a : allocs) cudaFree(a);
    if (h_st) cudaFreeHost(h_st);
    if (h_tol2) cudaFreeHost(h_tol2);
    if (h_vec) cudaFreeHost(h_vec);
    if (h_iters) cudaFreeHost(h_iters);
  }
};

namespace {

bcg_status validate_common(int32_t k, int32_t *p, int32_t sub, int32_t prec, int *global) {
  if (k < 1 || k > kNT) return fail(BCG_ERR_INVALID_ARG, "k=%d out of range 1..%d", k, kNT);
  switch (sub) {
    case BCG_SUB_HYBRID: *global = 0; break;
    case BCG_SUB_GLOBAL: *global = 1; break;
    case BCG_SUB_PARALLEL: *global = 0; *p = 1; break;
    case BCG_SUB_CLASSICAL: *global = 0; *p = k; break;
    default: return fail(BCG_ERR_INVALID_ARG, "unknown subalgebra %d", sub);
  }
  if (*p < 1 || k % *p != 0) return fail(BCG_ERR_INVALID_ARG, "p=%d must divide k=%d", *p, k);
  if (*p > kMaxP && (*p % 32 != 0 || *p > kNT))
    return fail(BCG_ERR_INVALID_ARG, "p=%d: blocks wider than %d must be a multiple of 32 (and <= %d)", *p, kMaxP, kNT);
  if (prec != BCG_FP64 && prec != BCG_FP32_REFINE && prec != BCG_FP64_DF)
    return fail(BCG_ERR_INVALID_ARG, "unknown precision %d", prec);
  return BCG_OK;
}

// Workspace common to both matrix forms; called once A64 is filled in.
bcg_status setup_workspace(bcg_ctx *h) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(small_prepare(h->p));
  CK(stream_grids<double>(h->opkind, h->n, h->k, h->p, h->global, h->nsm, &h->g64));
  // partial rows: every grid that writes them (K0, K1, K2, and K3 for the recomputed rho)
  auto grids_max = [](const StreamGrids &g) {
    return std::max(std::max(std::max(std::max(g.op, g.res), std::max(g.upd, g.upd_zs)), std::max(g.pup, g.pup_zs)),
                    std::max(g.upd_df, g.upd_zs_df));
  };
  int np = grids_max(h->g64);
  if (h->prec == BCG_FP32_REFINE) {
    CK(stream_grids<float>(h->opkind, h->n, h->k, h->p, h->global, h->nsm, &h->g32));
    np = std::max(np, grids_max(h->g32));
  }
  h->nparts = np;
  const size_t nk = (size_t)h->n * h->k;
  const size_t E = (size_t)h->k * h->p;
  const size_t pp = (size_t)h->nblk * h->p * h->p;
  if (h->prec != BCG_FP32_REFINE) {
    // P (and Q, which trades places with P for p > 32) also hold the halo rows of a row-sharded handle
    const size_t nck = (size_t)std::max(h->ncols, h->n) * h->k;
    CKS(h->alloc(&h->R, nk));
    CKS(h->alloc(&h->P, nck));
    CKS(h->alloc(&h->Q, nck));
  } else {
    CKS(h->alloc(&h->Q, nk));   // FP64 outer residual / true-residual scratch
    CKS(h->alloc(&h->R32, nk));
    CKS(h->alloc(&h->P32, nk));
    CKS(h->alloc(&h->Q32, nk));
    CKS(h->alloc(&h->D32, nk));
  }
  CKS(h->alloc(&h->partA, (size_t)np * E));
  CKS(h->alloc(&h->partR, (size_t)np * E));
  CKS(h->alloc(&h->partRho, (size_t)np * E));
  CKS(h->alloc(&h->partN, (size_t)np * h->k));
  CKS(h->alloc(&h->lam, pp));
  CKS(h->alloc(&h->beta, pp));
  CKS(h->alloc(&h->rho_rec, pp));
  CKS(h->alloc(&h->r0n2, h->k));
  CKS(h->alloc(&h->rn2, h->k));
  CKS(h->alloc(&h->rtn2, h->k));
  CKS(h->alloc(&h->outer0, h->k));
  CKS(h->alloc(&h->active, h->nblk));
  CKS(h->alloc(&h->block_iters, h->nblk));
  CKS(h->alloc(&h->sh, 3 * (size_t)h->k));
  CK(cudaMemsetAsync(h->sh, 0, 3 * sizeof(int) * h->k, h->stream));
  CKS(h->alloc(&h->opmax, 2));
  CKS(h->alloc(&h->tmp2k, 2 * (size_t)h->k));
  CKS(h->alloc(&h->bdot_sh, 2 * (size_t)h->k));
  if (h->prec == BCG_FP32_REFINE) CKS(h->alloc(&h->msig, h->k));
  if (small_needs_gws(h->p)) CKS(h->alloc(&h->gws, (size_t)h->nblk * small_ws_doubles(h->p)));
  if (tc_ok(h->k, h->p)) {   // FP64 products and updates; the mixed form's FP32 process uses the products
    CKS(h->alloc(&h->tc_cs, tc_workspace_bytes(h->nblk, h->p) / sizeof(uint16_t)));
    CKS(h->alloc(&h->tc_cexp, (size_t)h->nblk * h->p));
    CKS(h->alloc(&h->tc_ecol, 2 * (size_t)h->k));
    // digit images of the large-block iteration (16 bytes per value each, 4 of them: about 64 n k bytes)
    const size_t ib = std::max(tc_row_image_size(h->n, h->k), tc_col_image_size(h->n, h->k));
    for (int i = 0; i < 4; ++i) CKS(h->alloc(&h->tc_img[i], ib));
    CKS(h->alloc(&h->tc_erow, 2 * (size_t)((h->n + 127) / 128) * 128 * (h->k / h->p)));
  }
  if (h->prec == BCG_FP64 && (tc_pair_ok(h->k, h->p) || tc_b32_ok(h->k, h->p))) {
    // blocks of 32, paired into 64-column tiles where 64 divides k, else in 32-column tiles: the block updates'
    // row images of P and Q (16 bytes per value each) and the digit images of lambda / beta
    h->tc_small = 1;
    if (tc_pair_ok(h->k, h->p)) {
      const int nout = h->global ? 1 : h->k / 64;
      CKS(h->alloc(&h->tc_pair, (size_t)nout * 64 * 64));
      CKS(h->alloc(&h->tc_cs, tc_workspace_bytes(nout, 64) / sizeof(uint16_t)));
      CKS(h->alloc(&h->tc_cexp, (size_t)nout * 64));
    } else {
      CKS(h->alloc(&h->tc_cs, tc_workspace_bytes(h->nblk, h->p) / sizeof(uint16_t)));
      CKS(h->alloc(&h->tc_cexp, (size_t)h->nblk * h->p));
    }
    for (int i = 2; i < 4; ++i) CKS(h->alloc(&h->tc_img[i], tc_row_image_size(h->n, h->k)));
    CKS(h->alloc(&h->tc_erow, 2 * (size_t)((h->n + 127) / 128) * 128 * (h->k / h->p)));
  }
  if (h->prec != BCG_FP32_REFINE) {
    CKS(h->alloc(&h->dr_C, pp));
    CKS(h->alloc(&h->dr_xi, pp));
    CKS(h->alloc(&h->dr_psiinv, pp));
    CKS(h->alloc(&h->dr_phi, pp));
  }
  CKS(h->alloc(&h->dinv64, (size_t)h->n));
  if (h->prec == BCG_FP32_REFINE) CKS(h->alloc(&h->dinv32, (size_t)h->n));
  CKS(h->alloc(&h->st, 1));
  CKS(h->alloc(&h->tol2_dev, 1));
  CK(cudaMallocHost(&h->h_tol2, sizeof(double)));
  CK(cudaMallocHost(&h->h_st, sizeof(DevStatus)));
  CK(cudaMallocHost(&h->h_vec, 3 * sizeof(double) * h->k));
  CK(cudaMallocHost(&h->h_iters, sizeof(int) * h->nblk));
  h->last_block_iters.assign(h->nblk, 0);
  return BCG_OK;
}

bcg_status make_fp32_copy(bcg_ctx *h) {
  CK(launch_inv_diag(h->A64, h->n, h->dinv64, h->opmax, h->nsm, h->stream));
  if (h->dinv32) CK(launch_cast_to_float(h->dinv64, h->dinv32, h->n, h->nsm, h->stream));
  if (h->prec != BCG_FP32_REFINE) return BCG_OK;
  h->A32 = h->A64;
  if (h->ncoef > 0) {
    if (h->vals32 == nullptr) {
      float *v = nullptr;
      CKS(h->alloc(&v, h->ncoef));
      h->vals32 = v;
    }
    const bool by_entry = h->opkind == OP_CSR || h->opkind == OP_SELL;
    const double *src = static_cast<const double *>(by_entry ? h->A64.vals : h->A64.faces);
    CK(launch_cast_to_float(src, static_cast<float *>(h->vals32), h->ncoef, h->nsm, h->stream));
    if (by_entry) h->A32.vals = h->vals32;
    else h->A32.faces = h->vals32;
  }
  return BCG_OK;
}

// Gram shifts of a solve in precision T: the FP64 form keeps them with its column norms; FP32 operands are
// accumulated unshifted.
template <typename T>
ShiftCtl shifts_of(const bcg_ctx *h) {
  ShiftCtl sc;
  if (sizeof(T) == 8) {
    sc.sh = h->sh;
    sc.opmax = h->opmax;
    sc.precond = h->precond;
  }
  return sc;
}

// The K2 / K3 grids of an iteration in precision T, and whether K2 sums R's update in double-float arithmetic
// (precision BCG_FP64_DF, where the shapes allow; the partial-row count of K2 follows the grid used).
template <typename T>
bool df_updates(const bcg_ctx *h, const StreamGrids &g) {
  return sizeof(T) == 8 && h->prec == BCG_FP64_DF && (h->precond ? g.upd_zs_df : g.upd_df) > 0;
}
template <typename T>
int grid_upd(const bcg_ctx *h, const StreamGrids &g) {
  if (df_updates<T>(h, g)) return h->precond ? g.upd_zs_df : g.upd_df;
  return h->precond ? g.upd_zs : g.upd;
}
template <typename T>
int grid_pup(const bcg_ctx *h, const StreamGrids &g) {
  return h->precond ? g.pup_zs : g.pup;
}

template <typename T>
const T *dinv_of(const bcg_ctx *h);
template <>
const double *dinv_of<double>(const bcg_ctx *h) { return h->precond ? h->dinv64 : nullptr; }
template <>
const float *dinv_of<float>(const bcg_ctx *h) { return h->precond ? h->dinv32 : nullptr; }

// The squared tolerance lives in device memory so that a captured batch of iterations serves every solve
// and every refinement step (their tolerances differ). Stream-ordered; the pinned staging value is only
// rewritten after the stream has been synchronised (every solve reads the status word before returning).
bcg_status set_tol2(bcg_ctx *h, double tol2) {
  *h->h_tol2 = tol2;
  CK(cudaMemcpyAsync(h->tol2_dev, h->h_tol2, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  return BCG_OK;
}

// With rho_k3 the first iteration's recomputed rho, <<P^1, R^0>>_S, is a BDOT after K0, on the K3 grid so that
// K4a reads every iteration's partials the same way (later iterations get it from K3).
template <typename T>
bcg_status first_rho_rec(bcg_ctx *h, const T *P, const T *R, const StreamGrids &g) {
  if (!g.rho_k3) return BCG_OK;
  const int *sh = shifts_of<T>(h).sh;
  CK(launch_bdot<T>(P, R, h->n, h->k, h->p, h->partR, grid_pup<T>(h, g), h->stream,
                    sh_role(sh, h->k, SH_P), sh_role(sh, h->k, SH_R)));
  return BCG_OK;
}

// ev: NULL, or 10 events recorded around the 5 launches (profiling)
template <typename T>
bcg_status launch_iteration(bcg_ctx *h, const OpDesc &A, T *X, T *R, T *P, T *Q, const StreamGrids &g,
                            cudaEvent_t *ev = nullptr) {
  cudaStream_t s = h->stream;
#define REC(i) do { if (ev) CK(cudaEventRecord(ev[i], s)); } while (0)
  const int gu = grid_upd<T>(h, g), gp = grid_pup<T>(h, g);
  const int df = df_updates<T>(h, g) ? 1 : 0;
  const ShiftCtl sc = shifts_of<T>(h);
  REC(0);
  {
    NvtxRange r_("K1 BOP + alpha");
    CK(launch_op_gram<T>(A, P, R, Q, h->n, h->k, h->p, h->global, h->active, h->partA, h->partR, h->st, g.op, s,
                         sc.sh));
  }
  REC(1); REC(2);
  {
    NvtxRange r_("K4a lambda");
    CK(launch_solve_lambda(h->partA, h->partR, g.op, g.rho_k3 ? gp : g.op, h->k, h->p, h->global, h->active, h->lam,
                           h->rho_rec, h->st, h->gws, g.alpha_circ, s));
  }
  REC(3); REC(4);
  {
    NvtxRange r_("K2 X, R update + rho");
    CK(launch_update_xr<T>(X, R, P, Q, h->n, h->k, h->p, h->global, h->lam, h->active, h->partRho, h->partN, h->st,
                           gu, s, dinv_of<T>(h), sc.sh, df));
  }
  REC(5); REC(6);
  {
    NvtxRange r_("K4b stop test + beta");
    CK(launch_solve_beta(h->partRho, h->partN, gu, gu, h->k, h->p, h->global, h->tol2_dev, h->r0n2, h->rn2,
                         h->active, h->block_iters, h->rho_rec, h->beta, h->st, h->gws, g.rho_circ, s, sc));
  }
  REC(7); REC(8);
  {
    NvtxRange r_("K3 P update");
    CK(launch_update_p<T>(P, R, h->n, h->k, h->p, h->global, h->beta, h->active, h->st, gp, s, dinv_of<T>(h),
                          h->partR, sc.sh));
  }
  REC(9);
#undef REC
  return BCG_OK;
}

// One large-block update OUT = BASE (x bscale per row) + sign Y C with the tiled FMA kernel.
template <typename T>
bcg_status lp_update(bcg_ctx *h, T *OUT, const T *BASE, const T *Y, const double *C, double sign, int bump,
                     const T *bscale) {
  CK(launch_lp_baxpy<T>(OUT, BASE, Y, C, h->n, h->k, h->p, h->global, sign, h->active, h->st, bump, h->stream,
                        bscale));
  return BCG_OK;
}

// Partials of a large-block product <<X, Y>>_S (X's rows times xscale if given) into `chunks` partial rows with the
// tiled Dot2 kernel.
template <typename T>
bcg_status lp_gram(bcg_ctx *h, const T *X, const T *Y, double *part, int chunks, const T *xscale, const int *shX,
                   const int *shY) {
  CK(launch_lp_gram<T>(X, Y, h->n, h->k, h->p, h->global, h->active, part, chunks, h->st, h->stream, xscale, shX,
                       shY));
  return BCG_OK;
}

// One FP64 iteration with large blocks on the tensor cores, from digit images (p a multiple of 64): every operand is
// cut once per use into images that the MMA kernels copy into shared memory whole (P twice: column images for the
// Grams, row images for the updates, the latter serving both X += P lambda and P = Z + P beta). The new P is
// written into Q's buffer; the caller swaps P and Q.
bcg_status ensure_events(bcg_ctx *h, int count);

// With option "profile": one tensor-core launch bracketed by CUDA events and read back at once (slot 6: block
// products, 7: block updates).
template <typename F>
bcg_status tc_timed(bcg_ctx *h, int slot, F &&launch) {
  if (!h->profile) {
    CK(launch());
    return BCG_OK;
  }
  CKS(ensure_events(h, 2));
  CK(cudaEventRecord(h->ev[0], h->stream));
  CK(launch());
  CK(cudaEventRecord(h->ev[1], h->stream));
  CK(cudaEventSynchronize(h->ev[1]));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
  h->prof_ms[slot] += ms;
  h->prof_count[slot] += 1;
  return BCG_OK;
}

bcg_status launch_iteration_tcimg(bcg_ctx *h, const OpDesc &A, double *X, double *R, double *P, double *Q,
                                  const StreamGrids &g) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const int k = h->k, p = h->p, gl = h->global, ch = g.op, nsm = h->nsm;
  const ShiftCtl sc = shifts_of<double>(h);
  const double *dinv = dinv_of<double>(h);
  unsigned char *G1 = h->tc_img[0], *G2 = h->tc_img[1], *RP = h->tc_img[2], *RQ = h->tc_img[3];
  int *ec1 = h->tc_ecol, *ec2 = h->tc_ecol + k;
  int *erP = h->tc_erow, *erQ = h->tc_erow + (size_t)((n + 127) / 128) * 128 * (k / p);
  CK(launch_lp_bop<double>(A, P, Q, n, k, h->st, nsm, s));
  // alpha = <<P, Q>> and the recomputed rho = <<P, R>> (P's column images serve both)
  CK(launch_tc_col_exp<double>(P, nullptr, n, k, ec1, nsm, s));
  CK(launch_tc_cut_cols<double>(P, nullptr, n, k, ec1, G1, nsm, s));
  CK(launch_tc_col_exp<double>(Q, nullptr, n, k, ec2, nsm, s));
  CK(launch_tc_cut_cols<double>(Q, nullptr, n, k, ec2, G2, nsm, s));
  CKS(tc_timed(h, 6, [&] { return launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partA, ch, ec1, ec2, h->st, s); }));
  CK(launch_tc_col_exp<double>(R, nullptr, n, k, ec2, nsm, s));   // stream order: after the alpha kernel read ec2 and G2
  CK(launch_tc_cut_cols<double>(R, nullptr, n, k, ec2, G2, nsm, s));
  CKS(tc_timed(h, 6, [&] { return launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partR, ch, ec1, ec2, h->st, s); }));
  CK(launch_solve_lambda(h->partA, h->partR, ch, ch, k, p, gl, h->active, h->lam, h->rho_rec, h->st, h->gws, 0, s));
  // X += P lambda, R -= Q lambda
  CK(launch_tc_slice(h->lam, h->nblk, p, h->tc_cs, h->tc_cexp, s));
  CK(launch_tc_cut_rows(P, n, k, p, RP, erP, s));
  CK(launch_tc_cut_rows(Q, n, k, p, RQ, erQ, s));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img(X, X, RP, erP, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 0, s, nullptr, nsm);
  }));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img(R, R, RQ, erQ, h->tc_cs, h->tc_cexp, n, k, p, gl, -1.0, h->active, h->st, 0, s, nullptr,
                               nsm);
  }));
  // rho = <<Z, R>>, Z = M^{-1} R formed in the cut
  CK(launch_tc_col_exp<double>(R, dinv, n, k, ec1, nsm, s));
  CK(launch_tc_cut_cols<double>(R, dinv, n, k, ec1, G1, nsm, s));
  if (dinv) {
    CK(launch_tc_col_exp<double>(R, nullptr, n, k, ec2, nsm, s));
    CK(launch_tc_cut_cols<double>(R, nullptr, n, k, ec2, G2, nsm, s));
    CKS(tc_timed(h, 6, [&] { return launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partRho, ch, ec1, ec2, h->st, s); }));
  } else {
    CKS(tc_timed(h, 6, [&] { return launch_tc_gram_img(G1, G1, n, k, p, gl, h->active, h->partRho, ch, ec1, ec1, h->st, s); }));
  }
  CK(launch_lp_colnorm<double>(R, n, k, h->partN, g.res, h->st, s, sh_role(sc.sh, k, SH_R)));
  CK(launch_solve_beta(h->partRho, h->partN, ch, g.res, k, p, gl, h->tol2_dev, h->r0n2, h->rn2, h->active,
                       h->block_iters, h->rho_rec, h->beta, h->st, h->gws, 0, s, sc));
  // P = Z + P beta into Q's buffer (P's row images are still those of this iteration's P)
  CK(launch_tc_slice(h->beta, h->nblk, p, h->tc_cs, h->tc_cexp, s));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img(Q, R, RP, erP, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 1, s, dinv, nsm);
  }));
  return BCG_OK;
}

// One iteration with large blocks (p > 32): the tiled FMA kernel for BOP; the block products and updates on the
// tensor cores where the handle has digit images (the mixed form's FP32 process), else the tiled Dot2 products and
// FMA updates (and FP64 with option "tensor_cores" 0). The direction update cannot run in place across
// column tiles, so it writes into the Q buffer (free at that point) and the caller swaps P and Q.
template <typename T>
bcg_status launch_iteration_lp(bcg_ctx *h, const OpDesc &A, T *X, T *R, T *P, T *Q, const StreamGrids &g) {
  cudaStream_t s = h->stream;
  const int ch = g.op;
  const int64_t n = h->n;
  const int k = h->k, p = h->p, gl = h->global, nsm = h->nsm;
  const ShiftCtl sc = shifts_of<T>(h);
  const int *shR = sh_role(sc.sh, h->k, SH_R), *shP = sh_role(sc.sh, h->k, SH_P), *shQ = sh_role(sc.sh, h->k, SH_Q);
  // the block products on the tensor cores from digit images where the handle has them (the mixed form's FP32
  // process; the FP64 form has launch_iteration_tcimg)
  const bool tc = h->tensor_cores && h->tc_img[0] != nullptr;
  unsigned char *G1 = h->tc_img[0], *G2 = h->tc_img[1];
  int *ec1 = h->tc_ecol, *ec2 = h->tc_ecol + k;
  CK(launch_lp_bop<T>(A, P, Q, h->n, h->k, h->st, h->nsm, s));
  if (tc) {   // alpha = <<P, Q>>, the recomputed rho = <<P, R>> (P's images serve both)
    CK(launch_tc_col_exp<T>(P, nullptr, n, k, ec1, nsm, s));
    CK(launch_tc_cut_cols<T>(P, nullptr, n, k, ec1, G1, nsm, s));
    CK(launch_tc_col_exp<T>(Q, nullptr, n, k, ec2, nsm, s));
    CK(launch_tc_cut_cols<T>(Q, nullptr, n, k, ec2, G2, nsm, s));
    CK(launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partA, ch, ec1, ec2, h->st, s));
    CK(launch_tc_col_exp<T>(R, nullptr, n, k, ec2, nsm, s));
    CK(launch_tc_cut_cols<T>(R, nullptr, n, k, ec2, G2, nsm, s));
    CK(launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partR, ch, ec1, ec2, h->st, s));
  } else {
    CKS(lp_gram<T>(h, P, Q, h->partA, ch, nullptr, shP, shQ));
    CKS(lp_gram<T>(h, P, R, h->partR, ch, nullptr, shP, shR));
  }
  CK(launch_solve_lambda(h->partA, h->partR, ch, ch, h->k, h->p, h->global, h->active, h->lam, h->rho_rec, h->st,
                         h->gws, 0, s));
  // X += P lambda, R -= Q lambda (tensor cores: from the row images of P and Q; P's also serve P = Z + P beta)
  unsigned char *RP = h->tc_img[2], *RQ = h->tc_img[3];
  int *erP = h->tc_erow, *erQ = h->tc_erow + (size_t)((n + 127) / 128) * 128 * (k / p);
  if (tc) {
    CK(launch_tc_slice(h->lam, h->nblk, p, h->tc_cs, h->tc_cexp, s));
    CK(launch_tc_cut_rows<T>(P, n, k, p, RP, erP, s));
    CK(launch_tc_cut_rows<T>(Q, n, k, p, RQ, erQ, s));
    CKS(tc_timed(h, 7, [&] {
      return launch_tc_baxpy_img<T>(X, X, RP, erP, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 0, s,
                                    nullptr, nsm);
    }));
    CKS(tc_timed(h, 7, [&] {
      return launch_tc_baxpy_img<T>(R, R, RQ, erQ, h->tc_cs, h->tc_cexp, n, k, p, gl, -1.0, h->active, h->st, 0, s,
                                    nullptr, nsm);
    }));
  } else {
    CKS(lp_update<T>(h, X, X, P, h->lam, 1.0, 0, nullptr));
    CKS(lp_update<T>(h, R, R, Q, h->lam, -1.0, 0, nullptr));
  }
  // rho = <<Z, R>> with Z = M^{-1} R formed on the fly
  if (tc) {
    const T *dv = dinv_of<T>(h);
    CK(launch_tc_col_exp<T>(R, dv, n, k, ec1, nsm, s));
    CK(launch_tc_cut_cols<T>(R, dv, n, k, ec1, G1, nsm, s));
    if (dv) {
      CK(launch_tc_col_exp<T>(R, nullptr, n, k, ec2, nsm, s));
      CK(launch_tc_cut_cols<T>(R, nullptr, n, k, ec2, G2, nsm, s));
      CK(launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partRho, ch, ec1, ec2, h->st, s));
    } else {
      CK(launch_tc_gram_img(G1, G1, n, k, p, gl, h->active, h->partRho, ch, ec1, ec1, h->st, s));
    }
  } else {
    CKS(lp_gram<T>(h, R, R, h->partRho, ch, dinv_of<T>(h), shP, shR));
  }
  CK(launch_lp_colnorm<T>(R, h->n, h->k, h->partN, g.res, h->st, s, shR));   // a full-GPU grid, like K0's
  CK(launch_solve_beta(h->partRho, h->partN, ch, g.res, h->k, h->p, h->global, h->tol2_dev, h->r0n2, h->rn2,
                       h->active,
                       h->block_iters, h->rho_rec, h->beta, h->st, h->gws, 0, s, sc));
  if (tc) {
    CK(launch_tc_slice(h->beta, h->nblk, p, h->tc_cs, h->tc_cexp, s));
    CKS(tc_timed(h, 7, [&] {
      return launch_tc_baxpy_img<T>(Q, R, RP, erP, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 1, s,
                                    dinv_of<T>(h), nsm);
    }));
  } else {
    CKS(lp_update<T>(h, Q, R, P, h->beta, 1.0, 1, dinv_of<T>(h)));
  }
  return BCG_OK;
}

// One FP64 iteration with blocks of 32 columns whose block updates run on the tensor cores: K1 as in the fused path
// (BOP, alpha and the recomputed rho); X += P lambda and R -= Q lambda from row images of P and Q, with two blocks
// paired into each 64-column tile where 64 divides k (block-diagonal coefficient images, row exponents per block of
// 32), else in 32-column tiles; rho = <<Z, R>> and the column norms in passes of their own (the tiled Dot2 product
// and norm kernels);
// P = Z + P beta into Q's buffer (the caller swaps P and Q). Frozen blocks have lambda = beta = 0, so their X and R
// keep their values and their P becomes Z, as the warp-chunk kernels leave them.
bcg_status launch_iteration_tcpair(bcg_ctx *h, const OpDesc &A, double *X, double *R, double *P, double *Q,
                                   const StreamGrids &g) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const int k = h->k, p = h->p, gl = h->global, nsm = h->nsm;
  const ShiftCtl sc = shifts_of<double>(h);
  const double *dinv = dinv_of<double>(h);
  const int *shP = sh_role(sc.sh, k, SH_P), *shR = sh_role(sc.sh, k, SH_R);
  unsigned char *RP = h->tc_img[2], *RQ = h->tc_img[3];
  int *erP = h->tc_erow, *erQ = h->tc_erow + (size_t)((n + 127) / 128) * 128 * (k / p);
  const bool paired = h->tc_pair != nullptr;
  const int nout = gl ? 1 : k / 64, pt = paired ? 64 : p;   // pt: the block width of the update kernel's images
  auto coef = [&](const double *C) -> cudaError_t {   // digit images of lambda or beta
    if (!paired) return launch_tc_slice(C, h->nblk, p, h->tc_cs, h->tc_cexp, s);
    const cudaError_t e = launch_tc_pair_cmat(C, k, p, gl, h->tc_pair, s);
    return e != cudaSuccess ? e : launch_tc_slice(h->tc_pair, nout, 64, h->tc_cs, h->tc_cexp, s);
  };
  CK(launch_op_gram<double>(A, P, R, Q, n, k, p, gl, h->active, h->partA, h->partR, h->st, g.op, s, sc.sh));
  CK(launch_solve_lambda(h->partA, h->partR, g.op, g.op, k, p, gl, h->active, h->lam, h->rho_rec, h->st, h->gws,
                         g.alpha_circ, s));
  CK(coef(h->lam));
  CK(launch_tc_cut_rows<double>(P, n, k, p, RP, erP, s));
  CK(launch_tc_cut_rows<double>(Q, n, k, p, RQ, erQ, s));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img<double>(X, X, RP, erP, h->tc_cs, h->tc_cexp, n, k, pt, gl, 1.0, nullptr, h->st, 0, s,
                                       nullptr, nsm, p);
  }));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img<double>(R, R, RQ, erQ, h->tc_cs, h->tc_cexp, n, k, pt, gl, -1.0, nullptr, h->st, 0, s,
                                       nullptr, nsm, p);
  }));
  CK(launch_lp_gram<double>(R, R, n, k, p, gl, h->active, h->partRho, g.op, h->st, s, dinv, shP, shR));
  CK(launch_lp_colnorm<double>(R, n, k, h->partN, g.res, h->st, s, shR));
  CK(launch_solve_beta(h->partRho, h->partN, g.op, g.res, k, p, gl, h->tol2_dev, h->r0n2, h->rn2, h->active,
                       h->block_iters, h->rho_rec, h->beta, h->st, h->gws, 0, s, sc));
  CK(coef(h->beta));
  CKS(tc_timed(h, 7, [&] {
    return launch_tc_baxpy_img<double>(Q, R, RP, erP, h->tc_cs, h->tc_cexp, n, k, pt, gl, 1.0, nullptr, h->st, 1, s,
                                       dinv, nsm, p);
  }));
  return BCG_OK;
}

bcg_status ensure_events(bcg_ctx *h, int count) {
  while ((int)h->ev.size() < count) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->ev.push_back(e);
  }
  return BCG_OK;
}

// Accumulate the event timings of the first `executed` iterations of a profiled batch.
bcg_status collect_events(bcg_ctx *h, int executed) {
  for (int i = 0; i < executed; ++i) {
    for (int kk = 0; kk < 5; ++kk) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->ev[10 * i + 2 * kk], h->ev[10 * i + 2 * kk + 1]));
      h->prof_ms[kk] += ms;
      h->prof_count[kk] += 1;
    }
  }
  return BCG_OK;
}

// Every workspace buffer is followed by kGuardBytes bytes of kGuardByte. A kernel that writes past the end of a
// buffer changes them; with option "guards" the solves compare them after their work has finished.
bcg_status check_guards(bcg_ctx *h) {
  CK(cudaStreamSynchronize(h->stream));
  unsigned char g[kGuardBytes];
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    CK(cudaMemcpy(g, static_cast<unsigned char *>(h->allocs[i]) + h->alloc_bytes[i], kGuardBytes,
                  cudaMemcpyDeviceToHost));
    for (int b = 0; b < kGuardBytes; ++b)
      if (g[b] != kGuardByte)
        return fail(BCG_ERR_GUARD, "guard byte %d after workspace buffer %zu (%zu bytes) was overwritten", b, i,
                    h->alloc_bytes[i]);
  }
  return BCG_OK;
}

bcg_status read_status(bcg_ctx *h) {
  CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

// Run iterations until the device flags completion or `maxit` iterations were launched.
// On return h->h_st holds the final status word.
template <typename T>
bcg_status run_iterations(bcg_ctx *h, const OpDesc &A, T *X, T *R, T *P, T *Q, const StreamGrids &g, double tol2,
                          int maxit, cudaGraphExec_t *cached, int *cached_batch) {
  CKS(set_tol2(h, tol2));
  CKS(read_status(h));
  int launched = 0;
  const int batch = h->check_every;
  bool pair = false;   // FP64 blocks of 32 with their block updates on the tensor cores
  if constexpr (sizeof(T) == 8) pair = h->tensor_cores && h->tc_small && h->prec == BCG_FP64;
  if (pair) {   // plain launches, P and Q swap every iteration
    while (h->h_st->flags == 0 && launched < maxit) {
      const int nb = std::min(batch, maxit - launched);
      for (int i = 0; i < nb; ++i) {
        if constexpr (sizeof(T) == 8) CKS(launch_iteration_tcpair(h, A, X, R, P, Q, g));
        std::swap(P, Q);
      }
      launched += nb;
      CKS(read_status(h));
    }
    return BCG_OK;
  }
  if (h->p > kMaxP) {   // large blocks: plain launches, P and Q swap every iteration
    while (h->h_st->flags == 0 && launched < maxit) {
      const int nb = std::min(batch, maxit - launched);
      for (int i = 0; i < nb; ++i) {
        if constexpr (sizeof(T) == 8) {
          if (h->tensor_cores && h->tc_img[0] != nullptr) CKS(launch_iteration_tcimg(h, A, X, R, P, Q, g));
          else CKS(launch_iteration_lp<T>(h, A, X, R, P, Q, g));
        } else {
          CKS(launch_iteration_lp<T>(h, A, X, R, P, Q, g));
        }
        std::swap(P, Q);
      }
      launched += nb;
      CKS(read_status(h));
    }
    return BCG_OK;
  }
  struct Guard {   // a graph built for this call only is destroyed on every exit path
    cudaGraphExec_t exec = nullptr;
    bool own = false;
    ~Guard() { if (own && exec) cudaGraphExecDestroy(exec); }
  } gd;
  gd.exec = cached ? *cached : nullptr;
  cudaGraphExec_t &exec = gd.exec;
  bool &own_exec = gd.own;
  // stream capture is impossible on the legacy default stream: plain launches there
  const bool graphs = h->use_graph && h->stream != nullptr && !h->profile;
  if (h->profile) CKS(ensure_events(h, 10 * batch));
  while (h->h_st->flags == 0 && launched < maxit) {
    const int nb = std::min(batch, maxit - launched);
    if (graphs && nb == batch) {
      if (exec == nullptr || (cached && *cached_batch != batch)) {
        if (exec && (own_exec || cached)) cudaGraphExecDestroy(exec);
        exec = nullptr;
        if (cached) *cached = nullptr;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        bcg_status sc = BCG_OK;
        for (int i = 0; i < nb && sc == BCG_OK; ++i) sc = launch_iteration<T>(h, A, X, R, P, Q, g);
        cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
        if (sc != BCG_OK) {
          if (graph) cudaGraphDestroy(graph);
          return sc;
        }
        if (ec != cudaSuccess) return fail(BCG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ec != cudaSuccess) return fail(BCG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
        if (cached) {
          *cached = exec;
          *cached_batch = batch;
        } else {
          own_exec = true;
        }
      }
      CK(cudaGraphLaunch(exec, h->stream));
    } else {
      for (int i = 0; i < nb; ++i)
        CKS(launch_iteration<T>(h, A, X, R, P, Q, g, h->profile ? &h->ev[10 * i] : nullptr));
    }
    launched += nb;
    const int before = h->h_st->iter;
    CKS(read_status(h));
    if (h->profile) {
      // iterations that ran (the rest of the batch returned at entry once the status was set)
      int executed = h->h_st->iter - before;
      if (h->h_st->flags & (ST_BREAKDOWN | ST_NUMERIC)) executed += 1;
      CKS(collect_events(h, std::max(0, std::min(nb, executed))));
    }
  }
  return BCG_OK;
}

bcg_status fill_block_iters(bcg_ctx *h) {
  CK(cudaMemcpyAsync(h->h_iters, h->block_iters, sizeof(int) * h->nblk, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int j = 0; j < h->nblk; ++j) h->last_block_iters[j] = h->h_iters[j];
  return BCG_OK;
}

// copy k doubles from device to h->h_vec + off*k
bcg_status fetch_vec(bcg_ctx *h, const double *src, int off) {
  CK(cudaMemcpyAsync(h->h_vec + (size_t)off * h->k, src, sizeof(double) * h->k, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

double max_ratio(const double *num2, const double *den2, int k) {
  double m = 0.0;
  for (int c = 0; c < k; ++c) {
    const double r = den2[c] > 0 ? std::sqrt(num2[c] / den2[c]) : std::sqrt(num2[c]);
    if (!(r <= m)) m = r;   // propagates NaN
  }
  return m;
}

bcg_status status_from_flags(int flags, bool all_done) {
  if (flags & ST_TIMEOUT) return BCG_ERR_TIMEOUT;
  if (flags & ST_NUMERIC) return BCG_ERR_NUMERIC;
  if (flags & ST_BREAKDOWN) return BCG_ERR_BREAKDOWN;
  if (!all_done) return BCG_ERR_NOT_CONVERGED;
  return BCG_OK;
}

bcg_status solve_fp64(bcg_ctx *h, const double *B, double *X, double tol, int maxit, bcg_info *info) {
  cudaStream_t s = h->stream;
  const double tol2 = tol * tol;
  CK(launch_residual<double>(h->A64, X, B, h->R, h->P, nullptr, nullptr, h->n, h->k, h->partN, h->g64.res, s,
                             dinv_of<double>(h)));
  CK(launch_init_status(h->partN, h->g64.res, h->k, h->p, h->global, h->r0n2, h->rn2, h->active, h->block_iters,
                        h->lam, h->beta, h->st, s, shifts_of<double>(h)));
  CKS(first_rho_rec<double>(h, h->P, h->R, h->g64));
  CKS(run_iterations<double>(h, h->A64, X, h->R, h->P, h->Q, h->g64, tol2, maxit, nullptr, nullptr));
  const DevStatus fin = *h->h_st;
  CKS(fill_block_iters(h));
  // true residual B - A X, recomputed
  CK(launch_residual<double>(h->A64, X, B, h->Q, nullptr, nullptr, nullptr, h->n, h->k, h->partN, h->g64.res, s,
                             nullptr));
  CK(launch_reduce_norms(h->partN, h->g64.res, h->k, h->rtn2, s));
  CKS(fetch_vec(h, h->r0n2, 0));
  CKS(fetch_vec(h, h->rn2, 1));
  CKS(fetch_vec(h, h->rtn2, 2));
  const double *r0 = h->h_vec, *rn = h->h_vec + h->k, *rt = h->h_vec + 2 * h->k;
  const bcg_status st = status_from_flags(fin.flags, (fin.flags & ST_DONE) != 0);
  if (info) {
    info->status = st;
    info->iters = fin.iter;
    info->outer_iters = 0;
    info->breakdown_iter = (fin.flags & ST_BREAKDOWN) ? fin.breakdown_iter : -1;
    info->max_rel_res_recursive = max_ratio(rn, r0, h->k);
    info->max_rel_res_true = max_ratio(rt, r0, h->k);
  }
  if (st != BCG_OK) {
    const char *what = st == BCG_ERR_NUMERIC ? "non-finite value" : st == BCG_ERR_BREAKDOWN ? "breakdown" : "maxit reached";
    fail(st, "solve stopped: %s after %d iterations", what, fin.iter);
  }
  return st;
}

// Dubrulle's retooled block CG (option "retooled"; Electron. Trans. Numer. Anal. 12, 2001, the stability reference
// of Section 3), FP64, every subalgebra, M = I or Jacobi; the kernels and the recurrences are described in
// bcg_retooled.inc.
// p <= 32: Algorithm 1's K1 for W = A S and alpha, then two fused streaming updates, all in place (S, W, Q
// keep their buffers).
// p > 32: the tiled large-block kernels, unfused, and three n x k buffers rotate: W = A S is dead once
// T = Q - W xi is formed, so Q^+ = T psi^{-1} is written into it and S^+ = Q^+ + S psi^T into T's buffer (the
// tiled updates must not write a buffer they read by whole blocks of p columns). Q = T psi^{-1} is a product
// without a base term (a NULL base, or a zeroed output for the tiled update): T + T (psi^{-1} - I) would cancel
// digits in proportion to the column norms of R^0. Plain launches, a status read every check_every iterations.
bcg_status solve_retooled(bcg_ctx *h, const double *B, double *X, double tol, int maxit, bcg_info *info) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const int k = h->k, p = h->p, gl = h->global;
  const bool lp = p > kMaxP;
  const double *dinv = dinv_of<double>(h);
  const int np_g = lp ? h->g64.op : dr_grid_for(n, k, p, h->nsm, h->nparts, dinv != nullptr);
  // Gram shifts: R^0 is taken at the scale of its column norms (gamma^0 = <<M^{-1} R^0, R^0>>: M^{-1} R^0 in
  // the P role); afterwards every operand is of unit scale in the M^{-1} product (Q, S built from it) except
  // W = A S (role Q: the operator's offset)
  const ShiftCtl sc = shifts_of<double>(h);
  const int *shR = sh_role(sc.sh, k, SH_R), *shP = sh_role(sc.sh, k, SH_P), *shQ = sh_role(sc.sh, k, SH_Q);
  // partials of <<X, Y>> per column block; xs: X's rows times xs (the M^{-1} operand)
  auto gram = [&](const double *Xv, const double *Yv, double *part, const int *shx, const int *shy,
                  const double *xs) -> cudaError_t {
    return lp ? launch_lp_gram<double>(Xv, Yv, n, k, p, gl, h->active, part, np_g, h->st, s, xs, shx, shy)
              : launch_dr_gram(Xv, Yv, n, k, p, h->active, part, np_g, h->st, s, shx, shy, gl, xs);
  };
  // OUT = Y C (no base term)
  auto bmul = [&](double *OUT, const double *Yv, const double *Cm) -> cudaError_t {
    if (!lp) return launch_dr_baxpy(OUT, nullptr, Yv, Cm, n, k, p, 1.0, h->active, h->st, 0, h->nsm, s, gl, nullptr);
    cudaError_t e = cudaMemsetAsync(OUT, 0, sizeof(double) * (size_t)n * k, s);
    if (e != cudaSuccess) return e;
    return launch_lp_baxpy<double>(OUT, OUT, Yv, Cm, n, k, p, gl, 1.0, h->active, h->st, 0, s, nullptr);
  };
  auto baxpy = [&](double *OUT, const double *BASE, const double *Yv, const double *Cm, double sign, int bump,
                   const double *bscale) -> cudaError_t {
    return launch_lp_baxpy<double>(OUT, BASE, Yv, Cm, n, k, p, gl, sign, h->active, h->st, bump, s, bscale);
  };
  double *W = h->R, *S = h->P, *Qb = h->Q;
  double *partM = dinv ? h->partR : nullptr;   // <<T, M^{-1} T>> (K1's recomputed-rho partials are unused here)
  // wide blocks on the tensor cores (digit images) where the handle has them
  const bool tc = lp && h->tensor_cores && h->tc_img[0] != nullptr;
  unsigned char *G1 = h->tc_img[0], *G2 = h->tc_img[1], *RS = h->tc_img[2], *RT = h->tc_img[3];
  int *ec1 = h->tc_ecol, *ec2 = h->tc_ecol + k;
  int *erS = h->tc_erow, *erT = h->tc_erow + (size_t)((n + 127) / 128) * 128 * (k / p);
  // R^0 = B - A X^0 (in W's buffer) = Q^0 C^0, S^1 = M^{-1} Q^0
  CK(launch_residual<double>(h->A64, X, B, W, nullptr, nullptr, nullptr, n, k, h->partN, h->g64.res, s, nullptr));
  CK(launch_init_status(h->partN, h->g64.res, k, p, gl, h->r0n2, h->rn2, h->active, h->block_iters, h->lam,
                        h->beta, h->st, s, sc));
  CK(gram(W, W, h->partA, dinv ? shP : shR, shR, dinv));
  CK(launch_dr_start(h->partA, np_g, k, p, h->active, h->dr_C, h->dr_psiinv, h->st, h->gws, s, gl));
  CK(launch_fill_shifts(nullptr, k, sc, s));
  CK(bmul(Qb, W, h->dr_psiinv));
  CK(launch_dr_scale_rows(S, Qb, dinv, n, k, h->nsm, s));
  CKS(set_tol2(h, tol * tol));
  CKS(read_status(h));
  int launched = 0;
  while (h->h_st->flags == 0 && launched < maxit) {
    const int nb = std::min(h->check_every, maxit - launched);
    for (int i = 0; i < nb; ++i) {
      if (!lp) {
        // W = A S, alpha (K1; where K1 also forms a recomputed rho, it reads Q and the result is unused) |
        // xi, lambda | X += S lambda, T = Q - W xi, <<T, T>> (and <<T, M^{-1} T>>) | stop test, psi |
        // Q = T psi^{-1}, S = M^{-1} Q + S psi^T
        CK(launch_op_gram<double>(h->A64, S, Qb, W, n, k, p, gl, h->active, h->partA, h->partR, h->st, h->g64.op,
                                  s, sc.sh));
        CK(launch_dr_xi(h->partA, h->g64.op, k, p, h->active, h->dr_C, h->dr_xi, h->lam, h->st, h->gws,
                        h->g64.alpha_circ, s, gl));
        CK(launch_dr_update_xt(X, Qb, S, W, n, k, p, h->lam, h->dr_xi, h->active, h->partRho, np_g, h->st, s, gl,
                               dinv, partM));
        CK(launch_dr_psi(h->partRho, np_g, k, p, h->tol2_dev, h->r0n2, h->rn2, h->active, h->block_iters,
                         h->dr_C, h->dr_psiinv, h->dr_phi, h->st, h->gws, s, gl, partM));
        CK(launch_dr_update_qs(Qb, S, n, k, p, h->dr_psiinv, h->dr_phi, h->active, h->st, h->nsm, s, gl, dinv));
        continue;
      }
      if (tc) {   // the same steps on the tensor cores, from digit images
        CK(launch_lp_bop<double>(h->A64, S, W, n, k, h->st, h->nsm, s));                       // W = A S
        CK(launch_tc_col_exp<double>(S, nullptr, n, k, ec1, h->nsm, s));                       // alpha = <<S, W>>
        CK(launch_tc_cut_cols<double>(S, nullptr, n, k, ec1, G1, h->nsm, s));
        CK(launch_tc_col_exp<double>(W, nullptr, n, k, ec2, h->nsm, s));
        CK(launch_tc_cut_cols<double>(W, nullptr, n, k, ec2, G2, h->nsm, s));
        CK(launch_tc_gram_img(G1, G2, n, k, p, gl, h->active, h->partA, np_g, ec1, ec2, h->st, s));
        CK(launch_dr_xi(h->partA, np_g, k, p, h->active, h->dr_C, h->dr_xi, h->lam, h->st, h->gws, 0, s, gl));
        CK(launch_tc_slice(h->lam, h->nblk, p, h->tc_cs, h->tc_cexp, s));                     // X += S lambda
        CK(launch_tc_cut_rows(S, n, k, p, RS, erS, s));
        CK(launch_tc_baxpy_img(X, X, RS, erS, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 0, s, nullptr,
                               h->nsm));
        CK(launch_tc_slice(h->dr_xi, h->nblk, p, h->tc_cs, h->tc_cexp, s));                   // T = Q - W xi
        CK(launch_tc_cut_rows(W, n, k, p, RT, erT, s));
        CK(launch_tc_baxpy_img(Qb, Qb, RT, erT, h->tc_cs, h->tc_cexp, n, k, p, gl, -1.0, h->active, h->st, 0, s,
                               nullptr, h->nsm));
        CK(launch_tc_col_exp<double>(Qb, nullptr, n, k, ec1, h->nsm, s));                      // <<T, T>> per block
        CK(launch_tc_cut_cols<double>(Qb, nullptr, n, k, ec1, G1, h->nsm, s));
        CK(launch_tc_gram_img(G1, G1, n, k, p, gl, h->active, h->partRho, np_g, ec1, ec1, h->st, s));
        if (dinv) {                                                                             // <<M^{-1} T, T>>
          CK(launch_tc_col_exp<double>(Qb, dinv, n, k, ec2, h->nsm, s));
          CK(launch_tc_cut_cols<double>(Qb, dinv, n, k, ec2, G2, h->nsm, s));
          CK(launch_tc_gram_img(G2, G1, n, k, p, gl, h->active, partM, np_g, ec2, ec1, h->st, s));
        }
        CK(launch_dr_psi(h->partRho, np_g, k, p, h->tol2_dev, h->r0n2, h->rn2, h->active, h->block_iters, h->dr_C,
                         h->dr_psiinv, h->dr_phi, h->st, h->gws, s, gl, partM));
        CK(launch_tc_slice(h->dr_psiinv, h->nblk, p, h->tc_cs, h->tc_cexp, s));               // Q^+ = T psi^{-1}
        CK(launch_tc_cut_rows(Qb, n, k, p, RT, erT, s));
        CK(launch_tc_baxpy_img(W, nullptr, RT, erT, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 0, s,
                               nullptr, h->nsm));
        CK(launch_tc_slice(h->dr_phi, h->nblk, p, h->tc_cs, h->tc_cexp, s));                  // S^+ = M^{-1} Q^+ + S psi^T
        CK(launch_tc_baxpy_img(Qb, W, RS, erS, h->tc_cs, h->tc_cexp, n, k, p, gl, 1.0, h->active, h->st, 1, s, dinv,
                               h->nsm));
        double *old_s = S;
        S = Qb;
        Qb = W;
        W = old_s;
        continue;
      }
      CK(launch_lp_bop<double>(h->A64, S, W, n, k, h->st, h->nsm, s));   // W = A S
      CK(gram(S, W, h->partA, shP, shQ, nullptr));                       // alpha = <<S, W>>
      CK(launch_dr_xi(h->partA, np_g, k, p, h->active, h->dr_C, h->dr_xi, h->lam, h->st, h->gws, 0, s, gl));
      CK(baxpy(X, X, S, h->lam, 1.0, 0, nullptr));                       // X += S lambda, lambda = xi C
      CK(baxpy(Qb, Qb, W, h->dr_xi, -1.0, 0, nullptr));                  // T = Q - W xi
      CK(gram(Qb, Qb, h->partRho, shR, shR, nullptr));                   // <<T, T>> per column block
      if (dinv) CK(gram(Qb, Qb, partM, shP, shR, dinv));                 // <<M^{-1} T, T>>
      CK(launch_dr_psi(h->partRho, np_g, k, p, h->tol2_dev, h->r0n2, h->rn2, h->active, h->block_iters, h->dr_C,
                       h->dr_psiinv, h->dr_phi, h->st, h->gws, s, gl, partM));
      CK(bmul(W, Qb, h->dr_psiinv));                                     // Q^+ = T psi^{-1}
      CK(baxpy(Qb, W, S, h->dr_phi, 1.0, 1, dinv));                      // S^+ = M^{-1} Q^+ + S psi^T; ends it
      double *old_s = S;
      S = Qb;
      Qb = W;
      W = old_s;
    }
    launched += nb;
    CKS(read_status(h));
  }
  const DevStatus fin = *h->h_st;
  CKS(fill_block_iters(h));
  CK(launch_residual<double>(h->A64, X, B, W, nullptr, nullptr, nullptr, n, k, h->partN, h->g64.res, s, nullptr));
  CK(launch_reduce_norms(h->partN, h->g64.res, k, h->rtn2, s));
  CKS(fetch_vec(h, h->r0n2, 0));
  CKS(fetch_vec(h, h->rn2, 1));
  CKS(fetch_vec(h, h->rtn2, 2));
  const double *r0 = h->h_vec, *rn = h->h_vec + k, *rt = h->h_vec + 2 * k;
  const bcg_status st = status_from_flags(fin.flags, (fin.flags & ST_DONE) != 0);
  if (info) {
    info->status = st;
    info->iters = fin.iter;
    info->outer_iters = 0;
    info->breakdown_iter = (fin.flags & ST_BREAKDOWN) ? fin.breakdown_iter : -1;
    info->max_rel_res_recursive = max_ratio(rn, r0, k);
    info->max_rel_res_true = max_ratio(rt, r0, k);
  }
  if (st != BCG_OK) {
    const char *what = st == BCG_ERR_NUMERIC ? "non-finite value" : st == BCG_ERR_BREAKDOWN ? "breakdown" : "maxit reached";
    fail(st, "solve stopped: %s after %d iterations (retooled form)", what, fin.iter);
  }
  return st;
}

// FP32 block CG with FP64 residual replacement (refine = 1). One Krylov process in FP32 (BOP and block updates;
// Gram matrices FP64-accurate, p x p solves in FP64) accumulates a correction D; whenever its recursive
// residual has dropped by kReplaceDrop since the last replacement, and when every block has stopped, the
// correction is flushed into the FP64 iterate (X += D, D = 0) and the residual is replaced by the FP64 true
// residual B - A X. P is kept, and Algorithm 1 recomputes rho = <<P, R>>_S from the replaced residual in the
// next iteration, so the process continues instead of restarting. Converged when every column's true
// residual is below tol (relative to the initial one); blocks that stopped on their recursive residual before
// that are reopened; if a block's directions lose rank, a cycle stops making progress, or the process has run
// more iterations than the system has rows (in exact arithmetic it would have terminated: its directions are
// spent), the process restarts from the FP64 residual.
constexpr double kReplaceDrop = 0.1;
constexpr int kReplaceMinCycle = 64;   // shortest window after which a replacement cycle can count as stalled

bcg_status solve_replace(bcg_ctx *h, const double *B, double *X, double tol, int maxit, bcg_info *info) {
  cudaStream_t s = h->stream;
  const int64_t nk = h->n * h->k;
  const double tol2 = tol * tol;
  // (re)start of the Krylov process from the FP64 residual R: R32 = fl(R 2^-sigma), P32 = fl(M^{-1} R 2^-sigma),
  // D = 0, with sigma fixed per block until the next restart (launch_mixed_scale). The per-column stopping test
  // stays relative to the initial residual (r0n2 = the first start's norms, in the process's scale).
  auto start = [&](bool first) -> bcg_status {
    CK(launch_residual<double>(h->A64, X, B, h->Q, nullptr, nullptr, nullptr, h->n, h->k, h->partN, h->g64.res, s,
                               nullptr));
    CK(launch_reduce_norms(h->partN, h->g64.res, h->k, h->rtn2, s));
    if (first) CK(cudaMemcpyAsync(h->outer0, h->rtn2, sizeof(double) * h->k, cudaMemcpyDeviceToDevice, s));
    CK(launch_mixed_scale(h->rtn2, h->outer0, h->k, h->p, h->global, h->msig, h->partN, h->tmp2k, s));
    CK(launch_cast_scaled(h->Q, dinv_of<double>(h), h->msig, h->n, h->k, h->R32, h->P32, h->nsm, s));
    CK(launch_init_status(h->partN, 1, h->k, h->p, h->global, h->r0n2, h->rn2, h->active, h->block_iters, h->lam,
                          h->beta, h->st, s, shifts_of<float>(h)));
    CK(cudaMemcpyAsync(h->r0n2, h->tmp2k, sizeof(double) * h->k, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(h->D32, 0, sizeof(float) * nk, s));
    CKS(first_rho_rec<float>(h, h->P32, h->R32, h->g32));
    return BCG_OK;
  };
  CKS(start(true));
  CKS(fetch_vec(h, h->outer0, 0));
  bcg_status st = BCG_ERR_NOT_CONVERGED;
  int replaced = 0, restarts = 0, stalls = 0, brk = -1, base_iters = 0;
  double m_true = max_ratio(h->h_vec, h->h_vec, h->k) > 0 ? 1.0 : 0.0;   // relative to the initial residual
  double last2 = 1.0, best = INFINITY;
  int cycle_start = 0, longest = 0;   // iteration of the last replacement, longest cycle between replacements
  const int min_cycle = (int)std::min<int64_t>(kReplaceMinCycle, h->n);
  if (m_true == 0.0) st = BCG_OK;   // B - A X = 0 in every column
  while (st == BCG_ERR_NOT_CONVERGED) {
    CKS(run_iterations<float>(h, h->A32, h->D32, h->R32, h->P32, h->Q32, h->g32, tol2, h->check_every,
                              &h->graph32, &h->graph32_batch));
    const DevStatus fin = *h->h_st;
    const int iters = base_iters + fin.iter;
    if (fin.flags & ST_NUMERIC) { st = BCG_ERR_NUMERIC; break; }
    const bool broke = (fin.flags & ST_BREAKDOWN) != 0;
    if (broke && fin.breakdown_iter <= 1) { brk = iters; st = BCG_ERR_BREAKDOWN; break; }
    const bool done = (fin.flags & ST_DONE) != 0;
    CKS(fetch_vec(h, h->rn2, 1));
    CKS(fetch_vec(h, h->r0n2, 0));
    double rec2 = 0.0;   // squared max relative recursive residual
    for (int cc = 0; cc < h->k; ++cc) {
      const double r = h->h_vec[cc] > 0 ? h->h_vec[h->k + cc] / h->h_vec[cc] : 0.0;
      if (!(r <= rec2)) rec2 = r;
    }
    // a cycle running longer than twice the longest one so far (and at least min(kReplaceMinCycle, n)
    // iterations) gets a replacement too; if that shows no 10 % gain of the true residual, the kept directions
    // no longer help and the process restarts (below)
    const bool forced = iters - cycle_start > std::max(2 * longest, min_cycle);
    if (!(broke || done || forced || rec2 < kReplaceDrop * kReplaceDrop * last2 || iters >= maxit)) continue;
    longest = std::max(longest, iters - cycle_start);
    cycle_start = iters;
    // residual replacement: X += D 2^sigma, D = 0, R = B - A X in FP64 (R32 = fl(R 2^-sigma)); P and the Krylov
    // process stay
    CK(launch_add_correction(X, h->D32, nk, h->k, h->msig, h->nsm, s));
    CK(cudaMemsetAsync(h->D32, 0, sizeof(float) * nk, s));
    CK(launch_residual<double>(h->A64, X, B, h->Q, nullptr, h->R32, nullptr, h->n, h->k, h->partN, h->g64.res, s,
                               nullptr, h->msig));
    CK(launch_reduce_norms(h->partN, h->g64.res, h->k, h->rtn2, s));
    ++replaced;
    CKS(fetch_vec(h, h->outer0, 0));
    CKS(fetch_vec(h, h->rtn2, 2));
    const double m_prev = m_true;
    m_true = max_ratio(h->h_vec + 2 * h->k, h->h_vec, h->k);
    if (!std::isfinite(m_true)) { st = BCG_ERR_NUMERIC; break; }
    if (m_true <= tol) { st = BCG_OK; break; }
    if (iters >= maxit) break;
    const bool stuck = forced && !(m_true < 0.9 * m_prev);
    const bool spent = iters - base_iters > h->n;   // more iterations than rows since the process (re)started
    if (m_true >= 0.9 * best) {
      if (++stalls >= 3) break;
    } else {
      stalls = 0;
    }
    best = std::min(best, m_true);
    last2 = m_true * m_true;
    if (broke || stuck || spent) {
      // the FP32 directions of a block became dependent (its alpha or recomputed rho lost rank), the cycle
      // stalled, or the process outran the dimension of the system (the FP32 process has used up what its
      // directions can resolve): restart the Krylov process from the FP64 residual, as a restarted refinement
      // step would
      base_iters = iters;
      ++restarts;
      CKS(start(false));
    } else if (done) {
      // every block stopped on its recursive residual but some true residuals are still above the tolerance:
      // reopen those blocks with their directions
      CK(launch_reactivate(h->rtn2, h->outer0, tol2, h->k, h->p, h->global, h->active, h->st, s));
    }
  }
  CKS(read_status(h));
  const int iters = base_iters + h->h_st->iter;
  CKS(fill_block_iters(h));
  if (info) {
    info->status = st;
    info->iters = iters;
    info->outer_iters = replaced;
    info->breakdown_iter = brk;
    info->max_rel_res_recursive = m_true;
    info->max_rel_res_true = m_true;
  }
  if (st != BCG_OK)
    fail(st, "mixed-precision solve stopped with status %d after %d iterations, %d replacements, %d restarts", st,
         iters, replaced, restarts);
  return st;
}

// FP64 iterative refinement around FP32 inner block-CG solves (refine = 0): each step restarts the inner
// Krylov process from the FP64 residual.
bcg_status solve_refine(bcg_ctx *h, const double *B, double *X, double tol, int maxit, bcg_info *info) {
  cudaStream_t s = h->stream;
  const int64_t nk = h->n * h->k;
  int outer = 0, inner_total = 0, brk = -1;
  bcg_status st = BCG_ERR_NOT_CONVERGED;
  double last_max = INFINITY;
  int stalls = 0;
  for (;;) {
    // outer residual R in FP64; the inner right-hand side is R32 = fl(R 2^-sigma), P32 = fl(M^{-1} R 2^-sigma)
    // with a fresh scale per block (launch_mixed_scale)
    CK(launch_residual<double>(h->A64, X, B, h->Q, nullptr, nullptr, nullptr, h->n, h->k, h->partN, h->g64.res, s,
                               nullptr));
    CK(launch_reduce_norms(h->partN, h->g64.res, h->k, h->rtn2, s));
    if (outer == 0) CK(cudaMemcpyAsync(h->outer0, h->rtn2, sizeof(double) * h->k, cudaMemcpyDeviceToDevice, s));
    CKS(fetch_vec(h, h->outer0, 0));
    CKS(fetch_vec(h, h->rtn2, 2));
    const double *r0 = h->h_vec, *rt = h->h_vec + 2 * h->k;
    const double m = max_ratio(rt, r0, h->k);
    if (!std::isfinite(m)) { st = BCG_ERR_NUMERIC; break; }
    if (m <= tol) { st = BCG_OK; break; }
    if (outer >= h->max_outer) { st = BCG_ERR_NOT_CONVERGED; break; }
    if (m >= 0.9 * last_max) {
      if (++stalls >= 3) { st = BCG_ERR_NOT_CONVERGED; break; }
    } else {
      stalls = 0;
    }
    last_max = std::min(last_max, m);
    // inner FP32 solve of A D = fl(R) from D = 0, asked for the reduction still needed (with a factor-2
    // margin), but never for less than inner_tol (what FP32 block vectors can be trusted to deliver)
    const double itol = std::min(0.5, std::max(h->inner_tol, 0.5 * tol / m));
    const double itol2 = itol * itol;
    CK(cudaMemsetAsync(h->D32, 0, sizeof(float) * nk, s));
    CK(launch_mixed_scale(h->rtn2, nullptr, h->k, h->p, h->global, h->msig, h->partN, nullptr, s));
    CK(launch_cast_scaled(h->Q, dinv_of<double>(h), h->msig, h->n, h->k, h->R32, h->P32, h->nsm, s));
    CK(launch_init_status(h->partN, 1, h->k, h->p, h->global, h->r0n2, h->rn2, h->active, h->block_iters, h->lam,
                          h->beta, h->st, s, shifts_of<float>(h)));
    CKS(first_rho_rec<float>(h, h->P32, h->R32, h->g32));
    CKS(run_iterations<float>(h, h->A32, h->D32, h->R32, h->P32, h->Q32, h->g32, itol2, maxit, &h->graph32,
                              &h->graph32_batch));
    const DevStatus fin = *h->h_st;
    inner_total += fin.iter;
    if (fin.flags & ST_NUMERIC) { st = BCG_ERR_NUMERIC; break; }
    if ((fin.flags & ST_BREAKDOWN) && fin.breakdown_iter <= 1) {
      brk = inner_total;
      st = BCG_ERR_BREAKDOWN;
      break;
    }
    // a later inner breakdown or maxit still leaves a useful correction: apply it and refine on
    CK(launch_add_correction(X, h->D32, nk, h->k, h->msig, h->nsm, s));
    ++outer;
  }
  CKS(fill_block_iters(h));
  CKS(fetch_vec(h, h->outer0, 0));
  CKS(fetch_vec(h, h->rtn2, 2));
  const double *r0 = h->h_vec, *rt = h->h_vec + 2 * h->k;
  if (info) {
    info->status = st;
    info->iters = inner_total;
    info->outer_iters = outer;
    info->breakdown_iter = brk;
    info->max_rel_res_recursive = max_ratio(rt, r0, h->k);
    info->max_rel_res_true = info->max_rel_res_recursive;
  }
  if (st != BCG_OK) fail(st, "refinement stopped with status %d after %d outer / %d inner iterations", st, outer, inner_total);
  return st;
}

// ---------------------------------------------------------------------------------------------------
// Row-sharded iteration (one rank's rows). Each product's per-CTA partials collapse into one partial row
// (sums1 = [alpha | rho_rec] after phase 1, sums2 = [rho | column norms] after phase 2); the caller sums
// these over ranks (an allreduce) between the phases, so every rank runs the p x p solves on the same data.
// The caller also refreshes the halo rows of P before every phase 1.
bcg_status rows_phase(bcg_ctx *h, int phase) {
  cudaStream_t s = h->stream;
  const StreamGrids &g = h->g64;
  const int64_t E = (int64_t)h->k * h->p;
  const bool lp = h->p > kMaxP;
  const int gu = h->precond ? g.upd_zs : g.upd, gp = h->precond ? g.pup_zs : g.pup;
  const double *dinv = dinv_of<double>(h);
  const ShiftCtl sc = shifts_of<double>(h);
  const int *shR = sh_role(sc.sh, h->k, SH_R), *shP = sh_role(sc.sh, h->k, SH_P), *shQ = sh_role(sc.sh, h->k, SH_Q);
  if (phase == 1) {
    if (lp) {
      CK(launch_lp_bop<double>(h->A64, h->P, h->Q, h->n, h->k, h->st, h->nsm, s));
      CK(launch_lp_gram<double>(h->P, h->Q, h->n, h->k, h->p, h->global, h->active, h->partA, g.op, h->st, s,
                                nullptr, shP, shQ));
      CK(launch_lp_gram<double>(h->P, h->R, h->n, h->k, h->p, h->global, h->active, h->partR, g.op, h->st, s,
                                nullptr, shP, shR));
    } else {
      CK(launch_op_gram<double>(h->A64, h->P, h->R, h->Q, h->n, h->k, h->p, h->global, h->active, h->partA,
                                h->partR, h->st, g.op, s, sc.sh));
    }
    CK(launch_sum_partials(h->partA, g.op, E, h->sums1, h->nsm, s));
    // the recomputed rho: from this K1, or (rho_k3) already summed after the previous K3 / the start
    if (!g.rho_k3) CK(launch_sum_partials(h->partR, g.op, E, h->sums1 + E, h->nsm, s));
  } else if (phase == 2) {
    CK(launch_solve_lambda(h->sums1, h->sums1 + E, 1, 1, h->k, h->p, h->global, h->active, h->lam, h->rho_rec, h->st,
                           h->gws, lp ? 0 : g.alpha_circ, s));
    if (lp) {
      CK(launch_lp_baxpy<double>(h->X_rows, h->X_rows, h->P, h->lam, h->n, h->k, h->p, h->global, 1.0, h->active,
                                 h->st, 0, s, nullptr));
      CK(launch_lp_baxpy<double>(h->R, h->R, h->Q, h->lam, h->n, h->k, h->p, h->global, -1.0, h->active, h->st, 0, s,
                                 nullptr));
      CK(launch_lp_gram<double>(h->R, h->R, h->n, h->k, h->p, h->global, h->active, h->partRho, g.op, h->st, s,
                                dinv, shP, shR));
      CK(launch_lp_colnorm<double>(h->R, h->n, h->k, h->partN, g.res, h->st, s, shR));
      CK(launch_sum_partials(h->partRho, g.op, E, h->sums2, h->nsm, s));
      CK(launch_sum_partials(h->partN, g.res, h->k, h->sums2 + E, h->nsm, s));
    } else {
      CK(launch_update_xr<double>(h->X_rows, h->R, h->P, h->Q, h->n, h->k, h->p, h->global, h->lam, h->active,
                                  h->partRho, h->partN, h->st, gu, s, dinv, sc.sh));
      CK(launch_sum_partials(h->partRho, gu, E, h->sums2, h->nsm, s));
      CK(launch_sum_partials(h->partN, gu, h->k, h->sums2 + E, h->nsm, s));
    }
  } else {
    CK(launch_solve_beta(h->sums2, h->sums2 + E, 1, 1, h->k, h->p, h->global, h->tol2_dev, h->r0n2, h->rn2,
                         h->active,
                         h->block_iters, h->rho_rec, h->beta, h->st, h->gws, lp ? 0 : g.rho_circ, s, sc));
    if (lp) {
      CK(launch_lp_baxpy<double>(h->Q, h->R, h->P, h->beta, h->n, h->k, h->p, h->global, 1.0, h->active, h->st, 1, s,
                                 dinv));
      std::swap(h->P, h->Q);   // the new P was written into Q's buffer
    } else {
      CK(launch_update_p<double>(h->P, h->R, h->n, h->k, h->p, h->global, h->beta, h->active, h->st, gp, s, dinv,
                                 h->partR, sc.sh));
      if (g.rho_k3) CK(launch_sum_partials(h->partR, gp, E, h->sums1 + E, h->nsm, s));
    }
  }
  return BCG_OK;
}

bcg_status finish_create(bcg_ctx *h, bcg_handle *out) {
  bcg_status s = setup_workspace(h);
  if (s == BCG_OK) s = make_fp32_copy(h);
  if (s == BCG_OK && h->opkind == OP_CSR) {
    s = h->alloc(&h->rowidx, (size_t)h->nnz);
    if (s == BCG_OK) {
      cudaError_t e = launch_row_index(h->A64.rowptr, h->n, h->rowidx, h->nsm, h->stream);
      if (e != cudaSuccess) s = fail(BCG_ERR_CUDA, "row index: %s", cudaGetErrorString(e));
    }
  }
  if (s == BCG_OK) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = fail(BCG_ERR_CUDA, "create: %s", cudaGetErrorString(e));
  }
  if (s != BCG_OK) {
    delete h;
    return s;
  }
  *out = h;
  return BCG_OK;
}

}  // namespace

extern "C" {

bcg_status bcg_create_csr(bcg_handle *out, int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                          const double *vals, int32_t k, int32_t p, int32_t sub, int32_t prec, void *cuda_stream) {
  if (out == nullptr) return fail(BCG_ERR_INVALID_ARG, "handle pointer is NULL");
  *out = nullptr;
  if (n < 1 || nnz < 1) return fail(BCG_ERR_INVALID_ARG, "n=%lld nnz=%lld must be >= 1", (long long)n, (long long)nnz);
  if (n > INT32_MAX) return fail(BCG_ERR_INVALID_ARG, "n=%lld exceeds the int32 column index range", (long long)n);
  int global = 0;
  CKS(validate_common(k, &p, sub, prec, &global));
  if (!is_device_ptr(rowptr) || !is_device_ptr(colind) || !is_device_ptr(vals))
    return fail(BCG_ERR_INVALID_ARG, "rowptr, colind and vals must be device pointers");
  bcg_ctx *h = new (std::nothrow) bcg_ctx;
  if (h == nullptr) return fail(BCG_ERR_OOM, "host allocation failed");
  h->n = n; h->nnz = nnz; h->k = k; h->p = p; h->global = global; h->prec = prec;
  h->nblk = global ? 1 : k / p;
  h->opkind = OP_CSR;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->A64.kind = OP_CSR; h->A64.n = n; h->A64.rowptr = rowptr; h->A64.colind = colind; h->A64.vals = vals;
  h->ncoef = nnz;
  return finish_create(h, out);
}

bcg_status bcg_create_sell(bcg_handle *out, int64_t n, int64_t nent, const int64_t *chunkptr, const int32_t *rowlen,
                           const int32_t *colind, const double *vals, const int32_t *perm, int32_t k, int32_t p,
                           int32_t sub, int32_t prec, void *cuda_stream) {
  if (out == nullptr) return fail(BCG_ERR_INVALID_ARG, "handle pointer is NULL");
  *out = nullptr;
  if (n < 1 || nent < 1) return fail(BCG_ERR_INVALID_ARG, "n=%lld nent=%lld must be >= 1", (long long)n, (long long)nent);
  if (n > INT32_MAX) return fail(BCG_ERR_INVALID_ARG, "n=%lld exceeds the int32 column index range", (long long)n);
  int global = 0;
  CKS(validate_common(k, &p, sub, prec, &global));
  if (!is_device_ptr(chunkptr) || !is_device_ptr(rowlen) || !is_device_ptr(colind) || !is_device_ptr(vals) ||
      !is_device_ptr(perm))
    return fail(BCG_ERR_INVALID_ARG, "chunkptr, rowlen, colind, vals and perm must be device pointers");
  bcg_ctx *h = new (std::nothrow) bcg_ctx;
  if (h == nullptr) return fail(BCG_ERR_OOM, "host allocation failed");
  h->n = n; h->nnz = nent; h->k = k; h->p = p; h->global = global; h->prec = prec;
  h->nblk = global ? 1 : k / p;
  h->opkind = OP_SELL;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->A64.kind = OP_SELL; h->A64.n = n; h->A64.rowptr = chunkptr; h->A64.colind = colind; h->A64.vals = vals;
  h->A64.rowlen = rowlen;
  h->ncoef = nent;
  h->perm = perm;
  if (h->alloc(&h->Bp, (size_t)n * k) != BCG_OK || h->alloc(&h->Xp, (size_t)n * k) != BCG_OK) {
    delete h;
    return BCG_ERR_OOM;
  }
  return finish_create(h, out);
}

bcg_status bcg_create_stencil(bcg_handle *out, int32_t kind, int32_t nx, int32_t ny, int32_t nz, const double *coef,
                              double scale, int32_t k, int32_t p, int32_t sub, int32_t prec, void *cuda_stream) {
  if (out == nullptr) return fail(BCG_ERR_INVALID_ARG, "handle pointer is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(BCG_ERR_INVALID_ARG, "grid %d x %d x %d invalid", nx, ny, nz);
  if (!(scale > 0.0) || !std::isfinite(scale)) return fail(BCG_ERR_INVALID_ARG, "scale must be finite and > 0");
  int opk;
  switch (kind) {
    case BCG_STENCIL_5PT_2D: opk = OP_ST5; if (nz != 1) return fail(BCG_ERR_INVALID_ARG, "2D stencil needs nz = 1"); break;
    case BCG_STENCIL_7PT_3D: opk = OP_ST7; break;
    case BCG_STENCIL_7PT_3D_VARCOEF: opk = OP_ST7VC; break;
    default: return fail(BCG_ERR_INVALID_ARG, "unknown stencil kind %d", kind);
  }
  if (opk == OP_ST7VC && !is_device_ptr(coef)) return fail(BCG_ERR_INVALID_ARG, "varcoef stencil needs device faces");
  if (opk != OP_ST7VC && coef != nullptr) return fail(BCG_ERR_INVALID_ARG, "constant stencils take coef = NULL");
  const int64_t n = (int64_t)nx * ny * nz;
  int global = 0;
  CKS(validate_common(k, &p, sub, prec, &global));
  bcg_ctx *h = new (std::nothrow) bcg_ctx;
  if (h == nullptr) return fail(BCG_ERR_OOM, "host allocation failed");
  h->n = n; h->k = k; h->p = p; h->global = global; h->prec = prec;
  h->nblk = global ? 1 : k / p;
  h->opkind = opk;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->A64.kind = opk; h->A64.n = n; h->A64.nx = nx; h->A64.ny = ny; h->A64.nz = nz; h->A64.scale = scale;
  h->A64.faces = coef;
  h->ncoef = opk == OP_ST7VC ? (int64_t)nz * ny * (nx + 1) + (int64_t)nz * (ny + 1) * nx + (int64_t)(nz + 1) * ny * nx : 0;
  return finish_create(h, out);
}

bcg_status bcg_set_option(bcg_handle h, const char *key, double value) {
  if (h == nullptr || key == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle or key");
  if (!std::isfinite(value)) return fail(BCG_ERR_INVALID_ARG, "option value must be finite");
  if (!strcmp(key, "inner_tol")) {
    if (!(value > 0.0 && value < 1.0)) return fail(BCG_ERR_INVALID_ARG, "inner_tol must lie in (0, 1)");
    h->inner_tol = value;
  } else if (!strcmp(key, "max_outer")) {
    if (value < 1 || value > 1000) return fail(BCG_ERR_INVALID_ARG, "max_outer must lie in 1..1000");
    h->max_outer = (int)value;
  } else if (!strcmp(key, "check_every")) {
    if (value < 1 || value > 4096) return fail(BCG_ERR_INVALID_ARG, "check_every must lie in 1..4096");
    h->check_every = (int)value;
  } else if (!strcmp(key, "profile")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "profile must be 0 or 1");
    h->profile = (int)value;
    for (int i = 0; i < bcg_ctx::kKernels; ++i) { h->prof_ms[i] = 0.0; h->prof_count[i] = 0; }
  } else if (!strcmp(key, "refine")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "refine must be 0 (restart) or 1 (replace)");
    h->refine = (int)value;
  } else if (!strcmp(key, "precond")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "precond must be 0 (none) or 1 (Jacobi)");
    h->precond = (int)value;
    if (h->graph32) {   // captured graphs hold the preconditioner pointer
      cudaGraphExecDestroy(h->graph32);
      h->graph32 = nullptr;
    }
  } else if (!strcmp(key, "retooled")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "retooled must be 0 or 1");
    if (value == 1.0 && (h->prec != BCG_FP64 || h->rows_mode))
      return fail(BCG_ERR_INVALID_ARG, "the retooled form needs an FP64 handle (not row-sharded)");
    h->retooled = (int)value;
  } else if (!strcmp(key, "tensor_cores")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "tensor_cores must be 0 or 1");
    h->tensor_cores = (int)value;
  } else if (!strcmp(key, "guards")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "guards must be 0 or 1");
    h->guards = (int)value;
  } else if (!strcmp(key, "graph")) {
    if (value != 0.0 && value != 1.0) return fail(BCG_ERR_INVALID_ARG, "graph must be 0 or 1");
    h->use_graph = (int)value;
  } else {
    return fail(BCG_ERR_INVALID_ARG, "unknown option '%s'", key);
  }
  return BCG_OK;
}

bcg_status bcg_solve(bcg_handle h, const double *B, double *X, double tol, int32_t maxit, bcg_info *info) {
  NvtxRange range_("bcg_solve");
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (h->rows_mode) return fail(BCG_ERR_INVALID_ARG, "row-sharded handle: drive it with the bcg_rows_* calls");
  if (!is_device_ptr(B) || !is_device_ptr(X)) return fail(BCG_ERR_INVALID_ARG, "B and X must be device pointers");
  if (B == X) return fail(BCG_ERR_INVALID_ARG, "B and X must not alias");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(BCG_ERR_INVALID_ARG, "tol must be finite and > 0");
  if (maxit < 1) return fail(BCG_ERR_INVALID_ARG, "maxit must be >= 1");
  g_last_error.clear();
  auto run = [&](const double *Bs, double *Xs) {
    if (h->prec != BCG_FP32_REFINE) {
      if (h->retooled) return solve_retooled(h, Bs, Xs, tol, maxit, info);
      return solve_fp64(h, Bs, Xs, tol, maxit, info);
    }
    return h->refine ? solve_replace(h, Bs, Xs, tol, maxit, info) : solve_refine(h, Bs, Xs, tol, maxit, info);
  };
  auto guarded = [&](bcg_status st) {
    if (!h->guards || st == BCG_ERR_INVALID_ARG || st == BCG_ERR_CUDA || st == BCG_ERR_OOM) return st;
    const bcg_status g = check_guards(h);
    return g == BCG_OK ? st : g;
  };
  if (h->perm == nullptr) return guarded(run(B, X));
  // SELL-C-sigma handle: iterate on the permuted system (Pi A Pi^T)(Pi X) = Pi B
  CK(launch_permute_rows(B, h->perm, h->n, h->k, h->Bp, 0, h->nsm, h->stream));
  CK(launch_permute_rows(X, h->perm, h->n, h->k, h->Xp, 0, h->nsm, h->stream));
  const bcg_status st = run(h->Bp, h->Xp);
  if (st == BCG_ERR_INVALID_ARG || st == BCG_ERR_CUDA || st == BCG_ERR_OOM) return st;
  const std::string msg = g_last_error;
  CK(launch_permute_rows(h->Xp, h->perm, h->n, h->k, X, 1, h->nsm, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  g_last_error = msg;
  return guarded(st);
}

bcg_status bcg_solve_host(bcg_handle h, const double *B, double *X, double tol, int32_t maxit, bcg_info *info) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (h->rows_mode) return fail(BCG_ERR_INVALID_ARG, "row-sharded handle: drive it with the bcg_rows_* calls");
  if (B == nullptr || X == nullptr) return fail(BCG_ERR_INVALID_ARG, "B and X must not be NULL");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(BCG_ERR_INVALID_ARG, "tol must be finite and > 0");
  if (maxit < 1) return fail(BCG_ERR_INVALID_ARG, "maxit must be >= 1");
  const size_t bytes = sizeof(double) * (size_t)h->n * h->k;
  // each staging buffer is allocated once; a failed allocation leaves its pointer NULL, so the next call retries it
  if (h->stageB == nullptr) CKS(h->alloc(&h->stageB, (size_t)h->n * h->k));
  if (h->stageX == nullptr) CKS(h->alloc(&h->stageX, (size_t)h->n * h->k));
  CK(cudaMemcpyAsync(h->stageB, B, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->stageX, X, bytes, cudaMemcpyHostToDevice, h->stream));
  const bcg_status st = bcg_solve(h, h->stageB, h->stageX, tol, maxit, info);
  if (st == BCG_ERR_INVALID_ARG || st == BCG_ERR_CUDA || st == BCG_ERR_OOM) return st;
  const std::string msg = g_last_error;
  CK(cudaMemcpyAsync(X, h->stageX, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  g_last_error = msg;
  return st;
}

bcg_status bcg_block_iters(bcg_handle h, int32_t *out, int32_t cap) {
  if (h == nullptr || out == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL argument");
  if (cap < h->nblk) return fail(BCG_ERR_INVALID_ARG, "cap=%d < number of blocks %d", cap, h->nblk);
  for (int j = 0; j < h->nblk; ++j) out[j] = h->last_block_iters[j];
  return BCG_OK;
}

bcg_status bcg_grad_values(bcg_handle h, const double *Lambda, const double *X, double *grad) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (h->opkind != OP_CSR) return fail(BCG_ERR_INVALID_ARG, "gradient needs a CSR handle");
  if (!is_device_ptr(Lambda) || !is_device_ptr(X) || !is_device_ptr(grad))
    return fail(BCG_ERR_INVALID_ARG, "Lambda, X and grad must be device pointers");
  CK(launch_grad_values(h->rowidx, h->A64.colind, Lambda, X, h->nnz, h->k, grad, h->nsm, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

bcg_status bcg_update_values(bcg_handle h, const double *vals) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (h->ncoef == 0) return fail(BCG_ERR_INVALID_ARG, "constant stencils have no values");
  if (!is_device_ptr(vals)) return fail(BCG_ERR_INVALID_ARG, "vals must be a device pointer");
  if (h->opkind == OP_CSR || h->opkind == OP_SELL) h->A64.vals = vals;
  else h->A64.faces = vals;
  CKS(make_fp32_copy(h));
  if (h->graph32) {   // captured graphs hold the old operator descriptor
    cudaGraphExecDestroy(h->graph32);
    h->graph32 = nullptr;
  }
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

bcg_status bcg_bdot(bcg_handle h, const double *X, const double *Y, double *gamma) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (!is_device_ptr(X) || !is_device_ptr(Y) || !is_device_ptr(gamma))
    return fail(BCG_ERR_INVALID_ARG, "X, Y and gamma must be device pointers");
  // Gram shifts from the column maxima of X and of Y (a pass over each operand)
  int *shX = h->bdot_sh, *shY = h->bdot_sh + h->k;
  CK(launch_col_shifts(X, h->n, h->k, h->tmp2k, shX, h->nsm, h->stream));
  CK(launch_col_shifts(Y, h->n, h->k, h->tmp2k + h->k, shY, h->nsm, h->stream));
  if (h->p > kMaxP) {
    CK(launch_lp_gram<double>(X, Y, h->n, h->k, h->p, h->global, nullptr, h->partA, h->g64.op, nullptr, h->stream,
                              nullptr, shX, shY));
    CK(launch_finish_gram(h->partA, h->g64.op, h->k, h->p, h->global, gamma, h->gws, h->stream));
  } else {
    const int grid = std::min(h->nparts, bdot_grid<double>(h->n, h->k, h->p, h->nsm));
    CK(launch_bdot<double>(X, Y, h->n, h->k, h->p, h->partA, grid, h->stream, shX, shY));
    CK(launch_finish_gram(h->partA, grid, h->k, h->p, h->global, gamma, h->gws, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

bcg_status bcg_bdot_f32(bcg_handle h, const float *X, const float *Y, double *gamma) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (!is_device_ptr(X) || !is_device_ptr(Y) || !is_device_ptr(gamma))
    return fail(BCG_ERR_INVALID_ARG, "X, Y and gamma must be device pointers");
  if (h->p > kMaxP) {
    CK(launch_lp_gram<float>(X, Y, h->n, h->k, h->p, h->global, nullptr, h->partA, h->g64.op, nullptr, h->stream,
                             nullptr, nullptr, nullptr));
    CK(launch_finish_gram(h->partA, h->g64.op, h->k, h->p, h->global, gamma, h->gws, h->stream));
  } else {
    const int grid = std::min(h->nparts, bdot_grid<float>(h->n, h->k, h->p, h->nsm));
    CK(launch_bdot<float>(X, Y, h->n, h->k, h->p, h->partA, grid, h->stream, nullptr, nullptr));
    CK(launch_finish_gram(h->partA, grid, h->k, h->p, h->global, gamma, h->gws, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

bcg_status bcg_bop(bcg_handle h, const double *X, double *Y) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (!is_device_ptr(X) || !is_device_ptr(Y) || X == Y) return fail(BCG_ERR_INVALID_ARG, "X, Y: distinct device pointers");
  if (h->perm == nullptr) {
    CK(launch_bop<double>(h->A64, X, Y, h->n, h->k, h->g64.res, h->stream));
  } else {   // Y = Pi^T (Pi A Pi^T) Pi X
    CK(launch_permute_rows(X, h->perm, h->n, h->k, h->Xp, 0, h->nsm, h->stream));
    CK(launch_bop<double>(h->A64, h->Xp, h->Bp, h->n, h->k, h->g64.res, h->stream));
    CK(launch_permute_rows(h->Bp, h->perm, h->n, h->k, Y, 1, h->nsm, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return BCG_OK;
}

bcg_status bcg_profile(bcg_handle h, double *ms, int64_t *count, int32_t cap) {
  if (h == nullptr || ms == nullptr || count == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL argument");
  if (cap < bcg_ctx::kKernels) return fail(BCG_ERR_INVALID_ARG, "cap=%d < %d", cap, bcg_ctx::kKernels);
  for (int i = 0; i < bcg_ctx::kKernels; ++i) { ms[i] = h->prof_ms[i]; count[i] = h->prof_count[i]; }
  return BCG_OK;
}

bcg_status bcg_create_csr_rows(bcg_handle *out, int64_t n_local, int64_t n_cols, int64_t nnz, const int64_t *rowptr,
                               const int32_t *colind, const double *vals, int32_t k, int32_t p, int32_t sub,
                               void *cuda_stream) {
  if (out == nullptr) return fail(BCG_ERR_INVALID_ARG, "handle pointer is NULL");
  *out = nullptr;
  if (n_local < 1 || nnz < 1 || n_cols < n_local)
    return fail(BCG_ERR_INVALID_ARG, "n_local=%lld, n_cols=%lld, nnz=%lld: need n_local >= 1, nnz >= 1, "
                "n_cols >= n_local", (long long)n_local, (long long)n_cols, (long long)nnz);
  if (n_cols > INT32_MAX) return fail(BCG_ERR_INVALID_ARG, "n_cols exceeds the int32 column index range");
  int global = 0;
  CKS(validate_common(k, &p, sub, BCG_FP64, &global));
  if (!is_device_ptr(rowptr) || !is_device_ptr(colind) || !is_device_ptr(vals))
    return fail(BCG_ERR_INVALID_ARG, "rowptr, colind and vals must be device pointers");
  bcg_ctx *h = new (std::nothrow) bcg_ctx;
  if (h == nullptr) return fail(BCG_ERR_OOM, "host allocation failed");
  h->n = n_local; h->ncols = n_cols; h->nnz = nnz; h->k = k; h->p = p; h->global = global; h->prec = BCG_FP64;
  h->rows_mode = 1;
  h->nblk = global ? 1 : k / p;
  h->opkind = OP_CSR;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->A64.kind = OP_CSR; h->A64.n = n_local; h->A64.rowptr = rowptr; h->A64.colind = colind; h->A64.vals = vals;
  h->ncoef = nnz;
  return finish_create(h, out);
}

static bcg_status rows_handle(bcg_handle h) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (!h->rows_mode) return fail(BCG_ERR_INVALID_ARG, "not a row-sharded handle (bcg_create_csr_rows)");
  return BCG_OK;
}

bcg_status bcg_rows_bind(bcg_handle h, double *sums1, double *sums2) {
  CKS(rows_handle(h));
  if (!is_device_ptr(sums1) || !is_device_ptr(sums2) || sums1 == sums2)
    return fail(BCG_ERR_INVALID_ARG, "sums1 and sums2 must be distinct device pointers");
  h->sums1 = sums1;
  h->sums2 = sums2;
  return BCG_OK;
}

bcg_status bcg_rows_start(bcg_handle h, const double *B, double *X, double tol) {
  CKS(rows_handle(h));
  if (!is_device_ptr(B) || !is_device_ptr(X)) return fail(BCG_ERR_INVALID_ARG, "B and X must be device pointers");
  if (!(tol >= 0.0)) return fail(BCG_ERR_INVALID_ARG, "tol=%g must be >= 0", tol);
  if (h->sums1 == nullptr) return fail(BCG_ERR_INVALID_ARG, "bcg_rows_bind has not been called");
  h->X_rows = X;
  CKS(set_tol2(h, tol * tol));
  const int64_t E = (int64_t)h->k * h->p;
  CK(launch_residual<double>(h->A64, X, B, h->R, h->P, nullptr, nullptr, h->n, h->k, h->partN, h->g64.res, h->stream,
                             dinv_of<double>(h)));
  CK(launch_sum_partials(h->partN, h->g64.res, h->k, h->sums2 + E, h->nsm, h->stream));
  if (h->g64.rho_k3) {   // the first recomputed rho travels in sums1 with the first alpha
    // its Gram shifts from this rank's own column norms (the partial sums are unshifted, so ranks need not agree;
    // bcg_rows_start_status rewrites the shifts from the summed norms)
    CK(launch_fill_shifts(h->sums2 + E, h->k, shifts_of<double>(h), h->stream));
    CKS(first_rho_rec<double>(h, h->P, h->R, h->g64));
    CK(launch_sum_partials(h->partR, h->precond ? h->g64.pup_zs : h->g64.pup, E, h->sums1 + E, h->nsm, h->stream));
  }
  return BCG_OK;
}

bcg_status bcg_rows_start_status(bcg_handle h) {
  CKS(rows_handle(h));
  const int64_t E = (int64_t)h->k * h->p;
  CK(launch_init_status(h->sums2 + E, 1, h->k, h->p, h->global, h->r0n2, h->rn2, h->active, h->block_iters, h->lam,
                        h->beta, h->st, h->stream, shifts_of<double>(h)));
  return BCG_OK;
}

bcg_status bcg_rows_phase(bcg_handle h, int32_t phase) {
  CKS(rows_handle(h));
  if (phase < 1 || phase > 3) return fail(BCG_ERR_INVALID_ARG, "phase=%d must be 1, 2 or 3", phase);
  if (h->X_rows == nullptr) return fail(BCG_ERR_INVALID_ARG, "bcg_rows_start has not been called");
  return rows_phase(h, phase);
}

bcg_status bcg_rows_pack(bcg_handle h, const int32_t *rows, int64_t nrows, double *buf) {
  CKS(rows_handle(h));
  if (nrows < 0) return fail(BCG_ERR_INVALID_ARG, "nrows=%lld < 0", (long long)nrows);
  if (nrows == 0) return BCG_OK;
  if (!is_device_ptr(rows) || !is_device_ptr(buf)) return fail(BCG_ERR_INVALID_ARG, "rows and buf must be device pointers");
  CK(launch_gather_rows(h->P, rows, nrows, h->k, buf, h->nsm, h->stream));
  return BCG_OK;
}

bcg_status bcg_rows_unpack(bcg_handle h, const double *halo, int64_t nrows) {
  CKS(rows_handle(h));
  if (nrows != h->ncols - h->n)
    return fail(BCG_ERR_INVALID_ARG, "nrows=%lld, this rank has %lld halo rows", (long long)nrows,
                (long long)(h->ncols - h->n));
  if (nrows == 0) return BCG_OK;
  if (!is_device_ptr(halo)) return fail(BCG_ERR_INVALID_ARG, "halo must be a device pointer");
  CK(cudaMemcpyAsync(h->P + h->n * h->k, halo, sizeof(double) * nrows * h->k, cudaMemcpyDeviceToDevice, h->stream));
  return BCG_OK;
}

bcg_status bcg_rows_poll(bcg_handle h, int32_t *done) {
  CKS(rows_handle(h));
  if (!done) return fail(BCG_ERR_INVALID_ARG, "NULL output pointer");
  CKS(read_status(h));
  *done = h->h_st->flags != 0 ? 1 : 0;
  return BCG_OK;
}

bcg_status bcg_rows_finish(bcg_handle h, bcg_info *info) {
  CKS(rows_handle(h));
  CKS(read_status(h));
  const DevStatus fin = *h->h_st;
  CKS(fill_block_iters(h));
  CKS(fetch_vec(h, h->r0n2, 0));
  CKS(fetch_vec(h, h->rn2, 1));
  const bcg_status st = status_from_flags(fin.flags, (fin.flags & ST_DONE) != 0);
  if (info) {
    info->status = st;
    info->iters = fin.iter;
    info->outer_iters = 0;
    info->breakdown_iter = (fin.flags & ST_BREAKDOWN) ? fin.breakdown_iter : -1;
    info->max_rel_res_recursive = max_ratio(h->h_vec + h->k, h->h_vec, h->k);
    info->max_rel_res_true = NAN;   // needs the other ranks' rows of X: the caller recomputes it
  }
  h->X_rows = nullptr;
  if (h->guards) CKS(check_guards(h));
  return st;
}

const char *bcg_last_error(void) { return g_last_error.c_str(); }

bcg_status bcg_debug_poke_guard(bcg_handle h, int32_t index) {
  if (h == nullptr) return fail(BCG_ERR_INVALID_ARG, "NULL handle");
  if (index < 0 || (size_t)index >= h->allocs.size())
    return fail(BCG_ERR_INVALID_ARG, "index=%d, the handle has %zu workspace buffers", index, h->allocs.size());
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemset(static_cast<unsigned char *>(h->allocs[index]) + h->alloc_bytes[index], 0, 1));
  CK(cudaStreamSynchronize(0));
  return BCG_OK;
}

bcg_status bcg_debug_fail_alloc(int32_t nth) {
  if (nth < 0) return fail(BCG_ERR_INVALID_ARG, "nth=%d must be >= 0", nth);
  g_fail_alloc_in.store(nth);
  return BCG_OK;
}

void bcg_destroy(bcg_handle h) {
  if (h == nullptr) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  delete h;
}

}  // extern "C"
