// Host-side launchers of the device kernels (one translation unit per precision plus the small-solve
// unit); the C ABI in bcg_capi.cu only talks to these.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "bcg_kernels.cuh"

namespace bcgk {

// Largest p handled by the streaming kernels (per-thread Gram accumulators live in registers).
constexpr int kMaxP = 32;

// Exponent shifts of the FP64 Gram operands (bcg_kernels.cuh): a solver's shift array holds 3 k ints, one row
// of k per operand role -- R (the residual), P (directions and Z = M^{-1} R: R's shift plus the exponent of
// max|diag(A)^{-1}| under the Jacobi preconditioner), Q (A P: P's shift plus the exponent of A's largest
// absolute row sum). The small-solve kernels rewrite it from the column norms whenever those change.
enum ShiftRole { SH_R = 0, SH_P = 1, SH_Q = 2 };
inline const int *sh_role(const int *sh, int k, int role) { return sh ? sh + (size_t)role * k : nullptr; }

struct StreamGrids {
  int op;        // K1 CTAs
  int upd;       // K2 CTAs
  int pup;       // K3 CTAs
  int upd_zs;    // K2 CTAs, Jacobi-preconditioned instantiation
  int pup_zs;    // K3 CTAs, Jacobi-preconditioned instantiation
  int upd_df, upd_zs_df;   // K2 with double-float updates of R (0: not available)
  int res;       // K0 CTAs
  int alpha_circ;   // K1 stores alpha by circulant diagonals (symmetric product, half the terms)
  int rho_circ;     // K2 stores rho by circulant diagonals
  int rho_k3;       // the recomputed rho is formed by K3 (next iteration's) and a BDOT after K0, not by K1
};

// Sizes the grids for n rows from the occupancy of each kernel variant (capped to whole waves of SMs).
template <typename T>
cudaError_t stream_grids(int opkind, int64_t n, int k, int p, int global, int nsm, StreamGrids *out);

template <typename T>
cudaError_t launch_op_gram(const OpDesc &A, const T *P, const T *R, T *Q, int64_t n, int k, int p, int global,
                           const int *active, double *partA, double *partR, const DevStatus *st, int grid,
                           cudaStream_t s, const int *sh);
// dinv (optional, n values): inverse diagonal of the Jacobi preconditioner; Z = M^{-1} R is formed on the
// fly where Algorithm 1 needs it (NULL: M = I).
// df: the block updates in double-float arithmetic (FP64 data, 2 <= p <= 32 warp-chunk shapes; elsewhere the
// FP64 kernels run); grid must then be the df grid of StreamGrids.
template <typename T>
cudaError_t launch_update_xr(T *X, T *R, const T *P, const T *Q, int64_t n, int k, int p, int global,
                             const double *lam, const int *active, double *partRho, double *partN,
                             const DevStatus *st, int grid, cudaStream_t s, const T *dinv, const int *sh,
                             int df = 0);
template <typename T>
// partR: with rho_k3, the partials of the next iteration's recomputed rho <<P_new, R>>_S (one row per CTA)
cudaError_t launch_update_p(T *P, const T *R, int64_t n, int k, int p, int global, const double *beta,
                            const int *active, DevStatus *st, int grid, cudaStream_t s, const T *dinv,
                            double *partR, const int *sh);
template <typename T>
// sig (optional): R32 and P32 receive R 2^-sigma_c (the mixed form's scale)
cudaError_t launch_residual(const OpDesc &A, const T *X, const T *B, T *R, T *P, float *R32, float *P32, int64_t n,
                            int k, double *partN, int grid, cudaStream_t s, const T *dinv, const int *sig = nullptr);
// also the operator maxima behind the Gram shift offsets (opmax: 2 doubles, or NULL)
cudaError_t launch_inv_diag(const OpDesc &A, int64_t n, double *dinv, double *opmax, int nsm, cudaStream_t s);

template <typename T>
cudaError_t launch_bdot(const T *X, const T *Y, int64_t n, int k, int p, double *part, int grid, cudaStream_t s,
                        const int *shX, const int *shY);
template <typename T>
int bdot_grid(int64_t n, int k, int p, int nsm);
cudaError_t launch_finish_gram(const double *part, int nparts, int k, int p, int global, double *gamma, double *gws,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_bop(const OpDesc &A, const T *X, T *Y, int64_t n, int k, int grid, cudaStream_t s);

// large blocks (32 < p <= 256, p % 32 == 0): tiled products, see bcg_kernels_lp.cuh
int lp_chunks(int64_t n, int k, int p, int nsm);
template <typename T>
cudaError_t launch_lp_bop(const OpDesc &A, const T *P, T *Q, int64_t n, int k, const DevStatus *st, int nsm,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_lp_gram(const T *X, const T *Y, int64_t n, int k, int p, int global, const int *active,
                           double *part, int chunks, const DevStatus *st, cudaStream_t s, const T *xscale,
                           const int *shX, const int *shY);
template <typename T>
cudaError_t launch_lp_baxpy(T *OUT, const T *BASE, const T *Y, const double *C, int64_t n, int k, int p, int global,
                            double sign, const int *active, DevStatus *st, int bump, cudaStream_t s,
                            const T *bscale);
template <typename T>
cudaError_t launch_lp_colnorm(const T *R, int64_t n, int k, double *partN, int grid, const DevStatus *st,
                              cudaStream_t s, const int *shR);

// Tensor-core large-block products and updates (bcg_kernels_tc.cuh; FP64 data, or the mixed form's FP32 data; p a
// multiple of 64 up to 256).
// Every operand is first cut into bf16 digit images that are byte for byte the kernels' shared-memory stages:
// the p x p matrices with launch_tc_slice (C row-major per distinct block, Cs of tc_workspace_bytes(nblkC, p)
// bytes, Cexp nblkC * p ints); the Gram's operands into column images (an exponent per column:
// launch_tc_col_exp, then launch_tc_cut_cols; X times xscale per row if given); the BAXPY's Y into row images (an
// exponent per row of a block, written to erow: ceil(n / 128) * 128 * (k / p) ints). Then launch_tc_gram_img
// writes the partials of <<X, Y>>_S into `chunks` partial rows in the layout of launch_lp_gram, and
// launch_tc_baxpy_img forms OUT_j = BASE_j (x bscale) + sign Y_j C_j.
bool tc_ok(int k, int p);
// Blocks of 32 columns (k a multiple of 64) on the same kernels: launch_tc_pair_cmat writes the block-diagonal
// 64 x 64 matrices pairing consecutive blocks (k / 64 of them, one if global; 64 x 64 doubles each, row-major),
// which launch_tc_slice cuts with p = 64; launch_tc_cut_rows takes p = 32 (one exponent per row of each block);
// launch_tc_baxpy_img takes p = 64 and pe = 32.
bool tc_pair_ok(int k, int p);
// Blocks of 32 where 64 does not divide k: 32-column tiles (launch_tc_slice and launch_tc_baxpy_img with p = 32)
bool tc_b32_ok(int k, int p);
cudaError_t launch_tc_pair_cmat(const double *C, int k, int p, int global, double *out, cudaStream_t s);
size_t tc_workspace_bytes(int nblkC, int p);
cudaError_t launch_tc_slice(const double *C, int nblkC, int p, uint16_t *Cs, int *Cexp, cudaStream_t s);
size_t tc_row_image_size(int64_t n, int k);
size_t tc_col_image_size(int64_t n, int k);
// T = double or float (the mixed form's FP32 process: FP32 values are exact in the 48-bit cut)
template <typename T>
cudaError_t launch_tc_col_exp(const T *X, const T *xscale, int64_t n, int k, int *ecol, int nsm, cudaStream_t s);
template <typename T>
cudaError_t launch_tc_cut_cols(const T *X, const T *xscale, int64_t n, int k, const int *ecol, unsigned char *img,
                               int nsm, cudaStream_t s);
template <typename T>
cudaError_t launch_tc_cut_rows(const T *Y, int64_t n, int k, int p, unsigned char *img, int *erow, cudaStream_t s);
cudaError_t launch_tc_gram_img(const unsigned char *imgX, const unsigned char *imgY, int64_t n, int k, int p,
                               int global, const int *active, double *part, int chunks, const int *ecx,
                               const int *ecy, DevStatus *st, cudaStream_t s);
// T is deduced from OUT alone (BASE and bscale may be NULL)
template <typename T>
struct TcId {
  using type = T;
};
template <typename T>
cudaError_t launch_tc_baxpy_img(T *OUT, const typename TcId<T>::type *BASE, const unsigned char *imgY,
                                const int *erow, const uint16_t *Cs, const int *Cexp, int64_t n, int k, int p,
                                int global, double sign, const int *active, DevStatus *st, int bump, cudaStream_t s,
                                const typename TcId<T>::type *bscale, int nsm, int pe = 0);
// doubles of per-block workspace of the p x p solves; kept in global memory (gws) when too big for shared
size_t small_ws_doubles(int p);
bool small_needs_gws(int p);

cudaError_t small_prepare(int p);
// nparts: partial rows of alpha; nparts_r: partial rows of the recomputed rho
cudaError_t launch_solve_lambda(const double *partA, const double *partR, int nparts, int nparts_r, int k, int p,
                                int global, const int *active, double *lam, double *rho_rec, DevStatus *st,
                                double *gws, int alpha_circ, cudaStream_t s);
// nparts: partial rows of rho; nparts_n: partial rows of the column norms
cudaError_t launch_solve_beta(const double *partRho, const double *partN, int nparts, int nparts_n, int k, int p,
                              int global, const double *tol2, const double *r0n2, double *rn2, int *active,
                              int *block_iters,
                              const double *rho_rec, double *beta, DevStatus *st, double *gws, int rho_circ,
                              cudaStream_t s, const ShiftCtl &sc);
cudaError_t launch_init_status(const double *partN, int nparts, int k, int p, int global, double *r0n2, double *rn2,
                               int *active, int *block_iters, double *lam, double *beta, DevStatus *st,
                               cudaStream_t s, const ShiftCtl &sc);
// Rewrites sc.sh from the squared column norms n2 (NULL: every column's base shift 0, offsets only).
cudaError_t launch_fill_shifts(const double *n2, int k, const ShiftCtl &sc, cudaStream_t s);
cudaError_t launch_reduce_norms(const double *partN, int nparts, int k, double *out, cudaStream_t s);
cudaError_t launch_reactivate(const double *rtn2, const double *r0n2, double tol2, int k, int p, int global,
                              int *active, DevStatus *st, cudaStream_t s);
cudaError_t launch_sum_partials(const double *part, int nparts, int64_t E, double *out, int nsm, cudaStream_t s);
cudaError_t launch_gather_rows(const double *P, const int32_t *rows, int64_t nrows, int k, double *buf, int nsm,
                               cudaStream_t s);
cudaError_t launch_permute_rows(const double *src, const int32_t *perm, int64_t n, int k, double *dst, int scatter,
                                int nsm, cudaStream_t s);
// X += D 2^sigma_c with the mixed form's per-column scale exponents sig (NULL: 0)
cudaError_t launch_add_correction(double *X, const float *D, int64_t len, int k, const int *sig, int nsm,
                                  cudaStream_t s);
// Gram shifts of a standalone BDOT operand: sh[c] from max_r |X[r][c]| (cmax: k doubles of scratch)
cudaError_t launch_col_shifts(const double *X, int64_t n, int k, double *cmax, int *sh, int nsm, cudaStream_t s);
// the mixed form's FP32 scale per block from the squared column norms cur; cur_s, ref_s (optional) receive cur
// and ref in the scaled process's units
cudaError_t launch_mixed_scale(const double *cur, const double *ref, int k, int p, int global, int *sig,
                               double *cur_s, double *ref_s, cudaStream_t s);
// R32 = fl(R 2^-sigma), P32 = fl(M^{-1} R 2^-sigma) (P32, dinv optional)
cudaError_t launch_cast_scaled(const double *R, const double *dinv, const int *sig, int64_t n, int k, float *R32,
                               float *P32, int nsm, cudaStream_t s);
cudaError_t launch_cast_to_float(const double *src, float *dst, int64_t len, int nsm, cudaStream_t s);
cudaError_t launch_grad_values(const int32_t *rowidx, const int32_t *colind, const double *Lam, const double *X,
                               int64_t nnz, int k, double *grad, int nsm, cudaStream_t s);
cudaError_t launch_row_index(const int64_t *rowptr, int64_t n, int32_t *rowidx, int nsm, cudaStream_t s);

// Retooled block CG (bcg_retooled.inc), FP64, every subalgebra, M = I or Jacobi (dinv = 1 / diag(A), NULL: I):
// streaming kernels for p <= 32 (the large-block path uses launch_lp_*), and the Cholesky QR kernels. Cf (C),
// xi, lam, psiinv (psi^{-1}) and phi (psi^T) hold one row-major p x p matrix per coefficient block (q of them,
// or one for the global subalgebra). launch_dr_baxpy: BASE may be NULL (zero), rscale a row scale (or NULL).
// partial-row count of the gamma products of the streaming retooled path (<= cap, the partial buffers' rows)
int dr_grid_for(int64_t n, int k, int p, int nsm, int cap, int jac);
// partials of <<M^{-1} X, Y>> per column block (dinv NULL: <<X, Y>>)
cudaError_t launch_dr_gram(const double *X, const double *Y, int64_t n, int k, int p, const int *active,
                           double *part, int grid, const DevStatus *st, cudaStream_t s, const int *shX,
                           const int *shY, int global, const double *dinv);
// X += S lambda, Qb = Qb - W xi (= T), partials of <<T, T>> per column block, and (dinv) of <<T, M^{-1} T>>
cudaError_t launch_dr_update_xt(double *X, double *Qb, const double *S, const double *W, int64_t n, int k, int p,
                                const double *lam, const double *xi, const int *active, double *part, int grid,
                                const DevStatus *st, cudaStream_t s, int global, const double *dinv,
                                double *partM);
// Qb = Qb psiinv, S = M^{-1} Qb + S phi (in place); advances the iteration counter
cudaError_t launch_dr_update_qs(double *Qb, double *S, int64_t n, int k, int p, const double *psiinv,
                                const double *phi, const int *active, DevStatus *st, int nsm, cudaStream_t s,
                                int global, const double *dinv);
cudaError_t launch_dr_baxpy(double *OUT, const double *BASE, const double *Y, const double *C, int64_t n, int k,
                            int p, double sign, const int *active, DevStatus *st, int bump, int nsm,
                            cudaStream_t s, int global, const double *rscale);
cudaError_t launch_dr_scale_rows(double *OUT, const double *IN, const double *rs, int64_t n, int k, int nsm,
                                 cudaStream_t s);
cudaError_t launch_dr_start(const double *partG, int nparts, int k, int p, const int *active, double *Cf,
                            double *psiinv, DevStatus *st, double *gws, cudaStream_t s, int global);
// alpha_circ: the alpha partials are K1's circulant-diagonal storage
cudaError_t launch_dr_xi(const double *partA, int nparts, int k, int p, const int *active, const double *Cf,
                         double *xi, double *lam, DevStatus *st, double *gws, int alpha_circ, cudaStream_t s,
                         int global);
// stopping test from the per-column-block partials of <<T, T>> (partG); gamma from partGM (M^{-1} product) or,
// without it, from partG (summed over the column blocks for the global subalgebra)
cudaError_t launch_dr_psi(const double *partG, int nparts, int k, int p, const double *tol2, const double *r0n2,
                          double *rn2, int *active, int *block_iters, double *Cf, double *psiinv, double *phi,
                          DevStatus *st, double *gws, cudaStream_t s, int global, const double *partGM);

}  // namespace bcgk
