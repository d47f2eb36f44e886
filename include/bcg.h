/*
 * bcg.h -- C ABI of libbcg.so, a GB300 (sm_103a) implementation of the hot path of the generalized
 * Block Conjugate Gradients method (Dreier & Engwer, "Strategies for the vectorized Block Conjugate
 * Gradients method", arXiv 1912.11930).
 *
 * The library solves A X = B for a sparse symmetric positive definite A (n x n) and n x k blocks B, X
 * with Algorithm 1 of Section 3 (stabilised block CG, preconditioner M = I or Jacobi). Every block
 * product is restricted to one *-subalgebra S of R^{k x k} (Section 2, Definition "Relevant *-subalgebras"):
 *   hybrid    S_Hy^p = diag((R^{p x p})^q), q = k/p: q independent p x p Gram blocks;
 *   global    S_Gl^p = R^{p x p} (x) I_q: one p x p Gram summed over the q blocks, applied to each;
 *   parallel  S_Pl   = S_Hy^1: k independent CGs in lockstep;
 *   classical S_Cl   = S_Hy^k = S_Gl^k: O'Leary's block CG.
 * Column block j is the contiguous column range [j p, (j+1) p).
 *
 * Conventions for every function:
 *  - Block vectors are row-major n x k with leading dimension k: element (i, c) at i*k + c.
 *  - "device" pointers must be CUDA device (or managed) memory of the current device; "host" pointers
 *    ordinary or pinned host memory.
 *  - The caller owns every array it passes in. A handle BORROWS the matrix arrays given to
 *    bcg_create_* until bcg_destroy (they must stay valid and unchanged, except through
 *    bcg_update_values) and OWNS all of its workspace, allocated once at create time.
 *  - Every function returns a bcg_status and never aborts the process. Argument errors are detected on
 *    the host before any launch and leave all outputs untouched. bcg_last_error() describes the most
 *    recent failure of the calling thread.
 *  - Work is ordered on the handle's CUDA stream; bcg_solve returns after the final status is known.
 *  - A handle may be used by one thread at a time.
 *
 * Arithmetic of the FP64 form (BCG_FP64):
 *  - BOP (Y = A X), the block updates (BAXPY) and the p x p Cholesky/LU solves (BSOLVE) are IEEE FP64
 *    operations (fused multiply-adds), except for the block updates that the tensor-core path below forms.
 *  - Block products (BDOT: alpha, the recomputed rho, rho, the column norms of the stopping test) are not
 *    summed with FP64 operations. Each FP64 operand column c is first scaled by an exact power of two 2^-s_c
 *    (s_c from the column's latest 2-norm in the solver, from its largest entry in bcg_bdot), then every value
 *    is split into two floats hi + lo holding its leading 48 significant bits (|x - hi - lo| <= 2^-47 |x|).
 *    The products hi*hi (exactly, by TwoProd), hi*lo and lo*hi are accumulated as an unevaluated float pair
 *    per entry with error-free transformations (algorithm Dot2 of Ogita, Rump & Oishi, SIAM J. Sci. Comput.
 *    26(6), 2005); lo*lo (relative weight 2^-48) is dropped. Every 128 rows each pair is scaled back by
 *    2^(s_a + s_b) and added into FP64 sums, which are reduced over threads and CTAs in FP64 in a fixed
 *    order (bitwise repeatable).
 *  - Error: |computed - exact| <= about 2^-46 sum_r |x_ra y_rb| per entry (tested at 1e-13 of that sum), plus
 *    at most n 2^-100 max_r|x_ra| max_r|y_rb| from entries whose scaled product falls below FP32's range.
 *  - Range: any FP64 operands whose products and sums are finite in FP64 (tested with entries from 1e-300 to
 *    1e300 and exact zeros, and with B scaled by 1e+-30 and A by 1e+-10); within the solver a column may
 *    grow by about 2^50 or shrink by about 2^49 between two norm updates without loss.
 *  - Tensor cores (option "tensor_cores", on by default): with p a multiple of 64 (up to 256) the block products
 *    and block updates, and with p = 32 the block updates, are formed on the tensor
 *    cores instead (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012). Every operand value is truncated
 *    to 48 bits below an exponent shared along the contraction (per row of a block for the updated block Y,
 *    per column for lambda / beta and for the operands of the products) and cut into eight 6-bit digits held
 *    exactly in bf16. The 36 digit pairs of weight at least 2^-42 are multiplied and summed exactly in FP32
 *    (at most 512 terms before each read-out). The eight partial sums are combined with error-free float
 *    additions, and an update adds the result to its base with one FP64 addition. Error per entry: about
 *    2^-44 sum |u v| (truncation where the values sharing an exponent are of one magnitude; at most
 *    2^-47 max|u| sum|v| + 2^-47 max|v| sum|u|), plus about 2^-45 sum |u v| (the dropped pairs); FP64 FMAs
 *    give about K 2^-53 of it. Range: as the block products above (exponents are taken per row or column).
 */
#ifndef BCG_H
#define BCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcg_ctx *bcg_handle;

typedef enum {
  BCG_OK = 0,
  BCG_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or option; nothing was launched            */
  BCG_ERR_CUDA = 2,          /* a CUDA runtime call failed                                          */
  BCG_ERR_OOM = 3,           /* workspace allocation failed; nothing is leaked                      */
  BCG_ERR_BREAKDOWN = 4,     /* a p x p pivot <= 64 eps max|diag| or not finite (no deflation, the
                                method of Section 3 has none); X holds the last completed iterate    */
  BCG_ERR_NOT_CONVERGED = 5, /* maxit reached; X holds the last iterate, info is filled              */
  BCG_ERR_NUMERIC = 6,       /* a non-finite value in B, X0 or a residual norm                       */
  BCG_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                                  */
  BCG_ERR_GUARD = 8          /* option "guards": the guard bytes after a workspace buffer changed,
                                i.e. a kernel wrote past the end of a buffer                         */
} bcg_status;

typedef enum {
  BCG_SUB_HYBRID = 0,
  BCG_SUB_GLOBAL = 1,
  BCG_SUB_PARALLEL = 2,      /* same as hybrid with p = 1 (p is ignored) */
  BCG_SUB_CLASSICAL = 3      /* same as hybrid with p = k (p is ignored) */
} bcg_subalgebra;

typedef enum {
  BCG_FP64 = 0,              /* FP64 iteration vectors and updates, FP64-accurate block products (see
                                "Arithmetic of the FP64 form" above)                                  */
  BCG_FP32_REFINE = 1,       /* FP32 block CG inside FP64 residual recomputation: operator products
                                and block updates in FP32, Gram matrices FP64-accurate, p x p
                                Cholesky/LU solves, the solution and its residual in FP64; residual
                                replacement or restarted refinement (option "refine"). The FP32
                                process of block j runs on R_j 2^-sigma_j, an exact scaling with
                                sigma_j the exponent of the block's largest FP64 column norm, so
                                FP32's range never limits the scale of B or X                        */
  BCG_FP64_DF = 2            /* BCG_FP64 with the residual update R -= Q lambda (BAXPY) in double-
                                float arithmetic where the shapes allow it (2 <= p <= 16 with k | 32
                                or 32 | k, k even): its sum of p products is accumulated in float
                                pairs from 48-bit splits of its operands (on the FP32 pipes) and
                                added to the FP64 value with one FP64 addition, while X += P lambda
                                and P = Z + P beta keep their FP64 FMAs, so that the narrow FP64
                                pipe and the FP32 pipes share K2's products. Error of R's update
                                about 2^-46 sum_a |q_a l_ab|, against about p 2^-53 of it with FP64
                                FMAs; p + 1 instead of 2 p FP64 operations per element of K2. Other
                                shapes run BCG_FP64's updates. The retooled form is not available. */
} bcg_precision;

typedef enum {
  BCG_STENCIL_5PT_2D = 0,         /* scale * (4, -1, -1, -1, -1) on nx x ny, Dirichlet eliminated     */
  BCG_STENCIL_7PT_3D = 1,         /* scale * (6, -1 x 6) on nx x ny x nz                              */
  BCG_STENCIL_7PT_3D_VARCOEF = 2  /* scale * face-coefficient diffusion, see bcg_create_stencil       */
} bcg_stencil_kind;

typedef struct {
  int32_t status;                 /* bcg_status of the solve                                         */
  int32_t iters;                  /* FP64: products Q = A P performed (max over blocks);
                                     FP32_REFINE: total FP32 iterations                               */
  int32_t outer_iters;            /* FP32_REFINE: residual replacements or refinement steps (0: FP64) */
  int32_t breakdown_iter;         /* iteration of a breakdown, -1 if none                            */
  double max_rel_res_recursive;   /* max_s ||R_s|| / ||R_s^0|| of the recursive residual            */
  double max_rel_res_true;        /* max_s ||B_s - A X_s|| / ||B_s - A X_s^0||, recomputed in FP64   */
} bcg_info;

/*
 * bcg_create_csr -- solver for a CSR matrix (Section 3, kernel BOP "Y <- A X" on an assembled matrix).
 *   n, nnz        matrix order and number of stored entries (n >= 1, nnz >= 1)
 *   rowptr        device int64[n+1], rowptr[0] = 0, rowptr[n] = nnz
 *   colind        device int32[nnz], column of each entry, 0 <= colind < n
 *   vals          device double[nnz]; A must be symmetric positive definite
 *   k, p, sub     number of right-hand sides (1..256), block size (p divides k; p <= 32, or a
 *                 multiple of 32 up to 256 -- wide blocks use tiled block products and updates),
 *                 subalgebra (bcg_subalgebra)
 *   prec          bcg_precision
 *   cuda_stream   cudaStream_t to order all work on (NULL = legacy default stream)
 * Returns INVALID_ARG for bad sizes/pointers/enums, OOM if the workspace (about 4 n k scalars plus
 * small buffers) cannot be allocated.
 */
bcg_status bcg_create_csr(bcg_handle *h, int64_t n, int64_t nnz, const int64_t *rowptr,
                          const int32_t *colind, const double *vals, int32_t k, int32_t p,
                          int32_t sub, int32_t prec, void *cuda_stream);

/*
 * bcg_create_sell -- solver on an SELL-C-sigma matrix (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J.
 * Sci. Comput. 36(5), 2014; the sparse format Section 4 suggests against BOP's cache pressure at large k).
 * The matrix is stored for the permuted system A' = Pi A Pi^T, (Pi x)[s] = x[perm[s]]: rows sorted by
 * decreasing length inside windows of sigma rows, columns renumbered with the same permutation. Chunks of
 * C = 32 consecutive rows are stored column-major: entry j of row s at chunkptr[s / 32] + j*32 + s % 32,
 * rowlen[s] entries in row s, each chunk padded to its longest row (padding is never read).
 *   n         rows (>= 1, <= INT32_MAX)
 *   nent      stored entries including padding (length of colind and vals)
 *   chunkptr  device int64[ceil(n / 32)]: first entry of each chunk
 *   rowlen    device int32[n]
 *   colind    device int32[nent]: permuted column indices
 *   vals      device double[nent]
 *   perm      device int32[n]: the original row of permuted row s (a permutation of 0..n-1)
 * B and X of bcg_solve / bcg_solve_host stay in the original row order: the handle permutes them on entry
 * and X back on exit (two n x k buffers of workspace). bcg_bop applies A in the original order too.
 * bcg_update_values takes new values in the same padded layout; bcg_grad_values is not available.
 * Other arguments and ownership as for bcg_create_csr.
 */
bcg_status bcg_create_sell(bcg_handle *h, int64_t n, int64_t nent, const int64_t *chunkptr,
                           const int32_t *rowlen, const int32_t *colind, const double *vals,
                           const int32_t *perm, int32_t k, int32_t p, int32_t sub, int32_t prec,
                           void *cuda_stream);

/*
 * bcg_create_stencil -- matrix-free solver (BOP as a stencil, no assembled matrix).
 *   kind          bcg_stencil_kind; nz = 1 for the 2D stencil
 *   coef          NULL for the constant stencils. For BCG_STENCIL_7PT_3D_VARCOEF a device double
 *                 array of face coefficients: x-faces [nz][ny][nx+1], then y-faces [nz][ny+1][nx],
 *                 then z-faces [nz+1][ny][nx] (boundary faces included). Row i = x + nx*(y + ny*z) has
 *                 A_ii = scale * (sum of its six faces) and A_ij = -scale * (shared face).
 *   scale         multiplies the stencil (e.g. 1/h^2)
 * Other arguments as for bcg_create_csr. bcg_grad_values is not available on stencil handles.
 */
bcg_status bcg_create_stencil(bcg_handle *h, int32_t kind, int32_t nx, int32_t ny, int32_t nz,
                              const double *coef, double scale, int32_t k, int32_t p, int32_t sub,
                              int32_t prec, void *cuda_stream);

/*
 * bcg_set_option -- tune a handle. Keys:
 *   "refine"       FP32_REFINE strategy: 1 (default) residual replacement -- one FP32 block CG process whose
 *                  correction is flushed into the FP64 X, and whose residual is replaced by the FP64
 *                  B - A X, every time its residual has dropped tenfold (the process is restarted only if
 *                  a block's FP32 directions lose rank); 0 restarted iterative refinement -- every step
 *                  solves A D = R from D = 0 in FP32 and adds D to X in FP64
 *   "inner_tol"    FP32_REFINE with refine = 0: smallest relative residual reduction an inner solve is
 *                  asked for (default 3e-5); each inner solve targets the reduction still needed by the
 *                  outer tolerance (times 0.5), but not less than this
 *   "max_outer"    FP32_REFINE with refine = 0: maximum refinement steps (default 30)
 *   "check_every"  iterations launched between two host reads of the device status word (default 8;
 *                  converged iterations in between are skipped on the device at launch cost only)
 *   "graph"        1 = replay the batch of iterations as a captured CUDA graph, 0 = plain launches
 *                  (default 1; graphs need a non-NULL stream)
 *   "profile"      1 = time every iteration kernel with CUDA events (see bcg_profile), 0 = off;
 *                  setting it resets the counters
 *   "precond"      preconditioner M of Algorithm 1 (its steps P^1 = M^{-1} R^0 and Z = M^{-1} R; Section 3):
 *                  0 = identity (default), 1 = Jacobi, M = diag(A)
 *                  (Section 3 allows any SPD M; Z = M^{-1} R is formed on the fly by the kernels that
 *                  read R, from 1/diag(A) computed at create time and by bcg_update_values; the mixed
 *                  form uses an FP32 copy). Every diagonal entry must be positive.
 *   "retooled"     1 = Dubrulle's retooled block CG (Electron. Trans. Numer. Anal. 12, 2001; the stability
 *                  reference of Section 3) instead of Algorithm 1's recurrences: the residual is carried as
 *                  R = Q C with Q orthonormal in the S-product (a Cholesky QR per block) and the search
 *                  directions are built from Q; the same iterates in exact arithmetic, but a right-hand side
 *                  whose columns differ in scale by many orders factors like a well-scaled one. Each Cholesky
 *                  pivot is tested against its own diagonal entry. Every subalgebra (global: one factor shared
 *                  by the column blocks) and both preconditioners (Jacobi: Q orthonormal in the product
 *                  <<Q, M^{-1} Q>>, directions M^{-1} Q + S psi^T). FP64 handles that are not row-sharded
 *                  only (INVALID_ARG otherwise); 0 = Algorithm 1 (default).
 *   "tensor_cores" 1 (default) = the tcgen05 path described under "Arithmetic of the FP64 form": FP64 handles
 *                  with p a multiple of 64 take their block products and updates there, FP64 handles with
 *                  p = 32 their block updates (two blocks per 64-column tile where 64 divides k); the
 *                  mixed form's FP32 process with p a multiple of 64 takes both (its updates summed in FP64
 *                  and rounded once to FP32). 0 = FP64 FMA updates and Dot2 products everywhere.
 *   "guards"       1 = after each solve (bcg_solve, bcg_solve_host, bcg_rows_finish) compare the 16 guard
 *                  bytes that follow every workspace buffer of the handle with the pattern written at
 *                  allocation; a change returns BCG_ERR_GUARD naming the buffer. 0 = no check (default).
 * Unknown keys or out-of-range values return INVALID_ARG.
 */
bcg_status bcg_set_option(bcg_handle h, const char *key, double value);

/*
 * bcg_solve -- Algorithm 1 (Section 3) with M = I (or Jacobi, option "precond"; or Dubrulle's retooled
 * form of it, option "retooled") from X^0 = X to the stopping rule of Section 4's whole-solver experiment:
 * every column s with ||R_s|| <= tol ||R_s^0|| (recursive residual, 2-norm; the retooled form evaluates it
 * as (C^T gamma C)_ss from its factored residual R = Q C). Hybrid/parallel blocks stop updating once all
 * their columns pass; global/classical stop together.
 *   B      device double[n*k], row-major, not modified
 *   X      device double[n*k], row-major; in: X^0, out: the solution (or last iterate on error)
 *   tol    > 0 (FP32_REFINE: tolerance of the FP64 outer residual)
 *   maxit  >= 1; FP64: iteration cap; FP32_REFINE: cap on inner iterations per refinement step
 *   info   host, may be NULL
 * Returns OK, BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT, CUDA or INVALID_ARG.
 */
bcg_status bcg_solve(bcg_handle h, const double *B, double *X, double tol, int32_t maxit,
                     bcg_info *info);

/*
 * bcg_solve_host -- bcg_solve (Algorithm 1, Section 3) on HOST arrays: copies B and X^0 to the handle's device staging
 * buffers (allocated at the first call, 2 n k doubles), solves, and copies X back. Same arguments
 * and statuses as bcg_solve, with B and X in host memory.
 */
bcg_status bcg_solve_host(bcg_handle h, const double *B, double *X, double tol, int32_t maxit,
                          bcg_info *info);

/*
 * bcg_block_iters -- per distinct block (q for hybrid/parallel/classical, 1 for global) the
 * iteration at which it froze in the last solve (or the last iteration if it never did): the per-block
 * stopping of Section 4's rule in the hybrid subalgebra, whose blocks are independent solves (Section 3).
 * Statuses: OK, or INVALID_ARG for a NULL handle or output.
 * out: host int32[cap]; returns INVALID_ARG if cap is smaller than the number of blocks.
 */
bcg_status bcg_block_iters(bcg_handle h, int32_t *out, int32_t cap);

/*
 * bcg_grad_values -- gradient of a loss L(X) with respect to the stored CSR values, for
 * X = A^{-1} B: grad[e] = -Lambda_i . X_j for stored entry e = (i, j), where Lambda solves
 * A Lambda = dL/dX (an adjoint solve with the same handle, since A is symmetric).
 *   Lambda, X  device double[n*k]; grad: device double[nnz] (overwritten)
 * CSR handles only (INVALID_ARG otherwise). The paper has no differentiation; this is the adjoint
 * of BOP on the sparsity pattern.
 */
bcg_status bcg_grad_values(bcg_handle h, const double *Lambda, const double *X, double *grad);

/*
 * bcg_update_values -- rebind the operator of BOP (Section 3's kernel list, Y = A X): the CSR values
 * (same pattern) or the varcoef faces. vals is a device array of the same length as at create time; it is
 * borrowed from now on. 1/diag(A) (Jacobi) and the operator maxima behind the Gram shifts are recomputed.
 * Returns INVALID_ARG for a NULL handle, a non-device pointer or a constant-stencil handle, or CUDA.
 */
bcg_status bcg_update_values(bcg_handle h, const double *vals);

/*
 * bcg_bdot -- the BDOT kernel alone (Section 3; Section 2, Definition "Relevant *-subalgebras"):
 * gamma = <<X, Y>>_S for the handle's k, p and subalgebra, accumulated as described under "Arithmetic of the
 * FP64 form" (shifts from the column maxima of X and of Y, found by one extra pass over each), with per-CTA
 * partials in the handle's workspace summed in a fixed order.
 *   X, Y   device double[n*k], row-major
 *   gamma  device double[nblk*p*p], nblk = q (hybrid/parallel/classical) or 1 (global); block jb's entry
 *          (a, b) = sum_i X[i, jb*p + a] Y[i, jb*p + b] (global: summed over the q blocks) at jb*p*p + a*p + b
 */
bcg_status bcg_bdot(bcg_handle h, const double *X, const double *Y, double *gamma);

/*
 * bcg_bdot_f32 -- BDOT on FP32 block vectors with FP64-accurate accumulation: the block product exactly as
 * the FP32_REFINE inner solve forms it (products of FP32 values are exact in FP64; the sums carry FP64-class
 * accuracy). X, Y: device float[n*k]; gamma as for bcg_bdot (double).
 */
bcg_status bcg_bdot_f32(bcg_handle h, const float *X, const float *Y, double *gamma);

/*
 * bcg_bdot_noalloc -- bcg_bdot for callers that cannot allocate device memory. The paper has no
 * counterpart; this is a deployment variant of the BDOT kernel.
 *
 * Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being captured and must not
 * allocate, plug-ins whose host application owns every device allocation through its own pool, and
 * latency-critical paths where an allocation may block or fail. This entry point needs no handle (creating
 * one allocates) and allocates nothing: the column maxima and exponent shifts of X and Y and the per-CTA
 * partial sums live in one static device array of 262,144 doubles (2 MiB) that every GPU which loads the
 * library holds until the process exits. The caller passes the inputs and the output.
 *   n, k, p, sub  as for bcg_create_csr (1 <= k <= 256, p divides k, p <= 32; k*p <= 261,120)
 *   X, Y          device double[n*k], row-major
 *   gamma         device double[nblk*p*p], layout as for bcg_bdot
 *   cuda_stream   stream to order the work on; the call returns once it is enqueued
 * X, Y and gamma must live on the current device, whose copy of the array is used. The first call on a
 * device looks up that device's address of the array (cudaGetSymbolAddress) and should therefore come
 * before any stream capture. Every call shares the array: it clears the column maxima (a memset of the
 * array, which allocates nothing) and overwrites the partial sums it uses before reading them, so calls
 * that overlap on the GPU -- on different streams, or from several threads -- race and must be serialised
 * by the caller. The arithmetic is bcg_bdot's.
 * Returns INVALID_ARG (sizes beyond the limits, non-device pointers or pointers of another device, unknown
 * subalgebra) or CUDA.
 */
bcg_status bcg_bdot_noalloc(int64_t n, int32_t k, int32_t p, int32_t sub, const double *X, const double *Y,
                            double *gamma, void *cuda_stream);

/*
 * bcg_bop -- the BOP kernel alone (Section 3): Y = A X in FP64 with the handle's operator.
 *   X, Y  device double[n*k], row-major, must not overlap.
 */
bcg_status bcg_bop(bcg_handle h, const double *X, double *Y);

/*
 * bcg_profile -- live per-kernel timing. After bcg_set_option(h, "profile", 1) (which also resets the
 * counters) every iteration kernel of the following solves is bracketed by CUDA events on the handle's
 * stream (plain launches, no graph replay), counting only iterations that executed. Fills, for
 *   0 K1 (BOP + alpha + recomputed rho), 1 K4a (Cholesky solve), 2 K2 (X, R update + rho + norms),
 *   3 K4b (stopping test + LU solve), 4 K3 (P update), 5 reserved, 6 the tensor-core block products and
 *   7 the tensor-core block updates (FP64 blocks of 32 and wider; each launch timed alone, the host waiting for it),
 * the total milliseconds ms[i] and the launch count count[i]. ms, count: host arrays of cap >= 8.
 * Timing instrumentation, not part of the paper's method.
 */
bcg_status bcg_profile(bcg_handle h, double *ms, int64_t *count, int32_t cap);

/*
 * Row-sharded solves (several GPUs, one rank per GPU). The rows of A are split into contiguous ranges, one
 * per rank; a rank's handle holds its rows and iterates Algorithm 1 on them. Every block product is a sum
 * over rows, so a rank's share of alpha, the recomputed rho, rho and the column norms is a partial sum
 * that the ranks add up (an allreduce) before the p x p solves, which every rank then runs on identical
 * data (Section 3 notes that the reduction of one block product can travel with the previous one; here the
 * two products of K1 travel in one message, rho and the column norms in another). BOP needs the rows of P
 * that other ranks own and A references (the halo), refreshed before every phase 1. FP64 and CSR only.
 * The caller drives the iteration:
 *
 *   bcg_create_csr_rows(&h, n_local, n_cols, nnz, rowptr, colind, vals, k, p, sub, stream)
 *   bcg_rows_bind(h, sums1, sums2)      the caller's buffers of the sums exchanged between ranks
 *   bcg_rows_start(h, B, X, tol)        R = B - A X, P = M^{-1} R; norm partials -> sums2[k*p ..]
 *   allreduce(sums2[k*p .. k*p + k))    then bcg_rows_start_status(h)
 *   loop:  halo of P: bcg_rows_pack for every rank that needs rows of this one, exchange,
 *          bcg_rows_unpack of the received rows
 *          bcg_rows_phase(h, 1)         K1: Q = A P, alpha, rho_rec -> sums1
 *          allreduce(sums1)
 *          bcg_rows_phase(h, 2)         lambda, X += P lambda, R -= Q lambda, rho, norms -> sums2
 *          allreduce(sums2)
 *          bcg_rows_phase(h, 3)         stopping test, beta, P = Z + P beta
 *          every few iterations: bcg_rows_poll(h, &done)
 *   bcg_rows_finish(h, &info)
 *
 * Local numbering: rows 0..n_local-1 are this rank's rows; columns n_local..n_cols-1 are halo rows (other
 * ranks' rows that A references), so colind (int32, device) holds local indices < n_cols and the diagonal
 * entry of row r is column r. B is n_local x k; X has n_cols rows, the last n_cols - n_local being halo
 * rows (read once, by bcg_rows_start; only the first n_local rows are updated). All calls enqueue on the
 * handle's stream and return without waiting, except bcg_rows_poll and bcg_rows_finish. Options
 * (bcg_set_option) apply, including "precond".
 *
 * bcg_create_csr_rows   -- as bcg_create_csr for this rank's rows (FP64); n_cols >= n_local.
 * bcg_rows_bind         -- sums1 (2 k p doubles) and sums2 (k p + k doubles): device buffers owned by the
 *                          caller, written by the phases and summed over ranks by the caller.
 * bcg_rows_start        -- begin a solve from X towards the per-column stopping rule of bcg_solve (tol >= 0).
 * bcg_rows_start_status -- after the norm partials were summed over ranks: initial norms and status.
 * bcg_rows_phase        -- phase 1, 2 or 3 of one iteration (see above). After convergence, breakdown or a
 *                          non-finite value the kernels return at entry, so surplus phases are harmless.
 * bcg_rows_pack         -- buf[i*k + c] = P[rows[i]*k + c] for i < nrows (rows int32, buf: device): the
 *                          rows another rank needs.
 * bcg_rows_unpack       -- copy nrows = n_cols - n_local received rows (device, row-major, in local halo
 *                          order) into P's halo rows.
 * bcg_rows_poll         -- *done = 1 once the solve has stopped (converged, breakdown or non-finite);
 *                          waits for the stream.
 * bcg_rows_finish       -- status and iteration counts of the solve (info->max_rel_res_true is NaN: it needs
 *                          the other ranks' rows of X).
 * On a row-sharded handle bcg_solve and bcg_solve_host return INVALID_ARG.
 */
bcg_status bcg_create_csr_rows(bcg_handle *h, int64_t n_local, int64_t n_cols, int64_t nnz,
                               const int64_t *rowptr, const int32_t *colind, const double *vals, int32_t k,
                               int32_t p, int32_t sub, void *cuda_stream);
bcg_status bcg_rows_bind(bcg_handle h, double *sums1, double *sums2);
bcg_status bcg_rows_start(bcg_handle h, const double *B, double *X, double tol);
bcg_status bcg_rows_start_status(bcg_handle h);
bcg_status bcg_rows_phase(bcg_handle h, int32_t phase);
bcg_status bcg_rows_pack(bcg_handle h, const int32_t *rows, int64_t nrows, double *buf);
bcg_status bcg_rows_unpack(bcg_handle h, const double *halo, int64_t nrows);
bcg_status bcg_rows_poll(bcg_handle h, int32_t *done);
bcg_status bcg_rows_finish(bcg_handle h, bcg_info *info);

/* bcg_last_error -- message of the calling thread's most recent failure ("" if none). */
const char *bcg_last_error(void);

/*
 * bcg_debug_fail_alloc -- failure injection for tests of the error paths (not part of the paper's method): after
 * bcg_debug_fail_alloc(N), N >= 1, the N-th device workspace allocation made by the library from then on (in any
 * handle, any thread) fails as if cudaMalloc had run out of memory, so the call making it returns BCG_ERR_OOM
 * and frees everything it had allocated; the injection then disarms. N = 0 disarms it. Returns INVALID_ARG for
 * N < 0. Process-wide; meant for single-threaded tests.
 */
bcg_status bcg_debug_fail_alloc(int32_t nth);

/*
 * bcg_debug_poke_guard -- test hook for the guard check (not part of the paper's method): overwrite the first
 * guard byte after workspace buffer `index` of the handle (memory the handle allocated for its guards, so no
 * access leaves an allocation). With option "guards" the next solve then returns BCG_ERR_GUARD. INVALID_ARG for
 * an index outside the handle's buffers.
 */
bcg_status bcg_debug_poke_guard(bcg_handle h, int32_t index);

/* bcg_destroy -- free the handle's workspace; NULL-safe. */
void bcg_destroy(bcg_handle h);

#ifdef __cplusplus
}
#endif

#endif /* BCG_H */
