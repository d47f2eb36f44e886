"""CPU FP64 oracle of the generalized Block Conjugate Gradients method (Dreier & Engwer, arXiv 1912.11930).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this module: only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it. It shares no code with
the CUDA library; both are fed from ``paper_1912_11930_gb300.workloads`` (input generation only).

It is deliberately plain and slow: numpy/scipy FP64, every step of Algorithm 1 done in the paper's order,
no fusion, no blocking, no reordering. Library primitives used as single steps: the sparse product
``A @ P`` (scipy CSR), dense matmuls, LAPACK's LU with partial pivoting, triangular solves.

Paper passages followed:
* Section 2, Definition "Relevant *-subalgebras": the block products of the hybrid (S_Hy^p) and global
  (S_Gl^p) subalgebras; classical = S_Hy^k = S_Gl^k, parallel = S_Hy^1.
* Section 3, Algorithm 1 (preconditioned, stabilised BCG) with M = I or the Jacobi preconditioner
  M = diag(A), including the recomputation of rho^{i-1} as <<P^i, R^{i-1}>>_S (the stabilisation of
  Section 3), and the four kernels BDOT, BAXPY, BOP, BSOLVE listed after it.
* Section 4, whole-solver experiment: the stopping rule "2-norm of every residual column reduced by the
  factor tol".

Readings of places where the paper is silent, garbled or inconsistent:
* R1 sign of the direction update: Algorithm 1 prints P^{i+1} = Z - P beta. With beta = rho_{i-1}^{-1}
  rho_i > 0 at k = 1 this contradicts CG, so the oracle uses P^{i+1} = Z + P beta.
* R2 global product: the printed sum runs from 0 to q; the proof of the global-rate lemma stacks
  contiguous column blocks, so block j = columns [j p, (j+1) p) for j = 0..q-1 and the global product is
  sum_j X_j^T Y_j, applied to every block.
* R3 which rho^{i-1} enters beta: the recomputed one (it overwrites the old value), used both in
  lambda = alpha^{-1} rho^{i-1} and in beta = (rho^{i-1})^{-1} rho^i.
* R4 BSOLVE method: alpha (SPD) by Cholesky without pivoting, reading alpha's lower triangle; the
  recomputed rho (not symmetric in floating point) by LU with partial pivoting; breakdown when a pivot is
  <= 64 eps max|diag| or not finite.
* R5 stopping rule: after the residual update, column s has converged when ||R_s|| <= tol ||R_s^0||
  (recursive residual, 2-norm). Hybrid/parallel blocks freeze once all their columns have converged
  (their lambda and beta are zero from then on); global/classical stop all columns together. A zero
  column converges at iteration 0. The iteration count is the number of products Q = A P.
* R6 no deflation: a breakdown is reported (status BREAKDOWN), never hidden.

``solve_retooled`` is the retooled block CG that Section 3 points to for the stability of the method
(A. A. Dubrulle, "Retooling the method of block conjugate gradients", Electron. Trans. Numer. Anal. 12,
2001): the residual is carried as R = Q C with an orthonormal Q and a p x p factor C, and the search
directions are built from Q, so differently scaled residual columns do not make the small systems
ill-conditioned. Readings:
* R12 the QR factorisation of Dubrulle's method is taken within the subalgebra as a Cholesky QR: with
  gamma = <<T, T>>_S = L L^T, C-factor psi = L^T and Q = T psi^{-1}; restricted to the hybrid family
  (hybrid, parallel, classical), whose products give every column's norm.
* R13 a Cholesky pivot of the retooled form fails when it is <= 64 eps times its own diagonal entry
  (column-relative, so that a right-hand side scaled column by column factors like the unscaled one).
* R14 the stopping test uses ||R_s||^2 = (C^T gamma C)_ss (the old C and the new gamma, before psi is
  formed), so a block that has converged needs no further factorisation; a failure of the very first
  factorisation is a breakdown in iteration 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# status codes, numerically identical to the C enum bcg_status
OK, INVALID_ARG, CUDA_ERR, OOM, BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT = range(8)

EPS = np.finfo(np.float64).eps
PIVOT_FACTOR = 64.0


def canonical_subalgebra(sub: str, k: int, p: int) -> tuple[str, int]:
    """Map the four subalgebras of Section 2 onto (kind, p) with kind in {hybrid, global}:
    parallel = S_Hy^1, classical = S_Hy^k (= S_Gl^k)."""
    if sub == "parallel":
        return "hybrid", 1
    if sub == "classical":
        return "hybrid", k
    if sub not in ("hybrid", "global"):
        raise ValueError(f"unknown subalgebra {sub!r}")
    if p < 1 or k % p:
        raise ValueError(f"p={p} must divide k={k}")
    return sub, p


def block_product(X: np.ndarray, Y: np.ndarray, p: int, kind: str) -> np.ndarray:
    """BDOT, the S-product <<X, Y>>_S of Section 2 (Definition "Relevant *-subalgebras").

    Returns the element of S as its distinct p x p blocks: shape (q, p, p) for hybrid (block j is
    X_j^T Y_j), shape (1, p, p) for global (sum_j X_j^T Y_j, the same block for every j)."""
    n, k = X.shape
    q = k // p
    blocks = [X[:, j * p:(j + 1) * p].T @ Y[:, j * p:(j + 1) * p] for j in range(q)]
    if kind == "hybrid":
        return np.stack(blocks)
    total = blocks[0].copy()
    for j in range(1, q):
        total = total + blocks[j]
    return total[None]


def block_apply(Y: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """Y gamma for gamma in S given as its distinct blocks (the product inside BAXPY)."""
    n, k = Y.shape
    p = gamma.shape[1]
    q = k // p
    out = np.empty_like(Y)
    for j in range(q):
        g = gamma[j] if gamma.shape[0] == q else gamma[0]
        out[:, j * p:(j + 1) * p] = Y[:, j * p:(j + 1) * p] @ g
    return out


def baxpy(X: np.ndarray, Y: np.ndarray, gamma: np.ndarray, sign: float = 1.0) -> np.ndarray:
    """BAXPY: X + sign * Y gamma (Section 3, kernel list)."""
    return X + sign * block_apply(Y, gamma)


def bop(A: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    """BOP: the operator applied to a block of vectors, A X (Section 3, kernel list)."""
    return np.asarray(A @ X)


def cholesky_lower(G: np.ndarray):
    """Cholesky G = L L^T from G's lower triangle, no pivoting. Returns None on breakdown
    (a pivot <= 64 eps max|diag(G)| or not finite)."""
    p = G.shape[0]
    L = np.zeros_like(G)
    thresh = PIVOT_FACTOR * EPS * np.max(np.abs(np.diag(G)))
    for a in range(p):
        d = G[a, a] - L[a, :a] @ L[a, :a]
        if not (np.isfinite(d) and d > thresh):
            return None
        L[a, a] = np.sqrt(d)
        L[a + 1:, a] = (G[a + 1:, a] - L[a + 1:, :a] @ L[a, :a]) / L[a, a]
    return L


def bsolve_cholesky(alpha: np.ndarray, delta: np.ndarray, active: np.ndarray):
    """BSOLVE for lambda = alpha^{-1} delta in S, alpha SPD: one Cholesky per distinct block.
    Blocks that are not active get a zero result. Returns (result, ok)."""
    out = np.zeros_like(delta)
    for j in range(alpha.shape[0]):
        if not active[j]:
            continue
        L = cholesky_lower(alpha[j])
        if L is None:
            return out, False
        y = sla.solve_triangular(L, delta[j], lower=True)
        out[j] = sla.solve_triangular(L.T, y, lower=False)
        if not np.all(np.isfinite(out[j])):
            return out, False
    return out, True


def bsolve_lu(rho: np.ndarray, delta: np.ndarray, active: np.ndarray):
    """BSOLVE for beta = rho^{-1} delta in S by LU with partial pivoting (rho is not symmetric in
    floating point). Returns (result, ok)."""
    out = np.zeros_like(delta)
    for j in range(rho.shape[0]):
        if not active[j]:
            continue
        G = rho[j]
        if not np.all(np.isfinite(G)):
            return out, False
        thresh = PIVOT_FACTOR * EPS * np.max(np.abs(np.diag(G)))
        lu, piv = sla.lu_factor(G, check_finite=False)
        if np.any(np.abs(np.diag(lu)) <= thresh):
            return out, False
        out[j] = sla.lu_solve((lu, piv), delta[j], check_finite=False)
        if not np.all(np.isfinite(out[j])):
            return out, False
    return out, True


@dataclass
class Result:
    X: np.ndarray
    status: int
    iters: int                     # number of products Q = A P performed
    block_iters: np.ndarray        # per distinct block: iteration at which it froze (or the last one)
    breakdown_iter: int            # -1 if none
    relres_recursive: np.ndarray   # ||R_s|| / ||R_s^0|| per column (0 where R_s^0 = 0)
    relres_true: np.ndarray        # ||B_s - A X_s|| / ||B_s - A X_s^0|| per column
    history: dict = field(default_factory=dict)


def _preconditioner(A, precond: str):
    """z = M^{-1} r for M = I ("none") or M = diag(A) ("jacobi"); always a fresh array."""
    if precond == "jacobi":
        dinv = 1.0 / np.asarray(A.diagonal(), dtype=np.float64)
        return lambda M_: M_ * dinv[:, None]
    if precond == "none":
        return lambda M_: M_.copy()
    raise ValueError(f"unknown preconditioner {precond!r}")


def _column_norms(M: np.ndarray) -> np.ndarray:
    return np.sqrt(np.sum(M * M, axis=0))


def _converged_blocks(rn, r0, tol, kind, p, q):
    """Reading R5: a block has converged when every one of its columns has ||R_s|| <= tol ||R_s^0||; the global
    subalgebra has one block made of all columns."""
    col_ok = rn <= tol * r0
    if kind == "hybrid":
        return np.array([bool(np.all(col_ok[j * p:(j + 1) * p])) for j in range(q)])
    return np.array([bool(np.all(col_ok))])


def _step_length(P, AP, R, p, kind, active):
    """The S-valued step along P that makes the new residual S-orthogonal to P: lambda = <<P, A P>>^{-1} <<P, R>>.
    The second product is formed afresh from the current P and R (the recomputation of Section 3) and also
    returned, since the direction coefficient divides by it (reading R3). Returns (alpha, <<P, R>>, lambda, ok)."""
    curv = block_product(P, AP, p, kind)
    proj = block_product(P, R, p, kind)
    lam, ok = bsolve_cholesky(curv, proj, active)
    return curv, proj, lam, ok


def _direction_weight(proj, Z, R, p, kind, active):
    """The S-valued weight of the old direction in the new one: beta = <<P, R_old>>^{-1} <<Z, R>>, by LU with
    partial pivoting (reading R4). Returns (<<Z, R>>, beta, ok)."""
    zr = block_product(Z, R, p, kind)
    beta, ok = bsolve_lu(proj, zr, active)
    return zr, beta, ok


def solve(A, B: np.ndarray, X0: np.ndarray | None = None, p: int = 1, sub: str = "hybrid",
          tol: float = 1e-8, maxit: int = 1000, record: bool = False, precond: str = "none") -> Result:
    """Block CG in a *-subalgebra S (Algorithm 1 of Section 3), FP64.

    Conjugate directions in the S-module sense: from R = B - A X and the first direction P = M^{-1} R, every
    iteration applies A to P, moves X by P lambda and R by -(A P) lambda with the step lambda of _step_length, stops
    the blocks whose columns meet the stopping rule, and forms the next direction M^{-1} R + P beta with the weight
    of _direction_weight (the "+" of reading R1). All products are S-products (block_product); all coefficients are
    elements of S, given by their distinct p x p blocks.

    ``A`` is a scipy sparse matrix (or anything supporting ``A @ X``); B and X0 are n x k.
    ``precond``: "none" (M = I) or "jacobi" (M = diag(A))."""
    B = np.asarray(B, dtype=np.float64)
    n, k = B.shape
    kind, p = canonical_subalgebra(sub, k, p)
    q = k // p
    nblk = q if kind == "hybrid" else 1
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64, copy=True)
    minv = _preconditioner(A, precond)
    hist = {"X": [], "R": [], "P": [], "Q": [], "alpha": [], "rho_rec": [], "rho": []} if record else {}

    R = B - bop(A, X)
    P = minv(R)
    r0 = _column_norms(R)
    if not (np.all(np.isfinite(r0)) and np.all(np.isfinite(X))):
        return Result(X, NUMERIC, 0, np.zeros(nblk, dtype=np.int64), -1, r0 * np.nan, r0 * np.nan, hist)
    active = ~_converged_blocks(r0, r0, tol, kind, p, q)
    block_iters = np.zeros(nblk, dtype=np.int64)
    status, brk, it = OK, -1, 0
    if record:
        hist["X"].append(X.copy()); hist["R"].append(R.copy()); hist["P"].append(P.copy())

    while np.any(active) and it < maxit:
        it += 1
        block_iters[active] = it
        AP = bop(A, P)
        curv, proj, lam, ok = _step_length(P, AP, R, p, kind, active)
        if not ok:
            status, brk = BREAKDOWN, it
            break
        X = baxpy(X, P, lam, +1.0)
        R = baxpy(R, AP, lam, -1.0)
        rn = _column_norms(R)
        if not np.all(np.isfinite(rn)):
            status = NUMERIC
            break
        active = active & ~_converged_blocks(rn, r0, tol, kind, p, q)
        Z = minv(R)
        zr, beta, ok = _direction_weight(proj, Z, R, p, kind, active)
        if record:
            hist["Q"].append(AP.copy()); hist["alpha"].append(curv); hist["rho_rec"].append(proj)
            hist["rho"].append(zr)
        if not ok:
            status, brk = BREAKDOWN, it
            break
        P = baxpy(Z, P, beta, +1.0)
        if record:
            hist["X"].append(X.copy()); hist["R"].append(R.copy()); hist["P"].append(P.copy())

    if status == OK and np.any(active):
        status = NOT_CONVERGED
    rn = _column_norms(R)
    with np.errstate(invalid="ignore", divide="ignore"):
        rel_rec = np.where(r0 > 0, rn / np.where(r0 > 0, r0, 1.0), 0.0)
        rt = _column_norms(B - bop(A, X))
        rel_true = np.where(r0 > 0, rt / np.where(r0 > 0, r0, 1.0), rt)
    return Result(X, status, it, block_iters, brk, rel_rec, rel_true, hist)


def cholesky_lower_colrel(G: np.ndarray):
    """Cholesky G = L L^T from G's lower triangle, no pivoting; breakdown (None) when a pivot is
    <= 64 eps times its own diagonal entry G_aa, or not finite (reading R13)."""
    p = G.shape[0]
    L = np.zeros_like(G)
    for a in range(p):
        d = G[a, a] - L[a, :a] @ L[a, :a]
        if not (np.isfinite(d) and d > PIVOT_FACTOR * EPS * G[a, a]):
            return None
        L[a, a] = np.sqrt(d)
        L[a + 1:, a] = (G[a + 1:, a] - L[a + 1:, :a] @ L[a, :a]) / L[a, a]
    return L


def retooled_solution_coefficient(xi: np.ndarray, C: np.ndarray) -> np.ndarray:
    """lambda = xi C: the step along S that moves X by S alpha^{-1} <<S, R>> with <<S, R>> = C."""
    return xi @ C


def retooled_direction(Q: np.ndarray, S: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """S^{i+1} = Q^{i+1} + S^i psi^T (the retooled form of P^{i+1} = R^i + P^i beta)."""
    return Q + S @ psi.T


def solve_retooled(A, B: np.ndarray, X0: np.ndarray | None = None, p: int = 1, sub: str = "hybrid",
                   tol: float = 1e-8, maxit: int = 1000, record: bool = False, precond: str = "none") -> Result:
    """Dubrulle's retooled block CG (Electron. Trans. Numer. Anal. 12, 2001) in a *-subalgebra S of Section 2,
    FP64, step by step. The residual is carried as R = Q C with C in S (upper triangular blocks) and Q
    orthonormal for the product <<Q, M^{-1} Q>> = I; the directions are P = S C. Per iteration, for every
    block that has not converged:

        W = A S;  alpha = <<S, W>>;  xi = alpha^{-1};  X += S (xi C);  T = Q - W xi;
        ||R_s||^2 = (C^T <<T, T>>_Hy C)_ss  (stopping test, per column);
        gamma = <<T, M^{-1} T>> = psi^T psi (Cholesky);  C = psi C;  Q = T psi^{-1};  S = M^{-1} Q + S psi^T

    starting from <<R^0, M^{-1} R^0>> = C^T C, Q = R^0 C^{-1} and S = M^{-1} Q. These follow from Algorithm 1's
    recurrences with R^i = Q^i C^i and P^{i+1} = S^{i+1} C^i: lambda = C^{-1} xi C, so P lambda = S xi C; the
    new residual is (Q - W xi) C; rho = <<R, M^{-1} R>> = C^T gamma C; and beta = (C^T C)^{-1} C_new^T C_new
    turns P_new = M^{-1} R_new + P beta into S_new C_new with S_new = M^{-1} Q_new + S psi^T. For the global
    subalgebra the coefficients (C, xi, psi) are one p x p matrix shared by the q column blocks and the
    products sum over blocks; the column norms still take each block's own <<T_j, T_j>>. In exact arithmetic
    X^i is Algorithm 1's iterate with the same preconditioner.

    ``precond``: "none" (M = I) or "jacobi" (M = diag(A))."""
    B = np.asarray(B, dtype=np.float64)
    n, k = B.shape
    kind, p = canonical_subalgebra(sub, k, p)
    q = k // p
    nb = q if kind == "hybrid" else 1
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64, copy=True)
    minv = _preconditioner(A, precond)
    hist = {"X": [], "Q": [], "S": [], "C": []} if record else {}

    def cols(j):
        return slice(j * p, (j + 1) * p)

    def blk(j):   # which coefficient block serves column block j
        return j if kind == "hybrid" else 0

    def block_of(j):   # the stopping unit of column block j
        return j if kind == "hybrid" else 0

    R = B - bop(A, X)
    r0 = _column_norms(R)
    if not (np.all(np.isfinite(r0)) and np.all(np.isfinite(X))):
        return Result(X, NUMERIC, 0, np.zeros(nb, dtype=np.int64), -1, r0 * np.nan, r0 * np.nan, hist)
    rn = r0.copy()
    active = ~_converged_blocks(r0, r0, tol, kind, p, q)
    block_iters = np.zeros(nb, dtype=np.int64)
    status, brk, it = OK, -1, 0

    def chol_qr(G, act):
        """Per active coefficient block: the lower factor L of G = L L^T (column-relative pivot test); psi = L^T."""
        Ls = np.zeros((nb, p, p))
        for b in range(nb):
            if not act[b]:
                continue
            L = cholesky_lower_colrel(G[b])
            if L is None:
                return None
            Ls[b] = L
        return Ls

    def right_div(Y, L):
        """Y psi^{-1} = Y L^{-T}, by a triangular solve."""
        return sla.solve_triangular(L, Y.T, lower=True).T

    # R^0 = Q^0 C^0 with <<Q^0, M^{-1} Q^0>> = I, S^1 = M^{-1} Q^0
    C = np.zeros((nb, p, p))
    Q = np.zeros_like(B)
    Ls = chol_qr(block_product(R, minv(R), p, kind), active)
    if Ls is None:
        status, brk = BREAKDOWN, 1
    else:
        C = np.transpose(Ls, (0, 2, 1)).copy()
        for j in range(q):
            if active[block_of(j)]:
                Q[:, cols(j)] = right_div(R[:, cols(j)], Ls[blk(j)])
    S = minv(Q)
    if record and status == OK:
        hist["X"].append(X.copy()); hist["Q"].append(Q.copy()); hist["S"].append(S.copy())
        hist["C"].append(C.copy())

    while status == OK and np.any(active) and it < maxit:
        it += 1
        block_iters[active] = it
        Wm = bop(A, S)
        alpha = block_product(S, Wm, p, kind)
        xi = np.zeros((nb, p, p))
        lam = np.zeros((nb, p, p))
        for b in range(nb):
            if not active[b]:
                continue
            L = cholesky_lower_colrel(alpha[b])
            if L is None:
                status, brk = BREAKDOWN, it
                break
            Linv = sla.solve_triangular(L, np.eye(p), lower=True)
            xi[b] = Linv.T @ Linv
            lam[b] = retooled_solution_coefficient(xi[b], C[b])
        if status != OK:
            break
        X = baxpy(X, S, lam, +1.0)
        T = baxpy(Q, Wm, xi, -1.0)
        # column norms of R = T C from each column block's own <<T_j, T_j>>
        Gh = block_product(T, T, p, "hybrid")
        for j in range(q):
            if active[block_of(j)]:
                Cb = C[blk(j)]
                rn[cols(j)] = np.sqrt(np.diag(Cb.T @ Gh[j] @ Cb))
        if not np.all(np.isfinite(rn)):
            status = NUMERIC
            break
        active = active & ~_converged_blocks(rn, r0, tol, kind, p, q)
        # gamma = <<T, M^{-1} T>> = psi^T psi; C = psi C; Q = T psi^{-1}; S = M^{-1} Q + S psi^T
        Ls = chol_qr(block_product(T, minv(T), p, kind), active)
        if Ls is None:
            status, brk = BREAKDOWN, it
            break
        Qn = Q.copy()
        for j in range(q):
            if active[block_of(j)]:
                Qn[:, cols(j)] = right_div(T[:, cols(j)], Ls[blk(j)])
        Zq = minv(Qn)
        for j in range(q):
            b = block_of(j)
            if active[b]:
                S[:, cols(j)] = retooled_direction(Zq[:, cols(j)], S[:, cols(j)], Ls[blk(j)].T)
                Q[:, cols(j)] = Qn[:, cols(j)]
        for b in range(nb):
            if active[b]:
                C[b] = Ls[b].T @ C[b]
        if record:
            hist["X"].append(X.copy()); hist["Q"].append(Q.copy()); hist["S"].append(S.copy())
            hist["C"].append(C.copy())

    if status == OK and np.any(active):
        status = NOT_CONVERGED
    with np.errstate(invalid="ignore", divide="ignore"):
        rel_rec = np.where(r0 > 0, rn / np.where(r0 > 0, r0, 1.0), 0.0)
        rt = _column_norms(B - bop(A, X))
        rel_true = np.where(r0 > 0, rt / np.where(r0 > 0, r0, 1.0), rt)
    return Result(X, status, it, block_iters, brk, rel_rec, rel_true, hist)


def grad_values(rowptr: np.ndarray, colind: np.ndarray, Lam: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Gradient of a loss L(X), X = A^{-1} B, with respect to the stored CSR values of A:
    dL/dA_ij = -Lambda_i . X_j (row i of the adjoint solution Lambda = A^{-T} dL/dX dotted with row j of
    X), one value per stored entry (i, j). Follows from dX = -A^{-1} dA X."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return -np.einsum("ec,ec->e", Lam[rows], X[colind.astype(np.int64)])


def solve_and_grad(A, rowptr, colind, B, W, p=1, sub="hybrid", tol=1e-12, maxit=5000):
    """Forward solve X = A^{-1} B, loss L = sum(W * X), adjoint solve A Lambda = W (A symmetric),
    dL/dB = Lambda, dL/dvals from ``grad_values``."""
    fwd = solve(A, B, p=p, sub=sub, tol=tol, maxit=maxit)
    adj = solve(A, W, p=p, sub=sub, tol=tol, maxit=maxit)
    return fwd, adj, grad_values(rowptr, colind, adj.X, fwd.X)
