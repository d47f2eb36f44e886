"""Pins of the CPU oracle against things other than itself (no GPU needed).

* dense FP64 solves (numpy LAPACK) on tiny SPD systems, and finite termination of block CG;
* the closed form of the BCG iterate: X^i - X^0 is the A-norm-optimal (Galerkin) correction in the block
  Krylov space K^i_S(A, R^0) of Section 2 (Definition "Block Krylov subspace"), built here by block Lanczos
  with re-orthogonalisation and a dense solve -- a different characterisation from the oracle's
  recurrence;
* k = 1 and the parallel subalgebra against scipy's textbook CG, iterate by iterate;
* hybrid^p = q independent classical BCGs (Section 3, remark after O'Leary's theorem);
* global^p = classical BCG with p right-hand sides on the stacked block-diagonal system (Section 3,
  proof of the global-rate lemma);
* the Galerkin and A-conjugacy invariants of block CG in the S-product;
* the stopping rule, zero columns, breakdown and maxit semantics.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.linalg import cg

from oracle import bcg as O
from paper_1912_11930_gb300 import workloads as W


def _systems():
    a = W.poisson2d(6)
    b = W.dense_to_csr(W.random_spd_dense(40, seed=3, cond=50.0))
    c = W.poisson3d(4)
    d = W.stencil27(3, seed=1)
    return {"poisson2d_6": a, "spd40": b, "poisson3d_4": c, "s27_3": d}


SYSTEMS = _systems()

# systems large enough that block CG converges well before its Krylov space is exhausted (the method
# has no deflation, so near ceil(n/p) steps it may legitimately break down)
CONVERGE = {"poisson2d_10": W.poisson2d(10), "poisson3d_5": W.poisson3d(5),
            "spd120": W.dense_to_csr(W.random_spd_dense(120, seed=3, cond=30.0)),
            "s27_5": W.stencil27(5, seed=1)}


def _block_krylov_basis(A, R, m):
    """Orthonormal basis of span{R, A R, ..., A^{m-1} R} by block Lanczos with full re-orthogonalisation."""
    blocks = []
    V = np.linalg.qr(R)[0]
    for t in range(m):
        blocks.append(V)
        if t == m - 1:
            break
        Wt = A @ V
        for _ in range(2):
            for U in blocks:
                Wt = Wt - U @ (U.T @ Wt)
        V = np.linalg.qr(Wt)[0]
    return np.hstack(blocks)


def _galerkin_iterate(Ad, B, X0, p, kind, m):
    """X^m from the Krylov-space characterisation of block CG."""
    n, k = B.shape
    q = k // p
    R0 = B - Ad @ X0
    X = X0.copy()
    if kind == "hybrid":
        for j in range(q):
            blk = slice(j * p, (j + 1) * p)
            V = _block_krylov_basis(Ad, R0[:, blk], m)
            X[:, blk] += V @ np.linalg.solve(V.T @ Ad @ V, V.T @ R0[:, blk])
        return X
    Ahat = sla.block_diag(*([Ad] * q))
    Rhat = np.vstack([R0[:, j * p:(j + 1) * p] for j in range(q)])
    V = _block_krylov_basis(Ahat, Rhat, m)
    C = V @ np.linalg.solve(V.T @ Ahat @ V, V.T @ Rhat)
    for j in range(q):
        X[:, j * p:(j + 1) * p] += C[j * n:(j + 1) * n]
    return X


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [  # (sub, k, p)
    ("parallel", 4, 1), ("hybrid", 4, 2), ("hybrid", 8, 4), ("classical", 4, 4),
    ("global", 4, 2), ("global", 8, 4), ("global", 4, 1), ("hybrid", 6, 3),
]


@pytest.mark.parametrize("name", list(CONVERGE))
@pytest.mark.parametrize("sub,k,p", CASES)
def test_dense_solution(name, sub, k, p):
    """Converged X against a dense LAPACK solve, within the textbook bound
    ||x - x*|| / ||x*|| <= cond(A) ||b - A x|| / ||b|| per column."""
    M = CONVERGE[name]
    A = M.to_scipy()
    Ad = A.toarray()
    B = W.rhs(M.n, k, seed=11)
    tol = 1e-10
    res = O.solve(A, B, p=p, sub=sub, tol=tol, maxit=2000)
    assert res.status == O.OK
    assert np.all(res.relres_recursive <= tol)
    Xd = np.linalg.solve(Ad, B)
    ev = np.linalg.eigvalsh(Ad)
    cond = ev[-1] / ev[0]
    for s in range(k):
        true = np.linalg.norm(B[:, s] - Ad @ res.X[:, s]) / np.linalg.norm(B[:, s])
        assert true <= 2 * tol                      # recursive and true residual agree
        assert _rel(res.X[:, s], Xd[:, s]) <= 1.01 * cond * true + 1e-14


@pytest.mark.parametrize("n,cond", [(40, 50.0), (64, 100.0), (96, 20.0)])
def test_finite_termination_classical(n, cond):
    """Classical BCG with k right-hand sides spans n dimensions after ceil(n/k) steps in exact
    arithmetic; in FP64 it must be converged to near machine precision shortly after (random
    spectrum: matrices with heavily repeated eigenvalues exhaust some eigenspaces early and lose
    accuracy there, since the method has no deflation)."""
    M = W.dense_to_csr(W.random_spd_dense(n, seed=n, cond=cond))
    A = M.to_scipy()
    k = 8
    B = W.rhs(M.n, k, seed=5)
    steps = -(-M.n // k)
    res = O.solve(A, B, sub="classical", tol=0.0, maxit=steps + 2)
    Xd = np.linalg.solve(A.toarray(), B)
    assert _rel(res.X, Xd) < 1e-8


@pytest.mark.parametrize("name", ["poisson2d_6", "spd40", "s27_3"])
@pytest.mark.parametrize("sub,k,p", CASES)
@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_krylov_galerkin_closed_form(name, sub, k, p, m):
    M = SYSTEMS[name]
    A = M.to_scipy()
    Ad = A.toarray()
    B = W.rhs(M.n, k, seed=7)
    X0 = 0.1 * W.rhs(M.n, k, seed=8)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    res = O.solve(A, B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert res.iters == m
    Xg = _galerkin_iterate(Ad, B, X0, pp, kind, m)
    assert _rel(res.X - X0, Xg - X0) < 1e-9


@pytest.mark.parametrize("sub", ["hybrid", "global", "parallel", "classical"])
def test_k1_is_textbook_cg(sub):
    M = SYSTEMS["poisson2d_6"]
    A = M.to_scipy()
    b = W.rhs(M.n, 1, seed=2)[:, 0]
    xs = []
    cg(A, b, x0=np.zeros(M.n), rtol=0.0, atol=0.0, maxiter=25, callback=lambda x: xs.append(x.copy()))
    for m in (1, 2, 5, 10, 20):
        res = O.solve(A, b[:, None], p=1, sub=sub, tol=0.0, maxit=m)
        assert _rel(res.X[:, 0], xs[m - 1]) < 1e-10, m


def test_parallel_is_k_independent_cgs():
    M = CONVERGE["spd120"]
    A = M.to_scipy()
    Ad = A.toarray()
    k, tol = 5, 1e-8
    B = W.rhs(M.n, k, seed=4)
    res = O.solve(A, B, sub="parallel", tol=tol, maxit=500)
    assert res.status == O.OK
    for s in range(k):
        xs = []
        cg(A, B[:, s], x0=np.zeros(M.n), rtol=0.0, atol=0.0, maxiter=res.block_iters[s] + 3,
           callback=lambda x: xs.append(x.copy()))
        # the same iterate as CG at the column's own freeze iteration
        assert _rel(res.X[:, s], xs[res.block_iters[s] - 1]) < 1e-9
        # and that iteration is where CG's residual first drops below tol (+-1 at the threshold)
        rn = [np.linalg.norm(B[:, s] - Ad @ x) / np.linalg.norm(B[:, s]) for x in xs]
        first = 1 + next(i for i, r in enumerate(rn) if r <= tol)
        assert abs(first - res.block_iters[s]) <= 1


@pytest.mark.parametrize("k,p", [(8, 4), (6, 2), (8, 2)])
def test_hybrid_is_independent_classical(k, p):
    M = SYSTEMS["poisson3d_4"]
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=9)
    hy = O.solve(A, B, p=p, sub="hybrid", tol=1e-9, maxit=500)
    assert hy.status == O.OK
    for j in range(k // p):
        blk = slice(j * p, (j + 1) * p)
        cl = O.solve(A, B[:, blk], sub="classical", tol=1e-9, maxit=500)
        assert cl.iters == hy.block_iters[j]
        assert _rel(hy.X[:, blk], cl.X) < 1e-13


@pytest.mark.parametrize("k,p", [(8, 4), (6, 2), (4, 1)])
def test_global_is_classical_on_stacked_system(k, p):
    M = SYSTEMS["spd40"]
    A = M.to_scipy()
    q = k // p
    B = W.rhs(M.n, k, seed=10)
    for m in (1, 3, 8):
        gl = O.solve(A, B, p=p, sub="global", tol=0.0, maxit=m)
        Ahat = sp.block_diag([A] * q, format="csr")
        Bhat = np.vstack([B[:, j * p:(j + 1) * p] for j in range(q)])
        st = O.solve(Ahat, Bhat, sub="classical", tol=0.0, maxit=m)
        Xs = np.hstack([st.X[j * M.n:(j + 1) * M.n] for j in range(q)])
        assert _rel(gl.X, Xs) < 1e-12


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 8, 2), ("parallel", 4, 1)])
def test_galerkin_and_conjugacy_invariants(sub, k, p):
    M = SYSTEMS["spd40"]
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=12)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    res = O.solve(A, B, p=p, sub=sub, tol=0.0, maxit=5, record=True)
    H = res.history
    R, P = H["R"], H["P"]          # R[i] = R^i, P[i] = P^{i+1}

    def normalized(Xm, Ym):
        g = O.block_product(Xm, Ym, pp, kind)
        nx = np.sqrt(np.sum(Xm * Xm, axis=0))
        ny = np.sqrt(np.sum(Ym * Ym, axis=0))
        return np.max(np.abs(g)) / (np.max(nx) * np.max(ny))

    for i in range(1, 6):
        for j in range(1, i + 1):      # <<P^j, R^i>> = 0 for j <= i
            assert normalized(P[j - 1], R[i]) < 1e-9, (i, j)
        for j in range(0, i):          # <<R^j, R^i>> = 0 for j < i
            assert normalized(R[j], R[i]) < 1e-9, (i, j)
        for j in range(1, i):          # <<P^j, A P^i>> = 0 for j != i
            assert normalized(P[j - 1], A @ P[i - 1]) < 1e-9, (i, j)
    for i in range(len(H["alpha"])):
        a = H["alpha"][i]
        assert np.max(np.abs(a - np.swapaxes(a, 1, 2))) <= 1e-12 * np.max(np.abs(a))
        if i > 0:   # the recomputed rho^{i-1} equals the previous rho^{i-1} up to rounding
            assert np.max(np.abs(H["rho_rec"][i] - H["rho"][i - 1])) <= 1e-10 * np.max(np.abs(H["rho"][i - 1]))


def test_block_product_structure():
    """The S-products of the Definition in Section 2 as k x k matrices: hybrid = block-diagonal part of
    X^T Y; global = (sum of the diagonal blocks) repeated on the diagonal (R2); and the embedding
    Gl^p within Hy^p, Pl within Hy^p."""
    rng = np.random.default_rng(0)
    X, Y = rng.standard_normal((20, 8)), rng.standard_normal((20, 8))
    full = X.T @ Y
    for p in (1, 2, 4, 8):
        q = 8 // p
        hy = O.block_product(X, Y, p, "hybrid")
        gl = O.block_product(X, Y, p, "global")
        mask = np.kron(np.eye(q), np.ones((p, p)))
        assert np.allclose(sla.block_diag(*hy), full * mask, rtol=1e-14, atol=1e-13)
        s = sum(full[j * p:(j + 1) * p, j * p:(j + 1) * p] for j in range(q))
        assert np.allclose(np.kron(np.eye(q), gl[0]), np.kron(np.eye(q), s), rtol=1e-14, atol=1e-13)
        # BAXPY applies gamma blockwise: Y gamma with gamma in S
        g = hy
        assert np.allclose(O.block_apply(Y, g), Y @ sla.block_diag(*g), rtol=1e-13, atol=1e-13)
        assert np.allclose(O.block_apply(Y, gl), Y @ np.kron(np.eye(q), gl[0]), rtol=1e-13, atol=1e-13)


def test_small_solves_match_lapack():
    rng = np.random.default_rng(1)
    for p in (1, 3, 8, 16):
        G = rng.standard_normal((p, 2 * p))
        S = G @ G.T + 0.1 * np.eye(p)
        D = rng.standard_normal((p, p))
        lam, ok = O.bsolve_cholesky(S[None], D[None], np.array([True]))
        assert ok and np.allclose(lam[0], np.linalg.solve(S, D), rtol=1e-10, atol=1e-12)
        N = S + 0.01 * rng.standard_normal((p, p))
        bet, ok = O.bsolve_lu(N[None], D[None], np.array([True]))
        assert ok and np.allclose(bet[0], np.linalg.solve(N, D), rtol=1e-10, atol=1e-12)


def test_stopping_rule_and_counts():
    M = SYSTEMS["poisson3d_4"]
    A = M.to_scipy()
    B = W.rhs(M.n, 8, seed=13)
    tol = 1e-8
    res = O.solve(A, B, p=4, sub="hybrid", tol=tol, maxit=500)
    assert res.status == O.OK
    assert np.all(res.relres_recursive <= tol)
    assert res.iters == max(res.block_iters)
    for j in range(2):   # one iteration fewer for that block alone would not have converged
        blk = slice(4 * j, 4 * j + 4)
        early = O.solve(A, B[:, blk], sub="classical", tol=tol, maxit=int(res.block_iters[j]) - 1)
        assert early.status == O.NOT_CONVERGED


def test_zero_columns_and_zero_rhs():
    M = SYSTEMS["poisson2d_6"]
    A = M.to_scipy()
    B = W.rhs(M.n, 4, seed=14)
    B[:, 2] = 0.0
    res = O.solve(A, B, sub="parallel", tol=1e-8, maxit=500)
    assert res.status == O.OK
    assert res.block_iters[2] == 0 and np.all(res.X[:, 2] == 0.0)
    assert np.all(res.block_iters[[0, 1, 3]] > 0)
    Z = O.solve(A, np.zeros((M.n, 4)), p=2, sub="hybrid", tol=1e-8)
    assert Z.status == O.OK and Z.iters == 0 and np.all(Z.X == 0)


def test_breakdown_duplicate_columns_and_non_spd():
    M = SYSTEMS["poisson2d_6"]
    A = M.to_scipy()
    B = W.rhs(M.n, 4, seed=15)
    B[:, 1] = B[:, 0]
    res = O.solve(A, B, p=2, sub="hybrid", tol=1e-8)
    assert res.status == O.BREAKDOWN and res.breakdown_iter == 1
    neg = -sp.identity(M.n, format="csr")
    res = O.solve(neg, W.rhs(M.n, 2, seed=1), p=2, sub="hybrid", tol=1e-8)
    assert res.status == O.BREAKDOWN and res.breakdown_iter == 1


def test_nan_and_maxit():
    M = SYSTEMS["poisson2d_6"]
    A = M.to_scipy()
    B = W.rhs(M.n, 2, seed=16)
    Bn = B.copy()
    Bn[3, 1] = np.nan
    assert O.solve(A, Bn, p=1, sub="hybrid").status == O.NUMERIC
    r = O.solve(A, B, p=2, sub="hybrid", tol=1e-14, maxit=3)
    assert r.status == O.NOT_CONVERGED and r.iters == 3


def test_gradient_dense_and_finite_differences():
    """dL/dB = Lambda and dL/dA_ij = -Lambda_i . X_j for L = sum(W * X), against a dense FP64 gradient
    and central finite differences of the dense solve (symmetric pairs perturbed together, so A stays
    SPD)."""
    M = W.stencil27(3, seed=2)
    A = M.to_scipy()
    Ad = A.toarray()
    k = 3
    B = W.rhs(M.n, k, seed=3)
    Wt = W.loss_weights(M.n, k, seed=3)
    fwd, adj, g = O.solve_and_grad(A, M.rowptr, M.colind, B, Wt, p=k, sub="hybrid", tol=1e-14)
    X = np.linalg.solve(Ad, B)
    Lam = np.linalg.solve(Ad, Wt)
    assert _rel(adj.X, Lam) < 1e-10
    rows = np.repeat(np.arange(M.n), np.diff(M.rowptr))
    gd = -np.sum(Lam[rows] * X[M.colind], axis=1)
    assert _rel(g, gd) < 1e-10
    # central differences on a few entries
    pos = {(int(rows[e]), int(M.colind[e])): e for e in range(M.nnz)}
    rng = np.random.default_rng(0)
    for e in rng.choice(M.nnz, 12, replace=False):
        i, j = int(rows[e]), int(M.colind[e])
        h = 1e-6 * abs(Ad[i, j])
        Ap, Am = Ad.copy(), Ad.copy()
        Ap[i, j] += h; Am[i, j] -= h
        if i != j:
            Ap[j, i] += h; Am[j, i] -= h
        fd = (np.sum(Wt * np.linalg.solve(Ap, B)) - np.sum(Wt * np.linalg.solve(Am, B))) / (2 * h)
        an = g[e] + (g[pos[(j, i)]] if i != j else 0.0)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (i, j, fd, an)


# ---- Jacobi preconditioner (Algorithm 1 with M = diag(A)) --------------------------------------------------
def test_jacobi_k1_is_scipy_pcg():
    M = W.varcoef3d(6, 5, 4, seed=2)
    A = M.to_scipy()
    b = W.rhs(M.n, 1, seed=5)[:, 0]
    import scipy.sparse as sps
    Minv = sps.diags(1.0 / A.diagonal())
    xs = []
    cg(A, b, x0=np.zeros(M.n), rtol=0.0, atol=0.0, maxiter=20, M=Minv, callback=lambda x: xs.append(x.copy()))
    for m in (1, 3, 8, 15):
        res = O.solve(A, b[:, None], p=1, sub="hybrid", tol=0.0, maxit=m, precond="jacobi")
        assert _rel(res.X[:, 0], xs[m - 1]) < 1e-10, m


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 8, 4), ("classical", 4, 4)])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_jacobi_galerkin_closed_form(sub, k, p, m):
    """Preconditioned block CG: X^m - X^0 is the A-norm-optimal correction in the block Krylov space of
    M^{-1} A and M^{-1} R^0 (the subalgebra's space)."""
    Mx = W.varcoef3d(5, 4, 3, seed=3)
    A = Mx.to_scipy()
    Ad = A.toarray()
    dinv = 1.0 / np.diag(Ad)
    B = W.rhs(Mx.n, k, seed=6)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    res = O.solve(A, B, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
    q = k // pp
    Xg = np.zeros_like(B)
    if kind == "hybrid":
        for j in range(q):
            blk = slice(j * pp, (j + 1) * pp)
            V = _block_krylov_basis(dinv[:, None] * Ad, dinv[:, None] * B[:, blk], m)
            Xg[:, blk] = V @ np.linalg.solve(V.T @ Ad @ V, V.T @ B[:, blk])
    else:
        Ahat = sla.block_diag(*([Ad] * q))
        Dhat = np.concatenate([dinv] * q)
        Bhat = np.vstack([B[:, j * pp:(j + 1) * pp] for j in range(q)])
        V = _block_krylov_basis(Dhat[:, None] * Ahat, Dhat[:, None] * Bhat, m)
        C = V @ np.linalg.solve(V.T @ Ahat @ V, V.T @ Bhat)
        for j in range(q):
            Xg[:, j * pp:(j + 1) * pp] = C[j * Mx.n:(j + 1) * Mx.n]
    assert _rel(res.X, Xg) < 1e-9


def test_jacobi_converges_to_dense_solution():
    Mx = W.stencil27(6, seed=4)
    A = Mx.to_scipy()
    B = W.rhs(Mx.n, 8, seed=7)
    res = O.solve(A, B, p=4, sub="hybrid", tol=1e-11, maxit=500, precond="jacobi")
    assert res.status == O.OK
    assert _rel(res.X, np.linalg.solve(A.toarray(), B)) < 1e-8
    plain = O.solve(A, B, p=4, sub="hybrid", tol=1e-11, maxit=500)
    assert res.iters <= plain.iters + 2
