"""Pins of the oracle's retooled block CG (Dubrulle, Electron. Trans. Numer. Anal. 12, 2001; the stability
reference of Section 3), none of which re-types its formulas:

* its iterates are the block Krylov Galerkin iterates, computed here from an orthonormal Krylov basis
  (the same closed form that pins Algorithm 1), and at k = 1 they are scipy's CG iterates;
* the invariants the retooling is built on hold: <<Q, Q>> = I, <<S, Q>> = I, and Q C is the true residual;
* a right-hand side scaled column by column gives the scaled iterates and the same iteration count,
  where Algorithm 1's small systems become singular to working precision;
* breakdown and degenerate cases: duplicated columns, zero blocks, a zero column inside a live block;
* planted mistakes (on the CPU, through monkeypatch) in the orthonormalisation, the direction update and
  the solution update are caught.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.sparse.linalg import cg

from oracle import bcg as O
from paper_1912_11930_gb300 import workloads as W

from test_oracle_pins import SYSTEMS, CONVERGE, _galerkin_iterate, _rel

CASES = [("parallel", 4, 1), ("hybrid", 4, 2), ("hybrid", 8, 4), ("classical", 4, 4), ("hybrid", 6, 3)]


@pytest.mark.parametrize("name", ["poisson2d_6", "spd40", "s27_3"])
@pytest.mark.parametrize("sub,k,p", CASES)
@pytest.mark.parametrize("m", [1, 2, 4])
def test_retooled_krylov_galerkin_closed_form(name, sub, k, p, m):
    M = SYSTEMS[name]
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=7)
    X0 = 0.1 * W.rhs(M.n, k, seed=8)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    res = O.solve_retooled(A, B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert res.status == O.NOT_CONVERGED and res.iters == m
    Xg = _galerkin_iterate(A.toarray(), B, X0, pp, kind, m)
    assert _rel(res.X - X0, Xg - X0) < 1e-9


def test_retooled_k1_is_textbook_cg():
    M = SYSTEMS["poisson2d_6"]
    A = M.to_scipy()
    b = W.rhs(M.n, 1, seed=2)[:, 0]
    xs = []
    cg(A, b, x0=np.zeros(M.n), rtol=0.0, atol=0.0, maxiter=25, callback=lambda x: xs.append(x.copy()))
    for m in (1, 2, 5, 10, 20):
        res = O.solve_retooled(A, b[:, None], p=1, sub="parallel", tol=0.0, maxit=m)
        assert _rel(res.X[:, 0], xs[m - 1]) < 1e-10, m


@pytest.mark.parametrize("name", list(CONVERGE))
@pytest.mark.parametrize("sub,k,p", CASES)
def test_retooled_dense_solution_and_counts(name, sub, k, p):
    """Converged solution within the textbook bound against LAPACK, true residual at the tolerance, and
    the same iteration counts as Algorithm 1 (the two are one method in exact arithmetic)."""
    M = CONVERGE[name]
    A = M.to_scipy()
    Ad = A.toarray()
    B = W.rhs(M.n, k, seed=11)
    tol = 1e-10
    res = O.solve_retooled(A, B, p=p, sub=sub, tol=tol, maxit=2000)
    assert res.status == O.OK
    assert np.all(res.relres_true <= 2 * tol)
    ev = np.linalg.eigvalsh(Ad)
    Xd = np.linalg.solve(Ad, B)
    for s in range(k):
        assert _rel(res.X[:, s], Xd[:, s]) <= 1.01 * ev[-1] / ev[0] * res.relres_true[s] + 1e-14
    ref = O.solve(A, B, p=p, sub=sub, tol=tol, maxit=2000)
    assert abs(res.iters - ref.iters) <= 1
    assert np.all(np.abs(res.block_iters - ref.block_iters) <= 1)


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("classical", 6, 6), ("parallel", 3, 1)])
def test_retooled_invariants(sub, k, p):
    """<<Q, Q>> = I and <<S, Q>> = I in every block, and Q C = B - A X, through the first iterations."""
    M = CONVERGE["spd120"]
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=5)
    res = O.solve_retooled(A, B, p=p, sub=sub, tol=0.0, maxit=6, record=True)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    for X, Q, S, C in zip(res.history["X"], res.history["Q"], res.history["S"], res.history["C"]):
        R = B - A @ X
        for j in range(k // pp):
            cols = slice(j * pp, (j + 1) * pp)
            assert np.abs(Q[:, cols].T @ Q[:, cols] - np.eye(pp)).max() < 1e-10
            assert np.abs(S[:, cols].T @ Q[:, cols] - np.eye(pp)).max() < 1e-8
            assert np.allclose(np.triu(C[j]), C[j])      # the factor stays upper triangular
            assert _rel(Q[:, cols] @ C[j], R[:, cols]) < 1e-9


def test_retooled_first_factor_is_the_qr_factorisation():
    """The Cholesky QR of R^0 gives LAPACK's QR with a positive diagonal."""
    M = SYSTEMS["spd40"]
    A = M.to_scipy()
    B = W.rhs(M.n, 4, seed=9)
    res = O.solve_retooled(A, B, p=4, sub="classical", tol=0.0, maxit=1, record=True)
    Qr, Rr = np.linalg.qr(B)
    sgn = np.sign(np.diag(Rr))
    assert _rel(res.history["Q"][0], Qr * sgn) < 1e-12
    assert _rel(res.history["C"][0][0], sgn[:, None] * Rr) < 1e-12


@pytest.mark.parametrize("spread", [4, 8, 10])
def test_retooled_is_scale_invariant(spread):
    """B D (D diagonal, column scales 10^-spread .. 10^spread): X(B D) = X(B) D at every step and the same
    count. Algorithm 1 forms rho = R^T R with diagonal entries 10^(4 spread) apart, below the pivot test
    of its LU, and reports a breakdown in iteration 1."""
    M = CONVERGE["poisson2d_10"]
    A = M.to_scipy()
    k = 4
    B = W.rhs(M.n, k, seed=11)
    D = np.diag(10.0 ** np.linspace(-spread, spread, k))
    for m in (3, 10):
        a = O.solve_retooled(A, B, p=k, sub="classical", tol=0.0, maxit=m)
        b = O.solve_retooled(A, B @ D, p=k, sub="classical", tol=0.0, maxit=m)
        assert _rel(b.X @ np.linalg.inv(D), a.X) < 1e-9
    a = O.solve_retooled(A, B, p=k, sub="classical", tol=1e-10, maxit=500)
    b = O.solve_retooled(A, B @ D, p=k, sub="classical", tol=1e-10, maxit=500)
    assert a.status == b.status == O.OK and a.iters == b.iters
    assert np.all(b.relres_true <= 2e-10)
    ref = O.solve(A, B @ D, p=k, sub="classical", tol=1e-10, maxit=500)
    assert ref.status == O.BREAKDOWN and ref.breakdown_iter == 1


def test_retooled_degenerate_cases():
    M = CONVERGE["poisson2d_10"]
    A = M.to_scipy()
    B = W.rhs(M.n, 8, seed=3)
    # a zero block converges at iteration 0, the others solve as if alone
    Bz = B.copy()
    Bz[:, 4:] = 0.0
    r = O.solve_retooled(A, Bz, p=4, sub="hybrid", tol=1e-10, maxit=500)
    alone = O.solve_retooled(A, B[:, :4], p=4, sub="classical", tol=1e-10, maxit=500)
    assert r.status == O.OK and r.block_iters[1] == 0 and np.all(r.X[:, 4:] == 0.0)
    assert np.array_equal(r.X[:, :4], alone.X)
    # an all-zero right-hand side: nothing to do
    r = O.solve_retooled(A, np.zeros_like(B), p=4, sub="hybrid", tol=1e-10, maxit=5)
    assert r.status == O.OK and r.iters == 0
    # duplicated columns, or a zero column next to live ones: the first Cholesky QR fails
    for Bd in (np.hstack([B[:, :2], B[:, :2]]), np.hstack([B[:, :3], np.zeros((M.n, 1))])):
        r = O.solve_retooled(A, Bd, p=4, sub="classical", tol=1e-10, maxit=50)
        assert r.status == O.BREAKDOWN and r.breakdown_iter == 1 and r.iters == 0
    with pytest.raises(ValueError):
        O.solve_retooled(A, B, p=3, sub="global")


# ---- the global subalgebra and the Jacobi preconditioner ---------------------------------------------------
GLOBAL_CASES = [("global", 4, 2), ("global", 8, 4), ("global", 4, 1), ("global", 6, 3)]


@pytest.mark.parametrize("name", ["poisson2d_6", "spd40", "s27_3"])
@pytest.mark.parametrize("sub,k,p", GLOBAL_CASES)
@pytest.mark.parametrize("m", [1, 2, 4])
def test_retooled_global_krylov_galerkin_closed_form(name, sub, k, p, m):
    """S_Gl: the iterate is the Galerkin solution of the stacked block-diagonal system over its block Krylov
    space (the closed form that pins Algorithm 1's global form)."""
    M = SYSTEMS[name]
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=7)
    X0 = 0.1 * W.rhs(M.n, k, seed=8)
    res = O.solve_retooled(A, B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert res.status == O.NOT_CONVERGED and res.iters == m
    Xg = _galerkin_iterate(A.toarray(), B, X0, p, "global", m)
    assert _rel(res.X - X0, Xg - X0) < 1e-9


def test_retooled_global_with_one_block_is_classical():
    M = CONVERGE["spd120"]
    A = M.to_scipy()
    B = W.rhs(M.n, 4, seed=3)
    a = O.solve_retooled(A, B, p=4, sub="global", tol=1e-10, maxit=500)
    b = O.solve_retooled(A, B, p=4, sub="classical", tol=1e-10, maxit=500)
    assert a.status == b.status == O.OK and a.iters == b.iters and np.array_equal(a.X, b.X)


def _jacobi_scaled(A):
    d = A.diagonal()
    s = 1.0 / np.sqrt(d)
    import scipy.sparse as sp
    Dm = sp.diags(s)
    return s, (Dm @ A @ Dm).tocsr()


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("classical", 4, 4), ("global", 6, 2), ("parallel", 3, 1)])
@pytest.mark.parametrize("m", [1, 3, 8])
def test_retooled_jacobi_is_the_symmetrically_scaled_system(sub, k, p, m):
    """With M = diag(A) = D the preconditioned iterate is D^{-1/2} times the unpreconditioned iterate on
    D^{-1/2} A D^{-1/2} y = D^{-1/2} B from y^0 = D^{1/2} X^0 (a change of variables, not the same code)."""
    M = W.varcoef3d(5, 4, 6, seed=3)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=4)
    X0 = 0.1 * W.rhs(M.n, k, seed=5)
    s, At = _jacobi_scaled(A)
    a = O.solve_retooled(A, B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
    b = O.solve_retooled(At, B * s[:, None], X0=X0 / s[:, None], p=p, sub=sub, tol=0.0, maxit=m)
    assert a.status == b.status == O.NOT_CONVERGED
    assert _rel(a.X, b.X * s[:, None]) < 1e-10


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 8, 4), ("classical", 4, 4)])
def test_retooled_jacobi_counts_and_solution_match_algorithm1(sub, k, p):
    M = W.varcoef3d(6, 5, 7, seed=2)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=6)
    for m in (2, 6):
        a = O.solve_retooled(A, B, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
        r = O.solve(A, B, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
        assert _rel(a.X, r.X) < 1e-9
    a = O.solve_retooled(A, B, p=p, sub=sub, tol=1e-10, maxit=2000, precond="jacobi")
    r = O.solve(A, B, p=p, sub=sub, tol=1e-10, maxit=2000, precond="jacobi")
    assert a.status == r.status == O.OK and abs(a.iters - r.iters) <= 1
    assert np.all(a.relres_true <= 2e-10)


@pytest.mark.parametrize("sub,k,p,pre", [("global", 8, 4, "none"), ("hybrid", 8, 4, "jacobi"),
                                         ("global", 6, 3, "jacobi")])
def test_retooled_invariants_global_and_jacobi(sub, k, p, pre):
    """<<Q, M^{-1} Q>> = I in the subalgebra (global: summed over the column blocks), C upper triangular and
    Q C = B - A X, through the first iterations."""
    M = W.varcoef3d(5, 5, 5, seed=1)
    A = M.to_scipy()
    d = A.diagonal() if pre == "jacobi" else np.ones(M.n)
    B = W.rhs(M.n, k, seed=5)
    res = O.solve_retooled(A, B, p=p, sub=sub, tol=0.0, maxit=5, record=True, precond=pre)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    q = k // pp
    for X, Q, C in zip(res.history["X"], res.history["Q"], res.history["C"]):
        R = B - A @ X
        grams = [Q[:, j * pp:(j + 1) * pp].T @ (Q[:, j * pp:(j + 1) * pp] / d[:, None]) for j in range(q)]
        if kind == "global":
            assert np.abs(sum(grams) - np.eye(pp)).max() < 1e-10
        else:
            assert all(np.abs(g - np.eye(pp)).max() < 1e-10 for g in grams)
        for j in range(q):
            Cb = C[j if kind == "hybrid" else 0]
            assert np.allclose(np.triu(Cb), Cb)
            assert _rel(Q[:, j * pp:(j + 1) * pp] @ Cb, R[:, j * pp:(j + 1) * pp]) < 1e-9


def test_retooled_global_scale_invariance():
    """A column scaling that is one diagonal D shared by all column blocks commutes with S_Gl's elements:
    X(B (I_q (x) D)) = X(B) (I_q (x) D) and the same count, where Algorithm 1's global form breaks down."""
    M = CONVERGE["poisson2d_10"]
    A = M.to_scipy()
    k, p = 8, 4
    B = W.rhs(M.n, k, seed=12)
    D = np.diag(np.tile(10.0 ** np.linspace(-8, 8, p), k // p))
    for m in (3, 10):
        a = O.solve_retooled(A, B, p=p, sub="global", tol=0.0, maxit=m)
        b = O.solve_retooled(A, B @ D, p=p, sub="global", tol=0.0, maxit=m)
        assert _rel(b.X @ np.linalg.inv(D), a.X) < 1e-9
    a = O.solve_retooled(A, B, p=p, sub="global", tol=1e-10, maxit=500)
    b = O.solve_retooled(A, B @ D, p=p, sub="global", tol=1e-10, maxit=500)
    assert a.status == b.status == O.OK and a.iters == b.iters
    assert np.all(b.relres_true <= 2e-10)
    assert O.solve(A, B @ D, p=p, sub="global", tol=1e-10, maxit=500).status == O.BREAKDOWN


def test_retooled_global_zero_block_and_zero_rhs():
    """A zero column block inside the global subalgebra does not break the shared factorisation (its Gram
    contribution is zero); an all-zero right-hand side converges at iteration 0."""
    M = CONVERGE["poisson2d_10"]
    A = M.to_scipy()
    B = W.rhs(M.n, 8, seed=3)
    Bz = B.copy()
    Bz[:, 4:] = 0.0
    r = O.solve_retooled(A, Bz, p=4, sub="global", tol=1e-10, maxit=500)
    ref = O.solve(A, Bz, p=4, sub="global", tol=1e-10, maxit=500)
    assert r.status == ref.status
    r = O.solve_retooled(A, np.zeros_like(B), p=4, sub="global", tol=1e-10, maxit=5)
    assert r.status == O.OK and r.iters == 0


# ---- planted mistakes -----------------------------------------------------------------------------------
def _deviation(m=3):
    M = SYSTEMS["spd40"]
    A = M.to_scipy()
    B = W.rhs(M.n, 8, seed=7)
    res = O.solve_retooled(A, B, p=4, sub="hybrid", tol=0.0, maxit=m)
    return _rel(res.X, _galerkin_iterate(A.toarray(), B, np.zeros_like(B), 4, "hybrid", m))


def test_retooled_pins_pass_unmutated():
    assert _deviation() < 1e-9


def test_detects_psi_not_transposed(monkeypatch):
    """S = Q + S psi (psi instead of psi^T in the direction update)."""
    monkeypatch.setattr(O, "retooled_direction", lambda Q, S, psi: Q + S @ psi)
    assert _deviation() > 1e-6


def test_detects_missing_c_in_solution_update(monkeypatch):
    """X += S xi instead of X += S (xi C): the factor of the residual is dropped."""
    monkeypatch.setattr(O, "retooled_solution_coefficient", lambda xi, C: xi)
    assert _deviation() > 1e-6


def test_detects_unnormalised_basis(monkeypatch):
    """A Cholesky factor off by a constant leaves the iterates alone (the method only needs R = Q C) but
    breaks the orthonormality that the invariants test checks."""
    orig = O.cholesky_lower_colrel
    monkeypatch.setattr(O, "cholesky_lower_colrel", lambda G: None if orig(G) is None else 1.5 * orig(G))
    M = CONVERGE["spd120"]
    B = W.rhs(M.n, 4, seed=5)
    res = O.solve_retooled(M.to_scipy(), B, p=4, sub="classical", tol=0.0, maxit=3, record=True)
    Q = res.history["Q"][-1]
    assert np.abs(Q.T @ Q - np.eye(4)).max() > 0.1


def test_detects_wrong_sign_of_residual_basis_update(monkeypatch):
    """T = Q + W xi instead of Q - W xi."""
    orig = O.baxpy
    calls = {"n": 0}

    def mutated(X, Y, gamma, sign=1.0):
        calls["n"] += 1
        if calls["n"] % 2 == 0:   # the second BAXPY of each iteration forms T
            return orig(X, Y, gamma, -sign)
        return orig(X, Y, gamma, sign)

    monkeypatch.setattr(O, "baxpy", mutated)
    assert _deviation() > 1e-6


def _jacobi_deviation(m=4):
    M = W.varcoef3d(5, 4, 6, seed=3)
    A = M.to_scipy()
    B = W.rhs(M.n, 8, seed=4)
    s, At = _jacobi_scaled(A)
    a = O.solve_retooled(A, B, p=4, sub="hybrid", tol=0.0, maxit=m, precond="jacobi")
    b = O.solve_retooled(At, B * s[:, None], p=4, sub="hybrid", tol=0.0, maxit=m)
    return _rel(a.X, b.X * s[:, None])


def test_detects_unpreconditioned_basis_product(monkeypatch):
    """gamma = <<T, T>> instead of <<T, M^{-1} T>> under Jacobi (the preconditioner skipped on every call that
    forms gamma): the basis is orthonormal in the wrong product and the iterates leave Algorithm 1's."""
    assert _jacobi_deviation() < 1e-10
    calls = {"n": 0}
    orig_pre = O._preconditioner

    def pre(A, precond):
        f = orig_pre(A, precond)
        def g(X):
            calls["n"] += 1
            return X if calls["n"] % 2 == 1 and calls["n"] > 2 else f(X)   # gamma's M^{-1} T skipped
        return g
    monkeypatch.setattr(O, "_preconditioner", pre)
    assert _jacobi_deviation() > 1e-6
