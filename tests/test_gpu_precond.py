"""GPU parity of the Jacobi-preconditioned solve (Algorithm 1 with M = diag(A)) against the CPU oracle.

Same bars as the unpreconditioned parity tests: FP64 relative solution error <= 1e-9 at equal iteration
counts, converged counts within +-2, mixed precision <= 1e-8 against the FP64 oracle. With M = diag(A) the
oracle's own iterates move by < 1e-13 under a 1e-16 relative perturbation of B on every case below (the
log-normal variable-coefficient matrix included: Jacobi removes most of its coefficient contrast), so the
equal-iteration cases run 15-25 iterations. The cases cover every kernel variant that forms Z = M^{-1} R:
the initial residual, the per-element and warp-chunk X/R updates and search-direction updates, and the
large-block tiled Gram and update kernels; CSR and stencil operators.
"""
import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import bcg, workloads as W
from parity_check import assert_close, rel_fro as _rel

pytestmark = pytest.mark.gpu

NEVER = 1e-300


@pytest.fixture(scope="module")
def torch_dev(lib):
    import torch
    return torch, torch.device("cuda:0")


_MATS = {}


def mat(name):
    if name not in _MATS:
        _MATS[name] = {
            "p3d_30": lambda: W.poisson3d(30, 31, 29),
            "vc_20": lambda: W.varcoef3d(20, 17, 23, seed=4),
            "s27_15": lambda: W.stencil27(15, 14, 13, seed=5),
            "spd_200": lambda: W.dense_to_csr(W.random_spd_dense(200, seed=6, cond=40.0)),
        }[name]()
    return _MATS[name]


def gpu_solve(torch_dev, M, B, *, k, p, sub, prec="fp64", form="csr", tol=NEVER, maxit=30, X0=None,
              precond=1):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, form=form, device=dev)
    S.set_option("precond", precond)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Xt = None if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).to(dev)
    X, r = S.solve(Bt, Xt, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    out = X.cpu().numpy()
    S.close()
    return out, r


# (matrix, operator form, sub, k, p, iterations)
FIXED = [
    ("vc_20", "csr", "hybrid", 16, 16, 20), ("vc_20", "stencil", "hybrid", 16, 16, 20),
    ("vc_20", "csr", "hybrid", 64, 16, 10), ("vc_20", "csr", "parallel", 8, 1, 30),
    ("vc_20", "csr", "classical", 8, 8, 12), ("s27_15", "csr", "hybrid", 24, 12, 15),
    ("s27_15", "csr", "global", 12, 3, 20), ("spd_200", "csr", "hybrid", 16, 4, 12),
    ("p3d_30", "csr", "hybrid", 6, 3, 25), ("p3d_30", "stencil", "hybrid", 32, 8, 25),
    # large blocks: tiled Gram with Z formed on the fly, tiled P update with the scaled base
    ("vc_20", "csr", "hybrid", 128, 64, 5), ("s27_15", "csr", "global", 128, 64, 5),
    ("s27_15", "csr", "classical", 64, 64, 6),
]


@pytest.mark.parametrize("name,form,sub,k,p,m", FIXED)
def test_jacobi_fp64_equal_iterations(torch_dev, name, form, sub, k, p, m):
    M = mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, form=form, maxit=m, X0=X0)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("name,sub,k,p", [("vc_20", "hybrid", 16, 4), ("s27_15", "hybrid", 16, 16),
                                          ("vc_20", "parallel", 8, 1)])
def test_jacobi_converged_counts(torch_dev, name, sub, k, p):
    M = mat(name)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=3)
    tol = 1e-8
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=3000)
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub=sub, tol=tol, maxit=3000, precond="jacobi")
    assert ref.status == O.OK
    assert abs(r.iters - ref.iters) <= 2, (r.iters, ref.iters)
    assert np.all(np.abs(np.array(r.block_iters) - ref.block_iters) <= 2)
    res = np.linalg.norm(B - A @ Xg, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5 * tol)
    # the preconditioner pays on the log-normal coefficients: fewer iterations than M = I
    if name == "vc_20":
        plain = O.solve(A, B, p=p, sub=sub, tol=tol, maxit=3000)
        assert r.iters < plain.iters


@pytest.mark.parametrize("name,form,sub,k,p", [("vc_20", "stencil", "hybrid", 16, 16), ("s27_15", "csr", "hybrid", 24, 8),
                                               ("vc_20", "csr", "classical", 64, 64)])
def test_jacobi_mixed_precision(torch_dev, name, form, sub, k, p):
    M = mat(name)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=11)
    X, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, prec="fp32_refine", form=form, tol=1e-12, maxit=5000)
    assert r.ok, r
    true = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true <= 1.5e-12)
    ref = O.solve(A, B, p=p, sub=sub, tol=1e-13, maxit=5000, precond="jacobi")
    assert_close(X, ref.X, 1e-8)


def test_jacobi_option_toggles_and_update_values(torch_dev):
    """precond can be switched on a live handle (the captured FP32 graph is rebuilt), and bcg_update_values
    recomputes diag(A)^{-1}: after scaling the matrix by 2 the Jacobi iterates are those of the new matrix."""
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = mat("vc_20")
    A = M.to_scipy()
    k, p, m = 16, 8, 15
    B = W.rhs(M.n, k, seed=21)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec="fp64", device=dev)
    Bt = torch.from_numpy(B).to(dev)
    X_plain, _ = S.solve(Bt, tol=NEVER, maxit=m)
    S.set_option("precond", 1)
    X_jac, _ = S.solve(Bt, tol=NEVER, maxit=m)
    S.set_option("precond", 0)
    X_back, _ = S.solve(Bt, tol=NEVER, maxit=m)
    assert torch.equal(X_plain, X_back)
    assert_close(X_plain.cpu().numpy(), O.solve(A, B, p=p, sub="hybrid", tol=0.0, maxit=m).X, 1e-9)
    assert_close(X_jac.cpu().numpy(), O.solve(A, B, p=p, sub="hybrid", tol=0.0, maxit=m, precond="jacobi").X, 1e-9)
    S.set_option("precond", 1)
    S.update_values(torch.from_numpy(2.0 * M.vals).to(dev))
    X2, _ = S.solve(Bt, tol=NEVER, maxit=m)
    ref2 = O.solve(2.0 * A, B, p=p, sub="hybrid", tol=0.0, maxit=m, precond="jacobi")
    assert_close(X2.cpu().numpy(), ref2.X, 1e-9)
    with pytest.raises(bcg.BCGError, match="precond"):
        S.set_option("precond", 2)
    S.close()
    # the mixed form keeps its own FP32 copy of diag(A)^{-1}; graphs on and off agree bit for bit
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec="fp32_refine", device=dev)
    S.set_option("precond", 1)
    X_g, r_g = S.solve(Bt, tol=1e-10, maxit=5000)
    S.set_option("graph", 0)
    X_n, r_n = S.solve(Bt, tol=1e-10, maxit=5000)
    S.close()
    assert r_g.ok and torch.equal(X_g, X_n) and r_g.iters == r_n.iters


def test_jacobi_zero_diagonal_is_reported(torch_dev):
    """M = diag(A) needs a positive diagonal; a zero diagonal entry makes Z non-finite and the solve stops
    with NUMERIC (or BREAKDOWN), in both precisions and on large blocks, instead of iterating on garbage."""
    from paper_1912_11930_gb300 import bcg
    M = mat("p3d_30")
    vals = M.vals.copy()
    diag = np.nonzero(M.colind == np.repeat(np.arange(M.n), np.diff(M.rowptr)))[0]
    vals[diag[17]] = 0.0
    Z = W.CSRMatrix(M.n, M.rowptr, M.colind, vals)
    for prec, k, p in (("fp64", 8, 4), ("fp32_refine", 8, 4), ("fp64", 64, 64)):
        X, r = gpu_solve(torch_dev, Z, W.rhs(M.n, k, seed=13), k=k, p=p, sub="hybrid" if p < k else "classical",
                         prec=prec, tol=1e-8, maxit=200)
        assert r.status in (bcg.NUMERIC, bcg.BREAKDOWN), r
