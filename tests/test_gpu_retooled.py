"""GPU parity of the retooled block CG (option "retooled": Dubrulle's form, the stability reference of
Section 3) against the oracle's ``solve_retooled``, through the C ABI.

Bars as for Algorithm 1: FP64 relative solution error <= 1e-9 at equal iteration counts, converged counts
within +-2. Cases cover the streaming kernels for p <= 32 (odd and even k, blocks that straddle warps, the
32-wide accumulators) and the tiled large-block path (p = 64, 128), CSR, stencil and SELL operators; then
what the form is for -- right-hand sides whose columns differ in scale by 12 orders, where Algorithm 1
breaks down -- and its degenerate cases and argument checks.
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
            "p2d_37x29": lambda: W.poisson2d(37, 29),
            "p3d_30": lambda: W.poisson3d(30, 31, 29),
            "p3d_17": lambda: W.poisson3d(17, 19, 16),
            "vc_20": lambda: W.varcoef3d(20, 17, 23, seed=4),
            "s27_15": lambda: W.stencil27(15, 14, 13, seed=5),
            "spd_200": lambda: W.dense_to_csr(W.random_spd_dense(200, seed=6, cond=40.0)),
        }[name]()
    return _MATS[name]


def gpu_solve(torch_dev, M, B, *, k, p, sub, form="csr", tol=NEVER, maxit=30, X0=None, retooled=1, precond=0):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec="fp64", form=form, device=dev)
    S.set_option("retooled", retooled)
    S.set_option("precond", precond)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Xt = None if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).to(dev)
    X, r = S.solve(Bt, Xt, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    out = X.cpu().numpy()
    S.close()
    return out, r


# (matrix, operator form, sub, k, p, iterations): iteration counts where Algorithm 1's parity cases stay
# stable under rounding (the retooled form has the same iterates in exact arithmetic)
FIXED = [
    ("p2d_37x29", "csr", "hybrid", 8, 4, 30), ("p2d_37x29", "stencil", "parallel", 8, 1, 30),
    ("p2d_37x29", "csr", "classical", 8, 8, 20), ("p3d_30", "csr", "hybrid", 32, 8, 25),
    ("p3d_30", "stencil", "hybrid", 32, 8, 25), ("p3d_30", "csr", "hybrid", 6, 3, 25),
    ("p3d_30", "csr", "hybrid", 1, 1, 40), ("p3d_30", "csr", "classical", 32, 32, 12),
    ("p3d_30", "sell", "hybrid", 16, 4, 20), ("vc_20", "stencil", "hybrid", 16, 16, 10),
    ("s27_15", "csr", "hybrid", 24, 12, 15), ("spd_200", "csr", "parallel", 5, 1, 20),
    ("spd_200", "csr", "hybrid", 15, 5, 10),
    # large blocks: tiled Gram and block updates, p x p factorisations in global memory
    ("p3d_17", "csr", "classical", 64, 64, 6), ("p3d_17", "csr", "hybrid", 128, 64, 5),
    ("p3d_17", "stencil", "classical", 128, 128, 4),
]


@pytest.mark.parametrize("name,form,sub,k,p,m", FIXED)
def test_retooled_equal_iterations(torch_dev, name, form, sub, k, p, m):
    M = mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, form=form, maxit=m, X0=X0)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    ref = O.solve_retooled(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("name,sub,k,p", [("p2d_37x29", "hybrid", 8, 4), ("p3d_30", "hybrid", 32, 8),
                                          ("spd_200", "parallel", 5, 1), ("s27_15", "classical", 12, 12),
                                          ("p3d_17", "classical", 64, 64)])
def test_retooled_converged_counts(torch_dev, name, sub, k, p):
    from paper_1912_11930_gb300 import bcg
    M = mat(name)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=3)
    tol = 1e-8
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=3000)
    assert r.status == bcg.OK, r
    ref = O.solve_retooled(A, B, p=p, sub=sub, tol=tol, maxit=3000)
    assert ref.status == O.OK
    assert abs(r.iters - ref.iters) <= 2, (r.iters, ref.iters)
    assert np.all(np.abs(np.array(r.block_iters) - ref.block_iters) <= 2)
    res = np.linalg.norm(B - A @ Xg, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5 * tol)
    # Algorithm 1 on the GPU: the same counts (one method in exact arithmetic)
    _, r1 = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=3000, retooled=0)
    assert abs(r.iters - r1.iters) <= 2


@pytest.mark.parametrize("k,p,sub", [(4, 4, "classical"), (16, 8, "hybrid"), (64, 64, "classical")])
def test_retooled_badly_scaled_columns(torch_dev, k, p, sub):
    """Columns of B scaled from 1e-6 to 1e6 within every block: Algorithm 1's rho = R^T R spans 24 orders and
    its factorisation fails in iteration 1; the retooled form converges in the iterations of the unscaled
    right-hand side, to X(B) D."""
    from paper_1912_11930_gb300 import bcg
    M = mat("p3d_17") if p > 32 else mat("p2d_37x29")
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=5)
    d = np.tile(10.0 ** np.linspace(-6, 6, p), k // p)
    Bs = B * d[None, :]
    tol = 1e-8
    _, r1 = gpu_solve(torch_dev, M, Bs, k=k, p=p, sub=sub, tol=tol, maxit=2000, retooled=0)
    assert r1.status == bcg.BREAKDOWN and r1.breakdown_iter == 1
    Xs, rs = gpu_solve(torch_dev, M, Bs, k=k, p=p, sub=sub, tol=tol, maxit=2000)
    Xu, ru = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=2000)
    assert rs.status == bcg.OK and ru.status == bcg.OK
    assert abs(rs.iters - ru.iters) <= 2
    res = np.linalg.norm(Bs - A @ Xs, axis=0) / np.linalg.norm(Bs, axis=0)
    assert np.all(res <= 1.5 * tol)
    ref = O.solve_retooled(A, Bs, p=p, sub=sub, tol=tol, maxit=2000)
    assert ref.status == O.OK and abs(ref.iters - rs.iters) <= 2
    assert_close(Xs / d[None, :], Xu, 1e-5)   # both within cond(A) tol of A^{-1} B


def test_retooled_degenerate_cases_and_arguments(torch_dev):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = mat("p2d_37x29")
    B = W.rhs(M.n, 8, seed=3)
    # a zero block stops at iteration 0 and its X stays; the other block solves as if alone
    Bz = B.copy()
    Bz[:, 4:] = 0.0
    X, r = gpu_solve(torch_dev, M, Bz, k=8, p=4, sub="hybrid", tol=1e-10, maxit=500)
    assert r.status == bcg.OK and r.block_iters[1] == 0 and np.all(X[:, 4:] == 0.0)
    ref = O.solve_retooled(M.to_scipy(), Bz, p=4, sub="hybrid", tol=1e-10, maxit=500)
    assert abs(r.iters - ref.iters) <= 2
    assert_close(X, ref.X, 1e-8)
    # an all-zero right-hand side: nothing to do
    X, r = gpu_solve(torch_dev, M, np.zeros_like(B), k=8, p=4, sub="hybrid", tol=1e-10, maxit=5)
    assert r.status == bcg.OK and r.iters == 0 and np.all(X == 0.0)
    # duplicated columns and a zero column next to live ones: the first Cholesky QR fails in iteration 1
    for Bd in (np.hstack([B[:, :2], B[:, :2]]), np.hstack([B[:, :3], np.zeros((M.n, 1))])):
        X, r = gpu_solve(torch_dev, M, Bd, k=4, p=4, sub="classical", tol=1e-10, maxit=50)
        assert r.status == bcg.BREAKDOWN and r.breakdown_iter == 1 and r.iters == 0
    # argument checks: FP64 handles only
    S = bcg.Solver.from_matrix(M, k=8, p=4, sub="hybrid", prec="fp32_refine", device=dev)
    with pytest.raises(bcg.BCGError, match="retooled"):
        S.set_option("retooled", 1)
    S.close()
    # switching back to Algorithm 1 on the same handle
    S = bcg.Solver.from_matrix(M, k=8, p=4, sub="hybrid", prec="fp64", device=dev)
    S.set_option("retooled", 0)
    X1, r1 = S.solve(torch.from_numpy(B).to(dev), tol=1e-8, maxit=500)
    S.set_option("retooled", 1)
    X2, r2 = S.solve(torch.from_numpy(B).to(dev), tol=1e-8, maxit=500)
    S.close()
    assert r1.ok and r2.ok and abs(r1.iters - r2.iters) <= 2
    assert_close(X2.cpu().numpy(), X1.cpu().numpy(), 1e-7)


def test_retooled_full_size_against_oracle(torch_dev):
    """The retooled bench workload (128^3 Poisson, k = 32, hybrid p = 8, FP64): four iterations on the GPU
    against four iterations of the oracle's retooled form on the whole matrix, 1e-9."""
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = W.poisson3d(128)
    k, p, m = 32, 8, 4
    B = W.rhs(M.n, k, seed=0)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec="fp64", device=dev)
    S.set_option("retooled", 1)
    X, r = S.solve(torch.from_numpy(B).to(dev), tol=NEVER, maxit=m)
    S.close()
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    ref = O.solve_retooled(M.to_scipy(), B, p=p, sub="hybrid", tol=0.0, maxit=m)
    assert_close(X.cpu().numpy(), ref.X, 1e-9)


# ---- the global subalgebra and the Jacobi preconditioner ----
# (matrix, form, sub, k, p, iterations, Jacobi): the streaming kernels (p <= 32; global with one shared factor
# for all column blocks, Jacobi with the second Gram <<T, M^{-1} T>>) and the tiled large-block path
GJ_FIXED = [
    ("p2d_37x29", "csr", "global", 8, 4, 25, 0), ("p3d_30", "csr", "global", 32, 8, 20, 0),
    ("p3d_30", "stencil", "global", 12, 4, 20, 0), ("p3d_30", "csr", "global", 6, 3, 20, 0),
    ("vc_20", "csr", "hybrid", 16, 4, 8, 1), ("vc_20", "stencil", "hybrid", 32, 8, 8, 1),
    ("vc_20", "csr", "global", 16, 4, 8, 1), ("vc_20", "csr", "parallel", 8, 1, 10, 1),
    ("vc_20", "csr", "classical", 16, 16, 8, 1), ("s27_15", "csr", "hybrid", 32, 32, 8, 1),
    ("p3d_17", "csr", "global", 128, 64, 4, 0), ("p3d_17", "csr", "hybrid", 64, 64, 5, 1),
    ("p3d_17", "csr", "global", 128, 64, 4, 1),
]


@pytest.mark.parametrize("name,form,sub,k,p,m,jac", GJ_FIXED)
def test_retooled_global_and_jacobi_equal_iterations(torch_dev, name, form, sub, k, p, m, jac):
    M = mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, form=form, maxit=m, X0=X0, precond=jac)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m, r
    ref = O.solve_retooled(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m,
                           precond="jacobi" if jac else "none")
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("name,sub,k,p,jac", [("p3d_30", "global", 32, 8, 0), ("vc_20", "hybrid", 16, 4, 1),
                                             ("vc_20", "global", 16, 8, 1), ("p3d_17", "global", 128, 64, 1)])
def test_retooled_global_and_jacobi_converge(torch_dev, name, sub, k, p, jac):
    """Converged counts within the oracle's spread (+2) of the oracle's retooled form with the same
    preconditioner, and the true residual at the tolerance."""
    M = mat(name)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=3)
    tol = 1e-8
    pre = "jacobi" if jac else "none"
    X, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=3000, precond=jac)
    assert r.ok, r
    ref = O.solve_retooled(A, B, p=p, sub=sub, tol=tol, maxit=3000, precond=pre)
    spread = [O.solve_retooled(A, B * (1 + 1e-16 * np.random.default_rng(s).standard_normal(B.shape)), p=p,
                               sub=sub, tol=tol, maxit=3000, precond=pre).iters for s in range(2)]
    allow = 2 + max(spread + [ref.iters]) - min(spread + [ref.iters])
    assert abs(r.iters - ref.iters) <= allow, (r.iters, ref.iters, spread)
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5 * tol), res


def test_retooled_global_shared_column_scaling(torch_dev):
    """Global subalgebra, columns scaled 1e-8 .. 1e8 by one diagonal shared by the column blocks: the retooled
    form converges like the unscaled system (X scales with B), where Algorithm 1 breaks down."""
    M = mat("p3d_30")
    k, p = 16, 4
    B = W.rhs(M.n, k, seed=12)
    d = np.tile(10.0 ** np.linspace(-8, 8, p), k // p)
    X1, r1 = gpu_solve(torch_dev, M, B, k=k, p=p, sub="global", tol=1e-8, maxit=2000)
    X2, r2 = gpu_solve(torch_dev, M, B * d, k=k, p=p, sub="global", tol=1e-8, maxit=2000)
    assert r1.ok and r2.ok and abs(r1.iters - r2.iters) <= 1, (r1, r2)
    assert_close(X2 / d, X1, 1e-7)
    _, ra = gpu_solve(torch_dev, M, B * d, k=k, p=p, sub="global", tol=1e-8, maxit=2000, retooled=0)
    assert ra.status == bcg.BREAKDOWN
