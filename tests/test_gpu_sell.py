"""GPU parity of SELL-C-sigma handles (bcg_create_sell): the solve iterates on the permuted system, so its
iterate, mapped back to the original row order, must match the CPU oracle on the original CSR matrix at the
bars of the CSR handles (1e-9 at equal iterations in FP64, 1e-8 after refinement)."""
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


def sell_solve(torch_dev, M, B, *, k, p, sub, sigma, prec="fp64", tol=NEVER, maxit=30, X0=None, precond=0):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, form="sell", sigma=sigma, device=dev)
    if precond:
        S.set_option("precond", precond)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Xt = None if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).to(dev)
    X, r = S.solve(Bt, Xt, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    S.close()
    return X.cpu().numpy(), r


FIXED = [  # (matrix, sub, k, p, sigma, iterations): per-element (k = 1, 6) and warp-chunk (k = 8, 32) layouts,
           # large blocks (p = 64), rows sorted across chunks (sigma > 32)
    ("p3d_30", "parallel", 1, 1, 1, 40), ("p3d_30", "hybrid", 6, 3, 256, 25), ("p3d_30", "hybrid", 8, 4, 1, 30),
    ("p3d_30", "hybrid", 32, 8, 1024, 25), ("s27_15", "hybrid", 24, 12, 64, 15), ("s27_15", "global", 32, 8, 1, 15),
    ("vc_20", "hybrid", 16, 16, 4096, 10), ("spd_200", "hybrid", 16, 4, 8, 12), ("p3d_30", "classical", 64, 64, 512, 5),
]


@pytest.mark.parametrize("name,sub,k,p,sigma,m", FIXED)
def test_sell_fp64_equal_iterations(torch_dev, name, sub, k, p, sigma, m):
    M = mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    X, r = sell_solve(torch_dev, M, B, k=k, p=p, sub=sub, sigma=sigma, maxit=m, X0=X0)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert_close(X, ref.X, 1e-9)


def test_sell_bop_and_host_entry(torch_dev):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = mat("s27_15")
    k = 8
    X = W.rhs(M.n, k, seed=9)
    S = bcg.Solver.from_matrix(M, k=k, p=4, sub="hybrid", form="sell", sigma=256, device=dev)
    Y = S.bop(torch.from_numpy(X).to(dev)).cpu().numpy()
    assert_close(Y, M.to_scipy() @ X, 1e-14)
    B = W.rhs(M.n, k, seed=10)
    Xd, rd = S.solve(torch.from_numpy(B).to(dev), tol=1e-8)
    Xh, rh = S.solve_host(B, np.zeros_like(B), tol=1e-8)
    assert rd.ok and rh.iters == rd.iters and np.array_equal(Xh, Xd.cpu().numpy())
    S.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_sell_converged_and_mixed(torch_dev, precond):
    M = mat("vc_20")
    A = M.to_scipy()
    k, p = 16, 4
    B = W.rhs(M.n, k, seed=3)
    pre = "jacobi" if precond else "none"
    X, r = sell_solve(torch_dev, M, B, k=k, p=p, sub="hybrid", sigma=128, tol=1e-8, maxit=3000, precond=precond)
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub="hybrid", tol=1e-8, maxit=3000, precond=pre)
    spread = [O.solve(A, B * (1 + 1e-16 * np.random.default_rng(s).standard_normal(B.shape)), p=p, sub="hybrid",
                      tol=1e-8, maxit=3000, precond=pre).iters for s in range(2)]
    allow = 2 + max(spread + [ref.iters]) - min(spread + [ref.iters])
    assert abs(r.iters - ref.iters) <= allow, (r.iters, ref.iters, spread)
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8)
    Xm, rm = sell_solve(torch_dev, M, B, k=k, p=p, sub="hybrid", sigma=128, prec="fp32_refine", tol=1e-12,
                        maxit=5000, precond=precond)
    assert rm.ok
    ref12 = O.solve(A, B, p=p, sub="hybrid", tol=1e-13, maxit=5000, precond=pre)
    assert_close(Xm, ref12.X, 1e-8)


def test_sell_update_values(torch_dev):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg, formats as F
    M = mat("p3d_30")
    Sm = F.sell_from_csr(M.rowptr, M.colind, M.vals, 64)
    sell = tuple(torch.from_numpy(a).to(dev) for a in (Sm.chunkptr, Sm.rowlen, Sm.colind, Sm.vals, Sm.perm))
    S = bcg.Solver(k=8, p=4, sub="hybrid", sell=sell, device=dev)
    S.update_values(torch.from_numpy(3.0 * Sm.vals).to(dev))
    B = W.rhs(M.n, 8, seed=12)
    X, r = S.solve(torch.from_numpy(B).to(dev), tol=NEVER, maxit=12)
    S.close()
    ref = O.solve(3.0 * M.to_scipy(), B, p=4, sub="hybrid", tol=0.0, maxit=12)
    assert_close(X.cpu().numpy(), ref.X, 1e-9)
