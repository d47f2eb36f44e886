"""GPU parity of the double-float block updates (precision "fp64_df") against the CPU oracle.

The form differs from BCG_FP64 only in how the residual update R -= Q lambda sums its p products: in float
pairs from 48-bit splits (about 2^-46 of sum_a |q_a l_ab| per update against p 2^-53 of it with FP64 FMAs),
turned into one double with integer operations and added to R with one FP64 addition; X += P lambda and
P = Z + P beta keep their FP64 FMAs. The bars are the FP64 form's:
relative solution error <= 1e-9 against the oracle at equal iteration counts (Frobenius and element by
element), converged counts within +-2, the true residual at the tolerance; and, at 128^3, k = 32, p = 8 (the
bench workload), four iterations against the oracle on the whole matrix and a converged solve whose count
equals the FP64 form's within 2.
"""
import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import bcg, workloads as W
from parity_check import assert_close

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
            "vc_20": lambda: W.varcoef3d(20, 17, 23, seed=4),
            "s27_15": lambda: W.stencil27(15, 14, 13, seed=5),
        }[name]()
    return _MATS[name]


def gpu_solve(torch_dev, M, B, *, k, p, sub, prec="fp64_df", form="csr", tol=NEVER, maxit=30, X0=None,
              opts=None):
    torch, dev = torch_dev
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, form=form, device=dev)
    for key, v in (opts or {}).items():
        S.set_option(key, v)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Xt = None if X0 is None else torch.from_numpy(np.ascontiguousarray(X0)).to(dev)
    X, r = S.solve(Bt, Xt, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    out = X.cpu().numpy()
    S.close()
    return out, r


# (matrix, sub, k, p, iterations, Jacobi): every double-float width PM = 2..16 (and p = 32, which keeps the FP64
# updates), blocks inside and across
# warps, k below and above 32, the recomputed rho formed in K3 (p <= 16) or in K1 (p = 32)
FIXED = [
    ("p2d_37x29", "hybrid", 8, 4, 30, 0), ("p2d_37x29", "global", 8, 4, 30, 0), ("p2d_37x29", "classical", 8, 8, 20, 0),
    ("p3d_30", "hybrid", 32, 8, 25, 0), ("p3d_30", "hybrid", 32, 2, 25, 0), ("p3d_30", "hybrid", 16, 16, 20, 0),
    ("p3d_30", "global", 32, 16, 15, 0), ("p3d_30", "hybrid", 64, 16, 15, 0), ("p3d_30", "hybrid", 4, 2, 30, 0),
    ("s27_15", "hybrid", 32, 16, 15, 0), ("vc_20", "hybrid", 16, 4, 10, 0), ("vc_20", "hybrid", 32, 8, 8, 1),
    ("p3d_30", "global", 32, 8, 20, 1),
]


@pytest.mark.parametrize("name,sub,k,p,m,jac", FIXED)
def test_df_equal_iterations(torch_dev, name, sub, k, p, m, jac):
    M = mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, maxit=m, X0=X0, opts={"precond": jac})
    assert r.status == bcg.NOT_CONVERGED and r.iters == m, r
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi" if jac else "none")
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("name,sub,k,p", [("p2d_37x29", "hybrid", 8, 4), ("p3d_30", "hybrid", 32, 8),
                                          ("p3d_30", "global", 32, 32), ("s27_15", "hybrid", 16, 16)])
def test_df_converged_counts_and_frozen_blocks(torch_dev, name, sub, k, p):
    """Hybrid blocks freeze at their own iterations: counts within +-2 of the oracle's, per block too, each
    block's X against the oracle at its own count, and the true residual at the tolerance."""
    M = mat(name)
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=3)
    tol = 1e-8
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=tol, maxit=3000)
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub=sub, tol=tol, maxit=3000)
    assert ref.status == O.OK
    assert abs(r.iters - ref.iters) <= 2, (r.iters, ref.iters)
    assert np.all(np.abs(np.array(r.block_iters) - ref.block_iters) <= 2), (r.block_iters, ref.block_iters)
    res = np.linalg.norm(B - A @ Xg, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5 * tol), res
    kind, pp = O.canonical_subalgebra(sub, k, p)
    if kind == "hybrid":
        for j, it in enumerate(r.block_iters):
            blk = slice(j * pp, (j + 1) * pp)
            assert_close(Xg[:, blk], O.solve(A, B[:, blk], p=pp, sub="hybrid", tol=0.0, maxit=int(it)).X, 1e-9,
                         f"block {j}")
    else:
        assert_close(Xg, O.solve(A, B, p=p, sub=sub, tol=0.0, maxit=r.iters).X, 1e-9)


@pytest.mark.parametrize("sb,sa", [(1e-30, 1.0), (1e30, 1.0), (1e-20, 1e10), (1e20, 1e-10)])
@pytest.mark.parametrize("sub,k,p", [("hybrid", 32, 8), ("global", 8, 4)])
def test_df_scaled(torch_dev, sub, k, p, sb, sa):
    """The float pairs of the updates are shifted into FP32's range like the Gram operands."""
    from dataclasses import replace
    base = mat("p3d_30")
    M = replace(base, vals=base.vals * sa)
    B = sb * W.rhs(M.n, k, seed=4)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, maxit=20)
    assert r.status == bcg.NOT_CONVERGED and r.iters == 20, r
    ref = O.solve(M.to_scipy(), B, p=p, sub=sub, tol=0.0, maxit=20)
    assert_close(Xg, ref.X, 1e-9)


def test_df_shapes_without_the_layout_run_fp64_updates(torch_dev):
    """k = 6 (no warp-chunk layout) and p = 1 run the FP64 updates: bitwise the FP64 handle's result."""
    M = mat("p3d_30")
    for k, p, sub in ((6, 3, "hybrid"), (8, 1, "parallel")):
        B = W.rhs(M.n, k, seed=5)
        a, _ = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, prec="fp64_df", maxit=15)
        b, _ = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, prec="fp64", maxit=15)
        assert np.array_equal(a, b)


def test_df_full_size_poisson128(torch_dev):
    """128^3 Poisson, k = 32, hybrid p = 8 (the bench workload): four iterations against four oracle iterations on
    the whole matrix (1e-9), then a converged solve whose count equals the FP64 form's within 2, with the true
    residual recomputed on the host."""
    torch, dev = torch_dev
    M = W.poisson3d(128)
    k, p, m = 32, 8, 4
    B = W.rhs(M.n, k, seed=0)
    Bt = torch.from_numpy(B).to(dev)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec="fp64_df", device=dev)
    X, r = S.solve(Bt, tol=NEVER, maxit=m)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    A = M.to_scipy()
    ref = O.solve(A, B, p=p, sub="hybrid", tol=0.0, maxit=m)
    assert_close(X.cpu().numpy(), ref.X, 1e-9)
    X, r = S.solve(Bt, tol=1e-8, maxit=5000)
    S.close()
    assert r.ok, r
    S64 = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec="fp64", device=dev)
    X64, r64 = S64.solve(Bt, tol=1e-8, maxit=5000)
    S64.close()
    assert abs(r.iters - r64.iters) <= 2, (r.iters, r64.iters)
    Xh = X.cpu().numpy()
    res = np.linalg.norm(B - A @ Xh, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8), res
