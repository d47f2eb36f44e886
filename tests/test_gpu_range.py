"""Range of the GPU path: right-hand sides and matrices scaled far outside FP32's exponent range.

The block products of the method are defined on FP64 values (Section 2's S-products, Algorithm 1), and the
oracle computes them in FP64. The GPU accumulates them as float pairs (Dot2) after an exact power-of-two
shift per column, and the mixed form runs its FP32 process on an exactly scaled residual. These cases check
that neither narrows the range: B scaled by 1e-30 ... 1e30 and A by 1e-10 ... 1e10, for Algorithm 1 (every
subalgebra, CSR, stencil and large-block paths, Jacobi), the mixed form (both strategies) and the retooled
form, against the oracle on the same scaled system; and the BDOT entry point on entries spanning 1e-300 ...
1e300 with exact zeros.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import bcg, workloads as W
from parity_check import assert_close

pytestmark = pytest.mark.gpu

NEVER = 1e-300
SCALES = [(1e-30, 1.0), (1e-20, 1.0), (1e20, 1.0), (1e30, 1.0), (1.0, 1e-10), (1.0, 1e10), (1e-30, 1e10),
          (1e30, 1e-10)]


@pytest.fixture(scope="module")
def torch_dev(lib):
    import torch
    return torch, torch.device("cuda:0")


_BASE = {}


def base(name):
    if name not in _BASE:
        _BASE[name] = {
            "p3d_14": lambda: W.poisson3d(14, 13, 12),
            "vc_12": lambda: W.varcoef3d(12, 11, 13, seed=7),
            "p2d_37x29": lambda: W.poisson2d(37, 29),
        }[name]()
    return _BASE[name]


def scaled(M, sa):
    """sa A (CSR values and, for the matrix-free form, the stencil's scale factor)."""
    st = None if M.stencil is None else dict(M.stencil, scale=M.stencil["scale"] * sa)
    return replace(M, vals=M.vals * sa, stencil=st)


def gpu_solve(torch_dev, M, B, *, k, p, sub, prec="fp64", form="csr", tol=NEVER, maxit=20, opts=None):
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, form=form, device=dev)
    for key, v in (opts or {}).items():
        S.set_option(key, v)
    X, r = S.solve(torch.from_numpy(np.ascontiguousarray(B)).to(dev), tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    out = X.cpu().numpy()
    S.close()
    return out, r


# (sub, k, p, operator form): the streaming kernels (per-element and warp-chunk layouts), the matrix-free
# stencil and the tiled large-block path
ALG1 = [("hybrid", 8, 4, "csr"), ("global", 8, 4, "csr"), ("parallel", 8, 1, "csr"), ("hybrid", 32, 8, "csr"),
        ("hybrid", 6, 3, "csr"), ("hybrid", 8, 4, "stencil"), ("classical", 64, 64, "csr"), ("hybrid", 64, 32, "csr"),
        ("classical", 32, 32, "csr")]


@pytest.mark.parametrize("sb,sa", SCALES)
@pytest.mark.parametrize("sub,k,p,form", ALG1)
def test_fp64_scaled_equal_iterations(torch_dev, sub, k, p, form, sb, sa):
    """Algorithm 1 on sa A X = sb B: the same iterates as the oracle's (X^m at equal iteration counts)."""
    M = scaled(base("p3d_14"), sa)
    B = sb * W.rhs(M.n, k, seed=11)
    m = 12 if p == 64 else 20
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, form=form, maxit=m)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m, r   # NOT_CONVERGED after exactly m iterations: no breakdown, no NaN
    ref = O.solve(M.to_scipy(), B, p=p, sub=sub, tol=0.0, maxit=m)
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("sb,sa", [(1e-30, 1.0), (1e30, 1.0), (1e-20, 1e10), (1e20, 1e-10)])
@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 8, 4)])
def test_fp64_scaled_converges_like_the_oracle(torch_dev, sub, k, p, sb, sa):
    """To tol 1e-8: OK status, converged counts within +-2 of the oracle's, the true residual at the tolerance."""
    M = scaled(base("p3d_14"), sa)
    A = M.to_scipy()
    B = sb * W.rhs(M.n, k, seed=12)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, tol=1e-8, maxit=2000)
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub=sub, tol=1e-8, maxit=2000)
    assert ref.status == O.OK
    assert abs(r.iters - ref.iters) <= 2, (r.iters, ref.iters)
    res = np.linalg.norm(B - A @ Xg, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8), res


@pytest.mark.parametrize("sb,sa", [(1e-30, 1e10), (1e30, 1e-10), (1e20, 1e10)])
@pytest.mark.parametrize("name,sub,k,p", [("vc_12", "hybrid", 8, 4), ("p3d_14", "classical", 64, 64)])
def test_jacobi_scaled_equal_iterations(torch_dev, name, sub, k, p, sb, sa):
    """M = diag(A): the directions M^{-1} R and the products A P carry their own exponent offsets."""
    M = scaled(base(name), sa)
    B = sb * W.rhs(M.n, k, seed=13)
    m = 8 if name == "vc_12" else 10
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, maxit=m, opts={"precond": 1})
    assert r.status == bcg.NOT_CONVERGED and r.iters == m, r
    ref = O.solve(M.to_scipy(), B, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi")
    assert_close(Xg, ref.X, 1e-9)


@pytest.mark.parametrize("refine", [1, 0])
@pytest.mark.parametrize("sb,sa", [(1e-30, 1.0), (1e30, 1.0), (1e-20, 1e10), (1e20, 1e-10)])
@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 8, 4), ("parallel", 8, 1)])
def test_mixed_scaled_reaches_fp64_accuracy(torch_dev, sub, k, p, sb, sa, refine):
    """The mixed form (FP32 process on R 2^-sigma, FP64 residuals) to 1e-10: within 1e-8 of the FP64 oracle's
    tight solution, element by element, with the true residual at the tolerance."""
    M = scaled(base("p3d_14"), sa)
    A = M.to_scipy()
    B = sb * W.rhs(M.n, k, seed=14)
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, prec="fp32_refine", tol=1e-10, maxit=5000,
                      opts={"refine": refine})
    assert r.ok, r
    res = np.linalg.norm(B - A @ Xg, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-10), res
    ref = O.solve(A, B, p=p, sub=sub, tol=1e-13, maxit=5000)
    assert ref.status == O.OK
    assert_close(Xg, ref.X, 1e-8)


@pytest.mark.parametrize("sb,sa", [(1e-30, 1.0), (1e30, 1.0), (1e-20, 1e10), (1e20, 1e-10)])
@pytest.mark.parametrize("sub,k,p,jac", [("hybrid", 8, 4, 0), ("hybrid", 64, 64, 0), ("global", 16, 4, 0),
                                         ("hybrid", 8, 4, 1), ("global", 128, 64, 1)])
def test_retooled_scaled_equal_iterations(torch_dev, sub, k, p, jac, sb, sa):
    """Dubrulle's form: gamma^0 = <<M^{-1} R^0, R^0>> at the residual's scale, W = A S at the operator's."""
    M = scaled(base("p3d_14"), sa)
    B = sb * W.rhs(M.n, k, seed=15)
    m = 10 if p == 64 else 20
    Xg, r = gpu_solve(torch_dev, M, B, k=k, p=p, sub=sub, maxit=m, opts={"retooled": 1, "precond": jac})
    assert r.status == bcg.NOT_CONVERGED and r.iters == m, r
    ref = O.solve_retooled(M.to_scipy(), B, p=p, sub=sub, tol=0.0, maxit=m, precond="jacobi" if jac else "none")
    assert_close(Xg, ref.X, 1e-9)


def _wide(n, k, lo, hi, seed, spread=20.0, zeros=0.1):
    """N(0,1) entries times 10^(column exponent in [lo, hi]) times 10^U(-spread, spread) per entry, a fraction
    of exact zeros, and one all-zero column."""
    rng = np.random.default_rng(seed)
    col = rng.uniform(lo, hi, k)
    X = rng.standard_normal((n, k)) * 10.0 ** (col[None, :] + rng.uniform(-spread, spread, (n, k)))
    X[rng.random((n, k)) < zeros] = 0.0
    X[:, k // 2] = 0.0
    return X


@pytest.mark.parametrize("sub,k,p", [("hybrid", 8, 4), ("global", 32, 8), ("parallel", 16, 1),
                                     ("classical", 32, 32), ("classical", 64, 64)])
def test_bdot_wide_range(torch_dev, sub, k, p):
    """Entries from 1e-300 to 1e300 (X's columns at 10^-280 ... 10^280, Y's of moderate size) and products
    that are all finite: every entry of <<X, Y>>_S within 1e-13 of sum_r |x_ra y_rb| of the oracle's; then the
    reverse spread (Y wide, X moderate) and both wide with opposite column exponents."""
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = base("p2d_37x29")
    kind, pp = O.canonical_subalgebra(sub, k, p)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, device=dev)
    wide = _wide(M.n, k, -280, 275, seed=51)            # entries 1e-300 ... 1e295
    mid = _wide(M.n, k, -1, 1, seed=52, spread=2.0, zeros=0.0)
    rng = np.random.default_rng(53)
    e = rng.uniform(-100, 100, k)
    both_x = _wide(M.n, k, 0, 0, seed=54) * 10.0 ** e[None, :]
    both_y = _wide(M.n, k, 0, 0, seed=55) * 10.0 ** (-e[None, :] + rng.uniform(-30, 30, k)[None, :])
    for X, Y in ((wide, mid), (mid, wide), (both_x, both_y)):
        assert np.all(np.isfinite(np.abs(X).T @ np.abs(Y)))   # every product and sum is an FP64 number
        g = S.bdot(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)).cpu().numpy()
        ref = O.block_product(X, Y, pp, kind)
        absdot = O.block_product(np.abs(X), np.abs(Y), pp, kind)
        assert np.all(np.isfinite(g))
        err = np.abs(g - ref)
        assert np.all(err <= 1e-13 * absdot), float(np.max(err / np.where(absdot > 0, absdot, 1.0)))
    S.close()


def test_bdot_noalloc_wide_range(torch_dev):
    """The allocation-free BDOT takes its shifts from the same column maxima."""
    torch, dev = torch_dev
    from paper_1912_11930_gb300 import bcg
    M = base("p2d_37x29")
    k, p = 16, 8
    X = _wide(M.n, k, -280, 275, seed=61)
    Y = _wide(M.n, k, -1, 1, seed=62, spread=2.0, zeros=0.0)
    got = torch.full((k // p, p, p), float("nan"), dtype=torch.float64, device=dev)
    bcg.bcg_bdot_noalloc(M.n, k, p, "hybrid", torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev), got)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    ref = O.block_product(X, Y, p, "hybrid")
    absdot = O.block_product(np.abs(X), np.abs(Y), p, "hybrid")
    assert np.all(np.abs(g - ref) <= 1e-13 * absdot)
