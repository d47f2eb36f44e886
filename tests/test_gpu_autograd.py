"""Differentiable solve (adjoint with the same handle) on the GPU: against a dense FP64 gradient, against
central finite differences of the loss, and on the full 100^3 27-point workload through properties that
hold at any size (forward and adjoint residuals, sampled gradient entries recomputed on the host)."""
import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import workloads as W
from parity_check import assert_close

pytestmark = pytest.mark.gpu


def _setup(M, k, seed, dev, tol=1e-13):
    import torch
    from paper_1912_11930_gb300 import bcg
    vals = torch.from_numpy(M.vals.copy()).to(dev).requires_grad_(True)
    csr = (torch.from_numpy(M.rowptr).to(dev), torch.from_numpy(M.colind).to(dev), vals)
    S = bcg.Solver(k=k, p=k, sub="hybrid", csr=csr, device=dev)
    B = torch.from_numpy(W.rhs(M.n, k, seed=seed)).to(dev).requires_grad_(True)
    Wt = torch.from_numpy(W.loss_weights(M.n, k, seed=seed)).to(dev)
    return S, vals, B, Wt


def test_gradient_dense_and_finite_differences(lib):
    import torch
    from paper_1912_11930_gb300.autograd import bcg_solve_autograd
    dev = torch.device("cuda:0")
    M = W.stencil27(6, seed=3)
    k = 4
    S, vals, B, Wt = _setup(M, k, 5, dev)
    X = bcg_solve_autograd(vals, B, S, tol=1e-13)
    loss = (Wt * X).sum()
    loss.backward()
    Ad = M.to_scipy().toarray()
    Bn, Wn = B.detach().cpu().numpy(), Wt.cpu().numpy()
    Xd = np.linalg.solve(Ad, Bn)
    Lam = np.linalg.solve(Ad, Wn)
    rows = np.repeat(np.arange(M.n), np.diff(M.rowptr))
    g_dense = -np.sum(Lam[rows] * Xd[M.colind], axis=1)
    gv = vals.grad.cpu().numpy()
    assert np.linalg.norm(gv - g_dense) <= 1e-8 * np.linalg.norm(g_dense)
    assert np.linalg.norm(B.grad.cpu().numpy() - Lam) <= 1e-8 * np.linalg.norm(Lam)
    # the oracle's forward solve, adjoint solve and gradient formula, element by element
    fwd, adj, g_or = O.solve_and_grad(M.to_scipy(), M.rowptr, M.colind, Bn, Wn, p=k, sub="hybrid", tol=1e-13)
    assert fwd.status == O.OK and adj.status == O.OK
    assert_close(X.detach().cpu().numpy(), fwd.X, 1e-9, "X")
    assert_close(B.grad.cpu().numpy(), adj.X, 1e-9, "dL/dB")
    assert_close(gv, g_or, 1e-9, "dL/dvals")
    # central differences of the loss through the GPU solver itself, symmetric pairs perturbed together
    pos = {(int(rows[e]), int(M.colind[e])): e for e in range(M.nnz)}
    rng = np.random.default_rng(1)
    with torch.no_grad():
        for e in rng.choice(M.nnz, 10, replace=False):
            i, j = int(rows[e]), int(M.colind[e])
            pair = [e] if i == j else [e, pos[(j, i)]]
            h = 1e-5 * abs(M.vals[e])
            f = []
            for sgn in (1.0, -1.0):
                for ee in pair:
                    vals[ee] += sgn * h
                Xp, r = S.solve(B.detach().contiguous(), tol=1e-13)
                assert r.ok
                f.append(float((Wt * Xp).sum()))
                for ee in pair:
                    vals[ee] -= sgn * h
            fd = (f[0] - f[1]) / (2 * h)
            an = float(sum(gv[ee] for ee in pair))
            assert abs(fd - an) <= 1e-6 * abs(an), (i, j, fd, an)
    S.close()


def test_full_size_27pt_100_k16(lib):
    """100^3 27-point SPD matrix, k = 16, FP64: forward and adjoint solves converge (residuals recomputed on
    the host), dL/dB is the adjoint solution, and sampled dL/dvals entries equal -Lambda_i . X_j."""
    import torch
    from paper_1912_11930_gb300.autograd import bcg_solve_autograd
    dev = torch.device("cuda:0")
    M = W.stencil27(100, seed=0)
    k, tol = 16, 1e-10
    S, vals, B, Wt = _setup(M, k, 0, dev)
    X = bcg_solve_autograd(vals, B, S, tol=tol)
    (Wt * X).sum().backward()
    A = M.to_scipy()
    Xn, Bn, Wn = X.detach().cpu().numpy(), B.detach().cpu().numpy(), Wt.cpu().numpy()
    Lam = B.grad.cpu().numpy()
    res_f = np.linalg.norm(Bn - A @ Xn, axis=0) / np.linalg.norm(Bn, axis=0)
    res_a = np.linalg.norm(Wn - A @ Lam, axis=0) / np.linalg.norm(Wn, axis=0)
    assert np.all(res_f <= 1.5 * tol) and np.all(res_a <= 1.5 * tol)
    gv = vals.grad.cpu().numpy()
    rng = np.random.default_rng(2)
    rows = np.repeat(np.arange(M.n), np.diff(M.rowptr))
    for e in rng.choice(M.nnz, 500, replace=False):
        ref = -float(np.dot(Lam[rows[e]], Xn[M.colind[e]]))
        assert abs(gv[e] - ref) <= 1e-12 * max(1.0, abs(ref))
    # independent of the gradient formula: the directional derivative of the loss along a random symmetric
    # perturbation D of the stored values (D_ij = D_ji, so A stays symmetric), by central differences through
    # two further solves, against sum_e grad_e D_e
    key = rows.astype(np.int64) * M.n + M.colind   # entry (i, j) -> i n + j; its transpose is j n + i
    srt = np.argsort(key)
    swap = srt[np.searchsorted(key[srt], M.colind.astype(np.int64) * M.n + rows)]   # index of the transposed entry
    assert np.array_equal(key[swap], M.colind.astype(np.int64) * M.n + rows)
    tri = rng.standard_normal(M.nnz)
    D = 1e-7 * np.abs(M.vals) * (tri + tri[swap]) / 2.0
    f = []
    with torch.no_grad():
        base = vals.detach().clone()
        for sgn in (1.0, -1.0):
            vals.copy_(base + sgn * torch.from_numpy(D).to(dev))
            Xp, r = S.solve(B.detach().contiguous(), tol=1e-12)
            assert r.ok
            f.append(float((Wt * Xp).sum()))
        vals.copy_(base)
    fd = (f[0] - f[1]) / 2.0
    an = float(np.dot(gv, D))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    S.close()
