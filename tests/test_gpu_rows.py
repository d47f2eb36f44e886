"""Row-sharded solves on the GPU: the rows of one problem split over `world` ranks, each rank a handle
(bcg_create_csr_rows) driven through the phase calls, the ranks emulated as threads on one GPU whose
exchanges (sums over ranks, halo rows of P) are host-ordered copies -- no kernel waits on another. The
gathered iterate must match the CPU oracle on the whole matrix at the same bars as the one-rank solve."""
import threading

import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import bcg, workloads as W
from parity_check import assert_close, rel_fro as _rel

pytestmark = pytest.mark.gpu

NEVER = 1e-300


def sharded_solve(lib, M, B, *, world, k, p, sub, tol=NEVER, maxit=30, X0=None, precond=0):
    import torch
    from paper_1912_11930_gb300 import dist as D
    dev = torch.device("cuda:0")
    plans = D.make_plans(M, world)
    comms = D.ThreadComm.group(world)
    out, errs = [None] * world, []

    def rank(q):
        try:
            pl = plans[q]
            r0, r1 = pl.bounds[q], pl.bounds[q + 1]
            S = D.RowShardedSolver(pl, k=k, p=p, sub=sub, comm=comms[q], device=dev, precond=precond)
            Bq = torch.from_numpy(np.ascontiguousarray(B[r0:r1])).to(dev)
            Xq = torch.zeros(pl.n_cols, k, dtype=torch.float64, device=dev)
            if X0 is not None:
                Xq[:pl.n_local] = torch.from_numpy(X0[r0:r1]).to(dev)
            res = S.solve(Bq, Xq, tol=tol, maxit=maxit)
            torch.cuda.synchronize(dev)
            out[q] = (Xq[:pl.n_local].cpu().numpy(), res)
            S.close()
        except Exception as e:   # noqa: BLE001 -- reported below
            errs.append(e)
            comms[q].shared.barrier.abort()

    ths = [threading.Thread(target=rank, args=(q,)) for q in range(world)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errs:
        raise errs[0]
    X = np.vstack([o[0] for o in out])
    results = [o[1] for o in out]
    assert all(r.iters == results[0].iters and r.status == results[0].status for r in results)
    return X, results[0]


CASES = [  # (matrix, world, sub, k, p, iterations)
    ("p3d", 3, "hybrid", 8, 4, 25), ("p3d", 2, "global", 16, 4, 15), ("p3d", 4, "parallel", 5, 1, 30),
    ("p3d", 1, "hybrid", 32, 8, 20), ("s27", 3, "hybrid", 24, 12, 12), ("p3d", 3, "classical", 64, 64, 5),
]


def _mat(name):
    return {"p3d": lambda: W.poisson3d(30, 31, 29), "s27": lambda: W.stencil27(15, 14, 13, seed=5),
            "vc": lambda: W.varcoef3d(20, 17, 23, seed=4)}[name]()


@pytest.mark.parametrize("name,world,sub,k,p,m", CASES)
def test_rows_equal_iterations(lib, name, world, sub, k, p, m):
    M = _mat(name)
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    X, r = sharded_solve(lib, M, B, world=world, k=k, p=p, sub=sub, maxit=m, X0=X0)
    assert r.status == bcg.NOT_CONVERGED and r.iters == m
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert_close(X, ref.X, 1e-9)


@pytest.mark.parametrize("precond", [0, 1])
def test_rows_converged(lib, precond):
    M = _mat("vc")
    A = M.to_scipy()
    k, p = 16, 4
    B = W.rhs(M.n, k, seed=3)
    X, r = sharded_solve(lib, M, B, world=3, k=k, p=p, sub="hybrid", tol=1e-8, maxit=3000, precond=precond)
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub="hybrid", tol=1e-8, maxit=3000, precond="jacobi" if precond else "none")
    spread = [O.solve(A, B * (1 + 1e-16 * np.random.default_rng(s).standard_normal(B.shape)), p=p, sub="hybrid",
                      tol=1e-8, maxit=3000, precond="jacobi" if precond else "none").iters for s in range(2)]
    allow = 2 + max(spread + [ref.iters]) - min(spread + [ref.iters])
    assert abs(r.iters - ref.iters) <= allow, (r.iters, ref.iters, spread)
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8)


def test_rows_jacobi_equal_iterations(lib):
    M = _mat("vc")
    B = W.rhs(M.n, 16, seed=4)
    X, r = sharded_solve(lib, M, B, world=2, k=16, p=16, sub="hybrid", maxit=15, precond=1)
    ref = O.solve(M.to_scipy(), B, p=16, sub="hybrid", tol=0.0, maxit=15, precond="jacobi")
    assert_close(X, ref.X, 1e-9)


def test_rows_handle_rejects_misuse(lib):
    import torch
    from paper_1912_11930_gb300 import bcg, dist as D
    dev = torch.device("cuda:0")
    M = W.poisson2d(20)
    pl = D.make_plans(M, 2)[0]
    rp, ci, va = (torch.from_numpy(a).to(dev) for a in (pl.rowptr, pl.colind, pl.vals))
    with pytest.raises(bcg.BCGError, match="n_cols"):
        bcg.bcg_create_csr_rows(pl.n_local, pl.n_local - 1, len(pl.colind), rp, ci, va, 4, 2, "hybrid")
    h = bcg.bcg_create_csr_rows(pl.n_local, pl.n_cols, len(pl.colind), rp, ci, va, 4, 2, "hybrid")
    B = torch.zeros(pl.n_local, 4, dtype=torch.float64, device=dev)
    X = torch.zeros(pl.n_cols, 4, dtype=torch.float64, device=dev)
    with pytest.raises(bcg.BCGError, match="row-sharded"):
        bcg.bcg_solve(h, B, X, 1e-8, 10)
    with pytest.raises(bcg.BCGError, match="bcg_rows_bind"):
        bcg.bcg_rows_start(h, B, X, 1e-8)
    with pytest.raises(bcg.BCGError, match="halo rows"):
        bcg.bcg_rows_unpack(h, X, 3)
    bcg.bcg_destroy(h)


@pytest.fixture(scope="module")
def nccl_world1(lib):
    """A one-rank NCCL process group in this process (no peer: nothing waits on another GPU)."""
    import socket
    import torch
    import torch.distributed as dist
    if dist.is_initialized():
        pytest.skip("a process group already exists in this process")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    yield dist
    dist.destroy_process_group()


@pytest.mark.parametrize("sub,k,p,m", [("hybrid", 32, 8, 21), ("global", 16, 4, 17), ("classical", 64, 64, 10)])
def test_rows_on_stream_nccl_with_graphs(nccl_world1, sub, k, p, m):
    """The production driver: NCCL collectives enqueued on the handle's stream (StreamComm, no host wait inside
    a batch), eagerly and with each batch after the first captured into a CUDA graph and replayed. Both give
    bitwise the same iterate, which matches the oracle at the one-rank bars (1e-9 at equal iterations); a
    batch count that leaves an odd remainder (m = 21, 17) runs its last batch eagerly."""
    import torch
    from paper_1912_11930_gb300 import dist as D
    dist = nccl_world1
    dev = torch.device("cuda:0")
    M = _mat("p3d")
    B = W.rhs(M.n, k, seed=1)
    X0 = 0.01 * W.rhs(M.n, k, seed=2)
    plan = D.make_plans(M, 1)[0]
    out = {}
    for graph in (False, True):
        stream = torch.cuda.Stream(dev)
        S = D.RowShardedSolver(plan, k=k, p=p, sub=sub, comm=D.StreamComm(dist, stream), device=dev, graph=graph)
        Bq = torch.from_numpy(B).to(dev)
        Xq = torch.from_numpy(X0.copy()).to(dev)
        r = S.solve(Bq, Xq, tol=NEVER, maxit=m, check_every=4)
        torch.cuda.synchronize(dev)
        assert r.status == bcg.NOT_CONVERGED and r.iters == m, r
        assert bool(S._graphs) == graph
        out[graph] = Xq.cpu().numpy()
        # a second solve on the same handle replays the graph from its first batch on
        Xq.copy_(torch.from_numpy(X0))
        r2 = S.solve(Bq, Xq, tol=NEVER, maxit=m, check_every=4)
        torch.cuda.synchronize(dev)
        assert r2.iters == m and np.array_equal(Xq.cpu().numpy(), out[graph])
        S.close()
    assert np.array_equal(out[False], out[True])
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    assert_close(out[True], ref.X, 1e-9)


def test_rows_on_stream_converges(nccl_world1):
    import torch
    from paper_1912_11930_gb300 import dist as D
    dev = torch.device("cuda:0")
    M = _mat("vc")
    A = M.to_scipy()
    k, p = 16, 4
    B = W.rhs(M.n, k, seed=3)
    stream = torch.cuda.Stream(dev)
    S = D.RowShardedSolver(D.make_plans(M, 1)[0], k=k, p=p, sub="hybrid", comm=D.StreamComm(nccl_world1, stream),
                           device=dev, graph=True)
    X = torch.zeros(M.n, k, dtype=torch.float64, device=dev)
    r = S.solve(torch.from_numpy(B).to(dev), X, tol=1e-8, maxit=3000)
    S.close()
    assert r.ok, r
    ref = O.solve(A, B, p=p, sub="hybrid", tol=1e-8, maxit=3000)
    assert abs(r.iters - ref.iters) <= 2
    Xh = X.cpu().numpy()
    res = np.linalg.norm(B - A @ Xh, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8), res
