"""The multi-rank path on CPU (gloo, world size 2): column-block sharding of the hybrid subalgebra needs no
collective on the data path -- each rank solves its own blocks and the union equals the unsharded solve --
and the job time is the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1912_11930_gb300 import dist as D


def test_shard_columns_cover_whole_blocks():
    for k, p in ((32, 8), (12, 3), (8, 1), (16, 16)):
        for world in (1, 2, 3, 4, 5):
            ranges = [D.shard_columns(k, p, world, r) for r in range(world)]
            cols = [c for c0, c1 in ranges for c in range(c0, c1)]
            assert cols == list(range(k))
            assert all((c0 % p, c1 % p) == (0, 0) for c0, c1 in ranges)
            sizes = [c1 - c0 for c0, c1 in ranges]
            assert max(sizes) - min(sizes) <= p
    with pytest.raises(ValueError):
        D.shard_columns(10, 4, 2, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import bcg as O
    from paper_1912_11930_gb300 import workloads as W
    M = W.poisson2d(12)
    k, p = 8, 2
    B = W.rhs(M.n, k, seed=3)
    c0, c1 = D.shard_columns(k, p, world, rank)
    res = O.solve(M.to_scipy(), B[:, c0:c1], p=p, sub="hybrid", tol=1e-10, maxit=500)
    np.save(os.path.join(out, f"x{rank}.npy"), res.X)
    t = D.max_over_ranks(float(rank + 1), dist)
    np.save(os.path.join(out, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_solve_their_blocks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    from oracle import bcg as O
    from paper_1912_11930_gb300 import workloads as W
    M = W.poisson2d(12)
    B = W.rhs(M.n, 8, seed=3)
    full = O.solve(M.to_scipy(), B, p=2, sub="hybrid", tol=1e-10, maxit=500)
    X = np.hstack([np.load(tmp_path / f"x{r}.npy") for r in range(world)])
    assert np.array_equal(X, full.X)      # independent blocks: bitwise the same iterates
    assert all(np.load(tmp_path / f"t{r}.npy")[0] == 2.0 for r in range(world))


# ---- row-sharded solves: the split, its halo plan and the exchanges (host logic; the kernels run on GPUs) ----
def test_row_plans_reproduce_the_operator():
    """Every rank's local CSR applied to [own rows; halo rows] gives that rank's rows of A x, bitwise."""
    from paper_1912_11930_gb300 import workloads as W
    import scipy.sparse as sp
    for M in (W.poisson3d(7, 6, 5), W.stencil27(6, 5, 4, seed=1), W.poisson2d(9)):
        A = M.to_scipy()
        x = W.rhs(M.n, 3, seed=2)
        y = A @ x
        for world in (1, 2, 3, 4):
            plans = D.make_plans(M, world)
            assert [pl.n_local for pl in plans] == [b1 - b0 for b0, b1 in zip(plans[0].bounds, plans[0].bounds[1:])]
            for pl in plans:
                r0, r1 = pl.bounds[pl.rank], pl.bounds[pl.rank + 1]
                L = sp.csr_matrix((pl.vals, pl.colind, pl.rowptr), shape=(pl.n_local, pl.n_cols))
                xl = np.vstack([x[r0:r1], x[pl.halo_gids]])
                assert np.array_equal(L @ xl, y[r0:r1])
                assert np.all(np.diff(pl.halo_gids) > 0)                       # sorted, unique
                assert all(not (r0 <= g < r1) for g in pl.halo_gids)
                # what a rank sends is exactly what its peers asked for, in their halo order
                for q, rows in pl.send:
                    assert np.array_equal(rows + r0, plans[q].requests[pl.rank])


def _exchange_round(comm, plan, x, torch):
    r0 = plan.bounds[plan.rank]
    sends = {q: torch.from_numpy(x[rows + r0].copy()) for q, rows in plan.send}
    halo = torch.zeros(len(plan.halo_gids), x.shape[1], dtype=torch.float64)
    recvs = {q: halo[off:off + cnt] for q, off, cnt in plan.recv}
    comm.exchange(sends, recvs)
    t = torch.full((5,), float(plan.rank + 1), dtype=torch.float64)
    comm.allreduce_(t)
    return halo.numpy(), t.numpy()


def test_thread_comm_halo_and_allreduce():
    import threading
    import torch
    from paper_1912_11930_gb300 import workloads as W
    M = W.poisson3d(6, 6, 6)
    x = W.rhs(M.n, 4, seed=5)
    world = 3
    plans = D.make_plans(M, world)
    comms = D.ThreadComm.group(world)
    out = [None] * world
    def run(q):
        out[q] = _exchange_round(comms[q], plans[q], x, torch)
    ths = [threading.Thread(target=run, args=(q,)) for q in range(world)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for q in range(world):
        halo, s = out[q]
        assert np.array_equal(halo, x[plans[q].halo_gids])
        assert np.all(s == sum(range(1, world + 1)))


def _rows_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from paper_1912_11930_gb300 import workloads as W
    M = W.poisson3d(6, 5, 7)
    x = W.rhs(M.n, 3, seed=6)
    comm = D.TorchComm(dist)
    b = D.row_bounds(M.n, world)
    plan = D.local_plan(M.rowptr, M.colind, M.vals, b, rank)
    D.fill_sends(plan, comm.all_gather_object(plan.requests))
    halo, s = _exchange_round(comm, plan, x, torch)
    ref = D.make_plans(M, world)[rank]
    ok = (len(plan.send) == len(ref.send) and all(q == qr and np.array_equal(r, rr)
                                                   for (q, r), (qr, rr) in zip(plan.send, ref.send)))
    np.save(os.path.join(out, f"r{rank}.npy"), np.array([ok, np.array_equal(halo, x[plan.halo_gids]),
                                                         bool(np.all(s == world * (world + 1) / 2))]))
    dist.barrier()
    dist.destroy_process_group()


def test_torch_comm_two_ranks_row_split(tmp_path):
    """The production exchange (torch.distributed; gloo here on host tensors): each rank builds its own plan,
    learns its sends from an all-gather of the requests, and the halo rows it receives are its peers' rows."""
    world = 2
    mp.start_processes(_rows_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        assert np.load(tmp_path / f"r{r}.npy").all()


# ---- the row-sharded iteration schedule on host tensors (gloo, 2 and 3 ranks) ----
class _HostRankOps:
    """One rank's share of Algorithm 1 on its rows, on host tensors, from the oracle's primitives: the
    interface RowSchedule drives (pack, unpack, phase 1..3, sums1, sums2, halo). Partial block products over
    the rank's rows go into sums1 / sums2 and are complete only after the schedule has added them over ranks."""

    def __init__(self, plan, B, X0, k, p, sub, torch):
        import scipy.sparse as sp
        from oracle import bcg as O
        self.O, self.torch = O, torch
        self.kind, self.p = O.canonical_subalgebra(sub, k, p)
        self.q = k // self.p
        self.nl = plan.n_local
        self.A = sp.csr_matrix((plan.vals, plan.colind, plan.rowptr), shape=(plan.n_local, plan.n_cols))
        nb = self.q if self.kind == "hybrid" else 1
        self.E = nb * self.p * self.p
        self.shape = (nb, self.p, self.p)
        self.sums1 = torch.zeros(2 * self.E, dtype=torch.float64)
        self.sums2 = torch.zeros(self.E + k, dtype=torch.float64)
        self.halo = torch.zeros(len(plan.halo_gids), k, dtype=torch.float64)
        self.X = X0.copy()                          # n_cols x k: own rows, then X^0's halo rows
        self.R = B - self.A @ self.X
        self.P = np.zeros_like(self.X)
        self.P[:self.nl] = self.R
        self.active = np.ones(nb, dtype=bool)

    def pack(self, q, rows, buf):
        buf.copy_(self.torch.from_numpy(self.P[rows.numpy().astype(np.int64)]))

    def unpack(self):
        self.P[self.nl:] = self.halo.numpy()

    def phase(self, i):
        O, Pl = self.O, self.P[:self.nl]
        if i == 1:
            self.Q = self.A @ self.P
            self.sums1[:self.E] = self.torch.from_numpy(O.block_product(Pl, self.Q, self.p, self.kind).ravel())
            self.sums1[self.E:] = self.torch.from_numpy(O.block_product(Pl, self.R, self.p, self.kind).ravel())
        elif i == 2:
            curv = self.sums1[:self.E].numpy().reshape(self.shape)
            self.proj = self.sums1[self.E:].numpy().reshape(self.shape).copy()
            lam, ok = O.bsolve_cholesky(curv, self.proj, self.active)
            assert ok
            self.X[:self.nl] = O.baxpy(self.X[:self.nl], Pl, lam, +1.0)
            self.R = O.baxpy(self.R, self.Q, lam, -1.0)
            self.sums2[:self.E] = self.torch.from_numpy(O.block_product(self.R, self.R, self.p, self.kind).ravel())
            self.sums2[self.E:] = self.torch.from_numpy(np.sum(self.R * self.R, axis=0))
        else:
            zr = self.sums2[:self.E].numpy().reshape(self.shape)
            beta, ok = O.bsolve_lu(self.proj, zr, self.active)
            assert ok
            self.P[:self.nl] = O.baxpy(self.R, Pl, beta, +1.0)


def _schedule_worker(rank, world, port, out, sub, k, p, m):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from paper_1912_11930_gb300 import workloads as W
    M = W.poisson3d(7, 6, 8)
    B = W.rhs(M.n, k, seed=11)
    X0 = 0.01 * W.rhs(M.n, k, seed=12)
    comm = D.TorchComm(dist)
    plan = D.local_plan(M.rowptr, M.colind, M.vals, D.row_bounds(M.n, world), rank)
    D.fill_sends(plan, comm.all_gather_object(plan.requests))
    r0, r1 = plan.bounds[rank], plan.bounds[rank + 1]
    ops = _HostRankOps(plan, B[r0:r1], np.vstack([X0[r0:r1], X0[plan.halo_gids]]), k, p, sub, torch)
    send_rows = {q: torch.from_numpy(rows) for q, rows in plan.send}
    send_bufs = {q: torch.empty(len(rows), k, dtype=torch.float64) for q, rows in plan.send}
    recv_views = {q: ops.halo[off:off + cnt] for q, off, cnt in plan.recv}
    sched = D.RowSchedule(ops, comm, send_rows, send_bufs, recv_views)
    for _ in range(m):
        sched.iteration()
    np.save(os.path.join(out, f"x{rank}.npy"), ops.X[:plan.n_local])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,sub,k,p", [(2, "hybrid", 6, 3), (3, "global", 4, 2), (2, "classical", 4, 4)])
def test_row_schedule_over_gloo_ranks_matches_the_oracle(tmp_path, world, sub, k, p):
    """RowSchedule's order of steps (halo of P, phase 1, sum over ranks, phase 2, sum, phase 3), driven over
    gloo ranks whose shares are written from the oracle's primitives, reproduces the unsharded Algorithm 1:
    the iterates after m iterations equal the oracle's on the whole matrix up to the rounding of the partial
    sums' order."""
    from oracle import bcg as O
    from paper_1912_11930_gb300 import workloads as W
    m = 12
    mp.start_processes(_schedule_worker, args=(world, _free_port(), str(tmp_path), sub, k, p, m), nprocs=world,
                       start_method="spawn")
    M = W.poisson3d(7, 6, 8)
    B = W.rhs(M.n, k, seed=11)
    X0 = 0.01 * W.rhs(M.n, k, seed=12)
    ref = O.solve(M.to_scipy(), B, X0=X0, p=p, sub=sub, tol=0.0, maxit=m)
    X = np.vstack([np.load(tmp_path / f"x{r}.npy") for r in range(world)])
    err = np.abs(X - ref.X).max(axis=0) / np.abs(ref.X).max(axis=0)
    assert np.all(err <= 1e-11), err
