"""Multi-GPU helpers: sharding by independent column blocks, and job timing over ranks.

The hybrid subalgebra S_Hy^p (and the parallel one, p = 1) makes the q = k/p column blocks independent
problems (Section 3: the hybrid method is a data-parallel version of the classical method), so k
right-hand sides are split into contiguous groups of whole blocks, one group per rank, with no collective
on the data path; only the job time is reduced (max over ranks). The global and classical subalgebras
couple all columns and are not sharded this way.
"""
from __future__ import annotations


def shard_columns(k: int, p: int, world: int, rank: int) -> tuple[int, int]:
    """Column range [c0, c1) of `rank`: whole blocks of p columns, as even as possible (leading ranks get one
    block more). Ranks beyond the number of blocks get an empty range."""
    if p < 1 or k % p:
        raise ValueError(f"p={p} must divide k={k}")
    q = k // p
    base, extra = divmod(q, world)
    b0 = rank * base + min(rank, extra)
    nb = base + (1 if rank < extra else 0)
    return b0 * p, (b0 + nb) * p


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own right-hand sides in the weak-scaling benchmark."""
    return seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Job time: the slowest rank's value (a single scalar all-reduce; identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------------------------
# Row-sharded solves: one problem, its rows split over ranks (strong scaling). Every block product of
# Algorithm 1 is a sum over rows, so each rank contributes partial sums that the ranks add up before the
# p x p solves; BOP needs the rows of P that A couples across the split (the halo). The C ABI runs one rank's
# share (bcg_create_csr_rows, bcg_rows_*); this module builds the split and drives the exchanges.

from dataclasses import dataclass, field

import numpy as np


def row_bounds(n: int, world: int) -> list:
    """Contiguous row ranges, as even as possible: rank q owns [b[q], b[q+1])."""
    base, extra = divmod(n, world)
    b = [0]
    for q in range(world):
        b.append(b[-1] + base + (1 if q < extra else 0))
    return b


@dataclass
class RowPlan:
    """One rank's rows in local numbering (own rows first, then halo rows sorted by global index, which
    groups them by owner) and the row traffic of its halo exchange."""
    rank: int
    bounds: list
    rowptr: np.ndarray           # int64, n_local + 1
    colind: np.ndarray           # int32, local column indices < n_cols
    vals: np.ndarray             # float64
    halo_gids: np.ndarray        # int64: global row of local column n_local + i
    recv: list                   # (owner rank, first halo index, count), owners ascending
    requests: dict               # owner rank -> global rows this rank needs from it
    send: list = field(default_factory=list)   # (rank, int32 local rows it needs from this rank)

    @property
    def n_local(self):
        return self.bounds[self.rank + 1] - self.bounds[self.rank]

    @property
    def n_cols(self):
        return self.n_local + len(self.halo_gids)


def local_plan(rowptr, colind, vals, bounds, rank) -> RowPlan:
    """The plan of `rank` from the global CSR arrays (only its own rows are read)."""
    r0, r1 = bounds[rank], bounds[rank + 1]
    e0, e1 = int(rowptr[r0]), int(rowptr[r1])
    cols = np.asarray(colind[e0:e1], dtype=np.int64)
    inside = (cols >= r0) & (cols < r1)
    halo = np.unique(cols[~inside])
    loc = np.empty_like(cols)
    loc[inside] = cols[inside] - r0
    loc[~inside] = (r1 - r0) + np.searchsorted(halo, cols[~inside])
    owner = np.searchsorted(np.asarray(bounds), halo, side="right") - 1
    recv, requests = [], {}
    for q in np.unique(owner):
        idx = np.nonzero(owner == q)[0]
        recv.append((int(q), int(idx[0]), int(idx.size)))
        requests[int(q)] = halo[idx]
    return RowPlan(rank=rank, bounds=list(bounds), rowptr=np.asarray(rowptr[r0:r1 + 1], dtype=np.int64) - e0,
                   colind=loc.astype(np.int32), vals=np.ascontiguousarray(vals[e0:e1], dtype=np.float64),
                   halo_gids=halo, recv=recv, requests=requests)


def fill_sends(plan: RowPlan, all_requests: list) -> RowPlan:
    """all_requests[q] = rank q's `requests` dict; this rank sends q the rows q asked it for."""
    r0 = plan.bounds[plan.rank]
    plan.send = [(q, (np.asarray(req[plan.rank]) - r0).astype(np.int32))
                 for q, req in enumerate(all_requests) if q != plan.rank and plan.rank in req]
    return plan


def make_plans(M, world: int) -> list:
    """Plans of all ranks from a workloads.CSRMatrix (single-process setup, e.g. for an emulated split)."""
    b = row_bounds(M.n, world)
    plans = [local_plan(M.rowptr, M.colind, M.vals, b, q) for q in range(world)]
    reqs = [pl.requests for pl in plans]
    return [fill_sends(pl, reqs) for pl in plans]


class TorchComm:
    """Host-ordered exchanges through torch.distributed (gloo on host tensors, or NCCL): the caller's device
    work is finished before a collective starts, and the collective is finished when the call returns."""

    on_stream = False

    def __init__(self, dist):
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    @staticmethod
    def _sync(t):
        if t is not None and t.is_cuda:
            import torch
            torch.cuda.synchronize(t.device)

    def allreduce_(self, t):
        self._sync(t)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        self._sync(t)

    def exchange(self, sends, recvs):
        """sends: {rank: tensor}, recvs: {rank: tensor view to fill}."""
        for t in sends.values():
            self._sync(t)
        ops = [self.dist.P2POp(self.dist.isend, t, q) for q, t in sends.items()]
        ops += [self.dist.P2POp(self.dist.irecv, t, q) for q, t in recvs.items()]
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        for t in recvs.values():
            self._sync(t)

    def all_gather_object(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out


class StreamComm(TorchComm):
    """Exchanges enqueued on one CUDA stream (NCCL): each collective is ordered after the work already on
    `stream` and before the work enqueued after it, and the host never waits for it, so an iteration's phases
    and exchanges queue up back to back (and can be captured into one CUDA graph)."""

    on_stream = True

    def __init__(self, dist, stream):
        super().__init__(dist)
        self.stream = stream

    def allreduce_(self, t):
        import torch
        with torch.cuda.stream(self.stream):
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)

    def exchange(self, sends, recvs):
        import torch
        ops = [self.dist.P2POp(self.dist.isend, t, q) for q, t in sends.items()]
        ops += [self.dist.P2POp(self.dist.irecv, t, q) for q, t in recvs.items()]
        if not ops:
            return
        with torch.cuda.stream(self.stream):
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()   # NCCL: the stream waits, not the host


class ThreadComm:
    """`world` ranks as threads of one process (one GPU or the CPU): the exchanges are copies between the
    ranks' tensors, sums in rank order. Each rank's device work is finished before it is read."""

    on_stream = False

    class _Shared:
        def __init__(self, world):
            import threading
            self.world = world
            self.barrier = threading.Barrier(world, timeout=120)   # a failed rank breaks it instead of hanging
            self.slots = [None] * world

    def __init__(self, shared, rank):
        self.shared, self.rank, self.world = shared, rank, shared.world

    @classmethod
    def group(cls, world):
        sh = cls._Shared(world)
        return [cls(sh, q) for q in range(world)]

    def _sync(self, t):
        if t is not None and t.is_cuda:
            import torch
            torch.cuda.synchronize(t.device)

    def allreduce_(self, t):
        sh = self.shared
        self._sync(t)
        sh.slots[self.rank] = t
        sh.barrier.wait()
        if self.rank == 0:
            s = sh.slots[0].clone()
            for q in range(1, self.world):
                s += sh.slots[q]
            for q in range(self.world):
                sh.slots[q].copy_(s)
            self._sync(s)
        sh.barrier.wait()

    def exchange(self, sends, recvs):
        sh = self.shared
        for t in sends.values():
            self._sync(t)
        sh.slots[self.rank] = sends
        sh.barrier.wait()
        for q, view in recvs.items():
            view.copy_(sh.slots[q][self.rank])
            self._sync(view)
        sh.barrier.wait()

    def all_gather_object(self, obj):
        sh = self.shared
        sh.slots[self.rank] = obj
        sh.barrier.wait()
        out = list(sh.slots)
        sh.barrier.wait()
        return out


class RowSchedule:
    """The steps of one row-sharded iteration and their order (Algorithm 1 split over row ranges): BOP needs
    the halo rows of P, so the owners' rows are packed, exchanged and unpacked first; alpha and the recomputed
    rho (sums1) are sums over all rows, so they are added over ranks before lambda is solved; rho and the
    column norms (sums2) likewise before the stopping test and beta.

    `ops` runs one rank's share: pack(q, rows, buf), unpack(), phase(i) and the buffers sums1, sums2, halo;
    `comm` adds over ranks and exchanges rows (host-ordered, or enqueued on the handle's stream)."""

    def __init__(self, ops, comm, send_rows, send_bufs, recv_views):
        self.ops, self.comm = ops, comm
        self.send_rows, self.send_bufs, self.recv_views = send_rows, send_bufs, recv_views

    def halo(self):
        for q, rows in self.send_rows.items():
            self.ops.pack(q, rows, self.send_bufs[q])
        self.comm.exchange(self.send_bufs, self.recv_views)
        self.ops.unpack()

    def iteration(self):
        self.halo()
        self.ops.phase(1)
        self.comm.allreduce_(self.ops.sums1)
        self.ops.phase(2)
        self.comm.allreduce_(self.ops.sums2)
        self.ops.phase(3)


class _HandleOps:
    """One rank's share through the C ABI (bcg_rows_*): every call enqueues on the handle's stream."""

    def __init__(self, bcg, h, sums1, sums2, halo):
        self.bcg, self.h, self.sums1, self.sums2, self.halo = bcg, h, sums1, sums2, halo

    def pack(self, q, rows, buf):
        self.bcg.bcg_rows_pack(self.h, rows, rows.numel(), buf)

    def unpack(self):
        if self.halo.shape[0]:
            self.bcg.bcg_rows_unpack(self.h, self.halo, self.halo.shape[0])

    def phase(self, i):
        self.bcg.bcg_rows_phase(self.h, i)


class RowShardedSolver:
    """One rank's share of a row-sharded solve (FP64, CSR): a handle on this rank's rows plus the buffers of
    its exchanges. `comm` is a StreamComm (NCCL on the handle's stream: no host synchronisation inside a batch
    of iterations; with `graph`, each batch after the first is one CUDA graph replay), a TorchComm (host-
    ordered) or a ThreadComm (ranks as threads of one process)."""

    def __init__(self, plan: RowPlan, *, k, p=1, sub="hybrid", comm, device=None, precond=0, graph=False):
        import torch
        from . import bcg
        self.torch, self.bcg, self.plan, self.comm = torch, bcg, plan, comm
        self.device = torch.device(device or "cuda")
        self.stream = comm.stream if getattr(comm, "on_stream", False) else torch.cuda.Stream(device=self.device)
        self.graph = bool(graph) and getattr(comm, "on_stream", False)
        self._graphs, self._warm, self._parity = {}, False, 0
        self.k = k
        self.p = 1 if sub == "parallel" else (k if sub == "classical" else p)
        self.nblk = 1 if sub == "global" else k // self.p
        dev, f64 = self.device, torch.float64
        self._rowptr = torch.from_numpy(plan.rowptr).to(dev)
        self._colind = torch.from_numpy(plan.colind).to(dev)
        self._vals = torch.from_numpy(plan.vals).to(dev)
        E = k * self.p
        self.sums1 = torch.zeros(2 * E, dtype=f64, device=dev)
        self.sums2 = torch.zeros(E + k, dtype=f64, device=dev)
        self.norms = self.sums2[E:]
        self.halo = torch.zeros(len(plan.halo_gids), k, dtype=f64, device=dev)
        self.recv_views = {q: self.halo[off:off + cnt] for q, off, cnt in plan.recv}
        self.send_rows = {q: torch.from_numpy(rows).to(dev) for q, rows in plan.send}
        self.send_bufs = {q: torch.empty(len(rows), k, dtype=f64, device=dev) for q, rows in plan.send}
        torch.cuda.synchronize(dev)
        self.h = bcg.bcg_create_csr_rows(plan.n_local, plan.n_cols, len(plan.colind), self._rowptr, self._colind,
                                         self._vals, k, self.p, sub, self.stream)
        bcg.bcg_rows_bind(self.h, self.sums1, self.sums2)
        if precond:
            bcg.bcg_set_option(self.h, "precond", precond)
        self.schedule = RowSchedule(_HandleOps(bcg, self.h, self.sums1, self.sums2, self.halo), comm,
                                    self.send_rows, self.send_bufs, self.recv_views)

    def _halo_x(self, X):
        """The halo rows of X^0 from their owners (once per solve, on the handle's stream)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            for q, rows in self.send_rows.items():
                torch.index_select(X[:self.plan.n_local], 0, rows.long(), out=self.send_bufs[q])
        self.comm.exchange(self.send_bufs, self.recv_views)
        with torch.cuda.stream(self.stream):
            X[self.plan.n_local:].copy_(self.halo)

    def _batch(self, n, X):
        """n iterations: enqueued eagerly, or (graph) the replay of a graph captured for batches of n. The first
        batch runs eagerly, so that the communicators and the kernels' first-launch set-up exist before a
        capture. A graph fixes the host-side arguments of the calls it captured: the solution buffer X (set by
        bcg_rows_start) and, with blocks wider than 32, which of two buffers holds P (the library swaps P and Q
        once per iteration) -- so graphs are kept per (n, X, parity of the iterations run on the handle)."""
        torch = self.torch
        key = (n, X.data_ptr(), self._parity)
        g = self._graphs.get(key)
        if g is None and (not self.graph or not self._warm):
            for _ in range(n):
                self.schedule.iteration()
        else:
            if g is None:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.stream):
                    for _ in range(n):
                        self.schedule.iteration()
                self._graphs[key] = g
            with torch.cuda.stream(self.stream):   # a replay runs on the current stream: the handle's
                g.replay()
        self._warm = True
        self._parity ^= n & 1

    def solve(self, B, X, tol=1e-8, maxit=10000, check_every=8):
        """B: n_local x k; X: n_cols x k (rows beyond n_local are scratch for the halo of X^0). Returns the
        SolveResult of this rank (identical on every rank). The host waits once per `check_every` iterations
        (the stopping poll); the exchanges in between follow `comm`'s ordering."""
        bcg, torch = self.bcg, self.torch
        torch.cuda.synchronize(self.device)
        self._halo_x(X)
        bcg.bcg_rows_start(self.h, B, X, tol)
        self.comm.allreduce_(self.norms)
        bcg.bcg_rows_start_status(self.h)
        done = bcg.bcg_rows_poll(self.h)
        it = 0
        while not done and it < maxit:
            n = min(check_every, maxit - it)
            self._batch(n, X)
            it += n
            done = bcg.bcg_rows_poll(self.h)
        st, info = bcg.bcg_rows_finish(self.h)
        iters = bcg.bcg_block_iters(self.h, self.nblk)
        return bcg.SolveResult(st, info.iters, 0, info.breakdown_iter, info.max_rel_res_recursive, float("nan"),
                               iters)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.bcg.bcg_destroy(self.h)
            self.h = None
