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
