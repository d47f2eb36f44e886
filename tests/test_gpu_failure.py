"""Failure paths of the C ABI, exercised without any GPU fault: a device allocation that fails (injected on the
host by bcg_debug_fail_alloc, as if cudaMalloc had run out of memory) must give BCG_ERR_OOM with nothing leaked
and leave other handles usable."""
import numpy as np
import pytest

from paper_1912_11930_gb300 import bcg, workloads as W

pytestmark = pytest.mark.gpu


def _csr(M, dev):
    import torch
    return (torch.from_numpy(M.rowptr).to(dev), torch.from_numpy(M.colind).to(dev),
            torch.from_numpy(M.vals).to(dev))


@pytest.mark.parametrize("k,p,sub,prec", [(8, 4, "hybrid", "fp64"), (8, 4, "hybrid", "fp32_refine"),
                                         (64, 64, "classical", "fp64"), (8, 4, "global", "fp64_df")])
def test_injected_allocation_failure_gives_oom_and_leaks_nothing(lib, k, p, sub, prec):
    import torch
    dev = torch.device("cuda:0")
    M = W.poisson3d(16)
    rowptr, colind, vals = _csr(M, dev)
    stream = torch.cuda.Stream(dev)

    def create():
        return bcg.bcg_create_csr(M.n, M.nnz, rowptr, colind, vals, k, p, sub, prec, stream)

    bcg.bcg_destroy(create())   # every lazy initialisation of the context and the kernels happens here
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    failures = 0
    try:
        for nth in range(1, 200):
            bcg.bcg_debug_fail_alloc(nth)
            try:
                h = create()
            except bcg.BCGError as e:
                assert e.status == bcg.OOM and "injected" in str(e), str(e)
                failures += 1
            else:   # the handle needed fewer than nth allocations: every failure point has been covered
                bcg.bcg_debug_fail_alloc(0)
                bcg.bcg_destroy(h)
                break
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info(dev)[0] == free0, f"device memory leaked after a failure at allocation {nth}"
    finally:
        bcg.bcg_debug_fail_alloc(0)
    assert failures >= 10, failures
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0


def test_failure_of_the_host_entry_staging_leaves_the_handle_usable(lib):
    """bcg_solve_host allocates its device staging at its first call: a failure there returns OOM, and the same
    handle then solves (the next call allocates the staging)."""
    import torch
    dev = torch.device("cuda:0")
    M = W.poisson3d(16)
    k = 8
    S = bcg.Solver.from_matrix(M, k=k, p=4, sub="hybrid", device=dev)
    B = np.ascontiguousarray(W.rhs(M.n, k, seed=3))
    X = np.zeros_like(B)
    try:
        for nth in (1, 2):   # the first or the second of the two staging buffers
            bcg.bcg_debug_fail_alloc(nth)
            with pytest.raises(bcg.BCGError) as ei:
                bcg.bcg_solve_host(S.h, B, X, 1e-8, 1000)
            assert ei.value.status == bcg.OOM
    finally:
        bcg.bcg_debug_fail_alloc(0)
    st, info = bcg.bcg_solve_host(S.h, B, X, 1e-8, 1000)
    assert st == bcg.OK and info.max_rel_res_true <= 1.5e-8
    S.close()


def test_debug_hook_rejects_negative_counts(lib):
    with pytest.raises(bcg.BCGError):
        bcg.bcg_debug_fail_alloc(-1)
