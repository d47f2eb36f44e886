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


# ---- guard bytes after every workspace buffer (option "guards") ----
GUARD_CASES = [  # odd sizes and every form: (matrix, k, p, sub, prec, options)
    ("p3d_odd", 5, 5, "classical", "fp64", {}), ("p3d_odd", 6, 3, "hybrid", "fp64", {}),
    ("p3d_odd", 12, 4, "global", "fp64", {}), ("p3d_odd", 7, 1, "parallel", "fp64", {}),
    ("p3d_odd", 32, 8, "hybrid", "fp32_refine", {}), ("p3d_odd", 32, 8, "hybrid", "fp64_df", {}),
    ("p3d_odd", 64, 64, "classical", "fp64", {}), ("p3d_odd", 128, 64, "hybrid", "fp64", {"tensor_cores": 0}),
    ("p3d_odd", 24, 12, "hybrid", "fp64", {"retooled": 1}), ("vc_odd", 16, 4, "hybrid", "fp64", {"precond": 1}),
]


def _guard_mat(name):
    return {"p3d_odd": lambda: W.poisson3d(13, 11, 7), "vc_odd": lambda: W.varcoef3d(9, 11, 13, seed=2)}[name]()


@pytest.mark.parametrize("name,k,p,sub,prec,opts", GUARD_CASES)
def test_guard_bytes_intact_after_solves(lib, name, k, p, sub, prec, opts):
    """Odd shapes (n = 1001 and 1287 rows, ragged tails in every kernel's row split) through every form with the
    guard check on: no kernel writes past the end of any workspace buffer, and the solution still meets the
    tolerance; then one overwritten guard byte is reported as BCG_ERR_GUARD."""
    import torch
    dev = torch.device("cuda:0")
    M = _guard_mat(name)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, device=dev)
    S.set_option("guards", 1)
    for key, v in opts.items():
        S.set_option(key, v)
    B = W.rhs(M.n, k, seed=9)
    Bt = torch.from_numpy(B).to(dev)
    X, r = S.solve(Bt, tol=1e-8, maxit=3000)
    assert r.ok, r
    res = np.linalg.norm(B - M.to_scipy() @ X.cpu().numpy(), axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= 1.5e-8), res
    Xh = np.zeros_like(B)
    st, info = bcg.bcg_solve_host(S.h, np.ascontiguousarray(B), Xh, 1e-8, 3000)
    assert st == bcg.OK
    bcg.bcg_debug_poke_guard(S.h, 0)
    with pytest.raises(bcg.BCGError) as ei:
        S.solve(Bt, tol=1e-8, maxit=3000)
    assert ei.value.status == bcg.GUARD and "buffer 0" in str(ei.value)
    with pytest.raises(bcg.BCGError):
        bcg.bcg_debug_poke_guard(S.h, 100000)
    S.close()
