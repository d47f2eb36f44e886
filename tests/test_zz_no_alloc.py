"""bcg_bdot_noalloc, the allocation-free variant of the BDOT entry point, for callers that cannot call
cudaMalloc (graph-capture regions that must not allocate, hosts that own every device allocation,
latency-critical paths). Its partial sums live in a static device array shared by all calls, so this test
makes two calls in a row (the second reuses the array the first left behind) and checks both against the
allocating entry point bcg_bdot within the tolerance of the other Gram tests. It lives in a file of its own
that pytest collects last, and passes both alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from paper_1912_11930_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("hybrid", 8, 4), ("global", 32, 8), ("parallel", 16, 1), ("classical", 32, 32), ("hybrid", 256, 32)]


@pytest.mark.parametrize("sub,k,p", CASES)
def test_noalloc_bdot_matches_allocating_entry(lib, sub, k, p):
    import torch
    from paper_1912_11930_gb300 import bcg
    dev = torch.device("cuda:0")
    M = W.poisson3d(20, 21, 19)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, device=dev)
    torch.cuda.synchronize()
    scale = None
    for call in range(2):   # two calls in a row: the second finds the first one's partial sums in the array
        X = torch.from_numpy(W.rhs(M.n, k, seed=30 + call)).to(dev)
        Y = torch.from_numpy(W.rhs(M.n, k, seed=40 + call)).to(dev)
        ref = S.bdot(X, Y)
        got = torch.full_like(ref, float("nan"))
        stream = torch.cuda.current_stream(dev)
        bcg.bcg_bdot_noalloc(M.n, k, S.p, sub, X, Y, got, stream)
        torch.cuda.synchronize()
        scale = float(torch.linalg.norm(X) * torch.linalg.norm(Y)) / k
        assert torch.isfinite(got).all()
        assert float((got - ref).abs().max()) <= 1e-13 * scale, (call, float((got - ref).abs().max()), scale)
    S.close()


def test_noalloc_rejects_bad_sizes(lib):
    import torch
    from paper_1912_11930_gb300 import bcg
    dev = torch.device("cuda:0")
    X = torch.zeros(10, 64, dtype=torch.float64, device=dev)
    g = torch.zeros(1, 64, 64, dtype=torch.float64, device=dev)
    with pytest.raises(bcg.BCGError, match="p > 32"):
        bcg.bcg_bdot_noalloc(10, 64, 64, "hybrid", X, X, g)
    with pytest.raises(bcg.BCGError, match="divide"):
        bcg.bcg_bdot_noalloc(10, 64, 6, "hybrid", X, X, g)
    with pytest.raises(bcg.BCGError, match="device pointers"):
        bcg.bcg_bdot_noalloc(10, 64, 8, "hybrid", X.cpu(), X, g)
