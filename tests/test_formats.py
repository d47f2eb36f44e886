"""SELL-C-sigma conversion (host side): the stored chunks describe exactly Pi A Pi^T, the permutation sorts
rows by decreasing length inside each sigma window, and the chunk layout is the one the kernels read."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1912_11930_gb300 import formats as F
from paper_1912_11930_gb300 import workloads as W


def _unpack(S):
    rows, cols, vals = [], [], []
    for s in range(S.n):
        base = S.chunkptr[s // F.SELL_C] + s % F.SELL_C
        for j in range(S.rowlen[s]):
            rows.append(s)
            cols.append(S.colind[base + j * F.SELL_C])
            vals.append(S.vals[base + j * F.SELL_C])
    return sp.csr_matrix((vals, (rows, cols)), shape=(S.n, S.n))


MATS = {
    "p3d": lambda: W.poisson3d(7, 6, 5),
    "s27": lambda: W.stencil27(6, 5, 4, seed=1),
    "p2d": lambda: W.poisson2d(9),
    "spd": lambda: W.dense_to_csr(W.random_spd_dense(40, seed=1, cond=10.0)),
    "tiny": lambda: W.poisson2d(3),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("sigma", [1, 32, 100, 100000])
def test_sell_is_the_permuted_matrix(name, sigma):
    M = MATS[name]()
    A = M.to_scipy()
    S = F.sell_from_csr(M.rowptr, M.colind, M.vals, sigma)
    n = M.n
    assert sorted(S.perm.tolist()) == list(range(n))
    P = sp.csr_matrix((np.ones(n), (np.arange(n), S.perm)), shape=(n, n))
    assert abs(_unpack(S) - P @ A @ P.T).max() == 0.0
    lens = np.diff(M.rowptr)
    assert np.array_equal(S.rowlen, lens[S.perm])
    for w0 in range(0, n, sigma):   # sorted inside each window, stable, never across windows
        w = S.perm[w0:w0 + sigma]
        assert set(w.tolist()) == set(range(w0, min(n, w0 + sigma)))
        assert np.all(np.diff(S.rowlen[w0:w0 + sigma]) <= 0)
    if sigma == 1:
        assert np.array_equal(S.perm, np.arange(n))
    # chunk layout: consecutive chunks, each C x (longest row) entries, all indices in range
    nch = (n + F.SELL_C - 1) // F.SELL_C
    width = [int(S.rowlen[c * F.SELL_C:(c + 1) * F.SELL_C].max()) for c in range(nch)]
    assert S.chunkptr[0] == 0 and S.nent == F.SELL_C * sum(width)
    assert np.array_equal(np.diff(S.chunkptr), F.SELL_C * np.array(width[:-1]))
    assert S.colind.min() >= 0 and S.colind.max() < n


def test_sell_sorting_reduces_padding():
    """Rows of very different lengths: a sigma window larger than a chunk groups similar rows and pads less."""
    rng = np.random.default_rng(3)
    n = 4096
    lens = rng.integers(1, 60, size=n)
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    colind = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    vals = rng.standard_normal(rowptr[-1])
    f1 = F.sell_from_csr(rowptr, colind, vals, 1).fill
    f4k = F.sell_from_csr(rowptr, colind, vals, 4096).fill
    assert f4k < 1.05 < f1
