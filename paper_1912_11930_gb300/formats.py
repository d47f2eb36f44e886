"""Host-side conversion of a CSR matrix to SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J. Sci.
Comput. 36(5), 2014), the sparse format Section 4 suggests for BOP. Setup only: the solver's kernels read the
result (bcg_create_sell).

Layout (C = 32): rows are sorted by decreasing length inside windows of sigma consecutive rows (a stable sort,
so sigma = 1 keeps the order); the sorted rows are cut into chunks of C rows; a chunk is stored column-major
and padded to its longest row, entry j of sorted row s at chunkptr[s // C] + j*C + s % C. Column indices are
renumbered with the same permutation, so the stored matrix is Pi A Pi^T with (Pi x)[s] = x[perm[s]].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SELL_C = 32


@dataclass
class SellMatrix:
    n: int
    sigma: int
    chunkptr: np.ndarray   # int64 [nchunks]
    rowlen: np.ndarray     # int32 [n]
    colind: np.ndarray     # int32 [nent], permuted column indices (padding: the row itself)
    vals: np.ndarray       # float64 [nent] (padding: 0)
    perm: np.ndarray       # int32 [n]: original row of sorted row s

    @property
    def nent(self):
        return int(self.vals.size)

    @property
    def fill(self):
        """Stored entries (with padding) per nonzero."""
        return self.nent / max(int(self.rowlen.sum()), 1)


def sell_from_csr(rowptr, colind, vals, sigma: int = 1, C: int = SELL_C) -> SellMatrix:
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    n = rowptr.size - 1
    if sigma < 1:
        raise ValueError("sigma must be >= 1")
    lens = np.diff(rowptr)
    perm = np.empty(n, dtype=np.int64)
    for w0 in range(0, n, sigma):
        w1 = min(n, w0 + sigma)
        order = np.argsort(-lens[w0:w1], kind="stable")
        perm[w0:w1] = w0 + order
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    slen = lens[perm]
    nch = (n + C - 1) // C
    width = np.zeros(nch, dtype=np.int64)
    np.maximum.at(width, np.arange(n) // C, slen)
    chunkptr = np.zeros(nch, dtype=np.int64)
    if nch > 1:
        chunkptr[1:] = np.cumsum(width * C)[:-1]
    nent = int((width * C).sum())
    # padding entries point at their own row (any valid index would do: they are never read); lanes past the
    # last row of a partial chunk point at row 0
    chunk_of = np.repeat(np.arange(nch, dtype=np.int64), width * C)
    lane = (np.arange(nent, dtype=np.int64) - np.repeat(chunkptr, width * C)) % C
    pad_row = chunk_of * C + lane
    out_c = np.where(pad_row < n, pad_row, 0).astype(np.int32)
    out_v = np.zeros(nent, dtype=np.float64)
    # real entries
    s_all = np.arange(n)
    for s in range(0, n, 1 << 16):
        rows = s_all[s:s + (1 << 16)]
        r = perm[rows]
        cnt = lens[r]
        srows = np.repeat(rows, cnt)
        j = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        src = np.repeat(rowptr[r], cnt) + j
        pos = chunkptr[srows // C] + j * C + srows % C
        out_c[pos] = iperm[colind[src]]
        out_v[pos] = vals[src]
    return SellMatrix(n=n, sigma=sigma, chunkptr=chunkptr, rowlen=slen.astype(np.int32), colind=out_c, vals=out_v,
                      perm=perm.astype(np.int32))
