"""Seeded synthetic inputs for the block CG solver: sparse SPD matrices and blocks of right-hand sides.

This module only *generates* inputs. It holds none of the solver's arithmetic, so that the CPU oracle
(``oracle/``) and the CUDA path can both be fed from it without sharing any part of the method.

Every matrix is returned in CSR form (``rowptr`` int64, ``colind`` int32, ``vals`` float64, columns sorted
within a row, rows in natural lexicographic order x fastest) and, where the CUDA library has a matrix-free
form for it, with the parameters of that stencil form as well.

Workloads (the paper's whole-solver experiment in Section 4 uses a 2D heterogeneous Poisson problem with a
5-point finite-difference stencil and random right-hand sides; these are synthetic stand-ins for it):

* ``poisson2d``      5-point Laplacian on an nx x ny interior grid, Dirichlet boundary eliminated,
                     A = h^-2 (4, -1, -1, -1, -1) with h = 1/(nx+1).
* ``poisson3d``      7-point Laplacian on nx x ny x nz, A = h^-2 (6, -1 x 6), h = 1/(nx+1).
* ``varcoef3d``      7-point variable-coefficient diffusion: one coefficient per cell face (boundary faces
                     included) drawn i.i.d. exp(N(0, sigma^2)); A_ii = h^-2 * sum of the cell's six face
                     coefficients, A_ij = -h^-2 * (coefficient of the shared face).
* ``varcoef2d``      5-point variable-coefficient diffusion on nx x ny, the 2D form of ``varcoef3d`` (the
                     heterogeneous 2D Poisson problem of the whole-solver experiment): x-faces (ny, nx+1)
                     then y-faces (ny+1, nx), i.i.d. exp(N(0, sigma^2)); CSR only.
* ``stencil27``      27-point SPD matrix: one value -U(0.5, 1.5) per unordered neighbour pair (so A is
                     symmetric), diagonal = row sum of |off-diagonals| + 0.1 (strictly diagonally dominant).
* ``powerlaw_laplacian``  graph Laplacian + I of a random graph whose out-degrees follow a Pareto law
                     (row lengths from a few to thousands): not one of the paper's problems, only the
                     irregular-row case the SELL-C-sigma format is meant for.
* ``rhs``            n x k block, i.i.d. N(0, 1), row-major (element (i, c) at i*k + c).

Seeds: the right-hand side uses ``seed``, the loss weights of the autograd workload ``seed + 1`` and matrix
coefficients ``seed + 2``, each from its own ``numpy.random.default_rng`` (PCG64, identical on every
platform).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSRMatrix:
    n: int
    rowptr: np.ndarray  # int64, n+1
    colind: np.ndarray  # int32, nnz
    vals: np.ndarray    # float64, nnz
    # matrix-free description understood by bcg_create_stencil (None when only CSR exists)
    stencil: dict | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind.astype(np.int64), self.rowptr), shape=(self.n, self.n))


def _assemble(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> tuple:
    """Sort COO triplets by (row, col) and compress to CSR. No duplicates are expected."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols.astype(np.int32), vals.astype(np.float64)


def poisson2d(nx: int, ny: int | None = None) -> CSRMatrix:
    ny = nx if ny is None else ny
    h = 1.0 / (nx + 1)
    s = 1.0 / (h * h)
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % nx, idx // nx
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 4.0 * s)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
        r = idx[ok]
        rows.append(r)
        cols.append(r + dx + dy * nx)
        vals.append(np.full(r.shape[0], -s))
    rowptr, colind, v = _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return CSRMatrix(n, rowptr, colind, v,
                     stencil=dict(kind="5pt_2d", nx=nx, ny=ny, nz=1, scale=s, coef=None),
                     meta=dict(name=f"poisson2d_{nx}x{ny}", h=h))


def poisson3d(nx: int, ny: int | None = None, nz: int | None = None) -> CSRMatrix:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    h = 1.0 / (nx + 1)
    s = 1.0 / (h * h)
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols, vals = [idx], [idx], [np.full(n, 6.0 * s)]
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        ok = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
              & (iz + dz >= 0) & (iz + dz < nz))
        r = idx[ok]
        rows.append(r)
        cols.append(r + dx + dy * nx + dz * nx * ny)
        vals.append(np.full(r.shape[0], -s))
    rowptr, colind, v = _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return CSRMatrix(n, rowptr, colind, v,
                     stencil=dict(kind="7pt_3d", nx=nx, ny=ny, nz=nz, scale=s, coef=None),
                     meta=dict(name=f"poisson3d_{nx}x{ny}x{nz}", h=h))


def varcoef_faces(nx: int, ny: int, nz: int, seed: int = 0, sigma: float = 1.0) -> np.ndarray:
    """Face coefficients exp(N(0, sigma^2)), packed as one float64 array:
    x-faces (nz, ny, nx+1), then y-faces (nz, ny+1, nx), then z-faces (nz+1, ny, nx), each C-order.
    Face (z, y, i) of the x-family lies between cells i-1 and i of row (z, y); faces 0 and nx are on the
    Dirichlet boundary (likewise for y and z)."""
    rng = np.random.default_rng(seed + 2)
    nf = nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx
    return np.exp(sigma * rng.standard_normal(nf))


def split_faces(faces: np.ndarray, nx: int, ny: int, nz: int):
    a = nz * ny * (nx + 1)
    b = a + nz * (ny + 1) * nx
    fx = faces[:a].reshape(nz, ny, nx + 1)
    fy = faces[a:b].reshape(nz, ny + 1, nx)
    fz = faces[b:].reshape(nz + 1, ny, nx)
    return fx, fy, fz


def varcoef3d(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0,
              sigma: float = 1.0) -> CSRMatrix:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    h = 1.0 / (nx + 1)
    s = 1.0 / (h * h)
    faces = varcoef_faces(nx, ny, nz, seed, sigma)
    fx, fy, fz = split_faces(faces, nx, ny, nz)
    n = nx * ny * nz
    # per-cell sums of the six face coefficients
    diag = (fx[:, :, :-1] + fx[:, :, 1:] + fy[:, :-1, :] + fy[:, 1:, :] + fz[:-1] + fz[1:]).reshape(n)
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols, vals = [idx], [idx], [s * diag]
    # neighbour in -x uses face ix, +x uses face ix+1 (x-family), likewise for y and z
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        ok = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
              & (iz + dz >= 0) & (iz + dz < nz))
        r = idx[ok]
        x, y, z = ix[ok], iy[ok], iz[ok]
        if dx:
            f = fx[z, y, x + (1 if dx > 0 else 0)]
        elif dy:
            f = fy[z, y + (1 if dy > 0 else 0), x]
        else:
            f = fz[z + (1 if dz > 0 else 0), y, x]
        rows.append(r)
        cols.append(r + dx + dy * nx + dz * nx * ny)
        vals.append(-s * f)
    rowptr, colind, v = _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return CSRMatrix(n, rowptr, colind, v,
                     stencil=dict(kind="7pt_3d_varcoef", nx=nx, ny=ny, nz=nz, scale=s, coef=faces),
                     meta=dict(name=f"varcoef3d_{nx}x{ny}x{nz}", h=h, sigma=sigma, seed=seed))


def varcoef2d(nx: int, ny: int | None = None, seed: int = 0, sigma: float = 1.0) -> CSRMatrix:
    ny = nx if ny is None else ny
    h = 1.0 / (nx + 1)
    s = 1.0 / (h * h)
    rng = np.random.default_rng(seed + 2)
    fx = np.exp(sigma * rng.standard_normal(ny * (nx + 1))).reshape(ny, nx + 1)
    fy = np.exp(sigma * rng.standard_normal((ny + 1) * nx)).reshape(ny + 1, nx)
    n = nx * ny
    diag = (fx[:, :-1] + fx[:, 1:] + fy[:-1, :] + fy[1:, :]).reshape(n)
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % nx, idx // nx
    rows, cols, vals = [idx], [idx], [s * diag]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
        r = idx[ok]
        x, y = ix[ok], iy[ok]
        f = fx[y, x + (1 if dx > 0 else 0)] if dx else fy[y + (1 if dy > 0 else 0), x]
        rows.append(r)
        cols.append(r + dx + dy * nx)
        vals.append(-s * f)
    rowptr, colind, v = _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return CSRMatrix(n, rowptr, colind, v, meta=dict(name=f"varcoef2d_{nx}x{ny}", h=h, sigma=sigma, seed=seed))


_OFFSETS27 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if (dx, dy, dz) != (0, 0, 0)]
# the 13 "forward" offsets: lexicographically positive (dz, dy, dx)
_FORWARD27 = [o for o in _OFFSETS27 if (o[2], o[1], o[0]) > (0, 0, 0)]


def stencil27(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0) -> CSRMatrix:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    rng = np.random.default_rng(seed + 2)
    # one uniform per (forward offset, cell); only used where the neighbour exists
    u = 0.5 + rng.random((len(_FORWARD27), n))
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols, vals = [], [], []
    absrow = np.zeros(n)
    for t, (dx, dy, dz) in enumerate(_FORWARD27):
        ok = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
              & (iz + dz >= 0) & (iz + dz < nz))
        r = idx[ok]
        c = r + dx + dy * nx + dz * nx * ny
        w = u[t, ok]
        rows += [r, c]
        cols += [c, r]
        vals += [-w, -w]
        np.add.at(absrow, r, w)
        np.add.at(absrow, c, w)
    rows.append(idx)
    cols.append(idx)
    vals.append(absrow + 0.1)
    rowptr, colind, v = _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return CSRMatrix(n, rowptr, colind, v, stencil=None,
                     meta=dict(name=f"stencil27_{nx}x{ny}x{nz}", seed=seed))


def powerlaw_laplacian(n: int, seed: int = 0, shape: float = 1.5, scale: float = 3.0,
                       max_degree: int = 2000) -> CSRMatrix:
    """L + I for the symmetrised random graph where node i links to deg_i uniform targets, deg_i =
    min(max_degree, floor(scale (1 + Pareto(shape)))); SPD (diagonally dominant), rows of very uneven length."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed + 2)
    deg = np.minimum((rng.pareto(shape, size=n) + 1.0) * scale, max_degree).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = rng.integers(0, n, size=src.size)
    G = sp.coo_matrix((np.ones(src.size), (src, dst)), shape=(n, n)).tocsr()
    G = ((G + G.T) > 0).astype(np.float64)
    G.setdiag(0)
    G.eliminate_zeros()
    L = (sp.diags(np.asarray(G.sum(axis=1)).ravel() + 1.0) - G).tocsr()
    L.sort_indices()
    return CSRMatrix(n, L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64),
                     stencil=None, meta=dict(name=f"powerlaw_laplacian_{n}", seed=seed))


def rhs(n: int, k: int, seed: int = 0) -> np.ndarray:
    """Right-hand sides B, n x k, i.i.d. N(0, 1), row-major float64."""
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal((n, k)))


def loss_weights(n: int, k: int, seed: int = 0) -> np.ndarray:
    """W for the autograd workload loss = sum(W * X), i.i.d. N(0, 1)."""
    return np.ascontiguousarray(np.random.default_rng(seed + 1).standard_normal((n, k)))


def random_spd_dense(n: int, seed: int = 0, cond: float = 100.0) -> np.ndarray:
    """Small dense SPD matrix with eigenvalues log-spaced in [1, cond] (for tiny oracle pins)."""
    rng = np.random.default_rng(seed + 2)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    A = (Qm * lam) @ Qm.T
    return 0.5 * (A + A.T)


def dense_to_csr(A: np.ndarray, drop: float = 0.0) -> CSRMatrix:
    n = A.shape[0]
    r, c = np.nonzero(np.abs(A) > drop)
    rowptr, colind, v = _assemble(n, r.astype(np.int64), c.astype(np.int64), A[r, c])
    return CSRMatrix(n, rowptr, colind, v, stencil=None, meta=dict(name=f"dense_{n}"))


# The five workloads of the benchmark table, by name. Sizes are the full ones; tests shrink them.
WORKLOADS = {
    "poisson2d_64_k8": dict(matrix=("poisson2d", 64), k=8, p=4, sub="hybrid", prec="fp64", tol=1e-8),
    "poisson3d_128_k32": dict(matrix=("poisson3d", 128), k=32, p=8, sub="hybrid", prec="fp64", tol=1e-8),
    "varcoef3d_160_k64": dict(matrix=("varcoef3d", 160), k=64, p=16, sub="hybrid", prec="fp32_refine",
                              tol=1e-10),
    "stencil27_100_k16": dict(matrix=("stencil27", 100), k=16, p=16, sub="hybrid", prec="fp64", tol=1e-8),
    "poisson3d_96_sweep": dict(matrix=("poisson3d", 96), k=(1, 8, 32, 128, 256), p="1,k/8,k",
                               sub="hybrid", prec=("fp64", "fp32_refine"), tol=1e-8),
}


def make_matrix(kind: str, size: int, seed: int = 0) -> CSRMatrix:
    if kind == "poisson2d":
        return poisson2d(size)
    if kind == "poisson3d":
        return poisson3d(size)
    if kind == "varcoef3d":
        return varcoef3d(size, seed=seed)
    if kind == "stencil27":
        return stencil27(size, seed=seed)
    if kind == "varcoef2d":
        return varcoef2d(size, seed=seed)
    raise ValueError(kind)
