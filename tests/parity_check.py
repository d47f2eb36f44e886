"""Solution comparisons shared by the GPU parity tests.

Every solution is compared two ways: the relative Frobenius error ||X - X_ref|| / ||X_ref|| over the whole
block, and element by element, column by column, max_i |X_ic - X_ref,ic| / max_i |X_ref,ic|. A wrong tail row or
a single wrong entry hides in the first measure on a large block (67 M entries at 128^3, k = 32) but not in
the second."""
import numpy as np


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_elem(a, b):
    """Largest over columns of the max-norm error of the column relative to the column's max norm (columns
    where b is zero: the absolute error)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    if a.shape != b.shape:
        raise ValueError(f"shapes differ: {a.shape} {b.shape}")
    den = np.max(np.abs(b), axis=0)
    num = np.max(np.abs(a - b), axis=0)
    if not np.all(np.isfinite(num)):
        return float("inf")
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def assert_close(a, b, tol, what=""):
    """Both measures at most tol."""
    f, e = rel_fro(a, b), rel_elem(a, b)
    assert f <= tol and e <= tol, f"{what} relative error {f:.3e} (Frobenius), {e:.3e} (element-wise), bar {tol:g}"
