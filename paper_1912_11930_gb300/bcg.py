"""Thin Python binding of libbcg.so (include/bcg.h): the same entry points under the same names,
argument marshalling only. Every step of the solver runs in the library's CUDA kernels; this module
never computes anything itself and raises if the library is missing.

Tensors are torch CUDA tensors (float64 for matrices and block vectors, int64 row pointers, int32 column
indices); block vectors are row-major n x k and must be contiguous.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbcg.so")

OK, INVALID_ARG, CUDA_ERR, OOM, BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT, GUARD = range(9)
STATUS_NAMES = ["OK", "INVALID_ARG", "CUDA", "OOM", "BREAKDOWN", "NOT_CONVERGED", "NUMERIC", "TIMEOUT", "GUARD"]
SUBALGEBRA = {"hybrid": 0, "global": 1, "parallel": 2, "classical": 3}
PRECISION = {"fp64": 0, "fp32_refine": 1, "fp64_df": 2}
STENCIL = {"5pt_2d": 0, "7pt_3d": 1, "7pt_3d_varcoef": 2}

_lib = None


class bcg_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("breakdown_iter", ctypes.c_int32), ("max_rel_res_recursive", ctypes.c_double),
                ("max_rel_res_true", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BCGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status


def load():
    """Load libbcg.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "bcg_create_csr": [ctypes.POINTER(vp), i64, i64, vp, vp, vp, i32, i32, i32, i32, vp],
        "bcg_create_stencil": [ctypes.POINTER(vp), i32, i32, i32, i32, vp, dbl, i32, i32, i32, i32, vp],
        "bcg_set_option": [vp, ctypes.c_char_p, dbl],
        "bcg_solve": [vp, vp, vp, dbl, i32, ctypes.POINTER(bcg_info)],
        "bcg_solve_host": [vp, vp, vp, dbl, i32, ctypes.POINTER(bcg_info)],
        "bcg_block_iters": [vp, ctypes.POINTER(i32), i32],
        "bcg_grad_values": [vp, vp, vp, vp],
        "bcg_update_values": [vp, vp],
        "bcg_bop": [vp, vp, vp],
        "bcg_bdot": [vp, vp, vp, vp],
        "bcg_bdot_f32": [vp, vp, vp, vp],
        "bcg_bdot_noalloc": [i64, i32, i32, i32, vp, vp, vp, vp],
        "bcg_profile": [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64), i32],
        "bcg_create_sell": [ctypes.POINTER(vp), i64, i64, vp, vp, vp, vp, vp, i32, i32, i32, i32, vp],
        "bcg_create_csr_rows": [ctypes.POINTER(vp), i64, i64, i64, vp, vp, vp, i32, i32, i32, vp],
        "bcg_rows_bind": [vp, vp, vp],
        "bcg_rows_unpack": [vp, vp, i64],
        "bcg_rows_start": [vp, vp, vp, dbl],
        "bcg_rows_start_status": [vp],
        "bcg_rows_phase": [vp, i32],
        "bcg_rows_pack": [vp, vp, i64, vp],
        "bcg_rows_poll": [vp, ctypes.POINTER(i32)],
        "bcg_rows_finish": [vp, ctypes.POINTER(bcg_info)],
        "bcg_debug_fail_alloc": [i32],
        "bcg_debug_poke_guard": [vp, i32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bcg_last_error.argtypes = []
    lib.bcg_last_error.restype = ctypes.c_char_p
    lib.bcg_destroy.argtypes = [vp]
    lib.bcg_destroy.restype = None
    _lib = lib
    return lib


def bcg_debug_fail_alloc(nth: int):
    """Make the nth device workspace allocation from now on fail with OOM (0 disarms); for error-path tests."""
    _check(load().bcg_debug_fail_alloc(int(nth)))


def bcg_debug_poke_guard(h, index: int):
    """Overwrite one guard byte after workspace buffer `index` of handle h; for tests of option "guards"."""
    _check(load().bcg_debug_poke_guard(h, int(index)))


def bcg_last_error() -> str:
    return load().bcg_last_error().decode(errors="replace")


def _check(status: int, allow=()):
    if status != OK and status not in allow:
        raise BCGError(status, bcg_last_error())
    return status


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    return None if stream is None else ctypes.c_void_p(stream.cuda_stream)


def bcg_create_csr(n, nnz, rowptr, colind, vals, k, p, sub, prec, stream=None):
    h = ctypes.c_void_p()
    _check(load().bcg_create_csr(ctypes.byref(h), n, nnz, _ptr(rowptr), _ptr(colind), _ptr(vals), k, p,
                                 SUBALGEBRA.get(sub, sub), PRECISION.get(prec, prec), _stream(stream)))
    return h


def bcg_create_stencil(kind, nx, ny, nz, coef, scale, k, p, sub, prec, stream=None):
    h = ctypes.c_void_p()
    _check(load().bcg_create_stencil(ctypes.byref(h), STENCIL.get(kind, kind), nx, ny, nz, _ptr(coef), scale, k, p,
                                     SUBALGEBRA.get(sub, sub), PRECISION.get(prec, prec), _stream(stream)))
    return h


def bcg_create_sell(n, nent, chunkptr, rowlen, colind, vals, perm, k, p, sub, prec, stream=None):
    h = ctypes.c_void_p()
    _check(load().bcg_create_sell(ctypes.byref(h), n, nent, _ptr(chunkptr), _ptr(rowlen), _ptr(colind), _ptr(vals),
                                  _ptr(perm), k, p, SUBALGEBRA.get(sub, sub), PRECISION.get(prec, prec),
                                  _stream(stream)))
    return h


def bcg_create_csr_rows(n_local, n_cols, nnz, rowptr, colind, vals, k, p, sub, stream=None):
    h = ctypes.c_void_p()
    _check(load().bcg_create_csr_rows(ctypes.byref(h), n_local, n_cols, nnz, _ptr(rowptr), _ptr(colind), _ptr(vals),
                                      k, p, SUBALGEBRA.get(sub, sub), _stream(stream)))
    return h


def bcg_rows_bind(h, sums1, sums2):
    _check(load().bcg_rows_bind(h, _ptr(sums1), _ptr(sums2)))


def bcg_rows_unpack(h, halo, nrows):
    _check(load().bcg_rows_unpack(h, _ptr(halo), nrows))


def bcg_rows_start(h, B, X, tol):
    _check(load().bcg_rows_start(h, _ptr(B), _ptr(X), tol))


def bcg_rows_start_status(h):
    _check(load().bcg_rows_start_status(h))


def bcg_rows_phase(h, phase):
    _check(load().bcg_rows_phase(h, phase))


def bcg_rows_pack(h, rows, nrows, buf):
    _check(load().bcg_rows_pack(h, _ptr(rows), nrows, _ptr(buf)))


def bcg_rows_poll(h):
    done = ctypes.c_int32()
    _check(load().bcg_rows_poll(h, ctypes.byref(done)))
    return bool(done.value)


def bcg_rows_finish(h):
    info = bcg_info()
    st = _check(load().bcg_rows_finish(h, ctypes.byref(info)), allow=(BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT))
    return st, info


def bcg_set_option(h, key: str, value: float):
    _check(load().bcg_set_option(h, key.encode(), float(value)))


def bcg_solve(h, B, X, tol, maxit):
    """Returns (status, info); raises only for INVALID_ARG / CUDA / OOM."""
    info = bcg_info()
    st = _check(load().bcg_solve(h, _ptr(B), _ptr(X), tol, maxit, ctypes.byref(info)),
                allow=(BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT))
    return st, info


def bcg_solve_host(h, B, X, tol, maxit):
    """B, X: C-contiguous float64 numpy arrays (host memory, ideally pinned)."""
    info = bcg_info()
    st = _check(load().bcg_solve_host(h, ctypes.c_void_p(B.ctypes.data), ctypes.c_void_p(X.ctypes.data), tol, maxit,
                                      ctypes.byref(info)), allow=(BREAKDOWN, NOT_CONVERGED, NUMERIC, TIMEOUT))
    return st, info


def bcg_block_iters(h, nblk):
    out = (ctypes.c_int32 * nblk)()
    _check(load().bcg_block_iters(h, out, nblk))
    return list(out)


def bcg_grad_values(h, Lam, X, grad):
    _check(load().bcg_grad_values(h, _ptr(Lam), _ptr(X), _ptr(grad)))


def bcg_update_values(h, vals):
    _check(load().bcg_update_values(h, _ptr(vals)))


def bcg_bop(h, X, Y):
    _check(load().bcg_bop(h, _ptr(X), _ptr(Y)))


def bcg_bdot(h, X, Y, gamma):
    _check(load().bcg_bdot(h, _ptr(X), _ptr(Y), _ptr(gamma)))


def bcg_bdot_f32(h, X, Y, gamma):
    _check(load().bcg_bdot_f32(h, _ptr(X), _ptr(Y), _ptr(gamma)))


def bcg_bdot_noalloc(n, k, p, sub, X, Y, gamma, stream=None):
    """Allocation-free BDOT (static device scratch); stream-ordered, returns once enqueued."""
    _check(load().bcg_bdot_noalloc(n, k, p, SUBALGEBRA.get(sub, sub), _ptr(X), _ptr(Y), _ptr(gamma),
                                   _stream(stream)))


KERNEL_NAMES = ["op_gram", "solve_lambda", "update_xr", "solve_beta", "update_p", "residual", "tc_gram", "tc_baxpy"]


def bcg_profile(h):
    """{kernel: (total_ms, launches)} of the profiled iterations since profiling was enabled."""
    nk = len(KERNEL_NAMES)
    ms = (ctypes.c_double * nk)()
    cnt = (ctypes.c_int64 * nk)()
    _check(load().bcg_profile(h, ms, cnt, nk))
    return {KERNEL_NAMES[i]: (ms[i], cnt[i]) for i in range(nk)}


def bcg_destroy(h):
    if h is not None and h.value:
        load().bcg_destroy(h)


# ----------------------------------------------------------------------------------------------------
@dataclass
class SolveResult:
    status: int
    iters: int
    outer_iters: int
    breakdown_iter: int
    max_rel_res_recursive: float
    max_rel_res_true: float
    block_iters: list

    @property
    def ok(self):
        return self.status == OK


class Solver:
    """Owns a handle plus the tensors it borrows, and a private CUDA stream (so iteration batches can be
    replayed as CUDA graphs). Calls are ordered after torch's current stream and torch's current stream
    waits for them."""

    def __init__(self, *, k, p=1, sub="hybrid", prec="fp64", csr=None, stencil=None, sell=None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.stream = torch.cuda.Stream(device=self.device)
        self.k, self.sub, self.prec = k, sub, prec
        self.p = 1 if sub == "parallel" else (k if sub == "classical" else p)
        self.nblk = 1 if sub == "global" else k // self.p
        self._keep = []
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            if csr is not None:
                rowptr, colind, vals = csr
                self._keep += [rowptr, colind, vals]
                self.n = rowptr.numel() - 1
                self.nnz = colind.numel()
                self.h = bcg_create_csr(self.n, self.nnz, rowptr, colind, vals, k, p, sub, prec, self.stream)
            elif sell is not None:   # (chunkptr, rowlen, colind, vals, perm) device tensors
                chunkptr, rowlen, colind, vals, perm = sell
                self._keep += list(sell)
                self.n = rowlen.numel()
                self.nnz = vals.numel()
                self.h = bcg_create_sell(self.n, self.nnz, chunkptr, rowlen, colind, vals, perm, k, p, sub, prec,
                                         self.stream)
            else:
                kind, nx, ny, nz, coef, scale = stencil
                if coef is not None:
                    self._keep.append(coef)
                self.n = nx * ny * nz
                self.nnz = 0
                self.h = bcg_create_stencil(kind, nx, ny, nz, coef, scale, k, p, sub, prec, self.stream)

    @classmethod
    def from_matrix(cls, M, *, k, p=1, sub="hybrid", prec="fp64", form="csr", device=None, sigma=1):
        """M: a workloads.CSRMatrix; form 'csr', 'stencil' or 'sell' (SELL-C-sigma, sorting window sigma)."""
        import torch
        dev = torch.device(device or "cuda")
        if form == "sell":
            from .formats import sell_from_csr
            S = sell_from_csr(M.rowptr, M.colind, M.vals, sigma)
            sell = tuple(torch.from_numpy(a).to(dev) for a in (S.chunkptr, S.rowlen, S.colind, S.vals, S.perm))
            return cls(k=k, p=p, sub=sub, prec=prec, sell=sell, device=dev)
        if form == "csr":
            csr = (torch.from_numpy(M.rowptr).to(dev), torch.from_numpy(M.colind).to(dev),
                   torch.from_numpy(M.vals).to(dev))
            return cls(k=k, p=p, sub=sub, prec=prec, csr=csr, device=dev)
        s = M.stencil
        coef = None if s["coef"] is None else torch.from_numpy(s["coef"]).to(dev)
        return cls(k=k, p=p, sub=sub, prec=prec, stencil=(s["kind"], s["nx"], s["ny"], s["nz"], coef, s["scale"]),
                   device=dev)

    def set_option(self, key, value):
        bcg_set_option(self.h, key, value)

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def solve(self, B, X=None, tol=1e-8, maxit=10000) -> tuple:
        """Solve A X = B from X^0 = X (zeros if None). Returns (X, SolveResult)."""
        torch = self.torch
        if X is None:
            X = torch.zeros_like(B)
        self._enter()
        st, info = bcg_solve(self.h, B, X, tol, maxit)
        self._leave()
        return X, self._result(st, info)

    def solve_columns(self, B, X=None, tol=1e-8, maxit=10000):
        """Solve for K = r k right-hand sides with this k-column handle: r = K / k solves in sequence, one per
        group of k consecutive columns (the repetition schedule of the whole-solver experiment in Section 4,
        where 128 right-hand sides run as r = 128 / k block solves). B, X: n x K row-major device tensors;
        X is updated in place (zeros if None). Returns (X, [SolveResult per group])."""
        torch = self.torch
        K = B.shape[1]
        if K % self.k:
            raise BCGError(INVALID_ARG, f"{K} right-hand sides are not a multiple of the handle's k = {self.k}")
        if X is None:
            X = torch.zeros_like(B)
        results = []
        for g in range(K // self.k):
            cols = slice(g * self.k, (g + 1) * self.k)
            Xg = X[:, cols].contiguous()
            Xg, r = self.solve(B[:, cols].contiguous(), Xg, tol=tol, maxit=maxit)
            X[:, cols] = Xg
            results.append(r)
        return X, results

    def solve_host(self, B, X, tol=1e-8, maxit=10000):
        st, info = bcg_solve_host(self.h, B, X, tol, maxit)
        return X, self._result(st, info)

    def _result(self, st, info):
        return SolveResult(st, info.iters, info.outer_iters, info.breakdown_iter, info.max_rel_res_recursive,
                           info.max_rel_res_true, bcg_block_iters(self.h, self.nblk))

    def profile(self):
        return bcg_profile(self.h)

    def bop(self, X):
        Y = self.torch.empty_like(X)
        self._enter()
        bcg_bop(self.h, X, Y)
        self._leave()
        return Y

    def bdot(self, X, Y):
        """gamma = <<X, Y>>_S as a (nblk, p, p) float64 tensor."""
        g = self.torch.empty(self.nblk, self.p, self.p, dtype=self.torch.float64, device=self.device)
        self._enter()
        (bcg_bdot_f32 if X.dtype == self.torch.float32 else bcg_bdot)(self.h, X, Y, g)
        self._leave()
        return g

    def grad_values(self, Lam, X):
        g = self.torch.empty(self.nnz, dtype=self.torch.float64, device=self.device)
        self._enter()
        bcg_grad_values(self.h, Lam, X, g)
        self._leave()
        return g

    def update_values(self, vals):
        self._keep.append(vals)
        self._enter()
        bcg_update_values(self.h, vals)
        self._leave()

    def close(self):
        if getattr(self, "h", None) is not None:
            bcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
