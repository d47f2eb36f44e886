"""Writes oracle_regression.json: fixed small cases of the CPU oracle (Algorithm 1 in the four
subalgebras, with M = I and M = diag(A), and the retooled form), recorded so that any later change to the
oracle's arithmetic shows up as a difference against this file. Calls only ``oracle/`` and the input
generators. Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bcg as O                      # noqa: E402
from paper_1912_11930_gb300 import workloads as W  # noqa: E402

# (name, matrix, solver, sub, k, p, precond, tol, maxit)
CASES = [
    ("p2d8_hybrid_k4p2_m5", "poisson2d_8", "bcg", "hybrid", 4, 2, "none", 0.0, 5),
    ("p2d8_global_k4p2_m5", "poisson2d_8", "bcg", "global", 4, 2, "none", 0.0, 5),
    ("p2d8_parallel_k3_m5", "poisson2d_8", "bcg", "parallel", 3, 1, "none", 0.0, 5),
    ("p2d8_classical_k4_m4", "poisson2d_8", "bcg", "classical", 4, 4, "none", 0.0, 4),
    ("vc2d9x7_hybrid_k4p2_jacobi_conv", "varcoef2d_9x7", "bcg", "hybrid", 4, 2, "jacobi", 1e-10, 500),
    ("s27_3_hybrid_k6p3_conv", "stencil27_3", "bcg", "hybrid", 6, 3, "none", 1e-10, 500),
    ("p2d8_retooled_hybrid_k4p2_m5", "poisson2d_8", "retooled", "hybrid", 4, 2, "none", 0.0, 5),
    ("p3d4_retooled_classical_k4_conv", "poisson3d_4", "retooled", "classical", 4, 4, "none", 1e-10, 500),
]
SAMPLE = 7   # every SAMPLE-th entry of X (row-major) is stored


def matrix(name):
    return {"poisson2d_8": lambda: W.poisson2d(8), "varcoef2d_9x7": lambda: W.varcoef2d(9, 7, seed=1),
            "stencil27_3": lambda: W.stencil27(3, seed=1), "poisson3d_4": lambda: W.poisson3d(4)}[name]()


def run(case):
    _, mname, solver, sub, k, p, precond, tol, maxit = case
    M = matrix(mname)
    B = W.rhs(M.n, k, seed=5)
    if solver == "bcg":
        return O.solve(M.to_scipy(), B, p=p, sub=sub, tol=tol, maxit=maxit, precond=precond)
    return O.solve_retooled(M.to_scipy(), B, p=p, sub=sub, tol=tol, maxit=maxit)


def record(res):
    return {"status": int(res.status), "iters": int(res.iters), "block_iters": [int(v) for v in res.block_iters],
            "x_sample": [float(v) for v in res.X.ravel()[::SAMPLE]],
            "relres_recursive": [float(v) for v in res.relres_recursive]}


if __name__ == "__main__":
    out = {"sample_stride": SAMPLE, "cases": {c[0]: record(run(c)) for c in CASES}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
