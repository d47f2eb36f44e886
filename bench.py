#!/usr/bin/env python
"""Benchmark of the block CG hot path: time-to-tolerance of one solve (a "step" = one full solve from
X^0 = 0 to every column's relative residual <= 1e-8), per-iteration HBM traffic and the roofline of the
dominant kernel, measured live with CUDA events on the solver's stream.

Default workload: 3D 7-point Poisson 128^3 (n = 2,097,152, CSR), k = 32 right-hand sides i.i.d. N(0,1),
hybrid subalgebra p = 8, FP64, tol 1e-8. At N > 1 GPUs every rank solves its own 32 right-hand sides
(seed + rank; hybrid blocks are independent, so no data-path collective) and the job time is the max over
ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-variants]

--impl reference times the CPU oracle (the only reference this method has) on a bounded sample of the
same workload and prints the same line with "impl": "reference".
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BCG time-to-1e-8 rel. residual; HBM GB/s/iter vs roofline; mixed vs FP64"
NOMINAL_FP64_TFLOPS = 1.25          # GB300 FP64 (vector and tensor) per GPU, nominal
WORKLOAD = dict(name="poisson3d_128_csr_k32_hybrid_p8_fp64", grid=128, k=32, p=8, sub="hybrid", prec="fp64",
                tol=1e-8)
# Iterations the 128^3 / k = 32 / hybrid p = 8 FP64 solve takes to reach 1e-8 (measured on the GPU; the oracle
# agrees within +-2 on every size it can finish). Used only to extrapolate the oracle's per-iteration time
# to a time-to-tolerance in the reference arm.
REF_ITERS = 354
ORACLE_SAMPLE_ITERS = 3
# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture at 96^3 (profiles/<kernel>_poisson3d_96_*.md), scaled by rows to the 128^3 launch. Valid only for the
# device source the capture was taken on: sha256 prefix of the files that define the kernel (its body, the
# helpers it calls and its launcher), concatenated; reported as null once one of them changes.
UPDATE_XR_SOURCES = ("bcg_kernels.cuh", "bcg_kernels_wc.cuh", "bcg_stream.inc")
TRAFFIC = {("update_xr", "poisson3d_128_csr_k32_hybrid_p8_fp64"):
           (UPDATE_XR_SOURCES, "88cc6866fc22b045", 1.3264e9 * 2097152 / 884736)}


def kernel_source_sha(files):
    import hashlib
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_1912_11930_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6782.1)), "measured"
    except Exception:
        return 6800.0, "fallback"


def rho_in_k3(k, p, prec):
    """Where the library forms the recomputed rho (the dispatch rule rho_in_k3 of its streaming kernels):
    in K3 of the previous iteration for FP64 with 2 <= p <= 16 in the warp-chunk layout (k even, and k | 32,
    or 32 | k with k / 32 | 8 and p | 32); in K1 otherwise."""
    wc = k <= 256 and k % 2 == 0 and (32 % k == 0 or (k % 32 == 0 and 8 % (k // 32) == 0 and 32 % p == 0))
    return prec in ("fp64", "fp64_df") and 2 <= p <= 16 and wc


def kernel_model(n, k, p, z, s, a_bytes, rho_k3=False, df=False):
    """Algorithmic flops and bytes per launch of each iteration kernel (the paper's Table 1 omega and beta per
    kernel, fused as the kernels fuse them): K1 = BOP + BDOT alpha (+ BDOT of the recomputed rho, reading R),
    K2 = 2 BAXPY + BDOT + column norms, K3 = BAXPY (+ the next recomputed rho when rho_k3: R is read there
    anyway). `alu` is the part executed as native arithmetic of the block vectors' precision (BOP and
    BAXPY: FP64 FMAs in the FP64 form, FP32 FMAs in the mixed form); `gram` is the block-product part,
    which runs as error-free (Dot2) FP32 arithmetic with FP64-class accuracy in both forms. With `df` (the
    double-float residual update of precision fp64_df) K2's `alu` is X's FMAs plus one FP64 addition per
    element of R, and R's 2 n p k flops move to `df`, summed in float pairs on the FP32 pipes."""
    k1_grams = 1.0 if rho_k3 else 2.0
    upd_alu = 2.0 * n * p * k + n * k if df else 4.0 * n * p * k
    return {
        "op_gram": dict(alu=2.0 * k * z, gram=k1_grams * 2.0 * n * p * k,
                        bytes=a_bytes + (2.0 if rho_k3 else 3.0) * n * k * s),
        "update_xr": dict(alu=upd_alu, gram=2.0 * n * p * k + 2.0 * n * k, bytes=6.0 * n * k * s,
                          df=2.0 * n * p * k if df else 0.0),
        "update_p": dict(alu=2.0 * n * p * k, gram=2.0 * n * p * k if rho_k3 else 0.0, bytes=3.0 * n * k * s),
    }


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows)}


def oracle_sample(grid, k, p, sub, iters, seed, threads=1):
    """Time the CPU oracle on `iters` iterations of the workload in a fresh process limited to `threads` BLAS /
    OpenMP threads. Returns (seconds per iteration, seconds of the sample)."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
from oracle import bcg as O
from paper_1912_11930_gb300 import workloads as W
M = W.poisson3d({grid})
A = M.to_scipy()
B = W.rhs(M.n, {k}, seed={seed})
t0 = time.perf_counter()
O.solve(A, B, p={p}, sub={sub!r}, tol=0.0, maxit=1)
t1 = time.perf_counter()
O.solve(A, B, p={p}, sub={sub!r}, tol=0.0, maxit={1 + iters})
t2 = time.perf_counter()
print(json.dumps(dict(per_iter=((t2 - t1) - (t1 - t0)) / {iters}, first=t1 - t0, total=t2 - t0)))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = WORKLOAD
    iters_to_tol = REF_ITERS
    samples = []
    for _ in range(args.warmup + args.steps):
        samples.append(oracle_sample(w["grid"], w["k"], w["p"], w["sub"], 1, seed=0))
    timed = samples[args.warmup:]
    per_iter = sum(s["per_iter"] for s in timed) / len(timed)
    first = sum(s["first"] for s in timed) / len(timed)
    value = first + per_iter * iters_to_tol if iters_to_tol else None
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None if value is None else value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "n": w["grid"] ** 3, "k": w["k"], "p": w["p"],
                       "subalgebra": w["sub"], "tol": w["tol"]},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: 1 oracle iteration of the full workload (plus the initial "
                                       f"residual), single-threaded; time-to-tolerance = initial residual + "
                                       f"per-iteration time x {iters_to_tol} iterations"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------------
# Other workloads (not the default line): measured with `python bench.py --workload NAME`
EXTRA_WORKLOADS = ("poisson2d_64_k8", "varcoef3d_160_k64_mixed", "varcoef3d_160_k64_jacobi", "stencil27_100_k16_autograd",
                   "poisson3d_96_sweep", "sell_vs_csr", "large_blocks_64_k256", "blocks32_96_k256",
                   "retooled_128_k32", "repetitions_varcoef2d_512_128rhs")


def time_solve(bcg, torch, M, B, *, k, p, sub, prec, form="csr", tol=1e-8, reps=2, dev=None, opts=None, warm=True,
               maxit=20000):
    """Warm-up solve (unless warm=False), then the mean of `reps` timed solves from X0 = 0 (CUDA events on the
    solver's stream)."""
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec=prec, form=form, device=dev)
    for key, v in (opts or {}).items():
        S.set_option(key, v)
    X = torch.zeros_like(B)
    if warm:
        S.solve(B, X, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(S.stream)
    for _ in range(reps):
        with torch.cuda.stream(S.stream):
            X.zero_()
        X, r = S.solve(B, X, tol=tol, maxit=maxit)
    e1.record(S.stream)
    torch.cuda.synchronize()
    S.close()
    return e0.elapsed_time(e1) / reps / 1e3, r, X


def run_extra(name, args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_11930_gb300 import bcg, workloads as W
    dev = torch.device("cuda", 0)
    base = {"metric": METRIC, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    out = dict(base)
    if name == "poisson2d_64_k8":
        M = W.poisson2d(64)
        B = torch.from_numpy(W.rhs(M.n, 8, seed=0)).to(dev)
        rows = []
        for sub, p in (("hybrid", 4), ("global", 4), ("parallel", 1), ("classical", 8), ("hybrid", 1)):
            t, r, _ = time_solve(bcg, torch, M, B, k=8, p=p, sub=sub, prec="fp64", reps=args.steps, dev=dev)
            rows.append(dict(sub=sub, p=p, s=t, iterations=r.iters, status=bcg.STATUS_NAMES[r.status],
                             max_rel_res_true=r.max_rel_res_true))
        out.update(value=rows[0]["s"], dtype="f64", config={"workload": "poisson2d_64_csr_k8", "n": M.n, "k": 8},
                   results=rows)
    elif name == "varcoef3d_160_k64_mixed":
        M = W.varcoef3d(160, seed=0)
        k = 64
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows = []
        for prec, tol in (("fp32_refine", 1e-10), ("fp32_refine", 1e-8), ("fp64", 1e-8)):
            t, r, _ = time_solve(bcg, torch, M, B, k=k, p=16, sub="hybrid", prec=prec, form="stencil", tol=tol,
                                 reps=1, dev=dev)
            rows.append(dict(prec=prec, tol=tol, s=t, iterations=r.iters, outer=r.outer_iters,
                             status=bcg.STATUS_NAMES[r.status], max_rel_res_true=r.max_rel_res_true))
        out.update(value=rows[0]["s"], dtype="f32 inner, f64 refinement",
                   config={"workload": "varcoef3d_160_stencil_k64_hybrid_p16", "n": M.n, "k": k, "p": 16},
                   results=rows, mixed_vs_fp64_speedup_at_1e8=rows[2]["s"] / rows[1]["s"])
    elif name == "varcoef3d_160_k64_jacobi":
        # the log-normal coefficients' contrast is what a diagonal preconditioner removes: M = I against
        # M = diag(A), FP64 and the mixed form, time to 1e-8
        M = W.varcoef3d(160, seed=0)
        k = 64
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows = []
        for prec in ("fp64", "fp32_refine"):
            for pre in (0, 1):
                t, r, _ = time_solve(bcg, torch, M, B, k=k, p=16, sub="hybrid", prec=prec, form="stencil", tol=1e-8,
                                     reps=1, dev=dev, opts={"precond": pre})
                rows.append(dict(prec=prec, precond="jacobi" if pre else "none", s=t, iterations=r.iters,
                                 outer=r.outer_iters, status=bcg.STATUS_NAMES[r.status],
                                 max_rel_res_true=r.max_rel_res_true))
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        out.update(value=rows[1]["s"], dtype="f64 (and f32 inner, f64 refinement)",
                   config={"workload": "varcoef3d_160_stencil_k64_hybrid_p16_jacobi", "n": M.n, "k": k, "p": 16},
                   results=rows, jacobi_speedup_fp64=rows[0]["s"] / rows[1]["s"],
                   jacobi_speedup_mixed=rows[2]["s"] / rows[3]["s"])
    elif name == "sell_vs_csr":
        # BOP (inside K1) with the matrix in CSR and in SELL-C-sigma: the 128^3 Poisson matrix and an SPD matrix
        # with very uneven rows (2M rows, power-law degrees); K1 time per iteration from the live profile
        rows = []
        for mname, M in (("poisson3d_128", W.poisson3d(128)), ("powerlaw_2M", W.powerlaw_laplacian(1 << 21))):
            for k, p, sub in ((1, 1, "parallel"), (8, 8, "hybrid"), (32, 8, "hybrid")):
                B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
                for form, sigma in (("csr", 1), ("sell", 1), ("sell", 4096)):
                    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=sub, prec="fp64", form=form, device=dev, sigma=sigma)
                    X = torch.zeros_like(B)
                    S.solve(B, X, tol=1e-300, maxit=8)
                    S.set_option("profile", 1)
                    X.zero_()
                    S.solve(B, X, tol=1e-300, maxit=24)
                    tot, cnt = S.profile()["op_gram"]
                    S.close()
                    rows.append(dict(matrix=mname, k=k, p=p, format=form, sigma=sigma, k1_ms=tot / max(cnt, 1)))
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                del B
        out.update(value=rows[0]["k1_ms"] / 1e3, unit="s", dtype="f64",
                   config={"workload": "sell_vs_csr_k1_time", "iterations_profiled": 24}, results=rows,
                   note="value: K1 time of the first row (128^3 Poisson, k = 1, CSR), seconds per launch")
    elif name == "large_blocks_64_k256":
        # classical block CG with k = p = 256 (tiled kernels, p x p solves in global memory): 24 iterations of
        # each form, for the large-block launch profile
        M = W.poisson3d(64)
        k = 256
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows = []
        for prec, tc in (("fp64", 1), ("fp64", 0), ("fp32_refine", 1)):
            t, r, _ = time_solve(bcg, torch, M, B, k=k, p=k, sub="classical", prec=prec, tol=1e-300, reps=1, dev=dev,
                                 warm=False, maxit=24, opts={"tensor_cores": tc})
            rows.append(dict(prec=prec, tensor_cores=tc, s=t, iterations=r.iters, status=bcg.STATUS_NAMES[r.status],
                             ms_per_iteration=t * 1e3 / max(r.iters, 1)))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        # the tensor-core kernels alone (option "profile": each launch bracketed by CUDA events), 6 iterations, and
        # their throughput against the measured dense bf16 peak: each launch does 2 n p^2 FP64-accurate products
        # per block as 36 bf16 digit-pair products
        S = bcg.Solver.from_matrix(M, k=k, p=k, sub="classical", prec="fp64", device=dev)
        S.set_option("profile", 1)
        X = torch.zeros_like(B)
        S.solve(B, X, tol=1e-300, maxit=6)
        prof = S.profile()
        S.close()
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                bf16 = float(json.load(fh)["bf16_tflops"])
            src = "measured burst"
        except Exception:
            bf16, src = 1900.0, "fallback"
        flop = 2.0 * M.n * k * k * 36
        tc = {}
        for name in ("tc_gram", "tc_baxpy"):
            tot, cnt = prof[name]
            if cnt:
                avg = tot / cnt
                tc[name] = {"avg_ms": avg, "launches": cnt, "bf16_tflops": flop / (avg * 1e-3) / 1e12,
                            "frac_of_bf16_peak": flop / (avg * 1e-3) / 1e12 / bf16, "bf16_peak": bf16,
                            "peak_source": src}
        out.update(value=rows[0]["s"], dtype="f64 (and f32 with f64 residual replacement)",
                   config={"workload": "poisson3d_64_csr_k256_classical_24_iterations", "n": M.n, "k": k, "p": k},
                   results=rows, tensor_core_kernels=tc)
    elif name == "blocks32_96_k256":
        # hybrid blocks of 32 at k = 256 (FP64): 24 iterations with the block updates on the tensor cores (two blocks
        # per 64-column tile) and 24 on the warp-chunk FMA kernels, for the launch profile of that path
        M = W.poisson3d(96)
        k, p = 256, 32
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows = []
        for tc in (1, 0):
            t, r, _ = time_solve(bcg, torch, M, B, k=k, p=p, sub="hybrid", prec="fp64", tol=1e-300, reps=1, dev=dev,
                                 warm=False, maxit=24, opts={"tensor_cores": tc})
            rows.append(dict(prec="fp64", tensor_cores=tc, s=t, iterations=r.iters, status=bcg.STATUS_NAMES[r.status],
                             ms_per_iteration=t * 1e3 / max(r.iters, 1)))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        out.update(value=rows[0]["s"], dtype="f64",
                   config={"workload": "poisson3d_96_csr_k256_hybrid_p32_24_iterations", "n": M.n, "k": k, "p": p},
                   results=rows)
    elif name == "retooled_128_k32":
        # Dubrulle's retooled block CG against Algorithm 1 (FP64): the 128^3 Poisson solve to 1e-8, the same with
        # the right-hand side's columns scaled from 1e-6 to 1e6 inside every block of 8 (Algorithm 1 breaks down
        # there), and 24 iterations of the k = p = 256 classical solve at 64^3 (tiled large-block path)
        rows = []
        M = W.poisson3d(128)
        k, p = 32, 8
        B0 = W.rhs(M.n, k, seed=0)
        d = np.tile(10.0 ** np.linspace(-6, 6, p), k // p)
        for scaled in (False, True):
            B = torch.from_numpy(B0 * d[None, :] if scaled else B0).to(dev)
            for rt in (0, 1):
                t, r, _ = time_solve(bcg, torch, M, B, k=k, p=p, sub="hybrid", prec="fp64", reps=args.steps, dev=dev,
                                     opts={"retooled": rt})
                rows.append(dict(matrix="poisson3d_128", k=k, p=p, columns="scaled 1e-6..1e6" if scaled else "N(0,1)",
                                 form="retooled" if rt else "algorithm1", s=t, iterations=r.iters,
                                 status=bcg.STATUS_NAMES[r.status], breakdown_iter=r.breakdown_iter,
                                 ms_per_iteration=t * 1e3 / max(r.iters, 1), max_rel_res_true=r.max_rel_res_true))
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del B
        M = W.poisson3d(64)
        B = torch.from_numpy(W.rhs(M.n, 256, seed=0)).to(dev)
        for rt in (0, 1):
            t, r, _ = time_solve(bcg, torch, M, B, k=256, p=256, sub="classical", prec="fp64", tol=1e-300, reps=1,
                                 dev=dev, warm=False, maxit=24, opts={"retooled": rt})
            rows.append(dict(matrix="poisson3d_64", k=256, p=256, form="retooled" if rt else "algorithm1", s=t,
                             iterations=r.iters, ms_per_iteration=t * 1e3 / max(r.iters, 1)))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        out.update(value=rows[1]["s"], dtype="f64",
                   config={"workload": "poisson3d_128_csr_k32_hybrid_p8_retooled", "n": 128 ** 3, "k": k, "p": p},
                   results=rows, note="value: time to 1e-8 of the retooled form on the N(0,1) right-hand side")
    elif name == "repetitions_varcoef2d_512_128rhs":
        # the repetition study of Section 4: 128 right-hand sides solved as r = 128 / k block solves of k columns
        # (p = 16), on a 2D heterogeneous 5-point problem (512^2, log-normal face coefficients) with the Jacobi
        # preconditioner standing in for the paper's ILU; time to 1e-8 for all 128 columns
        M = W.varcoef2d(512, seed=0)
        K, p = 128, 16
        B = torch.from_numpy(W.rhs(M.n, K, seed=0)).to(dev)
        rows = []
        for prec in ("fp64", "fp32_refine"):
            for k in (16, 32, 64, 128):
                S = bcg.Solver.from_matrix(M, k=k, p=p, sub="hybrid", prec=prec, device=dev)
                S.set_option("precond", 1)
                S.solve_columns(B[:, :k], tol=1e-300, maxit=16)   # warm-up: kernels, graphs
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                X, res = S.solve_columns(B, tol=1e-8, maxit=20000)
                e1.record()
                torch.cuda.synchronize()
                S.close()
                rows.append(dict(prec=prec, k=k, p=p, r=K // k, s=e0.elapsed_time(e1) / 1e3,
                                 iterations=[x.iters for x in res], status=[bcg.STATUS_NAMES[x.status] for x in res],
                                 max_rel_res_true=max(x.max_rel_res_true for x in res)))
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        out.update(value=rows[0]["s"], dtype="f64 (and f32 inner, f64 residual replacement)",
                   config={"workload": "varcoef2d_512_csr_128rhs_hybrid_p16_jacobi_repetitions", "n": M.n,
                           "rhs": K, "p": p}, results=rows,
                   note="value: FP64, k = 16 (r = 8 solves); every row solves all 128 columns to 1e-8")
    elif name == "stencil27_100_k16_autograd":
        from paper_1912_11930_gb300.autograd import bcg_solve_autograd
        M = W.stencil27(100, seed=0)
        k = 16
        vals = torch.from_numpy(M.vals.copy()).to(dev).requires_grad_(True)
        csr = (torch.from_numpy(M.rowptr).to(dev), torch.from_numpy(M.colind).to(dev), vals)
        S = bcg.Solver(k=k, p=16, sub="hybrid", csr=csr, device=dev)
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev).requires_grad_(True)
        Wt = torch.from_numpy(W.loss_weights(M.n, k, seed=0)).to(dev)
        times = []
        for rep in range(1 + args.steps):
            vals.grad = None
            B.grad = None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X = bcg_solve_autograd(vals, B, S, tol=1e-8)
            loss = (Wt * X).sum()
            loss.backward()
            torch.cuda.synchronize()
            if rep:
                times.append(time.perf_counter() - t0)
        S.close()
        out.update(value=sum(times) / len(times), dtype="f64",
                   config={"workload": "stencil27_100_csr_k16_hybrid_p16_forward_backward", "n": M.n, "k": k,
                           "nnz": M.nnz}, note="one forward solve + adjoint solve + gradient kernel, tol 1e-8")
    elif name == "poisson3d_96_sweep":
        M = W.poisson3d(96)
        rows = []
        for k in (1, 8, 32, 128, 256):
            B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
            for p in sorted({1, max(1, k // 8), k}):
                for prec in ("fp64", "fp32_refine"):
                    sub = "hybrid"
                    t, r, _ = time_solve(bcg, torch, M, B, k=k, p=p, sub=sub, prec=prec, reps=1, dev=dev,
                                         warm=k * p <= 32 * 32)
                    rows.append(dict(k=k, p=p, prec=prec, s=t, iterations=r.iters, outer=r.outer_iters,
                                     status=bcg.STATUS_NAMES[r.status], max_rel_res_true=r.max_rel_res_true,
                                     s_per_rhs=t / k))
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del B
        out.update(value=next(x["s"] for x in rows if x["k"] == 32 and x["p"] == 4 and x["prec"] == "fp64"),
                   dtype="f64 and f32 inner/f64 refinement", config={"workload": "poisson3d_96_csr_sweep",
                                                                     "n": M.n}, results=rows)
    print(json.dumps(out), flush=True)


def config_variants(bcg, W, torch, dev, np):
    """The other configurations of the benchmark, one solve each (after the timed line; CUDA events on the solver's
    stream): 2D 64^2 in three subalgebras; the 160^3 variable-coefficient problem in the mixed form (to 1e-10 and
    1e-8) and in FP64 (to 1e-8); the differentiable 100^3 27-point solve (forward, adjoint, gradient); k = 256 at
    96^3 for p = 1, 32, 256 in FP64 and in the mixed form. Every mixed or double-float result carries its relative
    error against the FP64 solve of the same system (the FP64 form is parity-tested against the oracle)."""
    out = {}

    def rel_errs(Xa, Xb):
        a, b = Xa.cpu().numpy(), Xb.cpu().numpy()
        return {"rel_err_vs_fp64": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                "rel_err_vs_fp64_elementwise": float(np.max(np.max(np.abs(a - b), axis=0) /
                                                            np.maximum(np.max(np.abs(b), axis=0), 1e-300)))}

    def row(t, r, **kw):
        d = dict(kw, s=t, iterations=r.iters, outer=r.outer_iters, status=bcg.STATUS_NAMES[r.status],
                 max_rel_res_true=r.max_rel_res_true)
        print(json.dumps(d), file=sys.stderr, flush=True)
        return d

    def guarded(name, fn):
        try:
            out[name] = fn()
        except Exception as e:   # a failing variant must not take the default line with it
            out[name] = {"error": f"{type(e).__name__}: {e}"}

    def cfg1():
        M = W.poisson2d(64)
        B = torch.from_numpy(W.rhs(M.n, 8, seed=0)).to(dev)
        rows = []
        for sub, p in (("hybrid", 4), ("global", 4), ("parallel", 1)):
            t, r, _ = time_solve(bcg, torch, M, B, k=8, p=p, sub=sub, prec="fp64", reps=3, dev=dev)
            rows.append(row(t, r, sub=sub, p=p, prec="fp64", tol=1e-8))
        return {"workload": "poisson2d_64_csr_k8", "n": M.n, "results": rows}

    def cfg3():
        M = W.varcoef3d(160, seed=0)
        k, p = 64, 16
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows, X = [], {}
        for prec, tol in (("fp64", 1e-8), ("fp32_refine", 1e-8), ("fp32_refine", 1e-10)):
            t, r, Xr = time_solve(bcg, torch, M, B, k=k, p=p, sub="hybrid", prec=prec, form="stencil", tol=tol, reps=1,
                                  dev=dev, warm=False)
            rows.append(row(t, r, prec=prec, tol=tol))
            if prec != "fp64":
                rows[-1].update(rel_errs(Xr, X["fp64"]))
            else:
                X["fp64"] = Xr
        del B, X
        return {"workload": "varcoef3d_160_stencil_k64_hybrid_p16", "n": M.n, "results": rows,
                "mixed_vs_fp64_speedup_at_1e8": rows[0]["s"] / rows[1]["s"]}

    def cfg4():
        from paper_1912_11930_gb300.autograd import bcg_solve_autograd
        M = W.stencil27(100, seed=0)
        k = 16
        vals = torch.from_numpy(M.vals.copy()).to(dev).requires_grad_(True)
        csr = (torch.from_numpy(M.rowptr).to(dev), torch.from_numpy(M.colind).to(dev), vals)
        S = bcg.Solver(k=k, p=16, sub="hybrid", csr=csr, device=dev)
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev).requires_grad_(True)
        Wt = torch.from_numpy(W.loss_weights(M.n, k, seed=0)).to(dev)
        times = []
        for rep in range(2):
            vals.grad = None
            B.grad = None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X = bcg_solve_autograd(vals, B, S, tol=1e-8)
            (Wt * X).sum().backward()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        S.close()
        return {"workload": "stencil27_100_csr_k16_hybrid_p16_forward_adjoint_gradient", "n": M.n, "nnz": M.nnz,
                "s": times[-1], "note": "forward solve + adjoint solve + gradient kernel, tol 1e-8 (second run)"}

    def cfg5():
        M = W.poisson3d(96)
        k = 256
        B = torch.from_numpy(W.rhs(M.n, k, seed=0)).to(dev)
        rows = []
        for p, sub in ((1, "parallel"), (32, "hybrid"), (256, "classical")):
            X64 = None
            for prec in ("fp64", "fp32_refine"):
                t, r, Xr = time_solve(bcg, torch, M, B, k=k, p=p, sub=sub, prec=prec, reps=1, dev=dev, warm=False)
                rows.append(row(t, r, p=p, sub=sub, prec=prec, tol=1e-8))
                if prec == "fp64":
                    X64 = Xr
                else:
                    rows[-1].update(rel_errs(Xr, X64))
            del X64
        del B
        return {"workload": "poisson3d_96_csr_k256", "n": M.n, "results": rows}

    for name, fn in (("poisson2d_64_k8", cfg1), ("varcoef3d_160_k64", cfg3), ("stencil27_100_k16_autograd", cfg4),
                     ("poisson3d_96_k256", cfg5)):
        guarded(name, fn)
        torch.cuda.empty_cache()
    return out


def run_rows(args, rank, world, local):
    """`--mode rows`: the default workload as ONE problem whose rows are split over the ranks (strong scaling).
    Each rank runs bcg_create_csr_rows on its rows; the halo rows of P and the two sums of partial block
    products per iteration go through NCCL, enqueued on the handle's stream (no host wait inside a batch of 8
    iterations), and every batch after the first is one CUDA graph replay. value = the slowest rank's seconds
    to tolerance; e2e adds the per-step copies of each rank's rows of B (host -> device) and X (device ->
    host)."""
    import numpy as np
    import scipy.sparse as sp
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if "MASTER_ADDR" in os.environ:
        dist.init_process_group("nccl", device_id=dev)
    else:   # one rank without a launcher: a one-rank NCCL group on a free local port
        import socket
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1, device_id=dev)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    dist.barrier()
    from paper_1912_11930_gb300 import dist as D, workloads as W

    w = dict(WORKLOAD)
    if args.grid != w["grid"]:
        w["grid"] = args.grid
        w["name"] = w["name"].replace("128", str(args.grid))
    M = W.poisson3d(w["grid"])
    n, k, p = M.n, w["k"], w["p"]
    comm = D.TorchComm(dist)
    plan = D.local_plan(M.rowptr, M.colind, M.vals, D.row_bounds(n, world), rank)
    D.fill_sends(plan, comm.all_gather_object(plan.requests))
    r0, r1 = plan.bounds[rank], plan.bounds[rank + 1]
    B_host = np.ascontiguousarray(W.rhs(n, k, seed=0)[r0:r1])   # one problem: every rank its rows of it
    stream = torch.cuda.Stream(dev)
    S = D.RowShardedSolver(plan, k=k, p=p, sub=w["sub"], comm=D.StreamComm(dist, stream), device=dev, graph=True)
    B = torch.from_numpy(B_host).to(dev)
    X = torch.zeros(plan.n_cols, k, dtype=torch.float64, device=dev)

    def solve():
        with torch.cuda.stream(stream):
            X.zero_()
        return S.solve(B, X, tol=w["tol"], maxit=20000)

    for _ in range(args.warmup):
        res = solve()
        assert res.ok, res
    clocks = ClockSampler(local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [solve() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms_max = D.max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)

    # true residual of the gathered solution: each rank's rows of B - A X from X with its halo rows
    S._halo_x(X)
    torch.cuda.synchronize()
    L = sp.csr_matrix((plan.vals, plan.colind, plan.rowptr), shape=(plan.n_local, plan.n_cols))
    part = torch.from_numpy(np.concatenate([np.sum((B_host - L @ X.cpu().numpy()) ** 2, axis=0),
                                            np.sum(B_host ** 2, axis=0)])).to(dev)
    dist.all_reduce(part)
    part = part.cpu().numpy()
    rel_true = float(np.max(np.sqrt(part[:k] / part[k:])))

    # end to end: this rank's rows of B from pinned host memory, X back to pinned host memory, every step
    Bp = torch.from_numpy(B_host).pin_memory()
    Xp = torch.zeros(plan.n_local, k, dtype=torch.float64).pin_memory()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            B.copy_(Bp, non_blocking=True)
        solve()
        with torch.cuda.stream(stream):
            Xp.copy_(X[:plan.n_local], non_blocking=True)
        stream.synchronize()
    e2e = D.max_over_ranks((time.perf_counter() - t0) / args.steps, dist, dev)

    iters = results[-1].iters
    z = M.nnz
    model = kernel_model(n, k, p, z, 8, 12.0 * z + 8.0 * (n + 1), rho_k3=rho_in_k3(k, p, "fp64"))
    iter_bytes = sum(v["bytes"] for v in model.values())
    iter_s = ms_max * 1e-3 / max(iters, 1)
    hbm_peak, hbm_src = peaks()
    peers = len(plan.send)
    launched = int(math.ceil(iters / 8.0) * 8)
    line = {"metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"] + f"_rows{world}", "n": n, "nnz": z, "k": k, "p": p,
                       "subalgebra": w["sub"], "tol": w["tol"],
                       "l2": "inputs larger than L2 (537 MB per block vector at one rank)",
                       "parallelism": f"rows split over {world} ranks: NCCL halo + 2 allreduces per iteration on "
                                      "the handle's stream, CUDA graph per batch of 8 iterations"},
            "iterations": iters, "converged": all(r.ok for r in results), "max_rel_res_true": rel_true,
            "gb_per_iter_model": iter_bytes / 1e9,
            "roofline": {"bound": "hbm", "kernel": "whole iteration (all ranks)", "unit": "GB/s",
                         "achieved": iter_bytes / iter_s / 1e9, "peak": hbm_peak * world,
                         "frac": iter_bytes / iter_s / 1e9 / (hbm_peak * world), "traffic": None,
                         "peak_source": hbm_src,
                         "note": "modelled bytes of one iteration over the seconds per iteration; the FP64 pipe, "
                                 "not HBM, binds each rank's kernels"},
            "gpu_launches": args.steps * (launched * (8 + peers) + 6),
            "clocks": clk,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": (r1 - r0) * k * 8,
                    "d2h_bytes_per_step": (r1 - r0) * k * 8}}
    S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations after the variants")
    ap.add_argument("--grid", type=int, default=WORKLOAD["grid"],
                    help="Poisson grid edge (smaller grids only for profiling captures)")
    ap.add_argument("--prec", default=WORKLOAD["prec"], choices=["fp64", "fp32_refine", "fp64_df"],
                    help="precision of the timed solve (profiling captures of the mixed form)")
    ap.add_argument("--workload", default=None, choices=EXTRA_WORKLOADS,
                    help="measure one of the other workloads instead of the default line")
    ap.add_argument("--mode", default="columns", choices=["columns", "rows"],
                    help="columns: independent right-hand-side blocks per rank (weak scaling, the default line); "
                         "rows: one problem split by rows over the ranks (strong scaling, NCCL on stream)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload:
        return run_extra(args.workload, args)
    if args.mode == "rows":
        return run_rows(args, rank, world, int(os.environ.get("LOCAL_RANK", "0")))

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_1912_11930_gb300 import bcg, dist as D, workloads as W

    def barrier():
        if dist:
            dist.barrier()

    w = dict(WORKLOAD)
    if args.grid != w["grid"]:
        w["grid"] = args.grid
        w["name"] = w["name"].replace("128", str(args.grid))
    if args.prec != w["prec"]:
        w["prec"] = args.prec
        w["name"] = w["name"].replace("fp64", args.prec)
    M = W.poisson3d(w["grid"])
    n, k, p, z = M.n, w["k"], w["p"], M.nnz
    B_host = W.rhs(n, k, seed=D.rank_seed(0, rank))
    B = torch.from_numpy(B_host).to(dev)
    X = torch.zeros_like(B)
    S = bcg.Solver.from_matrix(M, k=k, p=p, sub=w["sub"], prec=w["prec"], device=dev)
    for _ in range(args.warmup):
        X.zero_()
        X, res = S.solve(B, X, tol=w["tol"], maxit=20000)
        assert res.ok, res
    S.set_option("profile", 1)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    e0.record(S.stream)
    for _ in range(args.steps):
        with torch.cuda.stream(S.stream):
            X.zero_()
        X, res = S.solve(B, X, tol=w["tol"], maxit=20000)
        results.append(res)
    e1.record(S.stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = D.max_over_ranks(ms, dist, dev)
    prof = S.profile()
    S.set_option("profile", 0)
    iters = results[-1].iters
    ok = all(r.ok and r.max_rel_res_true <= 1.5 * w["tol"] for r in results)

    # roofline of the dominant kernel
    # the profiled kernels are the FP64 iteration, or the FP32 inner iteration of the mixed form (FP32 block
    # vectors and an FP32 copy of the CSR values)
    fp64 = w["prec"] in ("fp64", "fp64_df")
    s_bytes = 8 if fp64 else 4
    a_bytes = (12.0 if fp64 else 8.0) * z + 8.0 * (n + 1)
    model = kernel_model(n, k, p, z, s_bytes, a_bytes, rho_k3=rho_in_k3(k, p, w["prec"]),
                         df=w["prec"] == "fp64_df" and rho_in_k3(k, p, w["prec"]))
    hbm_peak, hbm_src = peaks()
    per_kernel = {}
    for name, (tot, cnt) in prof.items():
        if cnt > 0:
            entry = {"avg_ms": tot / cnt, "launches": cnt, "share": None}
            if name in model:
                mdl = model[name]
                sec = tot / cnt * 1e-3
                entry["alg_gflop_fp64_pipe"] = mdl["alu"] / 1e9
                entry["alg_gflop_gram_dot2"] = mdl["gram"] / 1e9
                if mdl.get("df"):
                    entry["alg_gflop_double_float"] = mdl["df"] / 1e9
                entry["alg_gb"] = mdl["bytes"] / 1e9
                entry["fp64_tflops"] = mdl["alu"] / sec / 1e12
                entry["gbs"] = mdl["bytes"] / sec / 1e9
            per_kernel[name] = entry
    total_ms = sum(v["avg_ms"] * v["launches"] for v in per_kernel.values())
    for v in per_kernel.values():
        v["share"] = v["avg_ms"] * v["launches"] / total_ms if total_ms else None
    dom = max((nm for nm in per_kernel if nm in model), key=lambda nm: per_kernel[nm]["share"])
    d = per_kernel[dom]
    # FP64-pipe roofline of the dominant kernel: only the algorithmic flops that run as FP64 FMAs count
    # (the block products run as error-free FP32 arithmetic and are reported beside it)
    traffic = None
    ent = TRAFFIC.get((dom, w["name"]))
    if ent and ent[1] == kernel_source_sha(ent[0]):
        traffic = ent[2]
    roofline = {"bound": "alu", "kernel": dom, "achieved": d["fp64_tflops"], "peak": NOMINAL_FP64_TFLOPS,
                "unit": "TFLOP/s", "frac": d["fp64_tflops"] / NOMINAL_FP64_TFLOPS, "traffic": traffic,
                "counted": "algorithmic FP64-pipe flops of the kernel (BOP / BAXPY FMAs; with fp64_df, K2's X "
                           "FMAs and one addition per element of R); its block products (and fp64_df's R "
                           "products) run as error-free FP32 arithmetic and are listed under "
                           "kernels.*.alg_gflop_gram_dot2 (.alg_gflop_double_float)",
                "peak_source": "nominal FP64 (GB300 FP64 vector and tensor rate; the P0 DFMA probe measured 1.19)",
                "hbm_achieved_gbs": d["gbs"], "hbm_peak_gbs": hbm_peak, "hbm_frac": d["gbs"] / hbm_peak,
                "hbm_peak_source": hbm_src}
    iter_bytes = sum(model[nm]["bytes"] for nm in model)
    iter_ms = sum(per_kernel[nm]["avg_ms"] for nm in per_kernel)
    launched_iters = int(math.ceil(iters / 8.0) * 8)
    # per solve: K0, status reset, (FP64 with 2 <= p <= 16) the BDOT of the first recomputed rho, 5 kernels per
    # launched iteration (batches of 8), then K0 and a norm reduction for the true residual
    setup = 4 + (1 if rho_in_k3(k, p, w["prec"]) else 0)
    gpu_launches = args.steps * (setup + 5 * launched_iters)

    line = {"metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp64_df": "f64 (double-float residual update)"}.get(w["prec"],
                                                                                     "f32 inner, f64 refinement"),
            "data": "synthetic",
            "config": {"workload": w["name"], "n": n, "nnz": z, "k": k, "p": p, "subalgebra": w["sub"],
                       "tol": w["tol"], "rhs_per_rank": k, "l2": "inputs larger than L2 (537 MB per block vector)",
                       "parallelism": f"independent right-hand-side blocks per rank x{world}"},
            "iterations": iters, "converged": ok, "max_rel_res_true": max(r.max_rel_res_true for r in results),
            "gb_per_iter_model": iter_bytes / 1e9, "gbs_per_iter": iter_bytes / (iter_ms * 1e-3) / 1e9,
            "hbm_frac_per_iter": iter_bytes / (iter_ms * 1e-3) / 1e9 / hbm_peak,
            "kernels": per_kernel, "roofline": roofline, "gpu_launches": gpu_launches, "clocks": clk}

    # end-to-end through the public host-buffer entry point: B and X^0 host -> device, X device -> host
    if rank == 0 or world > 1:
        Bh = torch.from_numpy(B_host).pin_memory().numpy()
        Xh = torch.zeros(n, k, dtype=torch.float64).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Xh[:] = 0.0
            Xh, rh = S.solve_host(Bh, Xh, tol=w["tol"], maxit=20000)
        torch.cuda.synchronize()
        e2e = (time.perf_counter() - t0) / args.steps
        line["e2e"] = {"value": D.max_over_ranks(e2e, dist, dev), "unit": "s", "h2d_bytes_per_step": 2 * n * k * 8,
                       "d2h_bytes_per_step": n * k * 8}

    if rank == 0 and world == 1 and not args.no_variants:
        variants = {}
        X64 = X.cpu().numpy()   # the timed FP64 solve's solution (parity-tested against the oracle)
        for vname, sub, vp, prec in (("parallel_p1_fp64", "parallel", 1, "fp64"),
                                     ("global_p32_fp64", "global", 32, "fp64"),
                                     ("hybrid_p8_fp32_refine", "hybrid", 8, "fp32_refine"),
                                     ("hybrid_p8_fp64_df", "hybrid", 8, "fp64_df")):
            V = bcg.Solver.from_matrix(M, k=k, p=vp, sub=sub, prec=prec, device=dev)
            Xv = torch.zeros_like(B)
            V.solve(B, Xv, tol=w["tol"], maxit=20000)
            Xv.zero_()
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(V.stream)
            Xv, rv = V.solve(B, Xv, tol=w["tol"], maxit=20000)
            a1.record(V.stream)
            torch.cuda.synchronize()
            variants[vname] = {"s": a0.elapsed_time(a1) / 1e3, "iterations": rv.iters, "outer": rv.outer_iters,
                               "status": bcg.STATUS_NAMES[rv.status], "max_rel_res_true": rv.max_rel_res_true}
            if prec != "fp64" and w["prec"] == "fp64":
                # the variant's solution against the FP64 solve of the same system (both to 1e-8): relative error,
                # over the whole block and column by column in the max norm
                Xn = Xv.cpu().numpy()
                variants[vname]["rel_err_vs_fp64"] = float(np.linalg.norm(Xn - X64) / np.linalg.norm(X64))
                variants[vname]["rel_err_vs_fp64_elementwise"] = float(
                    np.max(np.max(np.abs(Xn - X64), axis=0) / np.max(np.abs(X64), axis=0)))
            V.close()
        variants["hybrid_p8_fp64"] = {"s": ms_max / 1e3, "iterations": iters}
        line["variants"] = variants
        line["mixed_vs_fp64_speedup"] = variants["hybrid_p8_fp64"]["s"] / variants["hybrid_p8_fp32_refine"]["s"]
        line["df_vs_fp64_speedup"] = variants["hybrid_p8_fp64"]["s"] / variants["hybrid_p8_fp64_df"]["s"]
        if not args.no_configs:
            line["configs"] = config_variants(bcg, W, torch, dev, np)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(w["grid"], k, p, w["sub"], ORACLE_SAMPLE_ITERS, seed=0)
        val = smp["first"] + smp["per_iter"] * iters
        line["cpu_baseline"] = {"value": val, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": f"{ORACLE_SAMPLE_ITERS} oracle iterations of the full workload "
                                          f"({smp['total']:.1f} s, single-threaded); time-to-tolerance = initial "
                                          f"residual + per-iteration time x the GPU's {iters} iterations",
                                "per_iter_s": smp["per_iter"]}
        ncores = len(os.sched_getaffinity(0))
        sma = oracle_sample(w["grid"], k, p, w["sub"], ORACLE_SAMPLE_ITERS, seed=0, threads=ncores)
        line["cpu_baseline_all_cores"] = {"value": sma["first"] + sma["per_iter"] * iters, "unit": "s",
                                          "cores": ncores, "kind": "oracle",
                                          "sample": f"as cpu_baseline with {ncores} BLAS / OpenMP threads (the oracle's "
                                                    f"sparse products are single-threaded in scipy; its dense block "
                                                    f"products use the threads) ({sma['total']:.1f} s)",
                                          "per_iter_s": sma["per_iter"]}
    S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
