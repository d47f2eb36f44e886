"""The oracle's pins must fail when a plausible mistake is planted in the oracle (on the CPU, through
monkeypatch): the printed minus sign of the direction update (Algorithm 1), a transposed lambda in
BAXPY, a global product that forgets blocks, a hybrid product that mixes blocks, a dropped residual
update term."""
import numpy as np
import pytest

from oracle import bcg as O
from paper_1912_11930_gb300 import workloads as W

from test_oracle_pins import _galerkin_iterate, _rel


def _deviation(sub, k, p, m=3):
    M = W.dense_to_csr(W.random_spd_dense(40, seed=3, cond=50.0))
    A = M.to_scipy()
    B = W.rhs(M.n, k, seed=7)
    kind, pp = O.canonical_subalgebra(sub, k, p)
    res = O.solve(A, B, p=p, sub=sub, tol=0.0, maxit=m)
    return _rel(res.X, _galerkin_iterate(A.toarray(), B, np.zeros_like(B), pp, kind, m))


def test_pins_pass_unmutated():
    for sub, k, p in (("hybrid", 8, 4), ("global", 8, 4), ("parallel", 4, 1)):
        assert _deviation(sub, k, p) < 1e-9


def test_detects_printed_minus_sign(monkeypatch):
    orig = O.baxpy
    calls = {"n": 0}

    def mutated(X, Y, gamma, sign=1.0):
        calls["n"] += 1
        # the third BAXPY of each iteration is the direction update P = R +- P beta
        if calls["n"] % 3 == 0:
            return orig(X, Y, gamma, -1.0)
        return orig(X, Y, gamma, sign)

    monkeypatch.setattr(O, "baxpy", mutated)
    assert _deviation("hybrid", 8, 4) > 1e-6


def test_detects_transposed_lambda(monkeypatch):
    orig = O.block_apply
    monkeypatch.setattr(O, "block_apply", lambda Y, g: orig(Y, np.swapaxes(g, 1, 2)))
    assert _deviation("hybrid", 8, 4) > 1e-6


def test_detects_global_product_missing_blocks(monkeypatch):
    orig = O.block_product

    def mutated(X, Y, p, kind):
        if kind == "global":   # forgets every block but the first
            return (X[:, :p].T @ Y[:, :p])[None]
        return orig(X, Y, p, kind)

    monkeypatch.setattr(O, "block_product", mutated)
    assert _deviation("global", 8, 4) > 1e-6


def test_detects_hybrid_blocks_mixed_up(monkeypatch):
    orig = O.block_product

    def mutated(X, Y, p, kind):
        g = orig(X, Y, p, kind)
        return g[::-1].copy() if kind == "hybrid" and g.shape[0] > 1 else g

    monkeypatch.setattr(O, "block_product", mutated)
    assert _deviation("hybrid", 8, 4) > 1e-6


def test_detects_dropped_residual_update(monkeypatch):
    orig = O.baxpy
    calls = {"n": 0}

    def mutated(X, Y, gamma, sign=1.0):
        calls["n"] += 1
        if calls["n"] % 3 == 2:      # R = R - Q lambda becomes R = R
            return X.copy()
        return orig(X, Y, gamma, sign)

    monkeypatch.setattr(O, "baxpy", mutated)
    assert _deviation("parallel", 4, 1) > 1e-6
