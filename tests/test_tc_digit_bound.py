"""The error bound that include/bcg.h states for the tensor-core block products and updates, checked on the CPU.

The scheme (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012, as the header describes it): every value of a
contraction operand is truncated to 48 bits below an exponent E shared along the contraction (2^E <= max |u| <
2^(E+1)) and cut into eight 6-bit digits, u ~ sgn(u) sum_i d_i 2^(E - 5 - 6 i); the contraction keeps the 36 digit
pairs with i + j <= 7. Written here from that definition with exact integer and rational arithmetic (no product code
is imported): the test pins the stated bound, at most 2^-47 max|u| sum|v| + 2^-47 max|v| sum|u| for the truncations
plus the dropped pairs (below K 2^-44 max|u| max|v|), and about 2^-44 sum |u v| where the values are of one size.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

DIGITS, BITS = 8, 6


def shared_exponent(x):
    m = float(np.max(np.abs(x)))
    return math.frexp(m)[1] - 1 if m > 0 else -1022   # 2^E <= m < 2^(E+1)


def digits(x, E):
    """Signs and the eight digits (most significant first) of floor(|x| 2^(47 - E)), exactly."""
    out = []
    for v in x:
        f = Fraction(abs(float(v))) * Fraction(2) ** (47 - E)
        fx = f.numerator // f.denominator
        assert fx < 2 ** 48
        out.append((-1 if v < 0 else 1, [(fx >> (42 - BITS * i)) & 63 for i in range(DIGITS)]))
    return out


def sliced_dot(u, v):
    """sum_k u_k v_k from the digit pairs with i + j <= 7, exactly: 2^(E + F - 10) sum_s 2^(-6 s) acc_s."""
    E, F = shared_exponent(u), shared_exponent(v)
    du, dv = digits(u, E), digits(v, F)
    acc = [0] * DIGITS
    for (su, a), (sv, b) in zip(du, dv):
        for s in range(DIGITS):
            acc[s] += su * sv * sum(a[i] * b[s - i] for i in range(s + 1))
    for s in range(DIGITS):   # each partial sum stays an integer below 2^24 for up to 512 terms: FP32-exact
        assert abs(acc[s]) < 2 ** 24
    return sum(Fraction(acc[s]) * Fraction(2) ** (E + F - 10 - BITS * s) for s in range(DIGITS))


def exact_dot(u, v):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, v))


def inputs(kind, K, seed):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal(K), rng.standard_normal(K)
    if kind == "wide":     # magnitudes over about 2^-20 .. 2^20 inside one operand
        return rng.standard_normal(K) * np.exp2(rng.integers(-20, 20, K)), rng.standard_normal(K)
    if kind == "zeros":    # exact zeros and one dominant entry
        u, v = rng.standard_normal(K), rng.standard_normal(K)
        u[::3] = 0.0
        v[0] = 1e6
        return u, v
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["normal", "wide", "zeros"])
@pytest.mark.parametrize("K", [16, 256, 512])
def test_digit_slice_error_within_stated_bound(kind, K):
    for seed in range(3):
        u, v = inputs(kind, K, seed)
        err = abs(float(sliced_dot(u, v) - exact_dot(u, v)))
        mu, mv = float(np.max(np.abs(u))), float(np.max(np.abs(v)))
        bound = 2.0 ** -47 * (mu * np.sum(np.abs(v)) + mv * np.sum(np.abs(u))) + K * 2.0 ** -44 * mu * mv
        assert err <= bound, (kind, K, seed, err, bound)


@pytest.mark.parametrize("K", [64, 512])
def test_digit_slice_error_relative_to_the_absolute_sum_for_one_size(K):
    """Values of one size (N(0,1)): the error is a few 2^-44 of sum |u v| or less, far below FP32 and near FP64."""
    for seed in range(3):
        u, v = inputs("normal", K, 10 + seed)
        err = abs(float(sliced_dot(u, v) - exact_dot(u, v)))
        assert err <= 2.0 ** -41 * float(np.sum(np.abs(u * v)))


def test_the_one_size_bound_fails_with_diagonals_dropped():
    """A mutation: keeping only the pairs with i + j <= 5 (two diagonals dropped) breaks the one-size bound, so that
    test can see a plausible slip in the scheme (the max-based bound above is a worst case and looser)."""
    u, v = inputs("normal", 256, 13)
    E, F = shared_exponent(u), shared_exponent(v)
    du, dv = digits(u, E), digits(v, F)
    acc = [0] * DIGITS
    for (su, a), (sv, b) in zip(du, dv):
        for s in range(DIGITS - 2):
            acc[s] += su * sv * sum(a[i] * b[s - i] for i in range(s + 1))
    approx = sum(Fraction(acc[s]) * Fraction(2) ** (E + F - 10 - BITS * s) for s in range(DIGITS))
    err = abs(float(approx - exact_dot(u, v)))
    assert err > 2.0 ** -41 * float(np.sum(np.abs(u * v)))
