"""CPU checks of the digit scheme behind spd_residual_tc (the float64-accurate
residual of Algorithm 1, lines 3/7, by exact digit products), in exact integer
arithmetic: the claims its error bound rests on.

- every entry of a row (column) is cut into ten balanced base-128 digits below
  2^e with e = ilogb(row max) + 2; the digits are at most 64 in magnitude and
  reproduce the entry up to its bits below 2^{e-70};
- a 64-wide chunk of any digit-product group sums to at most 2^22 in
  magnitude, so float32 accumulation of it is exact and the magic-number
  conversion to an integer is valid;
- keeping the products with p + q <= 11 errs by at most
  n 2^-64 max_j |a_ij| max_j |x_j| per residual entry (before the final
  rounding), on matrices whose rows decay, mix magnitudes over 2^+-40, or
  are dense and random.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

S, TMAX = 10, 11


def row_exp(vmax):
    return 0 if vmax == 0.0 else math.frexp(vmax)[1] - 1 + 2  # ilogb + 2


def digits(a, e):
    """Balanced base-128 digits d[0..9] (d[0] most significant) of
    sign(a) trunc(|a| 2^(70-e))."""
    f = int(abs(Fraction(a)) * Fraction(2) ** (70 - e))  # truncation toward zero
    d = []
    for _ in range(S - 1):
        t = f + 64
        d.append((t % 128) - 64)
        f = t // 128
    d.append(f)
    d = d[::-1]
    return [-x for x in d] if a < 0 else d


def value(d, e):
    return sum(Fraction(x) * Fraction(2) ** (e - 7 * (p + 1)) for p, x in enumerate(d))


def test_digits_bounded_and_exact_to_the_truncation():
    g = np.random.default_rng(0)
    for _ in range(3000):
        rowmax = math.ldexp(g.uniform(0.5, 1.0), int(g.integers(-1070, 1020)))
        e = row_exp(rowmax)
        for a in [rowmax, -rowmax, rowmax * g.uniform(-1, 1), rowmax * 2.0 ** -float(g.integers(0, 90))]:
            d = digits(a, e)
            assert all(abs(x) <= 64 for x in d)
            assert abs(value(d, e) - Fraction(a)) < Fraction(2) ** (e - 70)


def test_chunk_group_sums_fit_float32_exactly():
    # the worst case: every digit +-64 (same sign), every product pair of a
    # group present (10 pairs for t = 11), 64 terms per chunk
    worst = max(sum(64 * 64 for p in range(S) for q in range(S) if p + q + 2 == t) for t in range(2, TMAX + 1))
    assert worst * 64 <= 2 ** 22
    # and a random chunk stays within it
    g = np.random.default_rng(1)
    A = g.integers(-64, 65, (64, S))
    X = g.integers(-64, 65, (64, S))
    for t in range(2, TMAX + 1):
        tot = sum(int(A[j, p]) * int(X[j, q]) for j in range(64) for p in range(S) for q in range(S) if p + q + 2 == t)
        assert abs(tot) <= 2 ** 22


def product_by_groups(A, x):
    """sum_j a_ij x_j from the digit products with p + q <= 11, exactly."""
    n = A.shape[0]
    ex = row_exp(float(np.max(np.abs(x))))
    dx = [digits(float(v), ex) for v in x]
    out = []
    for i in range(n):
        ei = row_exp(float(np.max(np.abs(A[i]))))
        da = [digits(float(v), ei) for v in A[i]]
        groups = [0] * (TMAX + 1)
        for j in range(n):
            for p in range(S):
                if da[j][p] == 0:
                    continue
                for q in range(S):
                    t = p + q + 2
                    if t <= TMAX:
                        groups[t] += da[j][p] * dx[j][q]
        out.append(sum(Fraction(groups[t]) * Fraction(2) ** (ei + ex - 7 * t) for t in range(2, TMAX + 1)))
    return out


@pytest.mark.parametrize("kind", ["dense", "decaying", "spread"])
def test_truncated_products_within_the_stated_bound(kind):
    n = 48
    g = np.random.default_rng({"dense": 2, "decaying": 3, "spread": 4}[kind])
    if kind == "dense":
        A = g.standard_normal((n, n))
    elif kind == "decaying":  # the rows of a covariance: 1 on the diagonal, decaying away from it
        idx = np.arange(n)
        A = np.exp(-np.abs(idx[:, None] - idx[None, :]) / 1.5) * (1 + 0.1 * g.standard_normal((n, n)))
    else:
        A = g.standard_normal((n, n)) * np.exp2(g.uniform(-40, 40, (n, n)))
    x = g.standard_normal(n) * np.exp2(g.uniform(-20, 20, n))
    got = product_by_groups(A, x)
    xmax = float(np.max(np.abs(x)))
    for i in range(n):
        exact = sum(Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(n))
        bound = n * Fraction(2) ** -64 * Fraction(float(np.max(np.abs(A[i])))) * Fraction(xmax)
        assert abs(got[i] - exact) <= bound, float(abs(got[i] - exact) / bound)
