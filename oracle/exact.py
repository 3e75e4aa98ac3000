"""Correctly rounded residual R = B - A X -- TEST INFRASTRUCTURE.

The float64 residual of Algorithm 1 (lines 3 and 7) and Algorithm 2 (line 2)
is itself rounded; to judge a residual computed in other arithmetic (the
float32-pair residual of the CUDA path) the tests need the exact value.

* Every float64 product a*x is written exactly as a sum of four float64
  products of 26-bit halves (Veltkamp's splitting: a = a1 + a2 with a1
  holding the leading 26 significand bits), each of which is exact.
* Each entry b_i - sum_j a_ij x_j is then the exact sum of 4n + 1 float64
  numbers, which ``math.fsum`` (Shewchuk's algorithm) returns correctly
  rounded.

Valid while no product over- or underflows (|a|, |x| within about
[2^-400, 2^400]), which the tests respect.  ``residual_fraction`` is the
same quantity in rational arithmetic, for tiny cases.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_SPLITTER = 134217729.0  # 2^27 + 1


def split26(a):
    """Veltkamp's splitting a = hi + lo, both with at most 26 significant bits."""
    a = np.asarray(a, dtype=np.float64)
    c = _SPLITTER * a
    hi = c - (c - a)
    return hi, a - hi


def residual_exact(A, B, X):
    """R[i, c] = fl(B[i, c] - sum_j A[i, j] X[j, c]), correctly rounded."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[1], -1)
    a1, a2 = split26(A)
    R = np.empty_like(B)
    for c in range(B.shape[1]):
        x1, x2 = split26(X[:, c])
        terms = np.concatenate([-(a1 * x1), -(a1 * x2), -(a2 * x1), -(a2 * x2), B[:, c:c + 1]], axis=1)
        R[:, c] = [math.fsum(row) for row in terms.tolist()]
    return R


def residual_fraction(A, B, X):
    """The same residual in exact rational arithmetic, rounded once."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[1], -1)
    R = np.empty_like(B)
    for c in range(B.shape[1]):
        xs = [Fraction(float(v)) for v in X[:, c]]
        for i in range(A.shape[0]):
            s = Fraction(float(B[i, c]))
            for j in range(A.shape[1]):
                s -= Fraction(float(A[i, j])) * xs[j]
            R[i, c] = float(s)
    return R


def abs_product(A, X):
    """|A| |X| in float64 (the scale that residual error bounds refer to)."""
    return np.abs(np.asarray(A, dtype=np.float64)) @ np.abs(np.asarray(X, dtype=np.float64).reshape(A.shape[1], -1))
