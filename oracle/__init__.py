"""CPU float64 oracle for the mixed-precision SPD solver -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports or calls it, and it imports nothing from the
product.  The heavy loops live in ``oracle.c`` (plain textbook C); this module
marshals numpy arrays into it.

Every function states the passage of the paper it follows:

* ``potrf``          Section 3.1, eq. (cholesky): A = R^T R, R upper.
* ``potrs``          Section 3.1, eq. (cholesky): X = R^{-1} R^{-T} B.
* ``solve``          the two above: the float64 solution of A X = B (P1).
* ``potrf_f32`` / ``potrs_f32``  the same in IEEE single ("low precision",
  Section 3.1).
* ``residual``       R = B - A X (Alg. 1/Alg. 2 residual, high precision).
* ``berr``           normwise backward error ||b - Ax||_inf/(||A||_inf ||x||_inf).
* ``chol_ir``        Algorithm 1 with a supplied single-precision factor.
* ``chol_ir_f64``    Algorithm 1's loop with a perturbed float64 factor
  (the experiment behind Fig. 3b).
* ``cg``             textbook CG in float64.
* ``cg_ir``          Algorithm 2 in its nested low/high reading, optionally
  with the banded inner matrix of Section 4.1.
* ``spectral_solve`` the exact solution of A X = B for a matrix given by its
  eigendecomposition A = Q diag(lam) Q^T, Q a product of Householder
  reflections (the Section 5 test matrices with a prescribed spectrum): an
  O(n k m) reference at sizes where the dense oracle is too slow.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build
from .precision import ROUND, UNIT_ROUNDOFF  # noqa: F401

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, f, i, l = C.c_double, C.c_float, C.c_int, C.c_long
        P = C.c_void_p
        sig = {
            "oracle_potrf": (i, [i, P, l, P, l]),
            "oracle_potrs": (None, [i, i, P, l, P, l, P, l]),
            "oracle_potrf_f32": (i, [i, P, l, P, l]),
            "oracle_potrs_f32": (None, [i, i, P, l, P, l, P, l]),
            "oracle_residual": (None, [i, i, P, l, P, l, P, l, P, l]),
            "oracle_norm_inf": (d, [i, P, l]),
            "oracle_berr": (d, [i, i, P, l, P, l, P, l, P]),
            "oracle_chol_ir": (i, [i, i, P, l, P, l, P, l, P, l, d, i, i, P, P]),
            "oracle_chol_ir_f64": (i, [i, i, P, l, P, l, P, l, P, l, d, i, P, P]),
            "oracle_cg": (i, [i, i, P, l, P, l, P, l, d, i, P, P]),
            "oracle_cg_ir": (i, [i, i, P, l, P, l, i, P, l, P, l, d, i, d, i, i, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    """Column-major float64 copy/view of a 1-D or 2-D array."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return np.asfortranarray(a)


def _f32(a):
    a = np.asarray(a, dtype=np.float32)
    return np.asfortranarray(a)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _ld(a):
    return a.shape[0]


def potrf(A):
    """R (upper, float64) with A = R^T R; raises ValueError(info) if not SPD."""
    A = _f64(A)
    n = A.shape[0]
    R = np.zeros((n, n), order="F")
    info = lib().oracle_potrf(n, _p(A), _ld(A), _p(R), n)
    if info:
        raise ValueError(f"not positive definite at column {info}", info)
    return R


def potrs(R, B):
    R, B = _f64(R), _f64(B)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    lib().oracle_potrs(n, m, _p(R), _ld(R), _p(B), _ld(B), _p(X), n)
    return X


def solve(A, B):
    """float64 solution of A X = B by Cholesky and two substitutions."""
    return potrs(potrf(A), B)


def potrf_f32(A):
    A = _f64(A)
    n = A.shape[0]
    R = np.zeros((n, n), dtype=np.float32, order="F")
    info = lib().oracle_potrf_f32(n, _p(A), _ld(A), _p(R), n)
    if info:
        raise ValueError(f"not positive definite at column {info}", info)
    return R


def potrs_f32(R, B):
    R, B = _f32(R), _f64(B)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    lib().oracle_potrs_f32(n, m, _p(R), _ld(R), _p(B), _ld(B), _p(X), n)
    return X


def residual(A, B, X):
    A, B, X = _f64(A), _f64(B), _f64(X)
    n, m = B.shape
    Rr = np.zeros((n, m), order="F")
    lib().oracle_residual(n, m, _p(A), _ld(A), _p(B), _ld(B), _p(X), _ld(X), _p(Rr), n)
    return Rr


def norm_inf(A):
    A = _f64(A)
    return lib().oracle_norm_inf(A.shape[0], _p(A), _ld(A))


def berr(A, B, X, per_column=False):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf)."""
    A, B, X = _f64(A), _f64(B), _f64(X)
    n, m = B.shape
    pc = np.zeros(m)
    worst = lib().oracle_berr(n, m, _p(A), _ld(A), _p(B), _ld(B), _p(X), _ld(X), _p(pc))
    return pc if per_column else worst


def chol_ir(A, Rt, B, tol=1e-14, crit="berr", maxit=50):
    """Algorithm 1 with the single-precision factor Rt.  Returns (X, iters, err, ok)."""
    A, B = _f64(A), _f64(B)
    Rt = _f32(Rt)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    it = np.zeros(m, dtype=np.int32)
    err = np.zeros(m)
    c = 0 if crit == "abs2" else 1
    bad = lib().oracle_chol_ir(n, m, _p(A), _ld(A), _p(Rt), _ld(Rt), _p(B), _ld(B), _p(X), n,
                               float(tol), c, int(maxit), _p(it), _p(err))
    return X, it, err, not bad


def chol_ir_f64(A, Rp, B, tol=1e-14, maxit=200):
    """Algorithm 1's loop with a float64 (perturbed) factor Rp; backward-error stop."""
    A, B, Rp = _f64(A), _f64(B), _f64(Rp)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    it = np.zeros(m, dtype=np.int32)
    err = np.zeros(m)
    bad = lib().oracle_chol_ir_f64(n, m, _p(A), _ld(A), _p(Rp), _ld(Rp), _p(B), _ld(B), _p(X), n,
                                   float(tol), int(maxit), _p(it), _p(err))
    return X, it, err, not bad


def cg(A, B, tol_rel=1e-14, maxit=10000):
    """Textbook float64 CG from x0 = 0.  Returns (X, iters, relres, ok)."""
    A, B = _f64(A), _f64(B)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    it = np.zeros(m, dtype=np.int32)
    rr = np.zeros(m)
    bad = lib().oracle_cg(n, m, _p(A), _ld(A), _p(B), _ld(B), _p(X), n, float(tol_rel),
                          int(maxit), _p(it), _p(rr))
    return X, it, rr, not bad


def cg_ir(A, B, At=None, band=-1, tol=1e-14, crit="rel", eta=1e-3, maxit_in=5000, maxit_out=50):
    """Algorithm 2, nested reading.  At defaults to A rounded to single.

    Returns (X, iters_low, iters_high, final ||r||_2, ok).
    """
    A, B = _f64(A), _f64(B)
    At = _f32(A if At is None else At)
    n, m = B.shape
    X = np.zeros((n, m), order="F")
    lo = np.zeros(m, dtype=np.int32)
    hi = np.zeros(m, dtype=np.int32)
    fe = np.zeros(m)
    c = 0 if crit == "abs2" else 1
    bad = lib().oracle_cg_ir(n, m, _p(A), _ld(A), _p(At), _ld(At), int(band), _p(B), _ld(B),
                             _p(X), n, float(tol), c, float(eta), int(maxit_in), int(maxit_out),
                             _p(lo), _p(hi), _p(fe))
    return X, lo, hi, fe, not bad


def spectral_solve(V, lam, B):
    """X = Q diag(lam)^{-1} Q^T B for Q = H_1 H_2 ... H_k, H_i = I - 2 v_i v_i^T
    (v_i the unit columns of V): Q^T B = H_k ... H_1 B, a division by the
    eigenvalues, then Q Y = H_1 ... H_k Y.  Each reflection is applied as
    y - 2 v (v^T y), so the result errs by a few k units of roundoff relative
    to ||X||, whatever the condition number."""
    V = np.asarray(V, dtype=np.float64)
    Y = np.array(B, dtype=np.float64).reshape(V.shape[0], -1)
    for i in range(V.shape[1]):
        v = V[:, i:i + 1]
        Y -= 2.0 * v @ (v.T @ Y)
    Y /= np.asarray(lam, dtype=np.float64)[:, None]
    for i in reversed(range(V.shape[1])):
        v = V[:, i:i + 1]
        Y -= 2.0 * v @ (v.T @ Y)
    return Y


def cpu_threads() -> int:
    """Threads the OpenMP oracle may use on this host."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
