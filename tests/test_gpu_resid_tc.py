"""GPU parity of the tensor-core residual R = B - A X of Algorithm 1
(lines 3, 7) and Algorithm 2 (line 2): exact products of bf16 digits
(spd_residual_tc), judged against the correctly rounded residual of the
oracle; then Algorithm 1 and Algorithm 2 run end to end with it."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W
from oracle import exact as E

from tests.gpu_util import DEV, check, dev_cols, dev_sym, dev_zeros, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def matrix(kind, n):
    if kind == "householder":
        A, _, _ = W.householder_spectrum(n, 1e6, k=16, seed=n)
        return A
    if kind == "model":
        return W.model_covariance(n, 1.0)
    if kind == "matern":
        ell, nug = W.matern_family_params(n)
        return W.matern32_cov(n, ell, nug, n)[0]
    # symmetric, indefinite, entries spread over 2^-40 .. 2^40
    g = np.random.default_rng(n + 1)
    G = g.standard_normal((n, n)) * np.exp2(g.uniform(-40, 40, (n, n)))
    return np.tril(G) + np.tril(G, -1).T


def run(h, fn, A, B, X):
    n, m = B.shape
    R = dev_zeros(n, m)
    nrm = torch.zeros(3 * m, dtype=torch.float64, device=DEV)
    check(h, fn(h, dev_sym(A), dev_cols(B), dev_cols(X), R, nrm))
    return host(R), host(nrm)


def bound(A, X, r_ex):
    """The documented bound: 2^-53 |r_i| + n 2^-64 max_j |a_ij| max_j |x_jc|
    (the dropped digit products and the truncation below 2^{e - 70})."""
    n = A.shape[0]
    rowmax = np.max(np.abs(A), axis=1)[:, None]
    xmax = np.max(np.abs(X), axis=0)[None, :]
    return 2.0 ** -53 * np.abs(r_ex) + n * 2.0 ** -64 * rowmax * xmax


@pytest.mark.parametrize("kind", ["householder", "model", "matern", "spread"])
@pytest.mark.parametrize("n,m", [(300, 1), (1000, 3), (1337, 16), (2111, 20)])
def test_tc_residual_against_exact(h, kind, n, m):
    A = matrix(kind, n)
    g = np.random.default_rng(n * 31 + m)
    X = g.standard_normal((n, m))
    # near-solution right-hand sides: the residual cancels to ~1e-9 of |A||x|
    B = (A @ X) * (1.0 + 1e-9 * g.standard_normal((n, m)))
    R, nrm = run(h, spd.spd_residual_tc, A, B, X)
    R64, _ = run(h, spd.spd_residual, A, B, X)
    cols = sorted({0, m // 2, m - 1})  # the exact residual is slow: sample columns
    r_ex = E.residual_exact(A, B[:, cols], X[:, cols])
    err = np.abs(R[:, cols] - r_ex)
    assert np.all(err <= bound(A, X[:, cols], r_ex)), float(np.max(err / bound(A, X[:, cols], r_ex)))
    # in practice as accurate as the float64 residual: within a few units of
    # 2^-53 (|A||x|)_i where the float64 residual errs by up to n 2^-53
    scale = E.abs_product(A, X[:, cols]) + np.abs(B[:, cols])
    err64 = np.abs(R64[:, cols] - r_ex)
    assert np.max(err / scale) <= 2.0 ** -47, float(np.max(err / scale))
    assert np.all(err64 <= n * 2.0 ** -52 * scale)
    nr = nrm.reshape(m, 3)[cols]
    np.testing.assert_allclose(nr[:, 0], np.max(np.abs(r_ex), axis=0), rtol=1e-6, atol=8 * np.max(err))
    np.testing.assert_allclose(nr[:, 2], np.max(np.abs(X[:, cols]), axis=0), rtol=0, atol=0)


def test_tc_residual_is_deterministic(h):
    n, m = 1500, 5
    A = matrix("householder", n)
    X = np.random.default_rng(2).standard_normal((n, m))
    B = A @ X
    R1, _ = run(h, spd.spd_residual_tc, A, B, X)
    R2, _ = run(h, spd.spd_residual_tc, A, B, X)
    assert np.array_equal(R1, R2)


def test_tc_residual_exact_on_short_integers(h):
    """Integer A and X small enough that every product and sum is exact in
    float64: the residual must come out exactly."""
    n, m = 700, 4
    g = np.random.default_rng(3)
    A = g.integers(-2 ** 20, 2 ** 20, (n, n)).astype(np.float64)
    A = np.tril(A) + np.tril(A, -1).T
    X = g.integers(-2 ** 20, 2 ** 20, (n, m)).astype(np.float64)
    B = g.integers(-2 ** 50, 2 ** 50, (n, m)).astype(np.float64)
    R, _ = run(h, spd.spd_residual_tc, A, B, X)
    r_ex = E.residual_exact(A, B, X)
    assert np.array_equal(R, r_ex)


def test_tc_residual_special_entries(h):
    """Zeros, tiny and huge entries in one row, and columns of X scaled by
    1e200 and 1e-150 (the bound is relative to each row's and column's
    largest entry)."""
    n, m = 777, 4
    g = np.random.default_rng(9)
    A = g.standard_normal((n, n))
    A = np.tril(A) + np.tril(A, -1).T
    idx = g.choice(n * n, 600, replace=False)
    vals = np.concatenate([np.zeros(200), np.full(200, 1e-120), np.full(200, 3e40)])
    A.flat[idx] = vals * np.sign(g.standard_normal(600))
    A = np.tril(A) + np.tril(A, -1).T
    X = g.standard_normal((n, m))
    X[:, 1] *= 1e200
    X[:, 2] *= 1e-150
    X[::7, 3] = 0.0
    B = (A @ X) * (1.0 + 1e-6 * g.standard_normal((n, m)))
    R, _ = run(h, spd.spd_residual_tc, A, B, X)
    r_ex = E.residual_exact(A, B, X)
    err = np.abs(R - r_ex)
    assert np.all(err <= bound(A, X, r_ex)), float(np.max(err / bound(A, X, r_ex)))


def test_tc_residual_zero_rows_and_columns(h):
    n, m = 400, 3
    A = W.gram_shifted(n, 4)
    A[17, :] = 0.0
    A[:, 17] = 0.0
    X = np.random.default_rng(5).standard_normal((n, m))
    X[:, 1] = 0.0
    B = np.random.default_rng(6).standard_normal((n, m))
    R, _ = run(h, spd.spd_residual_tc, A, B, X)
    assert np.array_equal(R[:, 1], B[:, 1])
    assert R[17, 0] == B[17, 0] and R[17, 2] == B[17, 2]


def test_tc_residual_nonfinite_propagates(h):
    n, m = 260, 2
    A = W.gram_shifted(n, 2)
    A[5, 9] = A[9, 5] = np.nan
    X = np.random.default_rng(1).standard_normal((n, m))
    X[3, 1] = np.inf
    B = A @ np.nan_to_num(X, posinf=0.0)
    R, _ = run(h, spd.spd_residual_tc, np.array(A), B, X)
    assert np.all(np.isnan(R[:, 1]))
    assert np.isnan(R[5, 0]) and np.isnan(R[9, 0])
    assert np.sum(np.isnan(R[:, 0])) == 2


def test_tc_residual_empty_and_bad_arguments(h):
    Z = dev_zeros(0, 1)
    A0 = torch.zeros(0, 0, dtype=torch.float64, device=DEV)
    assert spd.spd_residual_tc(h, A0, Z, Z, Z) == spd.SPD_OK
    A = dev_sym(np.eye(4))
    B = dev_zeros(4, 1)
    assert spd.lib().spd_residual_tc(h, 4, 1, A.data_ptr(), 3, B.data_ptr(), 4, B.data_ptr(), 4,
                                     B.data_ptr(), 4, None) == spd.SPD_ERR_ARG


@pytest.mark.parametrize("kappa,prec", [(1e2, "fp16"), (1e6, "fp32"), (1e4, "bf16")])
def test_solve_ir_with_tc_residual(h, kappa, prec):
    """Algorithm 1 with every residual on the tensor cores: float64-level
    backward error judged by the exact residual, forward error as with
    float64 residuals."""
    n, m = 1500, 3
    A, _, _ = W.householder_spectrum(n, kappa, k=16, seed=4)
    x_true = W.gaussian_rhs(n, m, 8)
    B = A @ x_true
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, prec)
    check(h, st)
    sols, reps = {}, {}
    try:
        for resid in ["fp64", "tc"]:
            X = dev_zeros(n, m)
            st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X, {"tol": 1e-14, "resid": resid})
            check(h, st)
            assert rep.berr <= 1e-14
            sols[resid], reps[resid] = host(X), rep
    finally:
        spd.spd_factor_destroy(F)
    x = sols["tc"]
    r = E.residual_exact(A, B, x)
    berr = np.max(np.abs(r), axis=0) / (np.max(np.sum(np.abs(A), axis=1)) * np.max(np.abs(x), axis=0))
    assert np.all(berr <= 1e-14), berr
    xo = oracle.solve(A, B)
    fwd = lambda y: np.max(np.abs(y - xo)) / np.max(np.abs(xo))  # noqa: E731
    assert fwd(x) <= max(8 * fwd(sols["fp64"]), kappa * 2e-15), (fwd(x), fwd(sols["fp64"]))
    assert reps["tc"].iters_high <= reps["fp64"].iters_high + 1


def test_cg_ir_with_tc_residual(h):
    """Algorithm 2 (nested reading) with the outer residual on the tensor cores."""
    n, m = 1200, 2
    A = W.gram_shifted(n, 7, shift=0.1)
    B = W.gaussian_rhs(n, m, 3)
    X = dev_zeros(n, m)
    st, rep = spd.spd_cg(h, dev_sym(A), dev_cols(B), X, "fp32", "none",
                         opts={"tol": 1e-14, "crit": "rel2", "eta": 1e-4, "resid": "tc"})
    check(h, st)
    x = host(X)
    r = E.residual_exact(A, B, x)
    assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(B, axis=0) <= 1.5e-14)
    xo = oracle.solve(A, B)
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))
