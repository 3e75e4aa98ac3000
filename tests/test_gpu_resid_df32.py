"""GPU parity of the float32-pair ("DF32") residual: R = B - A X of
Algorithm 1 (lines 3, 7) and Algorithm 2 (line 2) computed on the float32
units, judged against the correctly rounded residual of the oracle and
against the float64 residual's own error; then Algorithm 1 and Algorithm 2
run end to end with it."""
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


def residuals(h, A, B, X):
    n, m = B.shape
    out = {}
    Ad, Bd, Xd = dev_sym(A), dev_cols(B), dev_cols(X)
    for name, fn in [("fp64", spd.spd_residual), ("df32", spd.spd_residual_df32)]:
        R = dev_zeros(n, m)
        nrm = torch.zeros(3 * m, dtype=torch.float64, device=DEV)
        check(h, fn(h, Ad, Bd, Xd, R, nrm))
        out[name] = (host(R), host(nrm))
    return out


@pytest.mark.parametrize("kind", ["householder", "model", "matern", "spread"])
@pytest.mark.parametrize("n,m", [(300, 1), (1000, 3), (1337, 16), (2111, 20)])
def test_df32_residual_against_exact(h, kind, n, m):
    A = matrix(kind, n)
    g = np.random.default_rng(n * 31 + m)
    X = g.standard_normal((n, m))
    # near-solution right-hand sides: the residual cancels to ~1e-9 of |A||x|
    B = (A @ X) * (1.0 + 1e-9 * g.standard_normal((n, m)))
    res = residuals(h, A, B, X)
    cols = sorted({0, m // 2, m - 1})  # the exact residual is slow: sample columns
    r_ex = E.residual_exact(A, B[:, cols], X[:, cols])
    scale = E.abs_product(A, X[:, cols]) + np.abs(B[:, cols])
    err_df = np.abs(res["df32"][0][:, cols] - r_ex)
    err_64 = np.abs(res["fp64"][0][:, cols] - r_ex)
    # elementwise: products within ~2^-47 |a||x| plus the pair sums'
    # rounding (~2^-43 of each 64-term run), inside 2^-40 |A||x|
    assert np.all(err_df <= 2.0 ** -40 * scale), float(np.max(err_df / scale))
    # the float64 residual, for scale: within n 2^-53 |A||x| (gamma_n)
    assert np.all(err_64 <= n * 2.0 ** -52 * scale)
    # the norms that feed the convergence test
    nr = res["df32"][1].reshape(m, 3)[cols]
    np.testing.assert_allclose(nr[:, 0], np.max(np.abs(r_ex), axis=0), rtol=1e-6, atol=8 * np.max(err_df))
    np.testing.assert_allclose(nr[:, 2], np.max(np.abs(X[:, cols]), axis=0), rtol=0, atol=0)


def test_df32_residual_special_entries(h):
    """Zeros, entries outside the split range [2^-100, 2^100) (float64
    branch), and columns of X scaled by 1e200 and 1e-150."""
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
    res = residuals(h, A, B, X)
    r_ex = E.residual_exact(A, B, X)
    scale = E.abs_product(A, X) + np.abs(B)
    err = np.abs(res["df32"][0] - r_ex)
    assert np.all(err <= 2.0 ** -40 * scale), float(np.max(err / scale))


def test_df32_residual_nonfinite_propagates(h):
    n, m = 260, 2
    A = W.gram_shifted(n, 2)
    A[5, 9] = A[9, 5] = np.nan
    X = np.random.default_rng(1).standard_normal((n, m))
    B = A @ np.nan_to_num(X)
    res = residuals(h, np.array(A), B, X)
    assert np.array_equal(np.isnan(res["df32"][0]), np.isnan(res["fp64"][0]))
    assert np.isnan(res["df32"][0][5, 0]) and np.isnan(res["df32"][0][9, 1])


def test_df32_residual_empty_and_bad_arguments(h):
    Z = dev_zeros(0, 1)
    A0 = torch.zeros(0, 0, dtype=torch.float64, device=DEV)
    assert spd.spd_residual_df32(h, A0, Z, Z, Z) == spd.SPD_OK
    A = dev_sym(np.eye(4))
    B = dev_zeros(4, 1)
    assert spd.lib().spd_residual_df32(h, 4, 1, A.data_ptr(), 3, B.data_ptr(), 4, B.data_ptr(), 4,
                                       B.data_ptr(), 4, None) == spd.SPD_ERR_ARG


@pytest.mark.parametrize("kappa,prec", [(1e2, "fp16"), (1e6, "fp32"), (1e4, "bf16")])
def test_solve_ir_with_df32_residual(h, kappa, prec):
    """Algorithm 1 with the hybrid residual (float32 pairs early, float64 to
    finish): same stopping rule, float64-level backward error judged by the
    exact residual, and a forward error as small as with float64 residuals
    throughout."""
    n, m = 1500, 3
    A, _, _ = W.householder_spectrum(n, kappa, k=16, seed=4)
    x_true = W.gaussian_rhs(n, m, 8)
    B = A @ x_true
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, prec)
    check(h, st)
    sols = {}
    try:
        for resid in ["fp64", "df32"]:
            X = dev_zeros(n, m)
            st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X, {"tol": 1e-14, "resid": resid})
            check(h, st)
            assert rep.berr <= 1e-14
            sols[resid] = host(X)
    finally:
        spd.spd_factor_destroy(F)
    x = sols["df32"]
    r = E.residual_exact(A, B, x)
    berr = np.max(np.abs(r), axis=0) / (np.max(np.sum(np.abs(A), axis=1)) * np.max(np.abs(x), axis=0))
    assert np.all(berr <= 1e-14), berr
    xo = oracle.solve(A, B)
    fwd = lambda y: np.max(np.abs(y - xo)) / np.max(np.abs(xo))  # noqa: E731
    assert fwd(x) <= max(8 * fwd(sols["fp64"]), kappa * 2e-15), (fwd(x), fwd(sols["fp64"]))


def test_cg_ir_with_df32_residual(h):
    """Algorithm 2 (nested reading) with the outer residual and the
    float64 products on the float32 units."""
    n, m = 1200, 2
    A = W.gram_shifted(n, 7, shift=0.1)
    B = W.gaussian_rhs(n, m, 3)
    X = dev_zeros(n, m)
    st, rep = spd.spd_cg(h, dev_sym(A), dev_cols(B), X, "fp32", "none",
                         opts={"tol": 1e-14, "crit": "rel2", "eta": 1e-4, "resid": "df32"})
    check(h, st)
    x = host(X)
    r = E.residual_exact(A, B, x)
    assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(B, axis=0) <= 1.5e-14)
    xo = oracle.solve(A, B)
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))


def test_resid_option_out_of_range_is_rejected(h):
    n = 64
    A = dev_sym(W.gram_shifted(n, 1))
    st, F, _ = spd.spd_factor(h, A, "fp32")
    check(h, st)
    try:
        for code in (4, -1):  # 0-3 are the residual kinds (3: automatic)
            st, _ = spd.spd_solve_ir(h, F, A, dev_cols(np.ones((n, 1))), dev_zeros(n, 1), {"resid": code})
            assert st == spd.SPD_ERR_ARG
    finally:
        spd.spd_factor_destroy(F)
