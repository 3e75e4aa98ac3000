"""AUTO's pre-factor condition bound: a few Lanczos steps on the scaled
float32 matrix give Ritz values inside its spectrum, so theta_max /
theta_min never exceeds kappa_2 of the scaled matrix; above 512 (kappa
u_fp16 > 1/4, the margin of eq. (iterref) the post-factor test uses) no FP16
factor is attempted.  Checked against the exact extreme eigenvalues of the
scaled matrix (numpy, float64)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

from tests.gpu_util import DEV, check, dev_cols, dev_sym, dev_zeros, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def scaled_kappa2(A):
    d = 1.0 / np.sqrt(np.diag(A))
    ev = np.linalg.eigvalsh(A * d[:, None] * d[None, :])
    return ev[-1] / ev[0]


@pytest.mark.parametrize("n,kappa,want", [(4096, 1e2, "fp16"), (4096, 1e4, "fp32"), (4133, 1e6, "fp32")])
def test_bound_below_kappa_and_precision_choice(h, n, kappa, want):
    A, _, _ = W.householder_spectrum(n, kappa, k=32, seed=3)
    k2 = scaled_kappa2(A)
    Ad = dev_sym(A)
    st, F, rep = spd.spd_factor(h, Ad, "auto")
    check(h, st)
    try:
        # a lower bound (float32 products: a relative slack of 1e-3)
        assert 0.0 < rep.cond_lower <= k2 * (1 + 1e-3), (rep.cond_lower, k2)
        assert spd.PREC_NAME[rep.prec_used] == want, (rep.cond_lower, rep.cond_est, k2)
        if rep.cond_lower > 512:
            assert rep.cond_est == 0.0  # no FP16 factor ran, so no estimate from one
        else:
            assert rep.cond_est > 0.0
        m = 2
        B = W.gaussian_rhs(n, m, 5)
        X = dev_zeros(n, m)
        st, r = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        check(h, st)
        assert oracle.berr(A, B, host(X)) <= 1e-14
    finally:
        spd.spd_factor_destroy(F)


def test_bound_on_a_covariance_matrix(h):
    """A model covariance (unit diagonal, dense): the bound stays below the
    exact kappa_2 and, where it is under 512, FP16 is still tried."""
    n = 4500
    A = W.model_covariance(n, 2)
    k2 = scaled_kappa2(A)
    st, F, rep = spd.spd_factor(h, dev_sym(A), "auto")
    check(h, st)
    spd.spd_factor_destroy(F)
    assert 0.0 < rep.cond_lower <= k2 * (1 + 1e-3), (rep.cond_lower, k2)
    if rep.cond_lower <= 512:
        assert rep.cond_est != 0.0


def test_no_bound_below_4096_or_outside_auto(h):
    A, _, _ = W.householder_spectrum(1000, 1e4, k=16, seed=1)
    st, F, rep = spd.spd_factor(h, dev_sym(A), "auto")
    check(h, st)
    spd.spd_factor_destroy(F)
    assert rep.cond_lower == 0.0
    A, _, _ = W.householder_spectrum(4096, 1e4, k=16, seed=1)
    st, F, rep = spd.spd_factor(h, dev_sym(A), "fp32")
    check(h, st)
    spd.spd_factor_destroy(F)
    assert rep.cond_lower == 0.0


def test_bound_is_profiled_as_its_own_phase():
    hh = spd.spd_create(torch.cuda.current_stream())
    try:
        spd.spd_profile_enable(hh, True)
        A, _, _ = W.householder_spectrum(4096, 1e2, k=16, seed=2)
        st, F, rep = spd.spd_factor(hh, dev_sym(A), "auto")
        check(hh, st)
        spd.spd_factor_destroy(F)
        ph = spd.spd_profile_read(hh, "estimate")
        assert ph["launches"] == 1 and ph["ms"] > 0.0  # one record per bound
        # sixteen symmetric products at most, 2 n^2 flops each
        assert 8 * 2.0 * 4096 ** 2 <= ph["flops"] <= 16 * 2.0 * 4096 ** 2
    finally:
        spd.spd_destroy(hh)
