"""GPU parity: factorisation, triangular solves, residual and Algorithm 1
through the C ABI, against the float64 CPU oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W
from oracle.precision import UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

from tests.gpu_util import DEV, check, dev_cols, dev_sym, dev_zeros, factor_L, host  # noqa: E402

SIZES = [1, 2, 3, 31, 33, 127, 128, 129, 300, 513, 1000]
PRECS = ["fp64", "fp32", "tf32", "bf16", "fp16", "fp8"]


@pytest.fixture(scope="module")
def h():
    import torch
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def scaled(A):
    d = 1.0 / np.sqrt(np.diag(A))
    return d, d[:, None] * A * d[None, :]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("prec", PRECS)
def test_factor_matches_oracle(h, n, prec):
    A = W.gram_shifted(n, seed=n, shift=0.5)
    st, F, rep = spd.spd_factor(h, dev_sym(A), prec)
    check(h, st)
    try:
        L, d, p = factor_L(F)
    finally:
        spd.spd_factor_destroy(F)
    d_ref, As = scaled(A)
    np.testing.assert_allclose(d, d_ref, rtol=4e-16, atol=0)
    R = oracle.potrf(As)                       # float64 factor of the scaled matrix
    u = 2.0 ** -53 if prec == "fp64" else max(UNIT_ROUNDOFF[prec], 2.0 ** -24)
    # backward: ||L L^T - As||_F / ||As||_F <= c n u  (u of the operand type)
    bw = np.linalg.norm(L @ L.T - As) / np.linalg.norm(As)
    assert bw <= 4 * max(n, 8) ** 0.5 * u, bw
    # forward against the oracle's factor
    kappa = np.linalg.cond(As)
    fw = np.max(np.abs(L - R.T)) / np.max(np.abs(R))
    assert fw <= 8 * kappa * max(n, 8) ** 0.5 * u, fw


@pytest.mark.parametrize("n", [129, 700, 2100])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "fp16", "fp8"])
def test_left_looking_and_recursive_schedules_agree(h, n, prec):
    """The default block-column (left-looking) schedule, its serial form and
    the recursive one compute the same factor up to rounding: all meet the
    backward bound of the operand type, the recursive one differs by no more
    than it allows, and the serial one is identical."""
    A = W.gram_shifted(n, seed=n + 1, shift=0.5)
    d_ref, As = scaled(A)
    Ls = []
    for flags in [spd.SPD_SCALE_DIAG, spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_RECURSIVE,
                  spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_SERIAL]:
        st, F, rep = spd.spd_factor(h, dev_sym(A), prec, flags)
        check(h, st)
        try:
            L, d, p = factor_L(F)
        finally:
            spd.spd_factor_destroy(F)
        u = max(UNIT_ROUNDOFF[prec], 2.0 ** -24)
        bw = np.linalg.norm(L @ L.T - As) / np.linalg.norm(As)
        assert bw <= 4 * max(n, 8) ** 0.5 * u, (flags, bw)
        Ls.append(L)
    kappa = np.linalg.cond(As)
    diff = np.max(np.abs(Ls[0] - Ls[1]))
    assert diff <= 8 * kappa * max(n, 8) ** 0.5 * max(UNIT_ROUNDOFF[prec], 2.0 ** -24), diff
    # the look-ahead only reorders independent work: the serial schedule
    # gives the same factor bit for bit
    assert np.array_equal(Ls[0], Ls[2])


@pytest.mark.parametrize("n", [3, 129, 700])
@pytest.mark.parametrize("m", [1, 5, 40])
def test_factor_solve_matches_oracle(h, n, m):
    """spd_factor_solve applies the GPU's own float32 factor; the oracle applies
    the same factor in float64 (Section 3.1, eq. (cholesky))."""
    A = W.gram_shifted(n, seed=7, shift=0.5)
    Rh = W.gaussian_rhs(n, m, 3)
    st, F, _ = spd.spd_factor(h, dev_sym(A), "fp32")
    check(h, st)
    try:
        L, d, _ = factor_L(F)
        Z = dev_zeros(n, m)
        check(h, spd.spd_factor_solve(h, F, dev_cols(Rh), Z))
    finally:
        spd.spd_factor_destroy(F)
    z_ref = d[:, None] * oracle.potrs(L.T, d[:, None] * Rh)
    kappa = np.linalg.cond(L) ** 2
    err = np.max(np.abs(host(Z) - z_ref)) / np.max(np.abs(z_ref))
    assert err <= 16 * n * kappa * 2.0 ** -24, err


@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (257, 1), (1000, 16), (1500, 17)])
def test_residual_matches_oracle(h, n, m):
    A = W.gram_shifted(n, seed=2)
    X = W.gaussian_rhs(n, m, 4)
    B = W.gaussian_rhs(n, m, 5)
    R = dev_zeros(n, m)
    import torch
    cn = torch.zeros(3 * m, dtype=torch.float64, device=DEV)
    check(h, spd.spd_residual(h, dev_sym(A), dev_cols(B), dev_cols(X), R, cn))
    R_ref = oracle.residual(A, B, X)
    scale = np.abs(A) @ np.abs(X) + np.abs(B)
    assert np.all(np.abs(host(R) - R_ref) <= 2 * n * 2.0 ** -53 * scale)
    cn = host(cn).reshape(m, 3)
    np.testing.assert_allclose(cn[:, 0], np.abs(R_ref).max(axis=0), rtol=1e-10)
    np.testing.assert_allclose(cn[:, 1], np.linalg.norm(R_ref, axis=0), rtol=1e-10)
    np.testing.assert_allclose(cn[:, 2], np.abs(X).max(axis=0), rtol=0)


@pytest.mark.parametrize("prec", [p for p in PRECS if p != "fp8"])
@pytest.mark.parametrize("n,m", [(1, 1), (2, 2), (129, 3), (300, 1), (1024, 1), (777, 16), (400, 33)])
def test_solve_ir_matches_oracle(h, prec, n, m):
    """Algorithm 1: low-precision factor, float64 refinement to backward error
    <= 1e-14; forward error within 10 kappa 1e-16 of the oracle's solution."""
    A = W.gram_shifted(n, seed=0, shift=0.1)
    x_true = W.gaussian_rhs(n, m, 1)
    B = A @ x_true
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, prec)
    check(h, st)
    X = dev_zeros(n, m)
    try:
        st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    Xg = host(X)
    assert oracle.berr(A, B, Xg) <= 1e-14
    assert rep.berr <= 1e-14
    Xo = oracle.solve(A, B)
    kappa = np.linalg.cond(A)
    fw = np.max(np.abs(Xg - Xo), axis=0) / np.max(np.abs(Xo), axis=0)
    assert np.all(fw <= 10 * kappa * 1e-16 * max(1.0, np.sqrt(n) / 8)), fw
    assert rep.iters_high == rep.iters_low and rep.iters_low >= 1


def test_solve_ir_host_buffers(h):
    n, m = 513, 4
    A = W.gram_shifted(n, seed=11, shift=0.1)
    B = np.asfortranarray(W.gaussian_rhs(n, m, 12))
    X = np.zeros((n, m), order="F")
    st, rep = spd.spd_solve_ir_host(h, np.ascontiguousarray(A), B, X, "bf16")
    check(h, st)
    assert oracle.berr(A, B, X) <= 1e-14


def test_solve_ir_host_buffers_grow_and_shrink():
    """The handle keeps the device copies between host-buffer calls: sizes
    that grow (the copies are reallocated), shrink (a prefix is reused) and
    grow again all solve correctly, with strided host A (lda > n)."""
    import torch
    hh = spd.spd_create(torch.cuda.current_stream())
    try:
        for n, m, seed in [(200, 1, 1), (700, 5, 2), (129, 3, 3), (700, 9, 4), (1000, 2, 5)]:
            A = W.gram_shifted(n, seed=seed, shift=0.1)
            # column-major with lda = n + 7: row j of Acm holds column j of A, then 7 pad entries
            Acm = np.zeros((n, n + 7))
            Acm[:, :n] = A.T
            B = np.asfortranarray(W.gaussian_rhs(n, m, seed + 10))
            X = np.zeros((n, m), order="F")
            st = spd.lib().spd_solve_ir_host(hh, n, m, Acm.ctypes.data, n + 7, B.ctypes.data, n,
                                             X.ctypes.data, n, spd.PREC["fp32"], None, None)
            check(hh, st)
            assert oracle.berr(A, B, X) <= 1e-14, (n, m)
    finally:
        spd.spd_destroy(hh)


def test_not_spd_reports_failing_column(h):
    n = 300
    for k in (30, 130, 255):
        A = np.eye(n)
        A[k, k + 1] = A[k + 1, k] = 2.0   # leading minor of order k+2 is indefinite
        st, F, rep = spd.spd_factor(h, dev_sym(A), "fp32")
        check(h, st, spd.SPD_ERR_NOT_SPD)
        assert F is None and rep.info == k + 2
    A = np.eye(40)
    A[17, 17] = -1.0
    st, F, rep = spd.spd_factor(h, dev_sym(A), "bf16")
    check(h, st, spd.SPD_ERR_NOT_SPD)
    assert rep.info == 18


def test_nonfinite_input_rejected(h):
    A = W.gram_shifted(64, seed=1)
    A[40, 3] = A[3, 40] = np.nan
    st, F, rep = spd.spd_factor(h, dev_sym(A), "fp32")
    check(h, st, spd.SPD_ERR_ARG)


def test_bad_arguments(h):
    import torch
    A = dev_sym(W.gram_shifted(8, seed=1))
    F = None
    st, F, rep = spd.spd_factor(h, A, "fp32")
    check(h, st)
    B = dev_zeros(8, 1)
    X = dev_zeros(7, 1)
    lib = spd.lib()
    st = lib.spd_solve_ir(h, F, 8, 1, A.data_ptr(), 8, B.data_ptr(), 8, X.data_ptr(), 7, None, None)
    assert st == spd.SPD_ERR_ARG
    st = lib.spd_factor(h, 8, A.data_ptr(), 8, 42, 1, None, None)
    assert st == spd.SPD_ERR_ARG
    spd.spd_factor_destroy(F)
    # n = 0 is a no-op
    st = lib.spd_solve_ir(h, None, 0, 1, None, 1, None, 1, None, 1, None, None)
    assert st in (spd.SPD_OK, spd.SPD_ERR_ARG)
    torch.cuda.synchronize()


def test_polish_off_meets_backward_error_only(h):
    n, m = 700, 3
    A = W.gram_shifted(n, seed=5, shift=0.1)
    B = W.gaussian_rhs(n, m, 6)
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, "fp16")
    check(h, st)
    X = dev_zeros(n, m)
    st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X, {"polish": 0})
    spd.spd_factor_destroy(F)
    check(h, st)
    assert oracle.berr(A, B, host(X)) <= 1e-14


def test_auto_precision_picks_per_matrix(h):
    """AUTO keeps FP16 for a well-conditioned matrix and moves to FP32 when
    the estimated kappa_1 / sqrt(n) u_fp16 exceeds 1/4; both reach
    berr <= 1e-14."""
    n, m = 640, 2
    for kappa, want in [(1e2, "fp16"), (1e6, "fp32")]:
        A, lam, V = W.householder_spectrum(n, kappa, k=32, seed=1)
        B = W.gaussian_rhs(n, m, 2)
        Ad = dev_sym(A)
        st, F, frep = spd.spd_factor(h, Ad, "auto")
        check(h, st)
        assert spd.PREC_NAME[frep.prec_used] == want, (kappa, frep.cond_est)
        if want == "fp16":  # the estimate exists when the FP16 factor did not break down
            assert 0.2 * kappa <= frep.cond_est <= 10 * n * kappa
        X = dev_zeros(n, m)
        st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        spd.spd_factor_destroy(F)
        check(h, st)
        assert oracle.berr(A, B, host(X)) <= 1e-14


def test_iterref_planted_perturbation_on_gpu(h):
    """eq. (iterref) / Fig. 3b on the GPU: refine A x = b with the factor of
    A + dA.  Small ||A^{-1} dA|| converges without help and the sweep count
    grows with the perturbation; dA = -0.6 A makes the plain loop diverge,
    and the stagnation fallback (float64 CG preconditioned by the factor)
    still reaches berr <= 1e-14."""
    n, m = 384, 2
    A = W.gram_shifted(n, seed=3, shift=0.5)
    B = W.gaussian_rhs(n, m, 4)
    Ad, Bd = dev_sym(A), dev_cols(B)
    g = np.random.default_rng(5)
    G = g.standard_normal((n, n))
    P = G @ G.T / n
    Ainv = np.linalg.inv(A)
    its = []
    for t in (1e-6, 1e-3, 1e-1):
        dA = P * (t / np.linalg.norm(Ainv @ P, np.inf))
        st, F, _ = spd.spd_factor(h, dev_sym(A + dA), "fp64")
        check(h, st)
        X = dev_zeros(n, m)
        st, rep = spd.spd_solve_ir(h, F, Ad, Bd, X, {"polish": 0})
        spd.spd_factor_destroy(F)
        check(h, st)
        assert rep.fell_back == 0
        assert oracle.berr(A, B, host(X)) <= 1e-14
        its.append(rep.iters_high)
    assert its == sorted(its) and its[-1] > its[0]
    st, F, _ = spd.spd_factor(h, dev_sym(0.4 * A), "fp32")
    check(h, st)
    X = dev_zeros(n, m)
    st, rep = spd.spd_solve_ir(h, F, Ad, Bd, X)
    spd.spd_factor_destroy(F)
    check(h, st)
    assert rep.fell_back == 1
    assert oracle.berr(A, B, host(X)) <= 1e-14


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
@pytest.mark.parametrize("n", [257, 1000, 2049])
def test_tensor_core_and_cuda_core_factors_agree(h, prec, n):
    """The tcgen05 trailing update and the CUDA-core reference engine use the
    same rounded operands; their factors differ only by float32 summation
    order."""
    A = W.gram_shifted(n, seed=n + 1, shift=0.5)
    Ad = dev_sym(A)
    st, F1, _ = spd.spd_factor(h, Ad, prec)
    check(h, st)
    st, F2, _ = spd.spd_factor(h, Ad, prec, spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_CUDA_CORES)
    check(h, st)
    try:
        L1, _, _ = factor_L(F1)
        L2, _, _ = factor_L(F2)
    finally:
        spd.spd_factor_destroy(F1)
        spd.spd_factor_destroy(F2)
    kappa = np.linalg.cond(L2) ** 2
    assert np.max(np.abs(L1 - L2)) <= 64 * kappa * n * 2.0 ** -24


@pytest.mark.parametrize("n,m", [(129, 3), (700, 1), (1100, 8), (2049, 2)])
def test_fp8_update_factor_refines_where_iterref_holds(h, n, m):
    """FP8 (e4m3) trailing-update operands put errors of about u = 2^-4 into
    the factor: eq. (iterref) holds for a well-conditioned matrix (kappa ~ 1.6
    here), so Algorithm 1 reaches backward error 1e-14 with no fallback; the
    sweeps needed are more than for FP16 operands but bounded."""
    A = np.eye(n) + 0.3 * W.gram_shifted(n, seed=n, shift=0.0)
    x_true = W.gaussian_rhs(n, m, 2)
    B = A @ x_true
    Ad = dev_sym(A)
    sweeps = {}
    for prec in ("fp8", "fp16"):
        st, F, _ = spd.spd_factor(h, Ad, prec)
        check(h, st)
        X = dev_zeros(n, m)
        try:
            st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X, {"fallback": 0})
            check(h, st)
        finally:
            spd.spd_factor_destroy(F)
        Xg = host(X)
        assert oracle.berr(A, B, Xg) <= 1e-14 and rep.fell_back == 0, prec
        Xo = oracle.solve(A, B)
        kappa = np.linalg.cond(A)
        fw = np.max(np.abs(Xg - Xo), axis=0) / np.max(np.abs(Xo), axis=0)
        assert np.all(fw <= 10 * kappa * 1e-16 * max(1.0, np.sqrt(n) / 8)), (prec, fw)
        sweeps[prec] = rep.iters_high
    assert sweeps["fp16"] <= sweeps["fp8"] <= 30, sweeps


def test_fp8_update_factor_falls_back_where_iterref_fails(h):
    """The exponential-kernel covariance matrix (n = 4096 points in the unit
    cube, ell = 0.1, nugget 1e-3): the FP8-update factor does not break down,
    but refinement with it stagnates (two sweeps in a row shrink the error by
    less than half: eq. (iterref) fails in practice); the fallback -- float64
    CG preconditioned by the same factor, Section 3.1: any inner solver that
    contracts will do -- takes over and reaches backward error 1e-14."""
    n = 4096
    A, _ = W.exp_kernel_cov(n, ell=0.1, nugget=1e-3, seed=0)
    B = W.gaussian_rhs(n, 2, 4)
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, "fp8")
    check(h, st)
    X = dev_zeros(n, 2)
    try:
        st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    assert rep.fell_back == 1
    assert oracle.berr(A, B, host(X)) <= 1e-14


@pytest.mark.parametrize("prec,kappa", [("fp8", 1e4), ("fp16", 1e6), ("bf16", 1e6)])
def test_shifted_factor_after_breakdown(h, prec, kappa):
    """A low-precision factor of a prescribed-spectrum matrix that breaks down
    (a non-positive pivot: the updates' rounding exceeds what is left of a
    pivot).  With SPD_FACTOR_SHIFT the factorisation is retried on the scaled
    matrix plus sigma I (sigma = 2u, 8u, 32u, ... of the update operands); the
    shifted factor drives the factor-preconditioned CG fallback to backward
    error 1e-14."""
    n = 1024
    A, lam, V = W.householder_spectrum(n, kappa, k=32, seed=1)
    B = W.gaussian_rhs(n, 2, 4)
    Ad = dev_sym(A)
    st, F, rep = spd.spd_factor(h, Ad, prec)
    check(h, st, spd.SPD_ERR_NOT_SPD)
    assert F is None and rep.info > 0
    st, F, rep = spd.spd_factor(h, Ad, prec, spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_SHIFT)
    check(h, st)
    u = UNIT_ROUNDOFF[prec]
    k = np.log2(rep.shift / (2 * u)) / 2  # sigma = 2u 4^k
    assert 0 < rep.shift <= 1 and k == round(k) and rep.info == 0
    X = dev_zeros(n, 2)
    try:
        st, srep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    assert srep.fell_back == 1
    assert oracle.berr(A, B, host(X)) <= 1e-14
