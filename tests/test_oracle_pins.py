"""Pins of the CPU oracle against facts fixed by the mathematics and the paper.

None of these re-types the oracle's own formulas: each checks the oracle
against a closed form, an exact rational computation, a library routine, an
invariant or the paper's own statements (Section 3, eq. (cholesky), eq.
(iterref), Algorithms 1 and 2, Fig. 3b, Section 4).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

U64 = 2.0 ** -53


# --------------------------------------------------------------------------
# Cholesky factor (Section 3.1, eq. (cholesky)): closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 17, 64])
def test_potrf_min_matrix_closed_form(n):
    # A_ij = min(i, j) (1-based) has R_ij = 1 for all i <= j.
    i = np.arange(1, n + 1)
    A = np.minimum(i[:, None], i[None, :]).astype(float)
    R = oracle.potrf(A)
    assert np.array_equal(R, np.triu(np.ones((n, n))))


@pytest.mark.parametrize("n", [2, 3, 10, 50])
def test_potrf_laplacian_closed_form(n):
    # tridiag(-1, 2, -1): R_kk = sqrt((k+1)/k), R_{k,k+1} = -sqrt(k/(k+1)), k 1-based.
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    R = oracle.potrf(A)
    k = np.arange(1, n + 1)
    np.testing.assert_allclose(np.diag(R), np.sqrt((k + 1) / k), rtol=4 * n * U64)
    np.testing.assert_allclose(np.diag(R, 1), -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=4 * n * U64)
    assert np.all(np.triu(R, 2) == 0) and np.all(np.tril(R, -1) == 0)


def test_potrf_identity_and_diagonal():
    assert np.array_equal(oracle.potrf(np.eye(7)), np.eye(7))
    d = np.array([4.0, 9.0, 0.25, 2.0])
    np.testing.assert_allclose(oracle.potrf(np.diag(d)), np.diag(np.sqrt(d)), rtol=0, atol=0)


def test_potrf_reads_only_lower_triangle():
    A = W.gram_shifted(40, seed=3)
    B = A.copy()
    B[np.triu_indices(40, 1)] = 1e300  # garbage above the diagonal
    assert np.array_equal(oracle.potrf(A), oracle.potrf(B))


@pytest.mark.parametrize("n", [33, 200])
def test_potrf_backward_invariant(n):
    A = W.gram_shifted(n, seed=1)
    R = oracle.potrf(A)
    rel = np.linalg.norm(R.T @ R - A) / np.linalg.norm(A)
    assert rel <= 2 * n * U64
    # agrees with LAPACK's factor (numpy: L lower with A = L L^T, so R = L^T)
    L = np.linalg.cholesky(A)
    np.testing.assert_allclose(R, L.T, rtol=0, atol=50 * n * U64 * np.abs(L).max())


U32 = 2.0 ** -24


@pytest.mark.parametrize("n", [1, 7, 17, 64])
def test_potrf_f32_min_matrix_closed_form(n):
    # every step of the single-precision factor of min(i, j) is exact in float32
    i = np.arange(1, n + 1)
    A = np.minimum(i[:, None], i[None, :]).astype(float)
    R = oracle.potrf_f32(A)
    assert R.dtype == np.float32
    assert np.array_equal(R, np.triu(np.ones((n, n), dtype=np.float32)))


@pytest.mark.parametrize("n", [33, 200])
def test_potrf_f32_backward_bound_and_lapack_single(n):
    import scipy.linalg as sl
    A = W.gram_shifted(n, seed=5)
    R = oracle.potrf_f32(A).astype(np.float64)
    # backward error of a single-precision Cholesky: ||R^T R - A|| <= c n u32 ||A||
    rel = np.linalg.norm(R.T @ R - A) / np.linalg.norm(A)
    assert rel <= 2 * n * U32
    # and it is a single-precision factor, not a float64 one rounded at the end
    R64 = oracle.potrf(A)
    assert np.max(np.abs(R - R64)) > 4 * U64 * np.abs(R64).max()
    # LAPACK's spotrf (scipy on a float32 matrix) agrees to the single-precision level
    Rl = sl.cholesky(A.astype(np.float32), lower=False).astype(np.float64)
    assert Rl.dtype == np.float64
    kappa = np.linalg.cond(A)
    np.testing.assert_allclose(R, Rl, rtol=0, atol=10 * n * U32 * kappa * np.abs(Rl).max())


def test_potrs_f32_exact_on_integer_factor():
    # R = triu(ones) (the factor of min(i, j)) with an integer right-hand side:
    # both substitutions stay in small integers, exact in float32
    n = 17
    i = np.arange(1, n + 1)
    A = np.minimum(i[:, None], i[None, :]).astype(float)
    x = np.arange(-8, 9, dtype=float)[:, None] * np.array([[1.0, -2.0]])
    R = np.triu(np.ones((n, n), dtype=np.float32))
    X = oracle.potrs_f32(R, A @ x)
    assert np.array_equal(X, x)


@pytest.mark.parametrize("n", [50, 300])
def test_potrs_f32_matches_float64_substitution_of_the_same_factor(n):
    import scipy.linalg as sl
    A = W.gram_shifted(n, seed=6)
    R = oracle.potrf_f32(A)
    B = W.gaussian_rhs(n, 3, 8)
    X = oracle.potrs_f32(R, B)
    R64 = R.astype(np.float64)
    Y = sl.solve_triangular(R64, B, trans="T", lower=False)
    X64 = sl.solve_triangular(R64, Y, lower=False)
    kappa = np.linalg.cond(R64) ** 2
    assert np.max(np.abs(X - X64)) <= 4 * n * U32 * kappa * np.max(np.abs(X64))
    # single-precision solves: they are not float64-accurate either
    assert np.max(np.abs(X - X64)) > 4 * U64 * np.max(np.abs(X64))


def test_potrf_not_spd_reports_column():
    A = np.eye(5)
    A[3, 3] = -1.0
    with pytest.raises(ValueError) as e:
        oracle.potrf(A)
    assert e.value.args[1] == 4  # 1-based, LAPACK convention


# --------------------------------------------------------------------------
# Solve X = R^{-1} R^{-T} B: exact rationals and a planted solution
# --------------------------------------------------------------------------
def _exact_solve(A_int, b_int):
    n = len(b_int)
    M = [[Fraction(int(A_int[i][j])) for j in range(n)] + [Fraction(int(b_int[i]))] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("n,seed", [(1, 0), (3, 1), (5, 2), (8, 3), (8, 4)])
def test_solve_matches_exact_rational_elimination(n, seed):
    g = np.random.default_rng(seed)
    G = g.integers(-3, 4, size=(n, n))
    A = G @ G.T + np.eye(n, dtype=np.int64)
    b = g.integers(-5, 6, size=n)
    x_exact = np.array([float(v) for v in _exact_solve(A.tolist(), b.tolist())])
    x = oracle.solve(A.astype(float), b.astype(float)[:, None])[:, 0]
    kappa = np.linalg.cond(A.astype(float))
    assert np.max(np.abs(x - x_exact)) <= 8 * n * kappa * U64 * np.max(np.abs(x_exact))


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_solve_planted_solution_known_eigendecomposition(kappa):
    n = 120
    A, lam, V = W.householder_spectrum(n, kappa, k=8, seed=5)
    # Q from its reflectors, built independently of the oracle
    Q = np.eye(n)
    for j in range(V.shape[1]):
        v = V[:, j:j + 1]
        Q = Q @ (np.eye(n) - 2 * v @ v.T)
    x_true = W.gaussian_rhs(n, 3, 11)
    b = Q @ (lam[:, None] * (Q.T @ x_true))
    x = oracle.solve(A, b)
    fwd = np.max(np.abs(x - x_true)) / np.max(np.abs(x_true))
    assert fwd <= 10 * kappa * 1e-16 * n ** 0.5


def test_berr_and_residual_hand_example():
    A = np.array([[4.0, 1.0], [1.0, 3.0]])
    x = np.array([[1.0], [2.0]])
    b = np.array([[6.0], [7.5]])  # A x = [6, 7]
    r = oracle.residual(A, b, x)
    np.testing.assert_array_equal(r, [[0.0], [0.5]])
    # ||r||_inf / (||A||_inf ||x||_inf) = 0.5 / (5 * 2)
    assert oracle.berr(A, b, x) == pytest.approx(0.05, rel=0, abs=1e-17)
    assert oracle.norm_inf(A) == 5.0


# --------------------------------------------------------------------------
# Conjugate gradients
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 5, 8])
def test_cg_terminates_in_n_steps(n):
    g = np.random.default_rng(n)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.linspace(1.0, 9.0, n)  # kappa <= 10
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    b = g.standard_normal((n, 1))
    X, it, rr, ok = oracle.cg(A, b, tol_rel=1e-13, maxit=n)
    assert ok and it[0] <= n
    np.testing.assert_allclose(X, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_cg_distinct_eigenvalues():
    # a diagonal matrix with 3 distinct eigenvalues: exact in 3 steps
    d = np.array([1.0, 1.0, 2.0, 2.0, 2.0, 5.0, 5.0, 1.0])
    A = np.diag(d)
    b = np.arange(1, 9, dtype=float)[:, None]
    X, it, rr, ok = oracle.cg(A, b, tol_rel=1e-14, maxit=8)
    assert ok and it[0] == 3
    np.testing.assert_allclose(X[:, 0], b[:, 0] / d, rtol=1e-13)


def test_cg_agrees_with_cholesky():
    A = W.gram_shifted(300, seed=0, shift=0.1)
    B = W.gaussian_rhs(300, 2, 4)
    X, it, rr, ok = oracle.cg(A, B, tol_rel=1e-14)
    assert ok
    Xc = oracle.solve(A, B)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - Xc)) <= 10 * kappa * 1e-14 * np.max(np.abs(Xc))


# --------------------------------------------------------------------------
# Algorithm 1 and eq. (iterref)
# --------------------------------------------------------------------------
def test_chol_ir_single_factor_reaches_double_accuracy():
    n = 256
    A = W.gram_shifted(n, seed=0, shift=0.1)
    x_true = W.gaussian_rhs(n, 1, 7)
    b = A @ x_true
    Rt = oracle.potrf_f32(A)
    X, it, err, ok = oracle.chol_ir(A, Rt, b, tol=1e-14)
    assert ok and err[0] <= 1e-14
    assert 1 <= it[0] <= 6
    # the float64 factor needs no sweep at all
    _, it0, _, ok0 = oracle.chol_ir_f64(A, oracle.potrf(A), b, tol=1e-14)
    assert ok0 and it0[0] == 0


def test_iterref_condition_planted_perturbation():
    """eq. (iterref): the inner solve is (A + dA) z = r.  The error obeys
    e' = (A + dA)^{-1} dA e, so refinement converges whenever
    ||A^{-1} dA|| < 1/2 for any sign of dA, and for every ||A^{-1} dA|| < 1
    when dA is positive semidefinite.  A negative dA with
    1/2 < ||A^{-1} dA|| < 1 can diverge: the printed bound is read as
    "less than one half" for indefinite perturbations."""
    n = 80
    A = W.gram_shifted(n, seed=2, shift=0.5)
    b = W.gaussian_rhs(n, 1, 3)
    Ainv = np.linalg.inv(A)
    g = np.random.default_rng(9)
    S = g.standard_normal((n, n))
    S = 0.5 * (S + S.T)                      # indefinite
    G = g.standard_normal((n, n))
    P = G @ G.T / n                          # positive semidefinite
    for E, target in [(S, 0.3), (S, 0.45), (P, 0.9)]:
        dA = E * (target / np.linalg.norm(Ainv @ E, np.inf))
        assert np.linalg.norm(Ainv @ dA, np.inf) == pytest.approx(target)
        X, it, err, ok = oracle.chol_ir_f64(A, oracle.potrf(A + dA), b, tol=1e-14, maxit=2000)
        assert ok, target
    # sufficient, not necessary: dA = 3A gives e' = (3/4) e
    X, it, err, ok = oracle.chol_ir_f64(A, oracle.potrf(4.0 * A), b, tol=1e-14, maxit=400)
    assert ok
    # dA = -0.6 A: ||A^{-1} dA|| = 0.6 < 1 yet e' = -1.5 e diverges
    X, it, err, ok = oracle.chol_ir_f64(A, oracle.potrf(0.4 * A), b, tol=1e-14, maxit=60)
    assert not ok


def test_perturbed_factor_sweep_fig3b():
    """Fig. 3b: a float64 factor perturbed by an upper-triangular E with
    ||E||_2 / ||R||_2 = 10^gamma still converges for every gamma in
    {-1, -3.25, -5.5, -7.75, -10}; the iteration count grows with gamma."""
    n = 150
    A = W.gram_shifted(n, seed=4, shift=1.0)
    b = W.uniform_rhs(n, 1, 0)
    R = oracle.potrf(A)
    g = np.random.default_rng(12)
    E0 = np.triu(g.standard_normal((n, n)))
    E0 /= np.linalg.norm(E0, 2)
    its = []
    for gamma in [-10, -7.75, -5.5, -3.25, -1]:
        Rp = R + (10.0 ** gamma) * np.linalg.norm(R, 2) * E0
        X, it, err, ok = oracle.chol_ir_f64(A, Rp, b, tol=1e-14, maxit=500)
        assert ok, gamma
        its.append(int(it[0]))
    assert its == sorted(its)
    assert its[-1] > its[0]


# --------------------------------------------------------------------------
# Algorithm 2 (nested reading) and Section 4's model covariance
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d", [1, 2, 4])
def test_model_covariance_is_spd(d):
    A = W.model_covariance(300, d)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0
    oracle.potrf(A)  # no breakdown


def test_cg_ir_paper_tolerance_and_decay_ordering():
    """Section 4: tolerance 1e-5 on U[0,1] right-hand sides; stronger decay
    (larger d) is easier for CG; the result is a solution of A x = b."""
    n = 1500
    lows = {}
    for d in (1, 4):
        A = W.model_covariance(n, d)
        b = W.uniform_rhs(n, 1, 0)
        X, lo, hi, fe, ok = oracle.cg_ir(A, b, tol=1e-5, crit="abs2", eta=0.0)
        assert ok and fe[0] < 1e-5
        assert np.linalg.norm(oracle.residual(A, b, X)) < 1e-5
        lows[d] = int(lo[0])
    assert lows[1] >= lows[4]


def test_banded_cg_ir_equals_dense_counts_at_strong_decay():
    """Section 4.1: at d = 4 the banded (bandwidth 33) inner solver needs the
    same low/high iteration counts as the dense one (at n = 70000).  At this
    small n the entries dropped from the band are relatively larger, so the
    pin is a band: low counts within 15 %, high counts within one."""
    n = 2000
    A = W.model_covariance(n, 4)
    b = W.uniform_rhs(n, 1, 0)
    _, lo_d, hi_d, _, ok1 = oracle.cg_ir(A, b, tol=1e-5, crit="abs2", eta=0.0)
    _, lo_b, hi_b, fe, ok2 = oracle.cg_ir(A, b, band=16, tol=1e-5, crit="abs2", eta=0.0)
    assert ok1 and ok2
    assert abs(int(lo_b[0]) - int(lo_d[0])) <= 0.15 * lo_d[0] and abs(int(hi_b[0]) - int(hi_d[0])) <= 1


def test_cg_ir_relative_target_reaches_double_accuracy():
    A = W.gram_shifted(400, seed=0, shift=0.1)
    b = W.gaussian_rhs(400, 1, 1)
    X, lo, hi, fe, ok = oracle.cg_ir(A, b, tol=1e-14, crit="rel", eta=1e-4)
    assert ok
    assert np.linalg.norm(oracle.residual(A, b, X)) <= 1e-14 * np.linalg.norm(b)
    assert hi[0] >= 2  # single-precision inner matvecs cannot get there in one sweep


# --------------------------------------------------------------------------
# Learned preconditioner oracle (no paper counterpart): definitions pinned
# against constructions whose answer is known
# --------------------------------------------------------------------------
def test_learned_oracle_exact_preconditioner_gives_zero_loss():
    """If Dh + Uh Uh^T equals the scaled matrix exactly, M = A^{-1} and the
    probe loss vanishes."""
    from oracle import learned as LO
    g = np.random.default_rng(0)
    n, H = 40, 8
    U = g.standard_normal((n, LO.RANK)) * 0.1
    dh = 1.0 - np.sum(U * U, axis=1)           # unit diagonal: diag(Dh + U U^T) = 1
    assert dh.min() > 0.2
    Ah = np.diag(dh) + U @ U.T
    t = 0.5 + g.random(n)
    A = t[:, None] * Ah * t[None, :]           # S = diag(A)^{-1/2} = 1/t, so S A S = Ah
    O = np.concatenate([np.log(np.expm1(dh - 1e-3))[:, None], U], axis=1)
    M = LO.precond(O, A)
    np.testing.assert_allclose(M @ A, np.eye(n), atol=1e-9)
    # a network whose last layer outputs O through its bias only
    count = H * LO.NFEAT + H + H * H + H + (1 + LO.RANK) * H + 1 + LO.RANK
    p = np.zeros(count)
    F = np.zeros((n, LO.NFEAT))
    Z = g.standard_normal((n, 3))
    assert LO.loss(p, H, A, F, Z) > 0.1            # M = S^2 here: not the inverse
    assert np.all(np.linalg.eigvalsh(LO.precond(LO.forward(p, F, H), A)) > 0)


def test_learned_oracle_features_on_a_known_matrix():
    from oracle import learned as LO
    A = np.array([[4.0, 2.0, 0.0], [2.0, 4.0, 1.0], [0.0, 1.0, 1.0]])
    coords = np.array([[0.0, 0.5], [0.25, 1.0], [1.0, 0.0]])
    F = LO.features(A, coords, 0.1, 1e-2)
    # scaled |A|: rows [1, .5, 0], [.5, 1, .5], [0, .5, 1]
    np.testing.assert_allclose(F[:, 12], [1.5 / 3, 2.0 / 3, 1.5 / 3])
    np.testing.assert_allclose(F[:, 14], [0.5, 0.5, 0.5])
    np.testing.assert_allclose(F[1, 4:8], [np.sin(np.pi / 4), np.cos(np.pi / 4), 0.0, -1.0], atol=1e-15)
    assert F[0, 2] == np.log(0.1) and F[0, 15] == 1.0


def test_learned_oracle_fd_gradient_matches_complex_step():
    """Central differences of the probe loss against the complex-step
    derivative Im L(p + i h v) / h, exact to rounding for an analytic L."""
    from oracle import learned as LO
    g = np.random.default_rng(4)
    n, H = 30, 6
    A = W.gram_shifted(n, 3, shift=0.5)
    F = g.standard_normal((n, LO.NFEAT))
    count = H * LO.NFEAT + H + H * H + H + (1 + LO.RANK) * H + 1 + LO.RANK
    p = g.standard_normal(count) * 0.2
    Z = g.standard_normal((n, 2))
    T = np.linalg.solve(A, Z[:, :1])
    for seed in range(3):
        v = np.random.default_rng(seed).standard_normal(count)
        h = 1e-30
        cs = np.imag(LO.loss(p + 1j * h * v, H, A, F, Z, T, 0.3)) / h
        fd = LO.fd_grad(p, H, A, F, Z, [v], T, 0.3, h=1e-5)[0]
        assert abs(fd - cs) <= 1e-6 * abs(cs) + 1e-12, (fd, cs)


# ---------------------------------------------------------------------------
# the correctly rounded residual (judge of the float32-pair residual)
# ---------------------------------------------------------------------------
def test_exact_residual_matches_rational_arithmetic():
    from oracle import exact as E
    g = np.random.default_rng(17)
    for n, m in [(1, 1), (7, 3), (33, 2)]:
        A = g.standard_normal((n, n)) * np.exp(g.uniform(-30, 30, (n, n)))
        X = g.standard_normal((n, m)) * np.exp(g.uniform(-10, 10, (n, m)))
        B = A @ X * (1 + 1e-9 * g.standard_normal((n, m)))  # heavy cancellation
        assert np.array_equal(E.residual_exact(A, B, X), E.residual_fraction(A, B, X))


def test_exact_residual_integer_inputs():
    """Integer data below 2^20: the residual is an exact integer."""
    from oracle import exact as E
    g = np.random.default_rng(3)
    A = g.integers(-2**20, 2**20, (25, 25))
    X = g.integers(-2**20, 2**20, (25, 2))
    B = g.integers(-2**40, 2**40, (25, 2))
    want = (B.astype(object) - A.astype(object).dot(X.astype(object))).astype(np.float64)
    got = E.residual_exact(A.astype(np.float64), B.astype(np.float64), X.astype(np.float64))
    assert np.array_equal(got, want)


def test_exact_residual_beats_float64_residual():
    """The plain float64 residual differs from the exact one by rounding only
    (bounded by gamma_n |A||x|), and the exact one is what fractions give."""
    from oracle import exact as E
    g = np.random.default_rng(5)
    n = 300
    A = g.standard_normal((n, n))
    x = g.standard_normal((n, 1))
    b = A @ x
    r_ex = E.residual_exact(A, b, x)
    r_64 = oracle.residual(A, b, x)
    gam = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
    assert np.all(np.abs(r_64 - r_ex) <= gam * (np.abs(b) + E.abs_product(A, x)))
    assert np.max(np.abs(r_64 - r_ex)) > 0  # the float64 residual really rounds
    i = 11
    assert r_ex[i, 0] == E.residual_fraction(A[i:i + 1], b[i:i + 1], x)[0, 0]


# --------------------------------------------------------------------------
# Reference solution from a known eigendecomposition (the prescribed-spectrum
# test matrices): pinned to LAPACK's solve and to two closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,k,kappa", [(300, 8, 1e4), (257, 32, 1e2), (64, 1, 1e6)])
def test_spectral_solve_matches_lapack(n, k, kappa):
    A, lam, V = W.householder_spectrum(n, kappa, k=k, seed=n)
    B = W.gaussian_rhs(n, 3, n + 1)
    X = oracle.spectral_solve(V, lam, B)
    Xl = np.linalg.solve(A, B)
    # both solve the assembled A up to its assembly error (a few k u ||A||),
    # amplified by kappa
    assert np.max(np.abs(X - Xl)) <= 1e-13 * kappa * np.max(np.abs(Xl))
    # and the residual against the assembled matrix is at that level too
    assert np.max(np.abs(B - A @ X)) <= 1e-13 * kappa * np.max(np.abs(B))


def test_spectral_solve_closed_forms():
    n = 50
    V = W.householder_vectors(n, 4, seed=3)
    B = W.gaussian_rhs(n, 2, 4)
    # all eigenvalues 1: A = Q Q^T = I
    assert np.allclose(oracle.spectral_solve(V, np.ones(n), B), B, rtol=0, atol=1e-14)
    # a single reflection H = I - 2 v v^T with eigenvalues lam: H diag(lam) H;
    # its inverse applied to B is H diag(1/lam) H B, formed densely here
    v = V[:, :1]
    H = np.eye(n) - 2.0 * v @ v.T
    lam = np.linspace(1.0, 7.0, n)
    ref = H @ (np.diag(1.0 / lam) @ (H @ B))
    assert np.allclose(oracle.spectral_solve(v, lam, B), ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))
