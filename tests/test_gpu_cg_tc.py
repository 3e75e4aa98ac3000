"""GPU parity of the tensor-core product of CG with several right-hand sides
(step C1 of Algorithm 2): the narrow fused-slice GEMM against the rounded
float32 product, without the bias of the tensor cores' own float32
accumulation (each K tile's sums are promoted to float32 registers), and
Algorithm 2 with its products on the tensor cores against the CUDA-core
products and the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

pytestmark = pytest.mark.gpu

from tests.gpu_util import DEV, check, dev_cols, dev_sym, dev_zeros, host  # noqa: E402


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def f32(x):
    return x.astype(np.float32).astype(np.float64)


def gemm(h, A, B, C0, **kw):
    At = torch.from_numpy(A.astype(np.float32)).to(DEV)
    Bt = torch.from_numpy(B.astype(np.float32)).to(DEV)
    Ct = torch.from_numpy(C0.astype(np.float32)).to(DEV)
    check(h, spd.spd_gemm_update(h, "fp32", At, Bt, Ct, **kw))
    return Ct.cpu().numpy().astype(np.float64)


# N spans one narrow tile (1, 5, 32), two widths (33, 64) and several column
# tiles (100); ragged M and K
@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (300, 1, 200), (1000, 5, 1000), (513, 33, 640),
                                   (2000, 64, 2048), (777, 100, 1500)])
@pytest.mark.parametrize("stream_k", [False, True])
def test_narrow_gemm_matches_rounded_product(h, M, N, K, stream_k):
    g = np.random.default_rng(M + 7 * N + 3 * K)
    A = g.uniform(-1, 1, (M, K)) * 2.0
    B = g.uniform(-1, 1, (N, K)) * 2.0
    C0 = f32(g.standard_normal((M, N)))
    ref = C0 - f32(A) @ f32(B).T
    got = gemm(h, A, B, C0, narrow=True, stream_k=stream_k)
    bound = (K + 8) * 2.0 ** -24 * (np.abs(f32(A)) @ np.abs(f32(B)).T) + 2.0 ** -24 * np.abs(C0)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.array_equal(got, gemm(h, A, B, C0, narrow=True, stream_k=stream_k))  # deterministic


def test_narrow_gemm_has_no_accumulation_bias(h):
    """Positive operands, K = 16384: a float32 sum that rounds toward zero at
    every step loses about K 2^-24 / 3 of the result (about 1e-4 here); with
    each 64-long K tile promoted to float32 registers (round to nearest) the
    mean relative error stays at the level of one K tile's sum."""
    M, N, K = 512, 32, 16384
    g = np.random.default_rng(7)
    A = g.uniform(0, 1, (M, K))
    B = g.uniform(0, 1, (N, K))
    C0 = np.zeros((M, N))
    exact = f32(A) @ f32(B).T
    got = -gemm(h, A, B, C0, narrow=True, stream_k=True)
    rel = (got - exact) / exact
    assert abs(rel.mean()) <= 2e-6, rel.mean()
    assert np.abs(rel).max() <= (K + 8) * 2.0 ** -24


def test_narrow_gemm_rejects_other_precisions_and_lower(h):
    A = torch.zeros(64, 64, dtype=torch.float32, device=DEV)
    assert spd.spd_gemm_update(h, "bf16", A, A, A, narrow=True) == spd.SPD_ERR_UNSUPPORTED
    assert spd.spd_gemm_update(h, "fp32", A, A, A, narrow=True, lower=True) == spd.SPD_ERR_UNSUPPORTED


@pytest.mark.parametrize("m", [8, 16, 32, 33, 70])
def test_cg_tensor_core_products_match_cuda_core_products(h, m):
    """Both product engines reach the relative target; the solutions agree
    with the oracle's within 10 kappa 1e-14 and the inner step counts are
    close (the products differ only in rounding)."""
    n = 1500
    A = W.gram_shifted(n, seed=m, shift=0.1)
    B = A @ W.gaussian_rhs(n, m, 2)
    Ad, Bd = dev_sym(A), dev_cols(B)
    Xo = oracle.solve(A, B)
    kappa = np.linalg.cond(A)
    reps = {}
    for cores in ("tensor", "cuda"):
        X = dev_zeros(n, m)
        st, rep = spd.spd_cg(h, Ad, Bd, X, "fp32",
                             opts={"tol": 1e-14, "crit": "rel2", "matvec_cores": cores})
        check(h, st)
        Xg = host(X)
        assert np.max(np.abs(Xg - Xo)) <= 10 * kappa * 1e-14 * np.max(np.abs(Xo)), cores
        reps[cores] = rep
    lo_t, lo_c = reps["tensor"].iters_low, reps["cuda"].iters_low
    assert abs(lo_t - lo_c) <= max(3, 0.15 * lo_c), (lo_t, lo_c)


@pytest.mark.parametrize("m", [1, 3])
def test_cg_tensor_core_products_for_few_right_hand_sides(h, m):
    n = 900
    A = W.gram_shifted(n, seed=40 + m, shift=0.1)
    B = W.gaussian_rhs(n, m, 3)
    X = dev_zeros(n, m)
    st, rep = spd.spd_cg(h, dev_sym(A), dev_cols(B), X, "fp32",
                         opts={"tol": 1e-14, "crit": "berr", "matvec_cores": "tensor"})
    check(h, st)
    assert oracle.berr(A, B, host(X)) <= 1e-14


def test_cg_paper_rule_many_rhs_on_tensor_cores(h):
    """Section 4 rule (absolute ||r||_2 < 1e-5, U[0,1] right-hand sides) with
    16 right-hand sides (the default engine for m >= 8 is the tensor cores):
    every column meets the rule and the inner step count matches the
    oracle's Algorithm 2 with float32 products."""
    n, m, d = 2000, 16, 4
    A = W.model_covariance(n, d)
    B = W.uniform_rhs(n, m, 0)
    X = dev_zeros(n, m)
    st, rep = spd.spd_cg(h, dev_sym(A), dev_cols(B), X, "fp32",
                         opts={"tol": 1e-5, "crit": "abs2", "eta": 0.0, "maxit_inner": 5000})
    check(h, st)
    assert np.all(np.linalg.norm(oracle.residual(A, B, host(X)), axis=0) < 1e-5)
    _, lo, hi, fe, ok = oracle.cg_ir(A, B, tol=1e-5, crit="abs2", eta=0.0)
    assert ok
    assert abs(rep.iters_low - int(lo.max())) <= max(3, 0.1 * lo.max())
    assert abs(rep.iters_high - int(hi.max())) <= 1


@pytest.mark.parametrize("m", [1, 3])
def test_auto_residual_in_both_algorithms(h, m):
    """SPD_RESID_AUTO (float64 fused multiply-adds for one right-hand side,
    the tensor-core residual for more) reaches the float64 target in
    Algorithm 1 and Algorithm 2; an unknown residual code is refused."""
    n = 700
    A = W.gram_shifted(n, seed=50 + m, shift=0.1)
    B = W.gaussian_rhs(n, m, 4)
    Ad, Bd = dev_sym(A), dev_cols(B)
    X = dev_zeros(n, m)
    st, rep = spd.spd_cg(h, Ad, Bd, X, "fp32", opts={"tol": 1e-14, "crit": "berr", "resid": "auto"})
    check(h, st)
    assert oracle.berr(A, B, host(X)) <= 1e-14
    st, F, _ = spd.spd_factor(h, Ad, "fp16")
    check(h, st)
    try:
        X2 = dev_zeros(n, m)
        st, rep = spd.spd_solve_ir(h, F, Ad, Bd, X2, {"resid": "auto"})
        check(h, st)
        assert oracle.berr(A, B, host(X2)) <= 1e-14
        st, _ = spd.spd_solve_ir(h, F, Ad, Bd, X2, {"resid": 4})
        assert st == spd.SPD_ERR_ARG
    finally:
        spd.spd_factor_destroy(F)


@pytest.mark.parametrize("mv,m,band", [("fp32", 1, -1), ("fp32", 16, -1), ("bf16", 3, -1), ("fp32", 2, 16)])
def test_cg_inner_steps_as_a_graph_match_direct_launches(mv, m, band):
    """Groups of inner steps replayed from a captured CUDA graph give the
    same iterates, bit for bit, as the same kernels launched one by one
    (profiling on: the library then launches directly)."""
    n = 1200
    A = W.model_covariance(n, 2)
    B = W.uniform_rhs(n, m, 5)
    Ad, Bd = dev_sym(A), dev_cols(B)
    opts = {"tol": 1e-5, "crit": "abs2", "eta": 0.0, "maxit_inner": 5000, "band": band}
    out = []
    for prof in (False, True):
        h = spd.spd_create(torch.cuda.current_stream())
        try:
            spd.spd_profile_enable(h, prof)
            X = dev_zeros(n, m)
            st, rep = spd.spd_cg(h, Ad, Bd, X, mv, opts=opts)
            check(h, st)
            out.append((host(X), rep.iters_low, rep.iters_high))
        finally:
            spd.spd_destroy(h)
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
