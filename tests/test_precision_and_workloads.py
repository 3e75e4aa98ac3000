"""Pins of the oracle's rounding helpers and of the seeded input generators."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import precision as P


def test_fp16_and_fp32_match_library_casts():
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-6, 4, 10000)
    np.testing.assert_array_equal(P.to_fp16(x), x.astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(P.to_fp32(x), x.astype(np.float32).astype(np.float64))


def test_bf16_matches_torch_rne():
    x = np.random.default_rng(2).standard_normal(20000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.to_bf16(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even fraction (1.0)
    assert P.to_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3*2^-8 lies halfway between 1+2^-7 and 1+2^-6: ties to 1 + 2^-6
    assert P.to_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_tf32_grid():
    # tf32 keeps 10 fraction bits: 1 + 2^-10 is representable, 1 + 2^-12 rounds to 1
    v = P.to_tf32(np.array([1.0 + 2.0 ** -10, 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -11]))
    assert v[0] == 1.0 + 2.0 ** -10 and v[1] == 1.0 and v[2] == 1.0 + 2.0 ** -9


def test_e4m3_values():
    g = P._E4M3
    assert g.max() == 448.0 and g[1] == 2.0 ** -9 and len(g) == 127
    assert P.to_e4m3(np.array([1e6]))[0] == 448.0          # saturating
    assert P.to_e4m3(np.array([1.0625]))[0] == 1.0         # tie between 1 and 1.125 -> even code
    assert P.to_e4m3(np.array([1.1875]))[0] == 1.25        # tie between 1.125 and 1.25 -> even code
    x = np.random.default_rng(3).uniform(-400, 400, 5000)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.to_e4m3(x), ref)


def test_generators_are_seeded_and_symmetric():
    A1 = W.gram_shifted(64, seed=0)
    A2 = W.gram_shifted(64, seed=0)
    assert np.array_equal(A1, A2) and np.array_equal(A1, A1.T)
    ev = np.linalg.eigvalsh(A1)
    assert ev.min() >= 0.1 - 1e-12


def test_householder_spectrum_matches_planted_eigenvalues():
    n = 96
    A, lam, V = W.householder_spectrum(n, 1e4, k=32, seed=0)
    assert np.array_equal(A, A.T)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), lam, rtol=1e-11)
    assert lam[0] == 1.0 and lam[-1] == pytest.approx(1e4)


def test_householder_spectrum_torch_assembly_agrees():
    A, lam, V = W.householder_spectrum(80, 1e2, k=8, seed=1)
    At, _, _ = W.householder_spectrum(80, 1e2, k=8, seed=1, device="cpu")
    np.testing.assert_allclose(At.numpy(), A, rtol=0, atol=1e-12)


def test_exp_kernel_and_matern_are_spd():
    A, _ = W.exp_kernel_cov(200, 0.1, 1e-3, seed=0)
    assert np.linalg.eigvalsh(A).min() > 0
    At, _ = W.exp_kernel_cov(200, 0.1, 1e-3, seed=0, device="cpu")
    np.testing.assert_allclose(At.numpy(), A, rtol=0, atol=1e-14)
    ell, nug = W.matern_family_params(3)
    assert 0.02 <= ell <= 0.5 and 1e-4 <= nug <= 1e-1
    M, _ = W.matern32_cov(150, ell, nug, seed=3)
    assert np.linalg.eigvalsh(M).min() > 0


def test_batched_sizes_and_systems():
    s = W.batched_sizes(4096)
    assert s.min() >= 32 and s.max() <= 512 and len(s) == 4096
    As, bs = W.batched_gram([33, 40])
    assert As[0].shape == (33, 33) and bs[1].shape == (40,)
    assert np.linalg.eigvalsh(As[1]).min() >= 0.05 - 1e-12


def test_model_covariance_definition_small():
    A = W.model_covariance(4, 2)
    exp = np.array([[2.0, 1.0, 0.25, 1 / 9],
                    [1.0, 1 + np.sqrt(2), 1.0, 0.25],
                    [0.25, 1.0, 1 + np.sqrt(3), 1.0],
                    [1 / 9, 0.25, 1.0, 3.0]])
    np.testing.assert_allclose(A, exp, rtol=1e-15)
