"""GPU parity of the tensor-core trailing update (step A3, tcgen05 + TMA)
against the oracle's float64 product of the same rounded operands."""
import numpy as np
import pytest

import paper_1405_4644_gb300 as spd
from oracle.precision import ROUND

pytestmark = pytest.mark.gpu

from tests.gpu_util import DEV, check  # noqa: E402

FP8_SCALE = 256.0


@pytest.fixture(scope="module")
def h():
    import torch
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def rounded(x, prec):
    if prec == "fp8":  # operands carry a 2^8 scale into e4m3
        return ROUND["fp8"](x * FP8_SCALE) / FP8_SCALE
    return ROUND[prec](ROUND["fp32"](x))


def run(h, prec, A, B, C0, lower=False):
    import torch
    At = torch.from_numpy(A.astype(np.float32)).to(DEV)
    Bt = At if lower else torch.from_numpy(B.astype(np.float32)).to(DEV)
    Ct = torch.from_numpy(C0.astype(np.float32)).to(DEV)
    check(h, spd.spd_gemm_update(h, prec, At, Bt, Ct, lower))
    return Ct.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "fp8"])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (128, 256, 128), (300, 500, 200), (1000, 1000, 1024),
                                   (37, 290, 1), (513, 129, 640)])
def test_gemm_update_matches_rounded_product(h, prec, M, N, K):
    g = np.random.default_rng(M * 7 + N * 3 + K)
    scale = 1.0 if prec == "fp8" else 2.0
    A = g.uniform(-1, 1, (M, K)) * scale
    B = g.uniform(-1, 1, (N, K)) * scale
    C0 = g.standard_normal((M, N)).astype(np.float32).astype(np.float64)
    Ar, Br = rounded(A, prec), rounded(B, prec)
    ref = C0 - Ar @ Br.T
    got = run(h, prec, A, B, C0)
    bound = 4 * K * 2.0 ** -23 * (np.abs(Ar) @ np.abs(Br).T) + 2.0 ** -22 * np.abs(C0) + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())
    if K >= 64:  # the operands really were rounded to the low-precision type
        A32, B32 = rounded(A, "fp32"), rounded(B, "fp32")
        unrounded = C0 - A32 @ B32.T
        if prec != "tf32" or K >= 128:
            assert np.max(np.abs(got - unrounded)) > 8 * np.max(err)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("M,K", [(256, 128), (700, 384)])
def test_gemm_update_lower_triangle(h, prec, M, K):
    g = np.random.default_rng(M + K)
    A = g.uniform(-1, 1, (M, K))
    C0 = g.standard_normal((M, M)).astype(np.float32).astype(np.float64)
    Ar = rounded(A, prec)
    ref = C0 - Ar @ Ar.T
    got = run(h, prec, A, None, C0, lower=True)
    iu = np.triu_indices(M, 1)
    assert np.array_equal(got[iu], C0[iu])  # strictly upper part untouched
    il = np.tril_indices(M)
    bound = 4 * K * 2.0 ** -23 * (np.abs(Ar) @ np.abs(Ar).T) + 2.0 ** -22 * np.abs(C0)
    assert np.all(np.abs(got[il] - ref[il]) <= bound[il])


@pytest.mark.parametrize("M,N,K", [(128, 256, 32), (300, 500, 200), (1000, 1000, 1024), (513, 129, 640)])
def test_gemm_update_fp32_three_bf16_slices(h, M, N, K):
    """FP32 operands split into three bf16 slices; the six slice products of
    order <= 2 give the float32 product to float32-class accuracy (dropped
    terms below 2^-23 |a||b|), far beyond one tf32 product."""
    g = np.random.default_rng(M + 5 * N + 11 * K)
    A = g.uniform(-1, 1, (M, K)) * 2.0
    B = g.uniform(-1, 1, (N, K)) * 2.0
    C0 = g.standard_normal((M, N)).astype(np.float32).astype(np.float64)
    A32, B32 = rounded(A, "fp32"), rounded(B, "fp32")
    ref = C0 - A32 @ B32.T
    got = run(h, "fp32", A, B, C0)
    mag = np.abs(A32) @ np.abs(B32).T
    err = np.abs(got - ref)
    bound = (K + 8) * 2.0 ** -24 * mag + 2.0 ** -24 * np.abs(C0)
    assert np.all(err <= bound), float((err / bound).max())
    tf = run(h, "tf32", A, B, C0)
    if K >= 64:
        assert np.max(np.abs(tf - ref)) > 16 * np.max(err)


def test_gemm_update_rejects_bad_arguments(h):
    import torch
    A = torch.zeros(8, 8, dtype=torch.float32, device=DEV)
    assert spd.spd_gemm_update(h, "fp64", A, A, A) == spd.SPD_ERR_UNSUPPORTED
    assert spd.lib().spd_gemm_update(h, spd.PREC["bf16"], 8, 8, 8, A.data_ptr(), 4, A.data_ptr(), 8,
                                     A.data_ptr(), 8, 0) == spd.SPD_ERR_ARG


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "fp8", "fp32"])
@pytest.mark.parametrize("M,N,K", [(300, 500, 1024), (1000, 1000, 1024), (129, 256, 4096), (37, 100, 2048)])
def test_gemm_update_stream_k_matches_rounded_product(h, prec, M, N, K):
    """Stream-K schedule (equal (tile, K tile) ranges per CTA, pieces of
    shared tiles added to C in K order by the fix-up kernel): same bounds as
    one CTA per tile, and the same result for every launch."""
    import torch
    g = np.random.default_rng(M * 5 + N + K)
    scale = 1.0 if prec == "fp8" else 2.0
    A = g.uniform(-1, 1, (M, K)) * scale
    B = g.uniform(-1, 1, (N, K)) * scale
    C0 = g.standard_normal((M, N)).astype(np.float32).astype(np.float64)
    Ar, Br = rounded(A, prec), rounded(B, prec)
    ref = C0 - Ar @ Br.T
    At = torch.from_numpy(A.astype(np.float32)).to(DEV)
    Bt = torch.from_numpy(B.astype(np.float32)).to(DEV)
    outs = []
    for _ in range(2):
        Ct = torch.from_numpy(C0.astype(np.float32)).to(DEV)
        check(h, spd.spd_gemm_update(h, prec, At, Bt, Ct, stream_k=True))
        outs.append(Ct.cpu().numpy().astype(np.float64))
    got = outs[0]
    assert np.array_equal(outs[0], outs[1])  # deterministic
    mag = np.abs(Ar) @ np.abs(Br).T
    if prec == "fp32":
        bound = (K + 8) * 2.0 ** -24 * mag + 2.0 ** -24 * np.abs(C0)
    else:
        bound = 4 * K * 2.0 ** -23 * mag + 2.0 ** -22 * np.abs(C0) + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("M,K", [(200, 2048), (256, 1024)])
def test_gemm_update_stream_k_lower(h, M, K):
    g = np.random.default_rng(M + 3 * K)
    A = g.uniform(-1, 1, (M, K))
    C0 = g.standard_normal((M, M)).astype(np.float32).astype(np.float64)
    Ar = rounded(A, "bf16")
    ref = C0 - Ar @ Ar.T
    import torch
    At = torch.from_numpy(A.astype(np.float32)).to(DEV)
    Ct = torch.from_numpy(C0.astype(np.float32)).to(DEV)
    check(h, spd.spd_gemm_update(h, "bf16", At, At, Ct, lower=True, stream_k=True))
    got = Ct.cpu().numpy().astype(np.float64)
    iu = np.triu_indices(M, 1)
    assert np.array_equal(got[iu], C0[iu])
    il = np.tril_indices(M)
    bound = 4 * K * 2.0 ** -23 * (np.abs(Ar) @ np.abs(Ar).T) + 2.0 ** -22 * np.abs(C0)
    assert np.all(np.abs(got[il] - ref[il]) <= bound[il])
