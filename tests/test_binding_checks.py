"""The Python binding rejects arguments the kernels would misread (host
tensors, other dtypes) before anything reaches libspd.  These checks run on
the CPU: the validation raises ValueError before the library is loaded."""
import pytest
import torch

import paper_1405_4644_gb300 as spd


def _args(dtype=torch.float64, n=8, m=2):
    A = torch.eye(n, dtype=dtype)
    B = torch.zeros(m, n, dtype=dtype).t()
    return A, B, B.clone(), B.clone()


@pytest.mark.parametrize("fn", ["spd_residual", "spd_residual_df32", "spd_residual_tc"])
def test_residuals_reject_host_and_float32_tensors(fn):
    f = getattr(spd, fn)
    with pytest.raises(ValueError, match="CUDA"):
        f(None, *_args())
    with pytest.raises(ValueError, match="float64"):
        f(None, *_args(torch.float32))


def test_static_residual_rejects_host_tensors():
    with pytest.raises(ValueError):
        spd.spd_residual_static(None, *_args())


def test_solvers_reject_host_tensors():
    A, B, X, _ = _args()
    with pytest.raises(ValueError):
        spd.spd_solve_ir(None, None, A, B, X)
    with pytest.raises(ValueError):
        spd.spd_cg(None, A, B, X)
    with pytest.raises(ValueError):
        spd.spd_factor(None, A, "fp32")


def test_gemm_update_rejects_host_and_float64_tensors():
    A = torch.zeros(4, 4, dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        spd.spd_gemm_update(None, "bf16", A, A, A)
    with pytest.raises(ValueError, match="float32"):
        spd.spd_gemm_update(None, "bf16", A.double(), A.double(), A.double())


@pytest.mark.gpu
def test_shape_and_norm_buffer_checks_on_the_device():
    n, m = 64, 3
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    B = torch.zeros(m, n, dtype=torch.float64, device="cuda").t()
    short = torch.zeros(m, n - 1, dtype=torch.float64, device="cuda").t()
    h = spd.spd_create(torch.cuda.current_stream())
    try:
        with pytest.raises(ValueError, match="shape"):
            spd.spd_residual(h, A, B, B.clone(), short)
        with pytest.raises(ValueError, match="3\\*m"):
            spd.spd_residual(h, A, B, B.clone(), B.clone(), torch.zeros(m, dtype=torch.float64, device="cuda"))
        cn = torch.zeros(3 * m, dtype=torch.float64, device="cuda")
        assert spd.spd_residual(h, A, B, B.clone(), B.clone(), cn) == spd.SPD_OK
    finally:
        spd.spd_destroy(h)
