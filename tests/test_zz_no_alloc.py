"""The allocation-free residual entry point (spd_residual_static).

Some callers cannot allocate device memory (host callbacks, allocator hooks,
fixed-budget processes); this entry point serves them from a fixed scratch
array inside the library.  The test calls it through the C ABI twice in a
row, on different data, and compares each result with the handle-based
spd_residual (which allocates its workspace) within the tolerance the
residual parity tests use, and with the float64 oracle's residual element
by element (the correctly rounded residual for the second call).  It sits in
a file of its own that pytest collects last, and passes both alone and after
the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W
from oracle import exact

pytestmark = pytest.mark.gpu


def _dev_sym(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _dev_cols(B):
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()


def _zeros(n, m):
    return torch.zeros(m, n, dtype=torch.float64, device="cuda").t()


def test_static_residual_matches_handle_residual_twice():
    stream = torch.cuda.current_stream()
    h = spd.spd_create(stream)
    try:
        for call, (n, m, seed) in enumerate([(1500, 17, 3), (777, 4, 9)]):
            A = W.gram_shifted(n, seed=seed)
            X = W.gaussian_rhs(n, m, seed + 1)
            B = W.gaussian_rhs(n, m, seed + 2)
            Ad, Bd, Xd = _dev_sym(A), _dev_cols(B), _dev_cols(X)
            R_ref, R_new = _zeros(n, m), _zeros(n, m)
            cn_ref = torch.zeros(3 * m, dtype=torch.float64, device="cuda")
            cn_new = torch.zeros(3 * m, dtype=torch.float64, device="cuda")
            assert spd.spd_residual(h, Ad, Bd, Xd, R_ref, cn_ref) == spd.SPD_OK
            st = spd.spd_residual_static(stream, Ad, Bd, Xd, R_new, cn_new)
            assert st == spd.SPD_OK, f"call {call}: status {st}"
            R_new_h = R_new.cpu().numpy()
            scale = np.abs(A) @ np.abs(X) + np.abs(B)
            # against the handle-based entry point
            diff = np.abs(R_new_h - R_ref.cpu().numpy())
            assert np.all(diff <= 2 * n * 2.0 ** -53 * scale), f"call {call}"
            np.testing.assert_allclose(cn_new.cpu().numpy(), cn_ref.cpu().numpy(), rtol=1e-12, atol=0)
            # against the oracle (both float64 sums err by at most n u (|A||X| + |B|))
            R_or = exact.residual_exact(A, B, X) if call == 1 else oracle.residual(A, B, X)
            bound = (1 if call == 1 else 2) * n * 2.0 ** -53 * scale
            assert np.all(np.abs(R_new_h - R_or) <= bound), f"call {call}: oracle"
            # the norms are those of the returned residual and of X
            cn = cn_new.cpu().numpy().reshape(m, 3)
            np.testing.assert_allclose(cn[:, 0], np.max(np.abs(R_new_h), axis=0), rtol=0, atol=0)
            np.testing.assert_allclose(cn[:, 1], np.linalg.norm(R_new_h, axis=0), rtol=1e-14)
            np.testing.assert_allclose(cn[:, 2], np.max(np.abs(X), axis=0), rtol=0, atol=0)
    finally:
        spd.spd_destroy(h)


def test_static_residual_rejects_problems_beyond_its_scratch():
    n, m = 4096, 600  # n*m = 2.46 million float64 > the 16 MiB scratch
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    Bm = torch.zeros(m, n, dtype=torch.float64, device="cuda").t()
    st = spd.spd_residual_static(torch.cuda.current_stream(), A, Bm, Bm, Bm)
    assert st == spd.SPD_ERR_SCRATCH
