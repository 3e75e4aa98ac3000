"""Failure handling without a GPU fault: a bounded device wait that runs out
(on a flag that nothing sets) returns SPD_ERR_TIMEOUT and leaves the handle
usable; a memory cap turns a too-large device request into SPD_ERR_OOM
before anything is allocated."""
import time

import numpy as np
import pytest

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

pytestmark = pytest.mark.gpu

from tests.gpu_util import check, dev_cols, dev_sym, dev_zeros, host  # noqa: E402


@pytest.fixture()
def h():
    import torch
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def test_expired_wait_reports_timeout_and_the_handle_stays_usable(h):
    check(h, spd.spd_set_wait_limit(h, 0.002))
    t0 = time.perf_counter()
    st = spd.spd_wait_probe(h)
    dt = time.perf_counter() - t0
    check(h, st, spd.SPD_ERR_TIMEOUT)
    assert "wait" in spd.spd_last_error_string(h)
    assert dt < 1.0
    # the status word was cleared: the same handle runs a full solve, its
    # sweeps waiting on real flags under a 1 s limit
    check(h, spd.spd_set_wait_limit(h, 1.0))
    n, m = 700, 3
    A = W.gram_shifted(n, seed=2, shift=0.1)
    B = W.gaussian_rhs(n, m, 3)
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, "fp16")
    check(h, st)
    X = dev_zeros(n, m)
    try:
        st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X)
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    assert oracle.berr(A, B, host(X)) <= 1e-14
    # and the probe times out again, as often as asked
    check(h, spd.spd_set_wait_limit(h, 0.001))
    check(h, spd.spd_wait_probe(h), spd.SPD_ERR_TIMEOUT)


def test_wait_limit_rejects_nonsense(h):
    check(h, spd.spd_set_wait_limit(h, 0.0), spd.SPD_ERR_ARG)
    check(h, spd.spd_set_wait_limit(h, -1.0), spd.SPD_ERR_ARG)
    check(h, spd.spd_set_wait_limit(h, 1e3), spd.SPD_ERR_ARG)


def test_memory_cap_gives_oom_before_allocating(h):
    import torch
    n, m = 1024, 2
    A = W.gram_shifted(n, seed=4, shift=0.1)
    Ad = dev_sym(A)
    free0 = torch.cuda.mem_get_info()[0]
    check(h, spd.spd_set_memory_cap(h, 64 << 10))  # 64 KiB: below every request at this size
    st, F, rep = spd.spd_factor(h, Ad, "fp32")
    check(h, st, spd.SPD_ERR_OOM)
    assert F is None and "cap" in spd.spd_last_error_string(h)
    # a float64 residual at this size needs a workspace above the cap too
    R = dev_zeros(n, m)
    B = dev_cols(W.gaussian_rhs(n, m, 5))
    check(h, spd.spd_residual(h, Ad, B, B, R), spd.SPD_ERR_OOM)
    # host-buffer solve: the device copies of A alone exceed the cap
    Bh = np.asfortranarray(W.gaussian_rhs(n, m, 6))
    Xh = np.zeros((n, m), order="F")
    st, _ = spd.spd_solve_ir_host(h, np.ascontiguousarray(A), Bh, Xh, "fp32")
    check(h, st, spd.SPD_ERR_OOM)
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    # lifting the cap restores every call
    check(h, spd.spd_set_memory_cap(h, 0))
    st, F, rep = spd.spd_factor(h, Ad, "fp32")
    check(h, st)
    X = dev_zeros(n, m)
    try:
        st, _ = spd.spd_solve_ir(h, F, Ad, B, X)
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    assert oracle.berr(A, host(B), host(X)) <= 1e-14
