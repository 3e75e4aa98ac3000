"""Algorithm 1 with the refinement's stop decision on the device
(spd_solve_ir_async): the same solution as the synchronous call, a report in
device memory, and a solve captured in a CUDA graph that replays correctly
for new right-hand sides in the same buffers."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

pytestmark = pytest.mark.gpu

from tests.gpu_util import check, dev_cols, dev_sym, dev_zeros, host  # noqa: E402


@pytest.mark.parametrize("prec,resid", [("fp16", "fp64"), ("fp32", "tc"), ("bf16", "fp64")])
def test_async_solve_matches_the_synchronous_one(prec, resid):
    h = spd.spd_create(torch.cuda.current_stream())
    try:
        n, m = 900, 5
        A = W.gram_shifted(n, seed=8, shift=0.1)
        B = W.gaussian_rhs(n, m, 9)
        Ad, Bd = dev_sym(A), dev_cols(B)
        st, F, _ = spd.spd_factor(h, Ad, prec)
        check(h, st)
        try:
            X1 = dev_zeros(n, m)
            st, rep = spd.spd_solve_ir(h, F, Ad, Bd, X1, {"resid": resid, "fallback": 0})
            check(h, st)
            X2 = dev_zeros(n, m)
            buf = spd.spd_report_dev_buffer()
            check(h, spd.spd_solve_ir_async(h, F, Ad, Bd, X2, buf, {"resid": resid, "maxit": 20}))
            r = spd.spd_report_dev_read(buf)
        finally:
            spd.spd_factor_destroy(F)
        assert r.status == spd.SPD_OK and r.active == 0 and r.dev_flags == 0
        assert r.sweeps == rep.iters_high - 1 and r.berr == rep.berr
        assert np.array_equal(host(X1), host(X2))  # the gated sweeps left the solution alone
        assert oracle.berr(A, B, host(X2)) <= 1e-14
    finally:
        spd.spd_destroy(h)


def test_async_solve_captured_in_a_graph_replays_for_new_right_hand_sides():
    s = torch.cuda.Stream()
    h = spd.spd_create(s)
    try:
        n, m = 1100, 3
        A = W.gram_shifted(n, seed=21, shift=0.1)
        Ad = dev_sym(A)
        Bd = dev_zeros(n, m)
        X = dev_zeros(n, m)
        buf = spd.spd_report_dev_buffer()
        opts = {"resid": "tc", "maxit": 12}
        with torch.cuda.stream(s):
            st, F, _ = spd.spd_factor(h, Ad, "fp16")
            check(h, st)
            Bd.copy_(dev_cols(W.gaussian_rhs(n, m, 1)))
            check(h, spd.spd_solve_ir_async(h, F, Ad, Bd, X, buf, opts))  # sizes the workspace
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            st = spd.spd_solve_ir_async(h, F, Ad, Bd, X, buf, opts)
        check(h, st)
        try:
            for seed in (2, 3, 4):
                Bh = W.gaussian_rhs(n, m, seed)
                with torch.cuda.stream(s):
                    Bd.copy_(dev_cols(Bh))
                    X.zero_()
                    g.replay()
                s.synchronize()
                r = spd.spd_report_dev_read(buf)
                assert r.status == spd.SPD_OK and r.active == 0, (seed, r.status, r.berr)
                assert 1 <= r.sweeps <= 12
                assert oracle.berr(A, Bh, host(X)) <= 1e-14, seed
        finally:
            spd.spd_factor_destroy(F)
    finally:
        spd.spd_destroy(h)


def test_async_solve_reports_no_convergence_within_maxit():
    h = spd.spd_create(torch.cuda.current_stream())
    try:
        n, m = 500, 2
        A = W.gram_shifted(n, seed=5, shift=0.1)
        B = W.gaussian_rhs(n, m, 6)
        Ad, Bd = dev_sym(A), dev_cols(B)
        st, F, _ = spd.spd_factor(h, Ad, "bf16")
        check(h, st)
        X = dev_zeros(n, m)
        buf = spd.spd_report_dev_buffer()
        try:
            check(h, spd.spd_solve_ir_async(h, F, Ad, Bd, X, buf, {"maxit": 1}))
            r = spd.spd_report_dev_read(buf)
        finally:
            spd.spd_factor_destroy(F)
        assert r.status == spd.SPD_ERR_NO_CONVERGENCE and r.active == m and r.sweeps == 1
        assert r.berr > 1e-14
    finally:
        spd.spd_destroy(h)
