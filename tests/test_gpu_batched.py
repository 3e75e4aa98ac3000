"""GPU parity of the batched persistent solves (many uneven systems, one
launch) against the float64 CPU oracle, system by system."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def make_batch(sizes, seed_base=1000, shift=0.05):
    As, bs = W.batched_gram(sizes, shift=shift, seed_base=seed_base)
    Ad = [torch.from_numpy(A).cuda() for A in As]
    bd = [torch.from_numpy(b).cuda() for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    return As, bs, Ad, bd, xd


SIZES = [1, 2, 31, 32, 33, 64, 100, 127, 128, 129, 255, 256, 300, 511, 512, 47, 200, 5, 400, 17]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_batched_chol_ir_matches_oracle(h, prec):
    As, bs, Ad, bd, xd = make_batch(SIZES)
    st, plan = spd.spd_batch_create(h, Ad, bd, xd)
    assert st == spd.SPD_OK
    try:
        st, rep, sts, be, it = spd.spd_batch_solve(plan, "chol_ir", prec, count=len(SIZES))
        assert st == spd.SPD_OK, spd.spd_last_error_string(h)
        info = spd.spd_batch_info(plan, "chol_ir")
        assert info["threads_per_cta"] in (256, 512)
    finally:
        spd.spd_batch_destroy(plan)
    assert np.all(sts == 0) and rep.berr <= 1e-14
    for A, b, x, bgpu in zip(As, bs, xd, be):
        xg = x.cpu().numpy()
        assert oracle.berr(A, b[:, None], xg[:, None]) <= 1e-14
        xo = oracle.solve(A, b[:, None])[:, 0]
        kappa = np.linalg.cond(A)
        assert np.max(np.abs(xg - xo)) <= 10 * kappa * 1e-16 * max(1.0, np.sqrt(len(b)) / 8) * np.max(np.abs(xo))


def test_batched_pcg_jacobi_matches_oracle(h):
    As, bs, Ad, bd, xd = make_batch(SIZES[:12])
    st, plan = spd.spd_batch_create(h, Ad, bd, xd)
    assert st == spd.SPD_OK
    try:
        st, rep, sts, be, it = spd.spd_batch_solve(plan, "pcg_jacobi", "fp64", count=12)
        assert st == spd.SPD_OK, spd.spd_last_error_string(h)
    finally:
        spd.spd_batch_destroy(plan)
    for A, b, x in zip(As, bs, xd):
        assert oracle.berr(A, b[:, None], x.cpu().numpy()[:, None]) <= 1e-14


def test_batched_breakdown_is_per_system_and_runs_are_reproducible(h):
    sizes = [40, 200, 64]
    As, bs, Ad, bd, xd = make_batch(sizes)
    bad = np.eye(200)
    bad[50, 51] = bad[51, 50] = 2.0
    Ad[1] = torch.from_numpy(bad).cuda()
    st, plan = spd.spd_batch_create(h, Ad, bd, xd)
    assert st == spd.SPD_OK
    try:
        st, rep, sts, be, it = spd.spd_batch_solve(plan, "chol_ir", "fp32", count=3)
        assert st == spd.SPD_ERR_NOT_SPD
        assert list(sts) == [0, spd.SPD_ERR_NOT_SPD, 0]
        x0 = xd[0].clone()
        st, rep, sts, be, it = spd.spd_batch_solve(plan, "chol_ir", "fp32", count=3)
        assert torch.equal(x0, xd[0])  # same system, same CTA-independent sequence: bitwise equal
    finally:
        spd.spd_batch_destroy(plan)


def test_batched_rejects_oversize(h):
    A = torch.eye(513, dtype=torch.float64, device="cuda")
    b = torch.ones(513, dtype=torch.float64, device="cuda")
    st, plan = spd.spd_batch_create(h, [A], [b], [b.clone()])
    assert st == spd.SPD_ERR_ARG and plan is None


def test_batched_graph_launched_by_the_caller(h):
    """spd_batch_graph hands out the captured graph; launched twice on the
    caller's own stream (the second time after the right-hand sides changed)
    it gives the same solutions as spd_batch_solve, bit for bit, and every
    system meets the tolerance against the oracle."""
    sizes = SIZES[:14]
    As, bs, Ad, bd, xd = make_batch(sizes, seed_base=2000)
    st, plan = spd.spd_batch_create(h, Ad, bd, xd)
    assert st == spd.SPD_OK
    try:
        st, rep, sts, be, it = spd.spd_batch_solve(plan, "chol_ir", "fp32", count=len(sizes))
        assert st == spd.SPD_OK
        ref = [x.cpu().numpy().copy() for x in xd]
        st, gx = spd.spd_batch_graph(plan, "chol_ir", "fp32")
        assert st == spd.SPD_OK and gx
        s = torch.cuda.Stream()
        for x in xd:
            x.zero_()
        torch.cuda.synchronize()
        assert spd.spd_graph_launch(gx, s) == spd.SPD_OK
        s.synchronize()
        st, rep2, sts2, be2, it2 = spd.spd_batch_results(plan, "chol_ir", "fp32", count=len(sizes))
        assert st == spd.SPD_OK and np.all(sts2 == 0)
        for x, r in zip(xd, ref):
            assert np.array_equal(x.cpu().numpy(), r)
        # new right-hand sides in the same buffers, the same graph
        bs2 = [b * 2.0 - 1.0 for b in bs]
        for b, b2 in zip(bd, bs2):
            b.copy_(torch.from_numpy(b2))
        torch.cuda.synchronize()
        assert spd.spd_graph_launch(gx, s) == spd.SPD_OK
        s.synchronize()
        st, rep3, sts3, _, _ = spd.spd_batch_results(plan, "chol_ir", "fp32", count=len(sizes))
        assert st == spd.SPD_OK and rep3.berr <= 1e-14
        for A, b2, x in zip(As, bs2, xd):
            assert oracle.berr(A, b2[:, None], x.cpu().numpy()[:, None]) <= 1e-14
    finally:
        spd.spd_batch_destroy(plan)
