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
