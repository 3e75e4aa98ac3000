"""GPU parity of the super-block triangular sweeps (step A4 of Algorithm 1
with explicit inverses of the diagonal super-blocks, the default once a
float32 factor has at least two super-blocks of eight 128-row blocks):
against the float64 oracle applying the GPU's own factor, against the
128-row block sweeps (SPD_FACTOR_BLOCK_SWEEPS) on the same factor, at ragged orders (a last
super-block of one block, a last block of one row) and right-hand-side counts
that span several column passes; and inside Algorithm 1, synchronous,
device-gated and replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W

pytestmark = pytest.mark.gpu

from tests.gpu_util import check, dev_cols, dev_sym, dev_zeros, factor_L, host  # noqa: E402

U32 = 2.0 ** -24
SB = spd.SPD_SCALE_DIAG
BLK = spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_BLOCK_SWEEPS


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def kappa_scaled(A):
    d = 1.0 / np.sqrt(np.diag(A))
    ev = np.linalg.eigvalsh(d[:, None] * A * d[None, :])
    return ev[-1] / ev[0]


def apply_factor(h, F, Rh):
    n, m = Rh.shape
    Z = dev_zeros(n, m)
    check(h, spd.spd_factor_solve(h, F, dev_cols(Rh), Z))
    return host(Z)


# 2048: two full super-blocks; 2049: a last super-block of one block of one
# row; 2100, 3000: ragged last blocks; 4097: five super-blocks, one ragged
@pytest.mark.parametrize("n", [2048, 2049, 2100, 3000, 4097])
@pytest.mark.parametrize("m", [1, 5, 16, 33])
def test_superblock_sweeps_match_oracle(h, n, m):
    A = W.gram_shifted(n, seed=n + m, shift=0.5)
    Rh = W.gaussian_rhs(n, m, 11)
    st, F, _ = spd.spd_factor(h, dev_sym(A), "fp32", SB)
    check(h, st)
    try:
        L, d, _ = factor_L(F)
        Z = apply_factor(h, F, Rh)
    finally:
        spd.spd_factor_destroy(F)
    z_ref = d[:, None] * oracle.potrs(L.T, d[:, None] * Rh)
    err = np.max(np.abs(Z - z_ref)) / np.max(np.abs(z_ref))
    assert err <= 16 * n * kappa_scaled(A) * U32, err


@pytest.mark.parametrize("n,m", [(2049, 3), (3000, 16), (4097, 17)])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_superblock_and_block_sweeps_agree(h, n, m, prec):
    """The flag changes only how the factor is applied: the factors are
    identical bit for bit, the two sweeps agree to float32 rounding."""
    A = W.gram_shifted(n, seed=3 * n, shift=0.5)
    Rh = W.gaussian_rhs(n, m, 12)
    out = []
    for flags in [SB, BLK]:
        st, F, _ = spd.spd_factor(h, dev_sym(A), prec, flags)
        check(h, st)
        try:
            L, _, _ = factor_L(F)
            out.append((L, apply_factor(h, F, Rh)))
        finally:
            spd.spd_factor_destroy(F)
    assert np.array_equal(out[0][0], out[1][0])
    z0, z1 = out[0][1], out[1][1]
    err = np.max(np.abs(z0 - z1)) / np.max(np.abs(z1))
    assert err <= 32 * n * kappa_scaled(A) * U32, err


@pytest.mark.parametrize("n,m", [(4097, 16), (9000, 40)])
def test_superblock_sweeps_repeat_bit_for_bit(h, n, m):
    """Every sum of the super-block sweeps is formed in an order fixed by the
    launch's grid (stream-K pieces added in CTA order), not by timing:
    repeated applications of one factor are identical."""
    A = W.gram_shifted(n, seed=7 * n + m, shift=0.5)
    Rh = W.gaussian_rhs(n, m, 13)
    st, F, _ = spd.spd_factor(h, dev_sym(A), "fp32", SB)
    check(h, st)
    try:
        Z = [apply_factor(h, F, Rh) for _ in range(3)]
    finally:
        spd.spd_factor_destroy(F)
    assert np.array_equal(Z[0], Z[1]) and np.array_equal(Z[0], Z[2])


def test_small_orders_keep_the_block_sweeps(h):
    """Below two super-blocks no inverses are formed: the flag changes nothing."""
    n, m = 1919, 4  # fifteen 128-row blocks
    A = W.gram_shifted(n, seed=5, shift=0.5)
    Rh = W.gaussian_rhs(n, m, 6)
    Z = []
    for flags in [SB, BLK]:
        st, F, _ = spd.spd_factor(h, dev_sym(A), "fp32", flags)
        check(h, st)
        try:
            Z.append(apply_factor(h, F, Rh))
        finally:
            spd.spd_factor_destroy(F)
    assert np.array_equal(Z[0], Z[1])


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_algorithm1_with_superblock_sweeps(h, prec):
    n, m = 3000, 16
    A = W.gram_shifted(n, seed=17, shift=0.1)
    B = W.gaussian_rhs(n, m, 18)
    Ad = dev_sym(A)
    st, F, _ = spd.spd_factor(h, Ad, prec, SB)
    check(h, st)
    try:
        X = dev_zeros(n, m)
        st, rep = spd.spd_solve_ir(h, F, Ad, dev_cols(B), X, {"resid": "tc", "fallback": 0})
        check(h, st)
    finally:
        spd.spd_factor_destroy(F)
    assert rep.iters_high <= 6
    assert oracle.berr(A, B, host(X)) <= 1e-14


def test_async_solve_with_superblock_sweeps_replays_from_a_graph():
    """The device-gated solve: the same answer as the synchronous call, and a
    captured graph (barrier words cleared by a captured memset) replayed for
    new right-hand sides."""
    s = torch.cuda.Stream()
    h = spd.spd_create(s)
    try:
        n, m = 2100, 3
        A = W.gram_shifted(n, seed=22, shift=0.1)
        Ad = dev_sym(A)
        B0 = W.gaussian_rhs(n, m, 1)
        Bd = dev_zeros(n, m)
        X = dev_zeros(n, m)
        X1 = dev_zeros(n, m)
        buf = spd.spd_report_dev_buffer()
        opts = {"resid": "tc", "maxit": 12}
        with torch.cuda.stream(s):
            st, F, _ = spd.spd_factor(h, Ad, "fp16", SB)
            check(h, st)
            Bd.copy_(dev_cols(B0))
            st, rep = spd.spd_solve_ir(h, F, Ad, Bd, X1, {"resid": "tc", "fallback": 0})
            check(h, st)
            check(h, spd.spd_solve_ir_async(h, F, Ad, Bd, X, buf, opts))  # sizes the workspace
        s.synchronize()
        r = spd.spd_report_dev_read(buf)
        assert r.status == spd.SPD_OK and r.sweeps == rep.iters_high - 1
        assert np.array_equal(host(X), host(X1))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            st = spd.spd_solve_ir_async(h, F, Ad, Bd, X, buf, opts)
        check(h, st)
        try:
            for seed in (2, 3):
                Bh = W.gaussian_rhs(n, m, seed)
                with torch.cuda.stream(s):
                    Bd.copy_(dev_cols(Bh))
                    X.zero_()
                    g.replay()
                s.synchronize()
                r = spd.spd_report_dev_read(buf)
                assert r.status == spd.SPD_OK and r.active == 0 and r.dev_flags == 0, (seed, r.status)
                assert oracle.berr(A, Bh, host(X)) <= 1e-14, seed
        finally:
            spd.spd_factor_destroy(F)
    finally:
        spd.spd_destroy(h)
