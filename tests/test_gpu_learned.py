"""GPU parity of the learned diagonal-plus-low-rank preconditioner: features,
network loss and gradient (against central finite differences of the
float64 oracle), the Woodbury apply, the training gain over Jacobi-PCG on
held-out systems, and the Cholesky-IR fallback."""
import numpy as np
import pytest
import torch

import oracle
import paper_1405_4644_gb300 as spd
import workloads as W
from oracle import learned as LO
from paper_1405_4644_gb300 import learned as trainer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    hh = spd.spd_create(torch.cuda.current_stream())
    yield hh
    spd.spd_destroy(hh)


def system(n, seed):
    ell, nug = W.matern_family_params(seed)
    pts = W.matern_points(n, seed)
    A, _ = W.matern32_cov(n, ell, nug, seed, points=pts)
    return A, pts, ell, nug


def test_features_match_oracle(h):
    A, pts, ell, nug = system(200, 3)
    F = torch.empty((200, 16), dtype=torch.float32, device="cuda")
    assert spd.spd_learned_features(h, torch.from_numpy(A).cuda(), torch.from_numpy(pts).cuda(), ell, nug, F) == 0
    np.testing.assert_allclose(F.cpu().numpy(), LO.features(A, pts, ell, nug), rtol=2e-6, atol=2e-6)


def _net(h, H, seed, bf16=False):
    st, net = spd.spd_mlp_create(h, H, seed, bf16)
    assert st == 0
    return net


def test_loss_and_gradient_match_oracle_finite_differences(h):
    n, H, p = 64, 16, 4
    A, pts, ell, nug = system(n, 5)
    net = _net(h, H, seed=1)
    try:
        cnt = spd.spd_mlp_params(net)
        params = np.zeros(cnt, dtype=np.float32)
        spd.spd_mlp_params(net, out=params)
        # move off the initialisation so every layer matters
        params += (np.random.default_rng(2).standard_normal(cnt) * 0.05).astype(np.float32)
        spd.spd_mlp_params(net, inp=params)
        Fg = torch.from_numpy(LO.features(A, pts, ell, nug).astype(np.float32)).cuda()
        Z = W.gaussian_rhs(n, p, 9)
        T = np.linalg.solve(A, Z[:, :1])
        Ad = torch.from_numpy(A).cuda()
        Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda().t()
        Td = torch.from_numpy(np.ascontiguousarray(T.T)).cuda().t()
        st, L = spd.spd_mlp_loss_grad(net, Ad, Fg, Zd, Td, 0.3)
        assert st == 0
        grad = np.zeros(cnt, dtype=np.float32)
        spd.spd_mlp_params(net, grad=grad)
    finally:
        spd.spd_mlp_destroy(net)
    p64 = params.astype(np.float64)
    F64 = Fg.cpu().numpy().astype(np.float64)
    L_ref = LO.loss(p64, H, A, F64, Z, T, 0.3)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    g = np.random.default_rng(3)
    dirs = [g.standard_normal(cnt) for _ in range(3)]
    big = np.argsort(-np.abs(grad))[:4]
    for k in big:
        e = np.zeros(cnt)
        e[k] = 1.0
        dirs.append(e)
    fd = LO.fd_grad(p64, H, A, F64, Z, dirs, T, 0.3, h=1e-4)
    an = np.array([grad.astype(np.float64) @ v for v in dirs])
    np.testing.assert_allclose(an, fd, rtol=2e-3, atol=1e-5 * np.abs(fd).max())


@pytest.mark.parametrize("n", [96, 700])  # one projection chunk; three, the last ragged
def test_woodbury_apply_matches_dense_inverse(h, n):
    H = 32
    A, pts, ell, nug = system(n, 8)
    net = _net(h, H, seed=4)
    try:
        cnt = spd.spd_mlp_params(net)
        params = np.zeros(cnt, dtype=np.float32)
        spd.spd_mlp_params(net, out=params)
        params += (np.random.default_rng(5).standard_normal(cnt) * 0.1).astype(np.float32)
        spd.spd_mlp_params(net, inp=params)
        Fg = torch.from_numpy(LO.features(A, pts, ell, nug).astype(np.float32)).cuda()
        st, P = spd.spd_lowrank_build(net, torch.from_numpy(A).cuda(), Fg)
        assert st == 0
        R = W.gaussian_rhs(n, 3, 6)
        Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda().t()
        Zd = torch.zeros((3, n), dtype=torch.float64, device="cuda").t()
        assert spd.spd_lowrank_apply(P, Rd, Zd) == 0
        spd.spd_lowrank_destroy(P)
    finally:
        spd.spd_mlp_destroy(net)
    M = LO.precond(LO.forward(params.astype(np.float64), Fg.cpu().numpy().astype(np.float64), H), A)
    np.testing.assert_allclose(Zd.cpu().numpy(), M @ R, rtol=1e-5, atol=1e-7 * np.abs(M @ R).max())


@pytest.mark.parametrize("n,m", [(700, 1), (700, 3), (1300, 2)])
def test_learned_pcg_fused_step_graph_and_direct_agree(n, m):
    """The learned PCG's inner step fuses the Woodbury apply into the CG
    update (projection partials) and the next dots: it reaches the relative
    target against the float64 solution, and the steps replayed from a CUDA
    graph give the iterates of the same kernels launched one by one
    (profiling on), bit for bit."""
    A, pts, ell, nug = system(n, 9)
    B = W.gaussian_rhs(n, m, 10)
    out = []
    for prof in (False, True):
        hh = spd.spd_create(torch.cuda.current_stream())
        net = _net(hh, 32, seed=6)
        try:
            spd.spd_profile_enable(hh, prof)
            Ad = torch.from_numpy(A).cuda()
            Fg = torch.from_numpy(LO.features(A, pts, ell, nug).astype(np.float32)).cuda()
            st, P = spd.spd_lowrank_build(net, Ad, Fg)
            assert st == 0
            X = torch.zeros((m, n), dtype=torch.float64, device="cuda").t()
            Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
            st, rep = spd.spd_cg(hh, Ad, Bd, X, "fp64", "lowrank", P,
                                 opts={"tol": 1e-10, "crit": "rel2", "eta": 1e-12, "maxit_inner": 5000})
            spd.spd_lowrank_destroy(P)
            assert st == 0
            out.append((X.cpu().numpy(), rep.iters_low))
        finally:
            spd.spd_mlp_destroy(net)
            spd.spd_destroy(hh)
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    x_ref = np.linalg.solve(A, B)
    assert np.max(np.abs(out[0][0] - x_ref)) <= 1e-7 * np.max(np.abs(x_ref))


def _pcg_iters(h, A, b, pc, P=None):
    Ad = torch.from_numpy(A).cuda()
    X = torch.zeros((1, len(b)), dtype=torch.float64, device="cuda").t()
    Bd = torch.from_numpy(b).cuda()[:, None]
    st, rep = spd.spd_cg(h, Ad, Bd, X, "fp64", pc, P, opts={"tol": 1e-10, "crit": "rel2", "eta": 1e-12,
                                                             "maxit_inner": 5000})
    assert st == 0
    return rep.iters_low, X.cpu().numpy()[:, 0]


def test_training_reduces_pcg_iterations_on_held_out_systems(h):
    """The method without the network (Jacobi-PCG) against PCG with the
    trained diagonal-plus-low-rank preconditioner, on systems the network
    never saw; solutions judged against the Cholesky oracle."""
    n = 256
    net = _net(h, 128, seed=11, bf16=True)
    try:
        hist = trainer.train(h, net, n, range(2000), W, probes=8, lr=3e-3, wsup=0.1, use_factor=True)
        assert np.mean(hist[-30:]) < 0.7 * np.mean(hist[:10])
        gains = []
        for seed in range(100000, 100008):
            A, pts, ell, nug = system(n, seed)
            b = W.gaussian_rhs(n, 1, seed)[:, 0]
            it_j, _ = _pcg_iters(h, A, b, "jacobi")
            Ad = torch.from_numpy(A).cuda()
            F = trainer.features(h, Ad, torch.from_numpy(pts).cuda(), ell, nug)
            st, P = spd.spd_lowrank_build(net, Ad, F)
            assert st == 0
            it_l, x = _pcg_iters(h, A, b, "lowrank", P)
            spd.spd_lowrank_destroy(P)
            xo = oracle.solve(A, b[:, None])[:, 0]
            assert np.max(np.abs(x - xo)) <= 1e-6 * np.max(np.abs(xo)) * np.linalg.cond(A) ** 0.5
            gains.append(it_j / max(it_l, 1))
    finally:
        spd.spd_mlp_destroy(net)
    assert np.median(gains) > 1.3, gains


def test_learned_solve_falls_back_to_cholesky_ir(h):
    """A useless network (and a tiny CG budget) still yields a float64-accurate
    solution through the float32 Cholesky-IR fallback."""
    n = 200
    A, pts, ell, nug = system(n, 21)
    net = _net(h, 32, seed=3)
    try:
        cnt = spd.spd_mlp_params(net)
        junk = (np.random.default_rng(0).standard_normal(cnt) * 3).astype(np.float32)
        spd.spd_mlp_params(net, inp=junk)
        Ad = torch.from_numpy(A).cuda()
        F = trainer.features(h, Ad, torch.from_numpy(pts).cuda(), ell, nug)
        st, P = spd.spd_lowrank_build(net, Ad, F)
        assert st == 0
        b = W.gaussian_rhs(n, 1, 1)
        X = torch.zeros((1, n), dtype=torch.float64, device="cuda").t()
        st, rep = spd.spd_solve_learned(h, P, Ad, torch.from_numpy(b).cuda(), X,
                                        {"tol": 1e-14, "maxit_inner": 3})
        spd.spd_lowrank_destroy(P)
    finally:
        spd.spd_mlp_destroy(net)
    assert st == 0 and rep.fell_back == 1
    assert oracle.berr(A, b, X.cpu().numpy()) <= 1e-14


def test_checkpoint_round_trip_resumes_training(h, tmp_path):
    """spd_learned_save / spd_learned_load: parameters and Adam state come
    back bit for bit, the loss of the reloaded network equals the original's,
    and one more Adam step from either gives identical parameters."""
    n, H, p = 96, 32, 4
    A, pts, ell, nug = system(n, 11)
    Ad = torch.from_numpy(A).cuda()
    Fg = torch.from_numpy(LO.features(A, pts, ell, nug).astype(np.float32)).cuda()
    Zd = torch.from_numpy(np.ascontiguousarray(W.gaussian_rhs(n, p, 3).T)).cuda().t()
    net = _net(h, H, seed=4)
    net2 = None
    try:
        for _ in range(3):
            st, _ = spd.spd_mlp_loss_grad(net, Ad, Fg, Zd)
            assert st == 0 and spd.spd_mlp_adam(net, 1e-3) == 0
        path = tmp_path / "net"
        assert spd.spd_learned_save(net, path) == 0
        assert (tmp_path / "net.json").exists() and (tmp_path / "net.bin").exists()
        st, net2 = spd.spd_learned_load(h, path)
        assert st == 0
        cnt = spd.spd_mlp_params(net)
        a, b = np.zeros(cnt, np.float32), np.zeros(cnt, np.float32)
        spd.spd_mlp_params(net, out=a)
        spd.spd_mlp_params(net2, out=b)
        assert np.array_equal(a, b)
        st, l1 = spd.spd_mlp_loss_grad(net, Ad, Fg, Zd)
        st2, l2 = spd.spd_mlp_loss_grad(net2, Ad, Fg, Zd)
        assert st == 0 and st2 == 0 and l1 == l2
        assert spd.spd_mlp_adam(net, 1e-3) == 0 and spd.spd_mlp_adam(net2, 1e-3) == 0
        spd.spd_mlp_params(net, out=a)
        spd.spd_mlp_params(net2, out=b)
        assert np.array_equal(a, b)
        # a truncated parameter file is refused
        raw = (tmp_path / "net.bin").read_bytes()
        (tmp_path / "net.bin").write_bytes(raw[:-4])
        st, bad = spd.spd_learned_load(h, path)
        assert st == spd.SPD_ERR_ARG and bad is None
    finally:
        spd.spd_mlp_destroy(net)
        if net2 is not None:
            spd.spd_mlp_destroy(net2)
