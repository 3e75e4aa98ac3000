"""float64 oracle of the learned diagonal-plus-low-rank preconditioner --
TEST INFRASTRUCTURE (the paper has no counterpart; this is the plain
definition the GPU kernels are checked against).

* ``features``  per-row features of A (16 per row)
* ``forward``   the 3-layer SiLU network, flat parameter layout
                [W1 (H x 16), b1 (H), W2 (H x H), b2 (H), W3 (33 x H), b3 (33)]
* ``precond``   M = S (Dh + Uh Uh^T)^{-1} S, S = diag(A)^{-1/2},
                Dh = softplus(O[:, 0]) + 1e-3, Uh = O[:, 1:33]
                (dense inverse: numpy's solver is the step used)
* ``loss``      (1/p) sum_c ||A M z_c - z_c||^2 / ||z_c||^2
                + w_sup ||M z_0 - t_0||^2 / ||t_0||^2
* ``fd_grad``   central finite differences of ``loss`` along given directions
                (pinned against the complex-step derivative, which every step of
                ``loss`` supports: parameters may be complex)
"""
from __future__ import annotations

import numpy as np

RANK = 32
NFEAT = 16


def features(A, coords, ell, nugget):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    s = 1.0 / np.sqrt(np.diag(A))
    Ah = np.abs(s[:, None] * A * s[None, :])
    off = Ah.copy()
    np.fill_diagonal(off, -np.inf)
    x, y = coords[:, 0], coords[:, 1]
    pi = np.pi
    F = np.stack([x, y, np.full(n, np.log(ell)), np.full(n, np.log(nugget)),
                  np.sin(pi * x), np.cos(pi * x), np.sin(pi * y), np.cos(pi * y),
                  np.sin(2 * pi * x), np.cos(2 * pi * x), np.sin(2 * pi * y), np.cos(2 * pi * y),
                  Ah.sum(axis=1) / n, np.sqrt((Ah ** 2).sum(axis=1) / n),
                  np.max(off, axis=1) if n > 1 else np.zeros(n), np.ones(n)], axis=1)
    return F


def unpack(params, H):
    p = np.asarray(params)
    if not np.iscomplexobj(p):  # complex parameters: the complex-step derivative of the tests
        p = p.astype(np.float64)
    o = 0
    W1 = p[o:o + H * NFEAT].reshape(H, NFEAT); o += H * NFEAT
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + (1 + RANK) * H].reshape(1 + RANK, H); o += (1 + RANK) * H
    b3 = p[o:o + 1 + RANK]; o += 1 + RANK
    assert o == len(p)
    return W1, b1, W2, b2, W3, b3


def silu(x):
    return x / (1.0 + np.exp(-x))


def forward(params, F, H):
    W1, b1, W2, b2, W3, b3 = unpack(params, H)
    h1 = silu(F @ W1.T + b1)
    h2 = silu(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def precond(O, A):
    s = 1.0 / np.sqrt(np.diag(A))
    dh = np.log1p(np.exp(O[:, 0])) + 1e-3
    U = O[:, 1:1 + RANK]
    Mh = np.linalg.inv(np.diag(dh) + U @ U.T)
    return s[:, None] * Mh * s[None, :]


def loss(params, H, A, F, Z, T=None, wsup=0.0):
    M = precond(forward(params, F, H), A)
    Y = M @ Z
    E = A @ Y - Z
    L = np.mean(np.sum(E ** 2, axis=0) / np.sum(Z ** 2, axis=0))
    if T is not None:
        L += wsup * np.sum((Y[:, 0] - T[:, 0]) ** 2) / np.sum(T[:, 0] ** 2)
    return L


def fd_grad(params, H, A, F, Z, directions, T=None, wsup=0.0, h=1e-5):
    """Directional derivatives d L(params + t v) / dt at t = 0, one per v."""
    out = []
    for v in directions:
        lp = loss(params + h * v, H, A, F, Z, T, wsup)
        lm = loss(params - h * v, H, A, F, Z, T, wsup)
        out.append((lp - lm) / (2 * h))
    return np.array(out)
