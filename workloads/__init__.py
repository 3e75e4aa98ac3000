"""Seeded synthetic inputs for the mixed-precision SPD solver.

This module only *synthesises inputs*: matrices, right-hand sides and planted
solutions.  It holds none of the solver's arithmetic (no factorisation, no
substitution, no refinement, no CG), so both the CPU oracle and the CUDA path
can draw their inputs from it without sharing any of the method.

All generators return float64 numpy arrays.  Matrices are exactly symmetric
and stored C-contiguous; because they are symmetric the same buffer is also
their column-major representation with leading dimension n.  Right-hand sides
are returned as (n, m) arrays; ``np.asfortranarray`` gives the column-major
layout the C-ABI takes.

Workload recipes (each cites where its shape comes from):

* ``model_covariance``  -- the paper's model covariance matrix (Section 4):
  A(i,j) = 1/|i-j|^d off the diagonal, 1 + sqrt(i) on it, i 1-based.
* ``gram_shifted``       -- A = G G^T / n + shift I, G i.i.d. N(0,1).
* ``householder_spectrum`` -- A = Q diag(lambda) Q^T, Q a product of random
  Householder reflectors, lambda log-spaced in [1, kappa].
* ``exp_kernel_cov``     -- exp(-|p_i - p_j| / ell) over uniform points in the
  unit cube plus a nugget on the diagonal.
* ``matern32_cov``       -- Matern-3/2 covariance over uniform points in the
  unit square plus a nugget.
* ``batched_gram``       -- many independent ``gram_shifted`` systems of
  uneven order.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "model_covariance",
    "uniform_rhs",
    "gram_shifted",
    "householder_vectors",
    "householder_spectrum",
    "exp_kernel_cov",
    "matern32_cov",
    "batched_sizes",
    "batched_gram",
    "gaussian_rhs",
]


def rng(seed: int) -> np.random.Generator:
    """The one random stream used everywhere: numpy PCG64 with an integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


# ---------------------------------------------------------------------------
# The paper's workload (Section 4): model covariance with decay d.
# ---------------------------------------------------------------------------
def model_covariance(n: int, d: float) -> np.ndarray:
    """Model covariance of Section 4 with 1-based index i.

    Off-diagonal entries decay as 1/|i-j|^d; the diagonal is 1 + sqrt(i) for
    i = 1..n.  With the 1-based reading the diagonal is at least 2 while the
    off-diagonal Toeplitz symbol of 1/|k|^d is bounded below by -2 ln 2
    (d=1), -pi^2/6 (d=2) and -(7/4) zeta(4) (d=4), so the matrix is SPD.
    """
    i = np.arange(n, dtype=np.float64)
    k = np.abs(i[:, None] - i[None, :])
    with np.errstate(divide="ignore"):
        A = np.where(k > 0, 1.0 / np.power(np.maximum(k, 1.0), d), 0.0)
    A[np.diag_indices(n)] = 1.0 + np.sqrt(i + 1.0)
    return A


def uniform_rhs(n: int, m: int, seed: int = 0) -> np.ndarray:
    """Right-hand sides with entries U[0,1] (Section 4); column j uses stream seed+j."""
    B = np.empty((n, m), dtype=np.float64)
    for j in range(m):
        B[:, j] = rng(seed + j).random(n)
    return B


def gaussian_rhs(n: int, m: int, seed: int) -> np.ndarray:
    """N(0,1) right-hand sides (or planted solutions), one (n, m) block from one stream."""
    return rng(seed).standard_normal((n, m))


# ---------------------------------------------------------------------------
# Gram matrices G G^T / n + shift I.
# ---------------------------------------------------------------------------
def gram_shifted(n: int, seed: int = 0, shift: float = 0.1) -> np.ndarray:
    """A = G G^T / n + shift * I with G (n x n) i.i.d. N(0,1) from ``rng(seed)``.

    The eigenvalues of G G^T / n follow Marchenko-Pastur on [0, 4], so the
    condition number is about (4 + shift) / shift.
    """
    G = rng(seed).standard_normal((n, n))
    A = (G @ G.T) / n
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] += shift
    return A


# ---------------------------------------------------------------------------
# A = Q diag(lambda) Q^T with Q = H_1 ... H_k (random Householder reflectors).
# ---------------------------------------------------------------------------
def householder_vectors(n: int, k: int = 32, seed: int = 0) -> np.ndarray:
    """k unit vectors (n x k) drawn N(0,1) and normalised; H_i = I - 2 v_i v_i^T."""
    V = rng(seed).standard_normal((n, k))
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    return V


def _compact_wy_T(V: np.ndarray) -> np.ndarray:
    """T (k x k, upper) with H_1 H_2 ... H_k = I - V T V^T for unit columns of V."""
    k = V.shape[1]
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 2.0
        if j:
            T[:j, j] = -2.0 * (T[:j, :j] @ (V[:, :j].T @ V[:, j]))
    return T


def householder_spectrum(n: int, kappa: float, k: int = 32, seed: int = 0,
                         device=None):
    """A = Q diag(lambda) Q^T, Q = H_1...H_k, lambda_i log-spaced in [1, kappa].

    Q is applied in compact-WY form Q = I - V T V^T, so that
    A = Lambda + [V W] C [V W]^T with W = Lambda V and a 2k x 2k core C; the
    assembly is one rank-2k update of a diagonal.  With ``device`` a torch
    device the assembly runs there in float64 (the random draws stay on the
    host, so every device sees the same V and lambda); the result is then a
    torch tensor.  Returns (A, lam, V).
    """
    lam = np.logspace(0.0, np.log10(kappa), n)
    V = householder_vectors(n, k, seed)
    T = _compact_wy_T(V)
    W = lam[:, None] * V
    VtW = V.T @ W
    # A = (I - V T V^T) Lam (I - V T^T V^T)
    #   = Lam - V T W^T - W T^T V^T + V (T VtW T^T) V^T
    C = np.zeros((2 * k, 2 * k))
    C[:k, :k] = T @ VtW @ T.T
    C[:k, k:] = -T
    C[k:, :k] = -T.T
    Y = np.concatenate([V, W], axis=1)
    if device is None:
        A = (Y @ C) @ Y.T
        A = 0.5 * (A + A.T)
        A[np.diag_indices(n)] += lam
        return A, lam, V
    import torch
    Yt = torch.from_numpy(Y).to(device)
    Ct = torch.from_numpy(C).to(device)
    A = (Yt @ Ct) @ Yt.T
    A = 0.5 * (A + A.T)
    A.diagonal().add_(torch.from_numpy(lam).to(device))
    return A, lam, V


# ---------------------------------------------------------------------------
# Kernel covariance matrices over random points.
# ---------------------------------------------------------------------------
def _pairwise_dist(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    diff = P[:, None, :] - Q[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=-1))


def exp_kernel_cov(n: int, ell: float = 0.1, nugget: float = 1e-3, seed: int = 0,
                   dim: int = 3, device=None, points=None):
    """A_ij = exp(-|p_i - p_j|_2 / ell) + nugget * delta_ij, p_i ~ U[0,1]^dim.

    With ``device`` the pairwise distances and exponentials are evaluated
    there (float64, row blocks) and a torch tensor is returned.
    Returns (A, points).
    """
    P = rng(seed).random((n, dim)) if points is None else points
    if device is None:
        A = np.exp(-_pairwise_dist(P, P) / ell)
        A[np.diag_indices(n)] += nugget
        return A, P
    import torch
    Pt = torch.from_numpy(P).to(device)
    A = torch.empty((n, n), dtype=torch.float64, device=device)
    blk = 2048
    for r in range(0, n, blk):
        d = torch.cdist(Pt[r:r + blk], Pt, compute_mode="donot_use_mm_for_euclid_dist")
        A[r:r + blk] = torch.exp(-d / ell)
    A = 0.5 * (A + A.T)
    A.diagonal().add_(nugget)
    return A, P


def matern32_cov(n: int, ell: float, nugget: float, seed: int, dim: int = 2,
                 points=None):
    """Matern-3/2: A_ij = (1 + sqrt3 r/ell) exp(-sqrt3 r/ell) + nugget delta_ij."""
    P = rng(seed).random((n, dim)) if points is None else points
    r = _pairwise_dist(P, P)
    s = np.sqrt(3.0) * r / ell
    A = (1.0 + s) * np.exp(-s)
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] += nugget
    return A, P


def matern_family_params(seed: int):
    """(ell, nugget) of one member of the Matern-3/2 family:
    ell ~ U[0.02, 0.5], nugget ~ logU[1e-4, 1e-1]."""
    g = rng(10_000_000 + int(seed))
    ell = 0.02 + 0.48 * g.random()
    nugget = 10.0 ** (-4.0 + 3.0 * g.random())
    return float(ell), float(nugget)


# ---------------------------------------------------------------------------
# Batched systems of uneven order.
# ---------------------------------------------------------------------------
def batched_sizes(count: int = 4096, nmin: int = 32, nmax: int = 512, seed: int = 0) -> np.ndarray:
    """System orders n_i ~ U{nmin..nmax} from ``rng(seed)``."""
    return rng(seed).integers(nmin, nmax + 1, size=count).astype(np.int64)


def batched_gram(sizes, shift: float = 0.05, seed_base: int = 1000):
    """System i: A_i = G G^T / n_i + shift I with G from ``rng(seed_base + i)``,
    and one N(0,1) right-hand side drawn from the same stream after G."""
    As, bs = [], []
    for i, n in enumerate(np.asarray(sizes)):
        g = rng(seed_base + i)
        G = g.standard_normal((int(n), int(n)))
        A = (G @ G.T) / n
        A = 0.5 * (A + A.T)
        A[np.diag_indices(int(n))] += shift
        As.append(A)
        bs.append(g.standard_normal(int(n)))
    return As, bs


def matern32_torch(points, ell: float, nugget: float, device):
    """Matern-3/2 covariance of the given points (numpy, n x dim) assembled
    in float64 on a torch device; same formula as ``matern32_cov``."""
    import torch
    P = torch.from_numpy(np.asarray(points, dtype=np.float64)).to(device)
    r = torch.cdist(P, P, compute_mode="donot_use_mm_for_euclid_dist")
    s = (3.0 ** 0.5) * r / ell
    A = (1.0 + s) * torch.exp(-s)
    A = 0.5 * (A + A.T)
    A.diagonal().add_(nugget)
    return A


def matern_points(n: int, seed: int, dim: int = 2):
    """Uniform points in the unit square (cube) for Matern system ``seed``."""
    return rng(seed).random((n, dim))
