"""Training loop of the learned diagonal-plus-low-rank preconditioner.

Host-side orchestration only: every step calls the library's kernels
through the C ABI (features, network forward/backward, probe loss, Adam;
the optional supervised target A^{-1} z_0 comes from the system's own
float32 Cholesky factor and two triangular solves).  Systems are drawn
from the Matern-3/2 family: points uniform in the unit square,
ell ~ U[0.02, 0.5], nugget ~ logU[1e-4, 1e-1].
"""
from __future__ import annotations

import numpy as np
import torch

from . import (PREC, SPD_OK, SpdError, colmajor, spd_factor, spd_factor_destroy, spd_factor_solve,
               spd_last_error_string, spd_learned_features, spd_mlp_adam, spd_mlp_loss_grad)


def make_system(n, seed, device, workloads):
    ell, nugget = workloads.matern_family_params(seed)
    pts = workloads.matern_points(n, seed)
    A = workloads.matern32_torch(pts, ell, nugget, device)
    coords = torch.from_numpy(np.ascontiguousarray(pts)).to(device)
    return A, coords, ell, nugget


def features(h, A, coords, ell, nugget):
    n = A.shape[0]
    F = torch.empty((n, 16), dtype=torch.float32, device=A.device)
    st = spd_learned_features(h, A, coords, ell, nugget, F)
    if st != SPD_OK:
        raise SpdError(st, spd_last_error_string(h))
    return F


def train(h, net, n, seeds, workloads, probes=8, lr=2e-3, wsup=0.1, use_factor=True, log_every=0,
          lr_final=0.05):
    """One Adam step per system seed (learning rate decays on a cosine from
    lr to lr * lr_final); returns the loss history."""
    dev = torch.device("cuda")
    hist = []
    seeds = list(seeds)
    steps = max(len(seeds), 1)
    for k, seed in enumerate(seeds):
        A, coords, ell, nugget = make_system(n, seed, dev, workloads)
        F = features(h, A, coords, ell, nugget)
        g = torch.Generator(device=dev)
        g.manual_seed(7919 * int(seed) + 1)
        Z = torch.randn((probes, n), dtype=torch.float64, device=dev, generator=g).t()
        T = None
        if use_factor:
            st, Fct, _ = spd_factor(h, A, "fp32")
            if st == SPD_OK:
                T = torch.zeros((1, n), dtype=torch.float64, device=dev).t()
                spd_factor_solve(h, Fct, Z[:, :1], T)
                spd_factor_destroy(Fct)
        st, L = spd_mlp_loss_grad(net, A, F, Z, T, wsup if T is not None else 0.0)
        if st != SPD_OK:
            raise SpdError(st, spd_last_error_string(h))
        frac = k / steps
        spd_mlp_adam(net, lr * (lr_final + (1.0 - lr_final) * 0.5 * (1.0 + np.cos(np.pi * frac))))
        hist.append(L)
        if log_every and (k + 1) % log_every == 0:
            print(f"step {k + 1}: loss {np.mean(hist[-log_every:]):.4g}", flush=True)
    return hist
