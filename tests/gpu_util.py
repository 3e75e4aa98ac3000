"""Helpers shared by the GPU parity tests (marshalling only, no solver arithmetic)."""
import numpy as np
import torch

import paper_1405_4644_gb300 as spd

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def dev_sym(A):
    return torch.from_numpy(np.ascontiguousarray(A)).to(DEV)


def dev_cols(B):
    """Column-major (n, m) device copy of a host (n, m) array."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    return torch.from_numpy(np.ascontiguousarray(B.T)).to(DEV).t()


def dev_zeros(n, m):
    return torch.zeros(m, n, dtype=torch.float64, device=DEV).t()


def host(t):
    return t.detach().cpu().numpy()


def factor_L(F):
    """(lower triangle of the factor as float64, scaling d, precision code)."""
    n, prec = spd.spd_factor_info(F)
    dt = np.float64 if prec == spd.PREC["fp64"] else np.float32
    L = np.zeros((n, max(n, 1)), dtype=dt)
    d = np.zeros(n)
    assert spd.spd_factor_copy(F, L, d) == spd.SPD_OK
    return np.tril(L).astype(np.float64), d, prec


def check(h, st, want=spd.SPD_OK):
    assert st == want, f"status {st} (want {want}): {spd.spd_last_error_string(h)}"
