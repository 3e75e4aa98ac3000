"""Small, fixed cases of single kernels families, for profiling one kernel at a
time (each case repeats its call so that a profiler can skip the first one):

    python -m paper_1405_4644_gb300.cases gemm        # tcgen05 update, BF16, M = N = K = 8192
    python -m paper_1405_4644_gb300.cases resid_fp64  # float64 residual, n = 8192, m = 16
    python -m paper_1405_4644_gb300.cases resid_tc    # tensor-core residual, n = 8192, m = 16
    python -m paper_1405_4644_gb300.cases sweeps      # triangular sweeps of an FP16 factor, n = 8192, m = 16
    python -m paper_1405_4644_gb300.cases convert     # scale + convert and factor, FP32, n = 8192

Inputs are seeded and synthetic (workloads); nothing is checked beyond the
status codes.  With --phases the library's per-phase records (launches, event
time, algorithmic flops and bytes, summed over the repetitions) are printed at
the end, for comparing a profiler's DRAM bytes with the algorithmic bytes.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["gemm", "resid_fp64", "resid_tc", "sweeps", "convert"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--phases", action="store_true")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_1405_4644_gb300 as spd
    import workloads as W

    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    n, m = a.n, a.m
    if a.phases:
        spd.spd_profile_enable(h, True)

    def ok(st):
        if st != spd.SPD_OK:
            raise RuntimeError(spd.spd_last_error_string(h))

    g = torch.Generator(device=dev).manual_seed(0)
    if a.case == "gemm":
        A = torch.rand(n, n, device=dev, generator=g) - 0.5
        C = torch.zeros(n, n, device=dev)
        for _ in range(a.reps):
            ok(spd.spd_gemm_update(h, "bf16", A, A, C))
    else:
        if a.case == "resid_fp64":
            A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
            A = A + A.T
        else:
            A, _, _ = W.householder_spectrum(n, 1e2, k=16, seed=0, device=dev)
        X = torch.randn(m, n, dtype=torch.float64, device=dev, generator=g).t()
        B = torch.randn(m, n, dtype=torch.float64, device=dev, generator=g).t()
        R = torch.zeros(m, n, dtype=torch.float64, device=dev).t()
        for _ in range(a.reps):
            if a.case == "resid_fp64":
                ok(spd.spd_residual(h, A, B, X, R))
            elif a.case == "resid_tc":
                ok(spd.spd_residual_tc(h, A, B, X, R))
            elif a.case == "convert":
                st, F, _ = spd.spd_factor(h, A, "fp32")
                ok(st)
                spd.spd_factor_destroy(F)
        if a.case == "sweeps":
            st, F, _ = spd.spd_factor(h, A, "fp16")
            ok(st)
            for _ in range(a.reps):
                ok(spd.spd_factor_solve(h, F, B, R))
            spd.spd_factor_destroy(F)
    torch.cuda.synchronize()
    if a.phases:
        for p in spd.PHASES:
            r = spd.spd_profile_read(h, p)
            if r["launches"]:
                print(f"phase {p}: launches {r['launches']} ms {r['ms']:.3f} flops {r['flops']:.6e} "
                      f"bytes {r['bytes']:.6e} (sum over {a.reps} repetitions)")
    spd.spd_destroy(h)
    print("ok", a.case, n, m)
    return 0


if __name__ == "__main__":
    sys.exit(main())
