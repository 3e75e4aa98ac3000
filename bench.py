#!/usr/bin/env python3
"""Benchmark: float64-accurate SPD solves per second (and joules per solve)
with mixed-precision Cholesky + iterative refinement (Algorithm 1), against
a float64 blocked Cholesky on the same GPU.

Workload (precision sweep): n = 16384, A = Q diag(lambda) Q^T with Q a
product of 32 random Householder reflectors and lambda log-spaced in
[1, kappa] for kappa in {1e2, 1e4, 1e6}; 16 N(0,1) right-hand sides; float64
storage.  One step = factor + refine all three systems to normwise backward
error <= 1e-14 (three solves).  Inputs (3 x 2.15 GB) are resident in HBM and
larger than L2.  Generation is untimed, as in the paper (Section 4.1).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-accurate SPD solves/s & J/solve: mixed-prec IR vs FP64 Cholesky, 1 GB300"
UNIT = "solves/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal dense tensor ratios to bf16 (fp16 1x, tf32 0.5x, fp8 2x); FP64 and
# FP32 CUDA-core peaks from the unit counts: 152 SMs x 2.07 GHz x (FP32: 128
# lanes x 2 flops; FP64: nominal 1.25 TFLOP/s for the part)
TENSOR_RATIO = {"fp16": 1.0, "bf16": 1.0, "tf32": 0.5, "fp8": 2.0}
FP32_SIMT_PEAK_TFLOPS = 152 * 2.07e9 * 128 * 2 / 1e12
FP64_PEAK_TFLOPS = 1.25


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# clocks / power during the timed region
# ---------------------------------------------------------------------------
class SmiSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "avg_power_w": statistics.mean(r[2] for r in rows), "samples": len(rows)}


class Nvml:
    """Read-only NVML access (total-energy counter) through the driver library."""

    def __init__(self, index):
        self.ok = False
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                return
            self.ok = self.energy_mj() is not None
        except OSError:
            pass

    def energy_mj(self):
        v = ctypes.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, ctypes.byref(v)) != 0:
            return None
        return v.value

    def power_w(self):
        v = ctypes.c_uint()
        if self.lib.nvmlDeviceGetPowerUsage(self.dev, ctypes.byref(v)) != 0:
            return None
        return v.value / 1000.0


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no collective on the data path)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_systems(n, m, kappas, dev):
    import numpy as np
    import torch
    import workloads as W
    systems = []
    for i, kappa in enumerate(kappas):
        A, lam, V = W.householder_spectrum(n, kappa, k=32, seed=i, device=dev)
        B = torch.from_numpy(np.ascontiguousarray(W.gaussian_rhs(n, m, 100 + i).T)).to(dev).t()
        systems.append((kappa, A, B))
    torch.cuda.synchronize()
    return systems


def run_step(spd, h, systems, precs, X, opts):
    reps = []
    for (kappa, A, B), prec in zip(systems, precs):
        st, F, frep = spd.spd_factor(h, A, prec)
        if st != spd.SPD_OK:
            raise RuntimeError(f"spd_factor({prec}, kappa={kappa}): {spd.spd_last_error_string(h)}")
        st, rep = spd.spd_solve_ir(h, F, A, B, X, opts)
        spd.spd_factor_destroy(F)
        if st != spd.SPD_OK:
            raise RuntimeError(f"spd_solve_ir kappa={kappa}: {spd.spd_last_error_string(h)}")
        reps.append((frep, rep))
    return reps


def cpu_oracle_sample(n_full, m, seconds_hint=20.0):
    """Time the float64 CPU oracle (Cholesky + substitution) on a bounded
    sample of the workload; scale to the full order by n^3."""
    import numpy as np
    import oracle
    import workloads as W
    ns = 3072
    A, lam, V = W.householder_spectrum(ns, 1e2, k=32, seed=0)
    B = W.gaussian_rhs(ns, m, 100)
    t0 = time.perf_counter()
    X = oracle.solve(A, B)
    t = time.perf_counter() - t0
    assert np.isfinite(X).all()
    scale = (n_full / ns) ** 3
    return {"value": 1.0 / (t * scale), "unit": UNIT, "cores": oracle.cpu_threads(), "kind": "oracle",
            "sample": f"one float64 oracle solve (Cholesky + substitution) at n={ns}, m={m}, kappa=1e2: "
                      f"{t:.2f} s, scaled by (n/{ns})^3 to n={n_full}"}


def reference_arm(args):
    """The oracle as it stands on the host cores, timed like our arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    samples = []
    for _ in range(args.warmup):
        cpu_oracle_sample(args.n, args.m)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(cpu_oracle_sample(args.n, args.m))
    wall = time.perf_counter() - t0
    v = statistics.mean(s["value"] for s in samples)
    cb = dict(samples[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"precision sweep n={args.n} m={args.m} kappa in {args.kappas}", "n": args.n,
                      "m": args.m},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--kappas", default="1e2,1e4,1e6")
    ap.add_argument("--precs", default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    args.kappas = [float(k) for k in args.kappas.split(",")]
    precs = args.precs.split(",")
    if len(precs) == 1:
        precs = precs * len(args.kappas)
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    h = spd.spd_create(stream)
    systems = make_systems(args.n, args.m, args.kappas, dev)
    X = torch.zeros(args.m, args.n, dtype=torch.float64, device=dev).t()
    opts = {"tol": 1e-14, "crit": "berr"}

    for _ in range(args.warmup):
        run_step(spd, h, systems, precs, X, opts)
    torch.cuda.synchronize()

    smi = SmiSampler(torch.cuda.current_device())
    nvml = Nvml(torch.cuda.current_device())
    spd.spd_profile_enable(h, True)
    launches0 = spd.spd_launch_count(h)
    barrier(world)
    torch.cuda.synchronize()
    smi.start()
    e0 = nvml.energy_mj() if nvml.ok else None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(args.steps):
        reps = run_step(spd, h, systems, precs, X, opts)
    ev1.record(stream)
    torch.cuda.synchronize()
    e1 = nvml.energy_mj() if nvml.ok else None
    barrier(world)
    clocks = smi.stop()
    ms = ev0.elapsed_time(ev1)
    launches = spd.spd_launch_count(h) - launches0
    phases = {p: spd.spd_profile_read(h, p) for p in spd.PHASES}
    spd.spd_profile_enable(h, False)
    ms_max = max_over_ranks(ms, world)
    solves = len(systems) * args.steps * world
    value = solves / (ms_max / 1e3)

    # dominant phase and its roofline
    peaks, peak_src = load_peaks()
    dom = max(phases, key=lambda p: phases[p]["ms"])
    ph = phases[dom]
    per_launch_ms = ph["ms"] / max(ph["launches"], 1)
    if dom == "trailing" and precs[0] in TENSOR_RATIO:
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * TENSOR_RATIO[precs[0]]
        roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": ph["flops"] / (ph["ms"] * 1e-3) / 1e12,
                "peak": peak, "peak_source": f"{peak_src} bf16 sustained x nominal {precs[0]} ratio"}
    elif dom in ("resid",):
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / (ph["ms"] * 1e-3) / 1e12,
                "peak": FP64_PEAK_TFLOPS, "peak_source": "nominal FP64 1.25 TFLOP/s (no measured FP64 peak)"}
    elif dom in ("trailing", "leaf"):
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / (ph["ms"] * 1e-3) / 1e12,
                "peak": FP32_SIMT_PEAK_TFLOPS, "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    else:
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": ph["bytes"] / (ph["ms"] * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "peak_source": f"{peak_src} copy bandwidth"}
    roof.update({"frac": roof["achieved"] / roof["peak"], "kernel_phase": dom, "launches": ph["launches"],
                 "avg_launch_ms": per_launch_ms, "traffic": None,
                 "algorithmic_per_launch": (ph["flops"] if roof["unit"] == "TFLOP/s" else ph["bytes"])
                 / max(ph["launches"], 1)})

    energy = None
    if e0 is not None and e1 is not None:
        j = (e1 - e0) / 1e3
        energy = {"j_per_solve": j / (len(systems) * args.steps), "avg_power_w": j / (ms / 1e3),
                  "source": "NVML total-energy counter, gross"}
    elif clocks:
        j = clocks["avg_power_w"] * ms / 1e3
        energy = {"j_per_solve": j / (len(systems) * args.steps), "avg_power_w": clocks["avg_power_w"],
                  "source": "nvidia-smi power.draw mean x time, gross"}

    per_kappa = [{"kappa": k, "prec": p, "factor_ms": fr.time_ms, "solve_ms": r.time_ms, "iters": r.iters_high,
                  "fell_back": r.fell_back, "berr": r.berr} for (k, _, _), p, (fr, r) in zip(systems, precs, reps)]

    # float64 blocked Cholesky on the same GPU (the plain baseline), one system
    fp64 = None
    if not args.no_fp64:
        kappa, A, B = systems[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (fr, r), = run_step(spd, h, [systems[0]], ["fp64"], X, opts)
        torch.cuda.synchronize()
        t_ours = time.perf_counter() - t0
        t0 = time.perf_counter()
        Lc = torch.linalg.cholesky(A)
        Xc = torch.cholesky_solve(B.contiguous(), Lc)
        torch.cuda.synchronize()
        t_cusolver = time.perf_counter() - t0
        del Lc, Xc
        best = min(t_ours, t_cusolver)
        fp64 = {"ms_per_solve_ours": 1e3 * t_ours, "ms_per_solve_cusolver": 1e3 * t_cusolver,
                "berr_ours": r.berr, "speedup_vs_faster": best / (ms / 1e3 / (len(systems) * args.steps))}

    e2e = None
    if not args.no_e2e:
        import numpy as np
        hostA = [torch.empty((args.n, args.n), dtype=torch.float64, pin_memory=True) for _ in systems]
        hostB = [torch.empty((args.m, args.n), dtype=torch.float64, pin_memory=True) for _ in systems]
        hostX = torch.empty((args.m, args.n), dtype=torch.float64, pin_memory=True)
        for (k, A, B), ha, hb in zip(systems, hostA, hostB):
            ha.copy_(A)
            hb.copy_(B.t())
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for (k, _, _), ha, hb, p in zip(systems, hostA, hostB, precs):
                st = spd.lib().spd_solve_ir_host(h, args.n, args.m, ha.data_ptr(), args.n, hb.data_ptr(),
                                                 args.n, hostX.data_ptr(), args.n, spd.PREC[p],
                                                 spd._opts(opts), ctypes.byref(spd.SpdReport()))
                if st != spd.SPD_OK:
                    raise RuntimeError("e2e: " + spd.spd_last_error_string(h))
        t = time.perf_counter() - t0
        t = max_over_ranks(t, world)
        e2e = {"value": len(systems) * e2e_steps * world / t, "unit": UNIT,
               "h2d_bytes_per_step": len(systems) * 8 * (args.n * args.n + args.n * args.m),
               "d2h_bytes_per_step": len(systems) * 8 * args.n * args.m}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(args.n, args.m)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "mixed: " + "/".join(sorted(set(precs))) + " factor, f64 refinement",
               "data": "synthetic",
               "config": {"workload": f"precision sweep n={args.n} m={args.m} kappa in {args.kappas}",
                          "n": args.n, "m": args.m, "kappas": args.kappas, "factor_prec": precs,
                          "l2": "inputs larger than L2 (3 x 8 n^2 bytes resident)", "tol_berr": 1e-14},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
               "energy": energy, "fp64_baseline": fp64, "per_kappa": per_kappa,
               "phases": {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in phases.items()}}
        print(json.dumps(out), flush=True)
    spd.spd_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
