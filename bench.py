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
import math
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

    def local_cpus(self):
        """The CPUs NVML lists as closest to the device (its CPU affinity
        mask), or None."""
        words = (os.cpu_count() or 64) // 64 + 1
        mask = (ctypes.c_ulong * words)()
        if self.lib.nvmlDeviceGetCpuAffinity(self.dev, words, mask) != 0:
            return None
        cpus = {64 * w + b for w in range(words) for b in range(64) if mask[w] >> b & 1}
        return cpus or None


def host_numa_info():
    """The memory nodes this process may allocate from (for the record of the
    end-to-end host copies)."""
    try:
        for line in open("/proc/self/status"):
            if line.startswith("Mems_allowed_list"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def bind_near_gpu(nvml):
    """Run this process (and the threads it starts later) on the CPUs next
    to the GPU, so that pinned host buffers, first touched here, sit in the
    GPU's local memory node: the host-to-device copies of the end-to-end
    measurement then cross one link, not the link between CPU sockets.  Only
    this process's CPU affinity changes.  Returns a description."""
    cpus = nvml.local_cpus() if nvml.ok else None
    if not cpus or not hasattr(os, "sched_setaffinity"):
        return {"bound": False}
    cpus &= os.sched_getaffinity(0)
    if not cpus:
        return {"bound": False}
    os.sched_setaffinity(0, cpus)
    return {"bound": True, "cpus": len(cpus)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no collective on the data path)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus):
    """rank, world size and local rank from the launcher's environment; for
    world > 1 a process group over NCCL (one GPU per rank), or over gloo
    where no GPU is visible (host-side tests of this plumbing)."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank does the same work)."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_systems(n, m, kappas, dev, spectra=None):
    """(kappa, A, B) on the device per kappa; with a list `spectra`, also
    (lam, V, B on the host) of each system, for its exact solution."""
    import numpy as np
    import torch
    import workloads as W
    systems = []
    for i, kappa in enumerate(kappas):
        A, lam, V = W.householder_spectrum(n, kappa, k=32, seed=i, device=dev)
        Bh = W.gaussian_rhs(n, m, 100 + i)
        B = torch.from_numpy(np.ascontiguousarray(Bh.T)).to(dev).t()
        systems.append((kappa, A, B))
        if spectra is not None:
            spectra.append((lam, V, Bh))
    torch.cuda.synchronize()
    return systems


def make_cov_systems(n, m, count, dev):
    """The covariance workload: A_ij = exp(-|p_i - p_j|_2 / 0.1) + 1e-3 delta_ij
    over n points uniform in the unit cube (seed 0), m N(0,1) right-hand
    sides (seed 100); `count` copies of (None, A, B) sharing A, one per
    precision compared."""
    import numpy as np
    import torch
    import workloads as W
    A, _ = W.exp_kernel_cov(n, ell=0.1, nugget=1e-3, seed=0, dim=3, device=dev)
    B = torch.from_numpy(np.ascontiguousarray(W.gaussian_rhs(n, m, 100).T)).to(dev).t()
    torch.cuda.synchronize()
    return [(None, A, B) for _ in range(count)]


def forward_errors(A_dev, X_gpu, lam, V, B, lapack=True):
    """Normwise forward errors max_c ||x_c - x*_c||_inf / ||x*_c||_inf of the
    GPU solution and (lapack) of LAPACK's float64 Cholesky solve of the same
    assembled matrix on the host, both against the exact solution x* of the
    prescribed spectrum (Q^T B by reflections, divided by lam, Q by
    reflections: accurate to roundoff whatever kappa is)."""
    import numpy as np
    import oracle
    Xs = oracle.spectral_solve(V, lam, B)
    den = np.max(np.abs(Xs), axis=0)
    fe = lambda X: float(np.max(np.max(np.abs(X - Xs), axis=0) / den))
    out = {"fwd_err": fe(X_gpu)}
    if lapack:
        import scipy.linalg as sl
        t0 = time.perf_counter()
        Ah = A_dev.cpu().numpy()
        Xl = sl.cho_solve(sl.cho_factor(Ah, lower=True, check_finite=False), B, check_finite=False)
        out["fwd_err_lapack"] = fe(Xl)
        out["lapack_s"] = time.perf_counter() - t0
    return out


def timed_repeats(fn, reps, nvml, stream):
    """One untimed call, then `reps` calls each bracketed by CUDA events on
    `stream`, inside one NVML energy window: (median ms, J per call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    times = []
    e0 = nvml.energy_mj() if nvml.ok else None
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    e1 = nvml.energy_mj() if nvml.ok else None
    j = (e1 - e0) / 1e3 / reps if e0 is not None and e1 is not None else None
    return statistics.median(times), j, sum(times) / 1e3


def idle_power(nvml, seconds=1.0):
    """Mean GPU power with nothing running (NVML), the baseline of net energy."""
    if not nvml.ok:
        return None
    vals = []
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end:
        v = nvml.power_w()
        if v is not None:
            vals.append(v)
        time.sleep(0.05)
    return statistics.mean(vals) if vals else None


FACTOR_FLAGS = {"flags": None}  # spd_factor flags of every benchmark solve (set from --shift)


def solve_one(spd, h, A, B, X, prec, opts, kappa):
    flags = FACTOR_FLAGS["flags"] if FACTOR_FLAGS["flags"] is not None else spd.SPD_SCALE_DIAG
    st, F, frep = spd.spd_factor(h, A, prec, flags)
    if st != spd.SPD_OK:
        raise RuntimeError(f"spd_factor({prec}, kappa={kappa}): {spd.spd_last_error_string(h)}")
    st, rep = spd.spd_solve_ir(h, F, A, B, X, opts)
    spd.spd_factor_destroy(F)
    if st != spd.SPD_OK:
        raise RuntimeError(f"spd_solve_ir kappa={kappa}: {spd.spd_last_error_string(h)}")
    return frep, rep


def run_step(spd, h, systems, precs, X, opts):
    """The systems one after another on one handle."""
    return [solve_one(spd, h, A, B, X, p, opts, k) for (k, A, B), p in zip(systems, precs)]


class Lanes:
    """Independent systems solved concurrently: one handle, stream, solution
    buffer and host thread per lane (the library calls release the GIL).  The
    latency-bound factorisation of one system overlaps the residuals and
    sweeps of another."""

    def __init__(self, spd, count, n, m, dev):
        import torch
        self.spd = spd
        # high priority: each solve's critical chain (rank-128 update, leaf,
        # panel, sweeps, residual) goes ahead of the bulk look-ahead updates,
        # which the library issues on a second stream of default priority
        self.streams = [torch.cuda.Stream(device=dev, priority=-1) for _ in range(count)]
        self.handles = [spd.spd_create(s) for s in self.streams]
        self.X = [torch.zeros(m, n, dtype=torch.float64, device=dev).t() for _ in range(count)]

    def run(self, systems, precs, opts, steps):
        """steps x len(systems) solves, taken from one shared queue (solve q
        is system q mod len(systems)): a lane that finishes takes the next
        solve, so cheap systems do not leave a lane idle while an expensive
        one runs.  Returns the report of each system's last solve."""
        import threading
        out = [None] * len(systems)
        err = []
        total = steps * len(systems)
        self.last_lane = [None] * len(systems)  # the lane (and X buffer) of each system's last solve
        nxt = [0]
        lock = threading.Lock()

        def work(lane):
            try:
                while True:
                    with lock:
                        q = nxt[0]
                        nxt[0] += 1
                    if q >= total or err:
                        return
                    i = q % len(systems)
                    k, A, B = systems[i]
                    out[i] = solve_one(self.spd, self.handles[lane], A, B, self.X[lane], precs[i], opts, k)
                    self.last_lane[i] = lane
            except Exception as e:  # noqa: BLE001 -- re-raised on the main thread
                err.append(e)

        th = [threading.Thread(target=work, args=(j,)) for j in range(len(self.handles))]
        for x in th:
            x.start()
        for x in th:
            x.join()
        if err:
            raise err[0]
        return out

    def fork(self, main_stream):
        """Make every lane stream wait for work queued so far on main_stream."""
        import torch
        ev = torch.cuda.Event()
        ev.record(main_stream)
        for s in self.streams:
            s.wait_event(ev)

    def join(self, main_stream):
        import torch
        for s in self.streams:
            ev = torch.cuda.Event()
            ev.record(s)
            main_stream.wait_event(ev)

    def destroy(self):
        for h in self.handles:
            self.spd.spd_destroy(h)


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
            "extrapolated": True,
            "sample": f"extrapolated: one float64 oracle solve (Cholesky + substitution) at n={ns}, m={m}, "
                      f"kappa=1e2 took {t:.2f} s; scaled by (n/{ns})^3 to n={n_full}"}


# FP32 instruction issue rate of the part: 152 SMs x 128 lanes x 2.07 GHz
FP32_OPS_PEAK_T = 152 * 2.07e9 * 128 / 1e12
# float32 instructions per multiply-add of the float32-pair residual
# (1 FMUL, 3 FFMA, 8 FADD: product, exact error, cross terms, TwoSum, pair)
DF32_OPS_PER_MADD = 12


# DRAM bytes (read + write, ncu) of a phase's launches, measured on a smaller
# case of the same kernels.  "solve": one forward + backward pair of the
# super-block sweeps at n = 8192, m = 16 moved 655 GB/s x 215 us + 586 GB/s x
# 240 us (DRAM throughput x duration of each launch); the sweeps stream the
# factor once each, so the bytes scale with n^2.  A phase in
# MEASURED_TRAFFIC_RATIO reports that ratio of DRAM bytes to algorithmic bytes
# (over a capture of its kernels) times its algorithmic bytes per launch.
MEASURED_TRAFFIC = {
    "solve": ((542379520 + 7653376 + 542446080 + 7765760) / 16384 ** 2,
              "ncu dram__bytes_read.sum + dram__bytes_write.sum of one forward + backward super-block sweep "
              "pair at n = 16384, m = 16 (two-phase kernel), per n^2"),
}
# FP32 rate of one SM: a one-CTA kernel's ceiling
FP32_SM_PEAK_TFLOPS = 128 * 2 * 2.07e9 / 1e12
MEASURED_TRAFFIC_RATIO = {
    # one stream-K bulk update of an n = 8192 FP32 factorisation (block
    # columns 32-33: M = 4096, N = 256, K = 3968, 152 CTAs): 99.76 MB read +
    # 3.28 MB written against 105.6 MB algorithmic (C read and written once,
    # three bf16 slices of each operand row once)
    "trailing_x3": ((99757568 + 3281152) / (8.0 * (256 * 4096 - 0.5 * 256 * 255) + 6.0 * 3968 * 4096),
                    "ncu DRAM bytes / algorithmic bytes of one stream-K FP32 bulk update at n = 8192, times this "
                    "phase's algorithmic bytes per launch"),
}


def phase_roofline(dom, ph, per_kappa, n=None):
    """Roofline of one phase (kernel family): achieved = its algorithmic work
    / its summed event time, against the peak of the unit that bounds it."""
    peaks, src = load_peaks()
    bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    bf16_burst = peaks["bf16_tflops"]
    sec = ph["ms"] * 1e-3
    low = sorted({k["prec_used"] for k in per_kappa} & set(TENSOR_RATIO))
    if dom == "trailing" and low:
        ratio = min(TENSOR_RATIO[p] for p in low)
        r = {"bound": "tensor", "unit": "TFLOP/s", "achieved": ph["flops"] / sec / 1e12, "peak": bf16_burst * ratio,
             "peak_source": f"{src} bf16 burst x nominal {'/'.join(low)} ratio {ratio} (kernels timed alone)",
             "frac_of_sustained": ph["flops"] / sec / 1e12 / (bf16 * ratio)}
    elif dom in ("trailing_x3", "trailing_last") and ph["flops"]:
        x3 = dom == "trailing_x3" or (low and low == ["fp32"])
        div = 6 if x3 else 1
        r = {"bound": "tensor", "unit": "TFLOP/s", "achieved": ph["flops"] / sec / 1e12, "peak": bf16_burst / div,
             "peak_source": f"{src} bf16 burst" + (" / 6 bf16 slice products per float32 product" if x3 else "")
                            + " (kernels timed alone)",
             "frac_of_sustained": ph["flops"] / sec / 1e12 / (bf16 / div)}
    elif dom == "resid":
        r = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / sec / 1e12, "peak": FP64_PEAK_TFLOPS,
             "peak_source": "nominal FP64 1.25 TFLOP/s of the part"}
    elif dom == "resid_df32":
        r = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / 2 * DF32_OPS_PER_MADD / sec / 1e12,
             "peak": FP32_OPS_PEAK_T,
             "peak_source": "float32 instructions/s: 152 SMs x 128 lanes x 2.07 GHz (one op per instruction)"}
    elif dom == "resid_tc":
        r = {"bound": "hbm", "unit": "GB/s", "achieved": ph["bytes"] / sec / 1e9, "peak": peaks["hbm_gbs"],
             "peak_source": f"{src} copy bandwidth (the digit planes stream from HBM)"}
    elif dom == "leaf":  # one CTA per 128 x 128 diagonal block, on the critical path
        r = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / sec / 1e12, "peak": FP32_SM_PEAK_TFLOPS,
             "peak_source": "one SM's 128 FP32 lanes x 2 x 2.07 GHz (each leaf is one CTA on one SM by design; "
                            "the concurrent lanes' work fills the other SMs)",
             "frac_of_gpu": ph["flops"] / sec / 1e12 / FP32_SIMT_PEAK_TFLOPS}
    elif dom in ("trailing", "panel", "inverses"):
        r = {"bound": "alu", "unit": "TFLOP/s", "achieved": ph["flops"] / sec / 1e12, "peak": FP32_SIMT_PEAK_TFLOPS,
             "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    else:
        r = {"bound": "hbm", "unit": "GB/s", "achieved": ph["bytes"] / sec / 1e9, "peak": peaks["hbm_gbs"],
             "peak_source": f"{src} copy bandwidth"}
    work = ph["flops"] if r["unit"] == "TFLOP/s" else ph["bytes"]
    if dom == "resid_df32":
        work = ph["flops"] / 2 * DF32_OPS_PER_MADD
    r.update({"frac": r["achieved"] / r["peak"], "kernel_phase": dom, "launches": ph["launches"],
              "avg_launch_ms": ph["ms"] / max(ph["launches"], 1),
              "traffic": (MEASURED_TRAFFIC[dom][0] * n * n if (dom in MEASURED_TRAFFIC and n)
                          else MEASURED_TRAFFIC_RATIO[dom][0] * ph["bytes"] / max(ph["launches"], 1)
                          if dom in MEASURED_TRAFFIC_RATIO else None),
              "traffic_source": (MEASURED_TRAFFIC[dom][1] if (dom in MEASURED_TRAFFIC and n)
                                 else MEASURED_TRAFFIC_RATIO[dom][1] if dom in MEASURED_TRAFFIC_RATIO else None),
              "algorithmic_per_launch": work / max(ph["launches"], 1)})
    return r


def roofline(phases, per_kappa, n=None):
    """Roofline of the phase that took the most device time, and of every
    phase that took at least 1 % of it (key "phases")."""
    dom = max(phases, key=lambda p: phases[p]["ms"])
    r = phase_roofline(dom, phases[dom], per_kappa, n)
    r["phases"] = {p: {k: v for k, v in phase_roofline(p, ph, per_kappa, n).items()
                       if k in ("bound", "unit", "achieved", "peak", "frac", "launches", "avg_launch_ms")}
                   for p, ph in phases.items() if ph["ms"] >= 0.01 * phases[dom]["ms"] and ph["launches"]}
    return r


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


def batched_leg(args):
    """Batched workload: 4096 systems, n_i ~ U{32..512}, A_i = G G^T / n_i +
    0.05 I, one N(0,1) right-hand side each, in one persistent graph launch.
    Matrices are drawn on the GPU (torch generator seeded 1000 + i; sizes
    from the seeded host stream)."""
    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd
    import workloads as W
    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    sizes = W.batched_sizes(args.count)
    As, bs, xs = [], [], []
    for i, n in enumerate(sizes):
        g = torch.Generator(device=dev)
        g.manual_seed(1000 + i)
        G = torch.randn((int(n), int(n)), dtype=torch.float64, device=dev, generator=g)
        A = G @ G.T / float(n)
        A = 0.5 * (A + A.T)
        A.diagonal().add_(0.05)
        As.append(A.contiguous())
        bs.append(torch.randn(int(n), dtype=torch.float64, device=dev, generator=g))
        xs.append(torch.zeros(int(n), dtype=torch.float64, device=dev))
    torch.cuda.synchronize()
    st, plan = spd.spd_batch_create(h, As, bs, xs)
    assert st == spd.SPD_OK, spd.spd_last_error_string(h)
    out = {"leg": "batched", "metric": "batched FP64-accurate SPD solves/s (one persistent launch)", "unit": "systems/s",
           "config": {"workload": f"batched: {args.count} systems, n ~ U{{32..512}}, A = G G^T/n + 0.05 I, 1 RHS",
                      "sum_n2": int(np.sum(sizes.astype(np.int64) ** 2)),
                      "sum_n3_over_3": float(np.sum(sizes.astype(np.float64) ** 3) / 3)}}
    sum8n2 = 8.0 * float(np.sum(sizes.astype(np.float64) ** 2))
    peaks, _ = load_peaks()
    for method, prec in [("chol_ir", "fp32"), ("chol_ir", "bf16"), ("pcg_jacobi", "fp64")]:
        st, rep, sts, be, it = spd.spd_batch_solve(plan, method, prec, count=len(sizes))  # warm-up (+ autotune)
        assert st == spd.SPD_OK, spd.spd_last_error_string(h)
        steps = max(1, args.steps if method == "chol_ir" else 1)
        ms = []
        for _ in range(steps):
            st, rep, sts, be, it = spd.spd_batch_solve(plan, method, prec, count=len(sizes))
            ms.append(rep.time_ms)
        t = float(np.median(ms))
        iters = float(np.mean(it))
        passes = 1.0 + iters if method == "chol_ir" else iters + 2.0   # float64 passes over every A
        fp64_flops = 2.0 * float(np.sum(sizes.astype(np.float64) ** 2)) * passes
        hbm = sum8n2 * passes / (t * 1e-3) / 1e9
        info = spd.spd_batch_info(plan, method)
        out[f"{method}_{prec}"] = {
            "value": len(sizes) / (t * 1e-3), "ms_per_launch": t, "max_berr": float(np.max(be)),
            "mean_iters": iters, "all_ok": bool(np.all(sts == 0)), "threads_per_cta": info["threads_per_cta"],
            "autotune_ms": info["tune_ms"],
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": fp64_flops / (t * 1e-3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "frac": fp64_flops / (t * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"],
                         "note": "float64 residual flops (2 n^2 per pass) and A bytes (8 n^2 per pass)"}}
    # the plain baseline: float64 Cholesky + solve per system, a sample of 128 systems scaled to the batch
    rng_ = np.random.default_rng(0)
    idx = rng_.choice(len(sizes), size=min(128, len(sizes)), replace=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in idx:
        stt, F, _ = spd.spd_factor(h, As[i], "fp64")
        X = torch.zeros((1, int(sizes[i])), dtype=torch.float64, device=dev).t()
        spd.spd_solve_ir(h, F, As[i], bs[i][:, None], X)
        spd.spd_factor_destroy(F)
    torch.cuda.synchronize()
    tl = time.perf_counter() - t0
    scale = float(np.sum(sizes.astype(np.float64) ** 3)) / float(np.sum(sizes[idx].astype(np.float64) ** 3))
    out["fp64_per_system_loop"] = {"value": len(sizes) / (tl * scale), "unit": "systems/s",
                                   "sample": f"{len(idx)} systems timed, scaled by sum n^3"}
    spd.spd_batch_destroy(plan)
    spd.spd_destroy(h)
    print(json.dumps(out), flush=True)
    return 0


def cg_leg(args):
    """CG (Algorithm 2, nested reading) on the paper's model covariance of
    Section 4: A(i,j) = 1/|i-j|^d off the diagonal, 1 + sqrt(i) on it (i
    1-based), d in {1, 2, 4}; 1 and 32 right-hand sides U[0, 1] (seed 0);
    stop at ||r||_2 <= 1e-5 as in Table 1; float32 matrix products, float64
    outer residual.  Per case: solves/s (library device time), the low and
    high iteration counts, and the matrix products' HBM rate (the bytes of
    A~ one product reads: 4 n^2 for the float32 copy on the CUDA cores, 6 n^2
    for its three bf16 slice planes on the tensor cores, which the library
    takes for m >= 8 unless --mv-cores says otherwise) against the measured
    copy bandwidth."""
    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd
    import workloads as W
    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    n = args.n_cg
    peaks, src = load_peaks()
    idx = torch.arange(n, dtype=torch.float64, device=dev)
    A = torch.empty((n, n), dtype=torch.float64, device=dev)
    base = {"tol": 1e-5, "crit": "abs2", "eta": 0.0, "maxit_inner": 5000, "matvec_cores": args.mv_cores}
    nvml = Nvml(torch.cuda.current_device())
    out = {"leg": "cg", "metric": "CG solves/s (Algorithm 2, float32 products, float64 outer residual)",
           "unit": "solves/s", "config": {"workload": f"model covariance (Section 4), n={n}, d in (1, 2, 4), "
                                                      "m in (1, 32), ||r||_2 <= 1e-5; dense and banded "
                                                      "(half-width 16, Section 4.1) inner products", "n": n}}
    for d in (1, 2, 4):
        for r0 in range(0, n, 4096):  # assembled in row blocks on the device (untimed)
            blk = A[r0:r0 + 4096]
            torch.sub(idx[r0:r0 + 4096, None], idx[None, :], out=blk)
            blk.abs_().clamp_min_(1.0).pow_(d).reciprocal_()
        A.diagonal().copy_(1.0 + torch.sqrt(idx + 1.0))
        for m in (1, 32):
            B = torch.from_numpy(np.ascontiguousarray(W.uniform_rhs(n, m, 0).T)).to(dev).t()
            X = torch.zeros(m, n, dtype=torch.float64, device=dev).t()
            for kind, opts in (("dense", base), ("band16", dict(base, band=16))):
                st, rep = spd.spd_cg(h, A, B, X, "fp32", opts=opts)  # warm-up
                if st != spd.SPD_OK:
                    raise RuntimeError(f"spd_cg d={d} m={m} {kind}: {spd.spd_last_error_string(h)}")
                ms = []
                spd.spd_profile_enable(h, True)
                torch.cuda.synchronize()
                e0 = nvml.energy_mj() if nvml.ok else None
                for _ in range(max(1, args.steps)):
                    X.zero_()
                    st, rep = spd.spd_cg(h, A, B, X, "fp32", opts=opts)
                    if st != spd.SPD_OK:
                        raise RuntimeError(f"spd_cg d={d} m={m} {kind}: {spd.spd_last_error_string(h)}")
                    ms.append(rep.time_ms)
                torch.cuda.synchronize()
                e1 = nvml.energy_mj() if nvml.ok else None
                mv = spd.spd_profile_read(h, "matvec")
                spd.spd_profile_enable(h, False)
                t = float(np.median(ms))
                gbs = mv["bytes"] / (mv["ms"] * 1e-3) / 1e9 if mv["ms"] > 0 else None
                out[f"d{d}_m{m}_{kind}"] = {
                    "value": 1e3 / t, "ms_per_solve": t, "iters_low": rep.iters_low, "iters_high": rep.iters_high,
                    "rel_resid": rep.rel_resid,
                    "j_per_solve": (e1 - e0) / 1e3 / len(ms) if e0 is not None and e1 is not None else None,
                    "matvec": {"launches": mv["launches"], "avg_launch_ms": mv["ms"] / max(mv["launches"], 1),
                               "share_of_solve": mv["ms"] / (t * len(ms)),
                               "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": gbs,
                                            "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                                            "peak_source": f"{src} copy bandwidth; float32 entries read per product"}}}
    spd.spd_destroy(h)
    print(json.dumps(out), flush=True)
    return 0


class PowerSampler:
    """NVML power samples (every 20 ms) on a background thread: the mean and
    its standard error over a measured window, as Table 1 reports them."""

    def __init__(self, nvml):
        self.nvml = nvml
        self.vals = []
        self.stop_flag = False
        self.th = None

    def __enter__(self):
        import threading
        self.vals, self.stop_flag = [], False

        def run():
            while not self.stop_flag:
                v = self.nvml.power_w() if self.nvml.ok else None
                if v is not None:
                    self.vals.append(v)
                time.sleep(0.02)

        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()
        return self

    def __exit__(self, *exc):
        self.stop_flag = True
        self.th.join()

    def stats(self):
        if len(self.vals) < 2:
            return None, None
        mean = statistics.mean(self.vals)
        return mean, statistics.stdev(self.vals) / math.sqrt(len(self.vals))


def table1_leg(args):
    """The paper's Table 1 (Section 4.1) on this GPU: the model covariance
    matrix of Section 4 (A(i,j) = 1/|i-j|^d off the diagonal, 1 + sqrt(i) on
    it, i 1-based), n = args.n_cg (70000 in the paper), d in {1, 2, 4};
    right-hand sides U[0,1] (seed 0), stop at ||r||_2 < 1e-5 as printed.
    Rows: Cholesky-IR with 32 right-hand sides (float32 factor, float64-
    accurate residual), CG with 1 and 32 (float32 products, float64-accurate
    outer residual), and CG whose inner products use the banded matrix
    (bandwidth 33).  The residual arithmetic is --resid when given, else
    the library's automatic choice: float64 fused multiply-adds for one
    right-hand side, exact products of bf16 digits on the tensor cores for
    32 (float64 fused multiply-adds are then bound by the FP64 rate).
    Per
    row: low/high iterations, seconds (device time of the library calls,
    repeated to fill at least one second), average power and its standard
    error (NVML samples), energy, and the paper's GFlops convention (CG:
    2 n^2 (low + high) m; banded: high iterations at 2 n^2, low ones at
    2 * 33 * n, per right-hand side; Cholesky: n^3 / 3) and GFlops/W.  The
    paper's numbers (IBM PS702, two POWER7) are printed beside each row."""
    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd
    import workloads as W
    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    n = args.n_cg
    nvml = Nvml(torch.cuda.current_device())
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                                       "table1_n70000.json")))
    paper = {(r[0], r[1], r[2]): dict(zip(gold["columns"], r)) for r in gold["rows"]}
    idx = torch.arange(n, dtype=torch.float64, device=dev)
    A = torch.empty((n, n), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    idle_w = idle_power(nvml, 2.0)
    crit = {"tol": 1e-5, "crit": "abs2"}
    # the leg's residual: the run's --resid when given, else float64 for one
    # right-hand side and the tensor-core residual for 32
    resid = args.resid if args.resid_given else "auto"
    rows = []
    for d in (1, 2, 4):
        for r0 in range(0, n, 4096):  # assembled in row blocks on the device (untimed, as in the paper)
            blk = A[r0:r0 + 4096]
            torch.sub(idx[r0:r0 + 4096, None], idx[None, :], out=blk)
            blk.abs_().clamp_min_(1.0).pow_(d).reciprocal_()
        A.diagonal().copy_(1.0 + torch.sqrt(idx + 1.0))
        for method, m in (("cholesky", 32), ("cg", 1), ("cg", 32), ("banded_cg", 1), ("banded_cg", 32)):
            B = torch.from_numpy(np.ascontiguousarray(W.uniform_rhs(n, m, 0).T)).to(dev).t()
            X = torch.zeros(m, n, dtype=torch.float64, device=dev).t()

            def run():
                if method == "cholesky":
                    st, F, fr = spd.spd_factor(h, A, "fp32")
                    if st != spd.SPD_OK:
                        raise RuntimeError(f"table1 factor d={d}: {spd.spd_last_error_string(h)}")
                    # the paper's rule: stop as soon as the tolerance holds (no polish sweep)
                    st, r = spd.spd_solve_ir(h, F, A, B, X, dict(crit, resid=resid, polish=0))
                    spd.spd_factor_destroy(F)
                    ms = fr.time_ms + r.time_ms
                else:
                    opts = dict(crit, eta=0.0, maxit_inner=20000, matvec_cores=args.mv_cores, resid=resid,
                                **({"band": 16} if method == "banded_cg" else {}))
                    st, r = spd.spd_cg(h, A, B, X, "fp32", opts=opts)
                    ms = r.time_ms
                if st != spd.SPD_OK:
                    raise RuntimeError(f"table1 {method} d={d} m={m}: {spd.spd_last_error_string(h)}")
                return ms, r

            run()  # warm-up (workspace, conversions)
            torch.cuda.synchronize()
            times, last = [], None
            e0 = nvml.energy_mj() if nvml.ok else None
            with PowerSampler(nvml) as ps:
                while not times or (sum(times) < 1000.0 and len(times) < 50):
                    X.zero_()
                    t, last = run()
                    times.append(t)
                torch.cuda.synchronize()
            e1 = nvml.energy_mj() if nvml.ok else None
            sec = statistics.median(times) / 1e3
            low, high = last.iters_low, last.iters_high
            if method == "cholesky":
                flops = n ** 3 / 3.0
            elif method == "cg":
                flops = 2.0 * n * n * (low + high) * m
            else:
                flops = (2.0 * n * n * high + 2.0 * 33 * n * low) * m
            pw, se = ps.stats()
            j = (e1 - e0) / 1e3 / len(times) if e0 is not None and e1 is not None else None
            row = {"method": method, "d": d, "rhs": m, "iters_low": low, "iters_high": high, "time_s": sec,
                   "avg_power_w": pw, "power_std_err_w": se, "energy_j": j,
                   "energy_j_net": (j - idle_w * sec) if (j is not None and idle_w is not None) else None,
                   "gflops": flops / sec / 1e9, "gflops_per_w": (flops / sec / 1e9 / pw) if pw else None,
                   "rel_resid_max": last.rel_resid, "repeats": len(times),
                   "paper": {k: paper[(method, d, m)][k] for k in ("iters_low", "iters_high", "time_s",
                                                                    "avg_power_w", "energy_kj", "gflops",
                                                                    "gflops_per_w")}}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del B, X
    spd.spd_destroy(h)
    out = {"leg": "table1", "metric": "Table 1 (Section 4.1): time, power and energy per row on one GB300",
           "config": {"workload": f"model covariance (Section 4), n={n}, d in (1, 2, 4), right-hand sides U[0,1], "
                                  "||r||_2 < 1e-5", "n": n, "idle_w": idle_w}, "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


def learned_leg(args):
    """Learned preconditioner on the Matern-3/2 family (n points uniform in the
    unit square, ell ~ U[0.02, 0.5], nugget ~ logU[1e-4, 1e-1]): train on
    seeds 0.., test on held-out seeds 100000..; PCG iterations and time with
    the learned M against Jacobi-PCG and float32 Cholesky-IR."""
    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd
    import workloads as W
    from paper_1405_4644_gb300 import learned as trainer
    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    n = args.n_learned
    st, net = spd.spd_mlp_create(h, 256, 11, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = trainer.train(h, net, n, range(args.train_systems), W, probes=8, lr=2e-3, wsup=0.1, use_factor=True)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {"jacobi": [], "learned": [], "chol_ir": []}
    opts = {"tol": 1e-14, "crit": "berr", "eta": 1e-12, "maxit_inner": 20000}
    for seed in range(100000, 100000 + args.test_systems):
        A, coords, ell, nug = trainer.make_system(n, seed, dev, W)
        b = torch.from_numpy(W.gaussian_rhs(n, 1, seed)).to(dev)
        X = torch.zeros((1, n), dtype=torch.float64, device=dev).t()
        st, rep = spd.spd_cg(h, A, b, X, "fp64", "jacobi", opts=opts)
        res["jacobi"].append((rep.iters_low, rep.time_ms, rep.berr, st))
        F = trainer.features(h, A, coords, ell, nug)
        tb0 = time.perf_counter()
        st, P = spd.spd_lowrank_build(net, A, F)
        torch.cuda.synchronize()
        tb = 1e3 * (time.perf_counter() - tb0)
        X.zero_()
        st, rep = spd.spd_solve_learned(h, P, A, b, X, opts)
        spd.spd_lowrank_destroy(P)
        res["learned"].append((rep.iters_low, rep.time_ms + tb, rep.berr, rep.fell_back))
        st, Fc, fr = spd.spd_factor(h, A, "fp32")
        X.zero_()
        st, rep = spd.spd_solve_ir(h, Fc, A, b, X)
        spd.spd_factor_destroy(Fc)
        res["chol_ir"].append((rep.iters_low, rep.time_ms + fr.time_ms, rep.berr, st))
    spd.spd_mlp_destroy(net)
    spd.spd_destroy(h)

    def summ(rows):
        a = np.array([r[:3] for r in rows], dtype=np.float64)
        return {"median_iters": float(np.median(a[:, 0])), "mean_ms": float(np.mean(a[:, 1])),
                "median_ms": float(np.median(a[:, 1])), "max_berr": float(np.max(a[:, 2]))}
    out = {"leg": "learned", "metric": "PCG iterations and ms per FP64-accurate solve, learned vs Jacobi",
           "config": {"workload": f"Matern-3/2 family, n={n}, {args.train_systems} training systems, "
                                  f"{args.test_systems} held-out", "n": n},
           "train": {"seconds": t_train, "systems_per_s": args.train_systems / t_train,
                     "loss_first10": float(np.mean(hist[:10])), "loss_last10": float(np.mean(hist[-10:]))},
           "jacobi_pcg": summ(res["jacobi"]), "learned_pcg": summ(res["learned"]),
           "learned_fallbacks": int(sum(r[3] for r in res["learned"])), "chol_ir_fp32": summ(res["chol_ir"]),
           "iteration_gain_median": float(np.median([j[0] / max(l[0], 1) for j, l in zip(res["jacobi"],
                                                                                       res["learned"])])),
           # per held-out system: Jacobi-PCG time / learned PCG time (the learned
           # time includes building M from the network's output)
           "time_gain_median": float(np.median([j[1] / max(l[1], 1e-9) for j, l in zip(res["jacobi"],
                                                                                    res["learned"])])),
           "learned_faster_systems": int(sum(l[1] < j[1] for j, l in zip(res["jacobi"], res["learned"])))}
    print(json.dumps(out), flush=True)
    return 0


def case_leg(args):
    """One kernel family at a time, for profilers (each case repeats its call
    so that a profiler can skip the first one); seeded synthetic inputs,
    nothing checked beyond the status codes.  With --phases the library's
    per-phase records (launches, event time, algorithmic flops and bytes,
    summed over the repetitions) are printed, for comparing a profiler's DRAM
    bytes with the algorithmic bytes.
      gemm        tcgen05 update C -= A B^T, BF16 operands, M = N = K = n
      resid_fp64  float64 residual, n x n, m right-hand sides
      resid_tc    tensor-core residual (digit planes and products)
      sweeps      triangular sweeps of an FP16 factor, m right-hand sides
                  (super-block sweeps; sweeps_block: the 128-block sweeps)
      convert     scale + convert and the whole FP32 factorisation
      factor      the factorisation in --precs (look-ahead schedule)
      factor_serial  the same on one stream (every kernel alone, for phase rates)
      cg          one Algorithm 2 solve on the model covariance (d = 2), m
                  right-hand sides, Table 1's rule (tensor-core products for m >= 8)"""
    import torch
    import paper_1405_4644_gb300 as spd
    import workloads as W

    dev = torch.device("cuda", 0)
    h = spd.spd_create(torch.cuda.current_stream())
    n, m = args.n, args.m
    if args.phases:
        spd.spd_profile_enable(h, True)

    def ok(st):
        if st != spd.SPD_OK:
            raise RuntimeError(spd.spd_last_error_string(h))

    g = torch.Generator(device=dev).manual_seed(0)
    if args.case == "gemm":
        A = torch.rand(n, n, device=dev, generator=g) - 0.5
        C = torch.zeros(n, n, device=dev)
        for _ in range(args.reps):
            ok(spd.spd_gemm_update(h, "bf16", A, A, C))
    elif args.case != "cg":
        if args.case == "resid_fp64":
            A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
            A = A + A.T
        else:
            A, _, _ = W.householder_spectrum(n, args.kappas[0], k=16, seed=0, device=dev)
        X = torch.randn(m, n, dtype=torch.float64, device=dev, generator=g).t()
        B = torch.randn(m, n, dtype=torch.float64, device=dev, generator=g).t()
        R = torch.zeros(m, n, dtype=torch.float64, device=dev).t()
        for _ in range(args.reps):
            if args.case == "resid_fp64":
                ok(spd.spd_residual(h, A, B, X, R))
            elif args.case == "resid_tc":
                ok(spd.spd_residual_tc(h, A, B, X, R))
            elif args.case in ("convert", "factor", "factor_serial"):
                prec = "fp32" if args.case == "convert" else args.precs.split(",")[0]
                flags = spd.SPD_SCALE_DIAG | (spd.SPD_FACTOR_SERIAL if args.case == "factor_serial" else 0)
                st, F, rep = spd.spd_factor(h, A, prec, flags)
                ok(st)
                print(f"factor {prec} n={n}: {rep.time_ms:.3f} ms")
                spd.spd_factor_destroy(F)
        if args.case in ("sweeps", "sweeps_block"):
            flags = spd.SPD_SCALE_DIAG | (spd.SPD_FACTOR_BLOCK_SWEEPS if args.case == "sweeps_block" else 0)
            st, F, _ = spd.spd_factor(h, A, "fp16", flags)
            ok(st)
            for _ in range(args.reps):
                ok(spd.spd_factor_solve(h, F, B, R))
            spd.spd_factor_destroy(F)
    if args.case == "cg":  # Algorithm 2 on the model covariance (d = 2), m right-hand sides, one solve
        idx = torch.arange(n, dtype=torch.float64, device=dev)
        Ac = (idx[:, None] - idx[None, :]).abs_().clamp_min_(1.0).pow_(2).reciprocal_()
        Ac.diagonal().copy_(1.0 + torch.sqrt(idx + 1.0))
        Bc = torch.rand(m, n, dtype=torch.float64, device=dev, generator=g).t()
        Xc = torch.zeros(m, n, dtype=torch.float64, device=dev).t()
        st, rep = spd.spd_cg(h, Ac, Bc, Xc, "fp32", opts={"tol": 1e-5, "crit": "abs2", "eta": 0.0,
                                                          "maxit_inner": 5000, "resid": "auto"})
        ok(st)
        print(f"cg n={n} m={m}: {rep.time_ms:.3f} ms, {rep.iters_low}/{rep.iters_high}")
        del Ac
    torch.cuda.synchronize()
    if args.phases:
        for p in spd.PHASES:
            r = spd.spd_profile_read(h, p)
            if r["launches"]:
                print(f"phase {p}: launches {r['launches']} ms {r['ms']:.3f} flops {r['flops']:.6e} "
                      f"bytes {r['bytes']:.6e} (sum over {args.reps} repetitions)")
    spd.spd_destroy(h)
    print("ok", args.case, n, m)
    return 0


FP64_REPS = 3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--kappas", default="1e2,1e4,1e6")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "cov"],
                    help="sweep: prescribed-spectrum matrices, one per kappa; cov: the exponential-kernel "
                         "covariance matrix, one solve per precision in --precs")
    ap.add_argument("--precs", default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-fwd", action="store_true", help="skip the forward errors against the exact solution")
    ap.add_argument("--shift", action="store_true",
                    help="factor with SPD_FACTOR_SHIFT (a shifted factor when the plain one breaks down)")
    ap.add_argument("--no-lapack", action="store_true", help="forward errors without LAPACK's host solve")
    ap.add_argument("--lanes", type=int, default=3,
                    help="systems solved concurrently (one handle, stream and host thread each)")
    ap.add_argument("--resid", default="tc", choices=["fp64", "df32", "tc", "auto"],
                    help="refinement residual: float64; float32 pairs until berr < 2^-36 then float64; "
                         "exact bf16 digit products on the tensor cores; or auto (float64 for one right-hand "
                         "side, tensor cores for more; the table1 leg's default)")
    ap.add_argument("--leg", default="main", choices=["main", "batched", "learned", "cg", "table1"])
    ap.add_argument("--n-cg", type=int, default=16384)
    ap.add_argument("--mv-cores", default="auto", choices=["auto", "cuda", "tensor"],
                    help="cg and table1 legs: where the float32 products run (auto: tensor cores for m >= 8)")
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--n-learned", type=int, default=4096)
    ap.add_argument("--train-systems", type=int, default=1000)
    ap.add_argument("--test-systems", type=int, default=32)
    ap.add_argument("--case", default=None,
                    choices=["gemm", "resid_fp64", "resid_tc", "sweeps", "sweeps_block", "convert", "factor",
                             "factor_serial", "cg"],
                    help="run one kernel family on a fixed case (for profilers) and exit")
    ap.add_argument("--reps", type=int, default=2, help="--case: repetitions")
    ap.add_argument("--phases", action="store_true", help="--case: print the library's phase records")
    args = ap.parse_args()
    args.resid_given = any(a == "--resid" or a.startswith("--resid=") for a in sys.argv[1:])
    args.kappas = [float(k) for k in args.kappas.split(",")]
    precs = args.precs.split(",")
    if len(precs) == 1 and args.workload == "sweep":
        precs = precs * len(args.kappas)
    if args.impl == "reference":
        return reference_arm(args)
    if args.case:
        return case_leg(args)
    if args.leg == "batched":
        return batched_leg(args)
    if args.leg == "cg":
        return cg_leg(args)
    if args.leg == "table1":
        return table1_leg(args)
    if args.leg == "learned":
        return learned_leg(args)

    import numpy as np
    import torch
    import paper_1405_4644_gb300 as spd

    if args.shift:
        FACTOR_FLAGS["flags"] = spd.SPD_SCALE_DIAG | spd.SPD_FACTOR_SHIFT
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    affinity = bind_near_gpu(Nvml(local))
    stream = torch.cuda.current_stream()
    h = spd.spd_create(stream)
    spectra = []
    if args.workload == "cov":
        systems = make_cov_systems(args.n, args.m, len(precs), dev)
        args.no_fwd = True  # no known exact solution for this matrix
    else:
        systems = make_systems(args.n, args.m, args.kappas, dev, spectra)
    # idle baseline of the energy figures: after the input generation has
    # drained and a short pause, before any solver work
    nvml = Nvml(torch.cuda.current_device())
    torch.cuda.synchronize()
    time.sleep(1.0)
    idle_w = idle_power(nvml, 2.0)
    X = torch.zeros(args.m, args.n, dtype=torch.float64, device=dev).t()
    opts = {"tol": 1e-14, "crit": "berr", "resid": args.resid}

    lanes = Lanes(spd, args.lanes, args.n, args.m, dev) if args.lanes > 1 else None
    handles = lanes.handles if lanes else [h]

    def step_all(k):
        if lanes:
            return lanes.run(systems, precs, opts, k)
        out = []
        for _ in range(k):
            out = run_step(spd, h, systems, precs, X, opts)
        return out

    if args.warmup:
        step_all(args.warmup)
    torch.cuda.synchronize()

    smi = SmiSampler(torch.cuda.current_device())
    # no profiling in the timed region: its events would sit between the
    # programmatically dependent launches and serialise them
    launches0 = sum(spd.spd_launch_count(hh) for hh in handles)
    barrier(world)
    torch.cuda.synchronize()
    smi.start()
    e0 = nvml.energy_mj() if nvml.ok else None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    if lanes:
        lanes.fork(stream)
    reps = step_all(args.steps)
    if lanes:
        lanes.join(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    e1 = nvml.energy_mj() if nvml.ok else None
    barrier(world)
    clocks = smi.stop()
    ms = ev0.elapsed_time(ev1)
    launches = sum(spd.spd_launch_count(hh) for hh in handles) - launches0
    ms_max = max_over_ranks(ms, world)
    value = job_rate(len(systems) * args.steps, world, ms_max / 1e3)

    # e2e right after the device-resident timing, before the extra roofline
    # step and the host-side forward errors (LAPACK threads on every core)
    e2e = None
    if not args.no_e2e:
        import numpy as np
        hostA = [torch.empty((args.n, args.n), dtype=torch.float64, pin_memory=True) for _ in systems]
        hostB = [torch.empty((args.m, args.n), dtype=torch.float64, pin_memory=True) for _ in systems]
        hostX = [torch.empty((args.m, args.n), dtype=torch.float64, pin_memory=True) for _ in handles]
        for (k, A, B), ha, hb in zip(systems, hostA, hostB):
            ha.copy_(A)
            hb.copy_(B.t())
        torch.cuda.synchronize()
        e2e_steps = max(1, args.steps)
        import threading

        def host_lane(j, errs, queue):
            # solves from one shared queue, as in the device-resident timing
            hh = handles[j]
            try:
                while True:
                    with queue["lock"]:
                        q = queue["next"]
                        queue["next"] += 1
                    if q >= queue["total"] or errs:
                        return
                    i = q % len(systems)
                    st = spd.lib().spd_solve_ir_host(hh, args.n, args.m, hostA[i].data_ptr(), args.n,
                                                     hostB[i].data_ptr(), args.n, hostX[j].data_ptr(), args.n,
                                                     spd.PREC[precs[i]], spd._opts(opts),
                                                     ctypes.byref(spd.SpdReport()))
                    if st != spd.SPD_OK:
                        raise RuntimeError("e2e: " + spd.spd_last_error_string(hh))
            except Exception as e:  # noqa: BLE001 -- re-raised below
                errs.append(e)

        def host_steps(steps):
            errs = []
            queue = {"lock": threading.Lock(), "next": 0, "total": steps * len(systems)}
            th = [threading.Thread(target=host_lane, args=(j, errs, queue)) for j in range(len(handles))]
            for x in th:
                x.start()
            for x in th:
                x.join()
            if errs:
                raise errs[0]

        host_steps(1)  # untimed: the handles' device copies of A, B, X are allocated here
        # the host link's rate for one pinned copy of each system's A, alone
        # (untimed; context for the number)
        tmp = torch.empty((args.n, args.n), dtype=torch.float64, device=dev)
        h2d_each = []
        for ha in hostA:
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            tmp.copy_(ha, non_blocking=True)
            torch.cuda.synchronize()
            h2d_each.append(8.0 * args.n * args.n / (time.perf_counter() - c0) / 1e9)
        h2d_gbs = h2d_each[0]
        del tmp
        barrier(world)
        smi_e2e = SmiSampler(torch.cuda.current_device())
        smi_e2e.start()
        t0 = time.perf_counter()
        host_steps(e2e_steps)
        t = time.perf_counter() - t0
        clocks_e2e = smi_e2e.stop()
        t = max_over_ranks(t, world)
        e2e = {"value": job_rate(len(systems) * e2e_steps, world, t), "unit": UNIT,
               "h2d_bytes_per_step": len(systems) * 8 * (args.n * args.n + args.n * args.m),
               "d2h_bytes_per_step": len(systems) * 8 * args.n * args.m,
               "h2d_gbs_one_copy": h2d_gbs, "h2d_gbs_each_system": h2d_each, "clocks": clocks_e2e,
               "cpu_affinity": affinity,
               "mems_allowed": host_numa_info()}

    # dominant phase and its roofline
    per_kappa = [{"kappa": k, "prec": p, "prec_used": spd.PREC_NAME.get(fr.prec_used, fr.prec_used),
                  "cond_est": fr.cond_est, "cond_lower": fr.cond_lower, "factor_ms": fr.time_ms, "solve_ms": r.time_ms, "iters": r.iters_high,
                  "iters_low": r.iters_low, "fell_back": r.fell_back, "berr": r.berr, "shift": fr.shift}
                 for (k, _, _), p, (fr, r) in zip(systems, precs, reps)]
    if True:
        # A launch's event time under concurrency (the lanes, and the factor's
        # look-ahead stream) includes sharing the SMs, so the kernel rooflines
        # come from one more step of the same workload with every kernel
        # running alone: one lane, the factor's serial schedule (CUDA events on
        # the launching stream).
        # The same pass gives each system's solution (bit-identical to the
        # timed region's: the serial schedule computes the same factor) for
        # its forward error, computed on the host after the pass.
        spd.spd_profile_enable(h, True)
        sols = []
        for (k, A, B), p in zip(systems, precs):
            base = FACTOR_FLAGS["flags"] if FACTOR_FLAGS["flags"] is not None else spd.SPD_SCALE_DIAG
            st, F, _ = spd.spd_factor(h, A, p, base | spd.SPD_FACTOR_SERIAL)
            if st != spd.SPD_OK:
                raise RuntimeError("roofline pass: " + spd.spd_last_error_string(h))
            st, _ = spd.spd_solve_ir(h, F, A, B, X, opts)
            spd.spd_factor_destroy(F)
            sols.append(X.cpu().numpy())
        roof_phases = {p: spd.spd_profile_read(h, p) for p in spd.PHASES}
        spd.spd_profile_enable(h, False)
        if not args.no_fwd:
            for pk, (k, A, B), Xg, (lam, V, Bh) in zip(per_kappa, systems, sols, spectra):
                fe = forward_errors(A, Xg, lam, V, Bh, lapack=not args.no_lapack)
                fe["bound"] = 10.0 * k * 1e-16
                if "fwd_err_lapack" in fe:
                    fe["within_bound_of_lapack"] = fe["fwd_err"] <= fe["fwd_err_lapack"] + fe["bound"]
                pk.update(fe)
        roof_note = ("phases of one extra step of the same workload with every kernel alone (one lane, serial "
                     "factor schedule); the timed region ran concurrent lanes and the look-ahead")
    roof = roofline(roof_phases, per_kappa, args.n)
    roof["measured_on"] = roof_note
    energy = None
    if e0 is not None and e1 is not None:
        j = (e1 - e0) / 1e3
        nsol = len(systems) * args.steps
        energy = {"j_per_solve": j / nsol, "avg_power_w": j / (ms / 1e3),
                  "source": "NVML total-energy counter, gross"}
        if idle_w is not None:
            energy.update({"idle_w": idle_w, "j_per_solve_net": (j - idle_w * ms / 1e3) / nsol})
    elif clocks:
        j = clocks["avg_power_w"] * ms / 1e3
        energy = {"j_per_solve": j / (len(systems) * args.steps), "avg_power_w": clocks["avg_power_w"],
                  "source": "nvidia-smi power.draw mean x time, gross"}

    # float64 blocked Cholesky on the same GPU (the plain baseline), one system
    fp64 = None
    if not args.no_fp64:
        # float64 Cholesky of the first system (kappa = 1e2; the float64
        # factor's cost does not depend on kappa): ours (blocked, CUDA cores,
        # then refinement with float64 residuals) and cuSOLVER's through
        # torch; one untimed solve, then FP64_REPS solves in one NVML window
        kappa, A, B = systems[0]
        rep_out = []
        t_ours, j_ours, s_ours = timed_repeats(
            lambda: rep_out.append(run_step(spd, h, [systems[0]], ["fp64"], X, dict(opts, resid="fp64"))[0]),
            FP64_REPS, nvml, stream)
        fr, r = rep_out[-1]

        def cusolver():
            Lc = torch.linalg.cholesky(A)
            torch.cholesky_solve(B.contiguous(), Lc)

        t_cus, j_cus, s_cus = timed_repeats(cusolver, FP64_REPS, nvml, stream)
        ms_mixed = ms / (len(systems) * args.steps)
        fast_t = min(t_ours, t_cus)
        fp64 = {"reps": FP64_REPS, "ms_per_solve_ours": t_ours, "ms_per_solve_cusolver": t_cus,
                "timing": "median of the repeats, CUDA events; one untimed solve first",
                "berr_ours": r.berr, "speedup_time_vs_faster": fast_t / ms_mixed}
        if j_ours is not None and j_cus is not None:
            fp64.update({"j_per_solve_ours": j_ours, "j_per_solve_cusolver": j_cus,
                         "energy_window_s": [s_ours, s_cus]})
            if energy is not None:
                fp64["speedup_energy_vs_lower"] = min(j_ours, j_cus) / energy["j_per_solve"]
                if idle_w is not None:
                    net = lambda j, sec: j - idle_w * sec / FP64_REPS
                    fp64["speedup_energy_net_vs_lower"] = (min(net(j_ours, s_ours), net(j_cus, s_cus))
                                                           / energy["j_per_solve_net"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(args.n, args.m)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "mixed: " + "/".join(sorted(set(precs))) + " factor, f64 refinement",
               "data": "synthetic",
               "config": {"workload": (f"precision sweep n={args.n} m={args.m} kappa in {args.kappas}"
                                       if args.workload == "sweep" else
                                       f"covariance n={args.n} m={args.m}: exp(-|p_i-p_j|/0.1) + 1e-3 I, "
                                       f"points U[0,1]^3, one solve per precision {precs}"),
                          "n": args.n, "m": args.m, "factor_prec": precs,
                          **({"kappas": args.kappas} if args.workload == "sweep" else {}),
                          "l2": f"inputs larger than L2 ({len(systems)} x 8 n^2 bytes resident)", "tol_berr": 1e-14,
                          "lanes": args.lanes,
                          "residual": {"fp64": "float64 throughout",
                                       "df32": "float32 pairs while berr > 2^-36, float64 to finish "
                                               "(convergence only accepted on a float64 residual)",
                                       "tc": "exact products of bf16 digits on the tensor cores (ten 7-bit "
                                             "digits per entry, 55 digit products), every residual"}[args.resid]},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
               "energy": energy, "fp64_baseline": fp64, "per_kappa": per_kappa,
               "phases": {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in roof_phases.items()},
               "phases_measured_on": roof_note}
        print(json.dumps(out), flush=True)
    if lanes:
        lanes.destroy()
    spd.spd_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
