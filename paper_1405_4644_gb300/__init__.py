"""paper_1405_4644_gb300 -- Python binding of libspd (include/spd.h).

A thin ctypes layer: every function here marshals torch tensors (device
memory) or numpy arrays (host memory) into the C ABI of the same name and
returns what it returns.  All arithmetic runs in libspd's CUDA kernels; if
the library is missing or cannot load, importing ``lib()`` raises -- there is
no fallback.

Layout convention: matrices are column-major, as in the C ABI.  A symmetric
C-contiguous (n, n) tensor is already its own column-major form.  An (n, m)
right-hand-side block must have stride(0) == 1 (build it as
``torch.empty(m, n).t()`` or use ``colmajor``); its leading dimension is
stride(1).  One-dimensional vectors are taken as (n, 1).
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB as _LIB_PATH

__all__ = [
    "SPD_OK", "SPD_ERR_ARG", "SPD_ERR_NOT_SPD", "SPD_ERR_NO_CONVERGENCE", "SPD_ERR_TIMEOUT", "SPD_ERR_CUDA",
    "SPD_ERR_OOM", "SPD_ERR_UNSUPPORTED", "PREC", "SPD_SCALE_DIAG", "SpdOpts", "SpdReport", "SpdError",
    "lib", "colmajor", "spd_create", "spd_destroy", "spd_last_error_string", "spd_opts_default", "spd_factor",
    "spd_factor_destroy", "spd_factor_info", "spd_factor_copy", "spd_solve_ir", "spd_solve_ir_host", "spd_factor_solve",
    "spd_residual", "spd_residual_df32", "spd_residual_tc", "RESID", "spd_cg", "spd_profile_enable", "spd_profile_read", "PHASES", "EXPORTED", "spd_launch_count", "spd_gemm_update", "spd_residual_static", "BATCH",
    "spd_batch_create", "spd_batch_solve", "spd_batch_info", "spd_batch_destroy",
    "spd_mlp_create", "spd_mlp_destroy", "spd_mlp_params", "spd_learned_features", "spd_mlp_loss_grad",
    "spd_mlp_adam", "spd_lowrank_build", "spd_lowrank_apply", "spd_lowrank_destroy", "spd_solve_learned",
    "spd_set_wait_limit", "spd_set_memory_cap", "spd_wait_probe", "spd_batch_graph", "spd_batch_results",
    "spd_graph_launch", "spd_learned_save", "spd_learned_load",
]

SPD_OK, SPD_ERR_ARG, SPD_ERR_NOT_SPD, SPD_ERR_NO_CONVERGENCE = 0, 1, 2, 3
SPD_ERR_TIMEOUT, SPD_ERR_CUDA, SPD_ERR_OOM, SPD_ERR_UNSUPPORTED = 4, 5, 6, 7
SPD_ERR_SCRATCH = 8
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "fp16": 4, "fp8": 5, "auto": 6}
PREC_NAME = {v: k for k, v in PREC.items()}
CRIT = {"berr": 0, "rel2": 1, "abs2": 2}
PC = {"none": 0, "jacobi": 1, "factor": 2, "lowrank": 3}
RESID = {"fp64": 0, "df32": 1, "tc": 2, "auto": 3}
BATCH = {"chol_ir": 0, "pcg_jacobi": 1}
SPD_SCALE_DIAG = 1
SPD_FACTOR_CUDA_CORES = 2
SPD_FACTOR_RECURSIVE = 4
SPD_FACTOR_SERIAL = 8
SPD_FACTOR_SHIFT = 16
SPD_FACTOR_BLOCK_SWEEPS = 32
MV_CORES = {"auto": 0, "cuda": 1, "tensor": 2}

# every symbol include/spd.h declares
EXPORTED = [
    "spd_create", "spd_destroy", "spd_last_error_string", "spd_opts_default", "spd_factor", "spd_factor_destroy",
    "spd_factor_info", "spd_factor_copy", "spd_solve_ir", "spd_solve_ir_host", "spd_factor_solve", "spd_residual", "spd_residual_df32", "spd_residual_tc", "spd_cg", "spd_profile_enable",
    "spd_profile_read", "spd_launch_count", "spd_gemm_update", "spd_residual_static", "spd_batch_create", "spd_batch_solve",
    "spd_batch_info", "spd_batch_destroy", "spd_mlp_create", "spd_mlp_destroy", "spd_mlp_params",
    "spd_learned_features", "spd_mlp_loss_grad", "spd_mlp_adam", "spd_lowrank_build", "spd_lowrank_apply",
    "spd_lowrank_destroy", "spd_solve_learned", "spd_set_wait_limit", "spd_set_memory_cap", "spd_wait_probe",
    "spd_batch_graph", "spd_batch_results", "spd_graph_launch", "spd_learned_save", "spd_learned_load",
    "spd_solve_ir_async",
]


class SpdOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("crit", C.c_int), ("maxit", C.c_int), ("maxit_inner", C.c_int),
                ("eta", C.c_double), ("band", C.c_int), ("fallback", C.c_int), ("resid", C.c_int),
                ("polish", C.c_int), ("matvec_cores", C.c_int)]


class SpdReport(C.Structure):
    _fields_ = [("status", C.c_int), ("info", C.c_int), ("iters_low", C.c_int), ("iters_high", C.c_int),
                ("prec_used", C.c_int), ("fell_back", C.c_int), ("berr", C.c_double), ("rel_resid", C.c_double),
                ("time_ms", C.c_double), ("cond_est", C.c_double), ("shift", C.c_double),
                ("cond_lower", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["prec_used"] = PREC_NAME.get(d["prec_used"], d["prec_used"])
        return d


class SpdReportDev(C.Structure):
    """Host view of the device-side report of spd_solve_ir_async."""
    _fields_ = [("status", C.c_int), ("active", C.c_int), ("sweeps", C.c_int), ("stagnated", C.c_int),
                ("dev_flags", C.c_int), ("pad", C.c_int), ("berr", C.c_double), ("rel_resid", C.c_double)]


class SpdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libspd status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libspd.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise SpdError(SPD_ERR_CUDA, f"libspd.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(_LIB_PATH)
    P, I, D, U = C.c_void_p, C.c_int, C.c_double, C.c_uint
    PP = C.POINTER(C.c_void_p)
    R = C.POINTER(SpdReport)
    O = C.POINTER(SpdOpts)
    sig = {
        "spd_create": (I, [PP, P]),
        "spd_destroy": (I, [P]),
        "spd_last_error_string": (C.c_char_p, [P]),
        "spd_opts_default": (None, [O]),
        "spd_factor": (I, [P, I, P, I, I, U, PP, R]),
        "spd_factor_destroy": (I, [P]),
        "spd_factor_info": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "spd_factor_copy": (I, [P, P, I, P]),
        "spd_solve_ir": (I, [P, P, I, I, P, I, P, I, P, I, O, R]),
        "spd_solve_ir_host": (I, [P, I, I, P, I, P, I, P, I, I, O, R]),
        "spd_factor_solve": (I, [P, P, I, I, P, I, P, I]),
        "spd_residual": (I, [P, I, I, P, I, P, I, P, I, P, I, P]),
        "spd_residual_df32": (I, [P, I, I, P, I, P, I, P, I, P, I, P]),
        "spd_residual_tc": (I, [P, I, I, P, I, P, I, P, I, P, I, P]),
        "spd_cg": (I, [P, I, I, P, I, I, I, P, P, I, P, I, O, R]),
        "spd_profile_enable": (I, [P, I]),
        "spd_launch_count": (I, [P, C.POINTER(C.c_longlong)]),
        "spd_gemm_update": (I, [P, I, I, I, I, P, I, P, I, P, I, I]),
        "spd_residual_static": (I, [P, I, I, P, I, P, I, P, I, P, I, P]),
        "spd_batch_create": (I, [P, I, P, P, P, P, P, PP]),
        "spd_batch_solve": (I, [P, I, I, O, R, P, P, P]),
        "spd_batch_info": (I, [P, I, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)]),
        "spd_batch_destroy": (I, [P]),
        "spd_mlp_create": (I, [P, I, C.c_ulonglong, I, PP]),
        "spd_mlp_destroy": (I, [P]),
        "spd_mlp_params": (I, [P, P, P, P, C.POINTER(C.c_long)]),
        "spd_learned_features": (I, [P, I, P, I, P, D, D, P]),
        "spd_mlp_loss_grad": (I, [P, I, P, I, P, I, P, P, D, C.POINTER(C.c_double)]),
        "spd_mlp_adam": (I, [P, D]),
        "spd_lowrank_build": (I, [P, I, P, I, P, PP]),
        "spd_lowrank_apply": (I, [P, I, P, I, P, I]),
        "spd_lowrank_destroy": (I, [P]),
        "spd_solve_learned": (I, [P, P, I, I, P, I, P, I, P, I, O, R]),
        "spd_profile_read": (I, [P, I, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
        "spd_set_wait_limit": (I, [P, D]),
        "spd_set_memory_cap": (I, [P, C.c_size_t]),
        "spd_wait_probe": (I, [P]),
        "spd_batch_graph": (I, [P, I, I, O, PP]),
        "spd_batch_results": (I, [P, I, I, R, P, P, P]),
        "spd_graph_launch": (I, [P, P]),
        "spd_learned_save": (I, [P, C.c_char_p]),
        "spd_learned_load": (I, [P, C.c_char_p, PP]),
        "spd_solve_ir_async": (I, [P, P, I, I, P, I, P, I, P, I, O, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def colmajor(t):
    """(pointer, leading dimension, rows, cols) of a column-major matrix view."""
    import torch
    if t.dim() == 1:
        return t.data_ptr(), max(t.shape[0], 1), t.shape[0], 1
    n, m = t.shape
    if m == 1 or n == 0:
        return t.data_ptr(), max(t.stride(1) if m > 1 else n, 1), n, m
    if t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride(0) == 1)")
    return t.data_ptr(), t.stride(1), n, m


def _need_dev(t, name, dtype="float64"):
    """Reject what the kernels would misread: a host tensor, another dtype,
    or a tensor on a device other than the current one."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor on the GPU")
    want = getattr(torch, dtype)
    if t.dtype != want:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be on a CUDA device")
    if t.device.index is not None and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def _cols(t, name, n, m=None, dtype="float64"):
    """colmajor() of a device block that must have n rows (and m columns)."""
    _need_dev(t, name, dtype)
    p, ld, rows, cols = colmajor(t)
    if rows != n or (m is not None and cols != m):
        raise ValueError(f"{name} has shape ({rows}, {cols}), expected ({n}, {m if m is not None else cols})")
    return p, ld, rows, cols


def _norms(colnorms, m):
    """Pointer of the optional per-column norm buffer: 3*m float64 values."""
    if colnorms is None:
        return None
    _need_dev(colnorms, "colnorms")
    if not colnorms.is_contiguous() or colnorms.numel() < 3 * m:
        raise ValueError(f"colnorms must be contiguous with at least 3*m = {3 * m} float64 values")
    return colnorms.data_ptr()


def _sym(A, dtype="float64"):
    """Pointer and lda of a symmetric matrix given as a C- or F-contiguous tensor."""
    _need_dev(A, "A", dtype)
    n = A.shape[0]
    if A.dim() != 2 or A.shape != (n, n):
        raise ValueError("A must be square")
    if A.is_contiguous():
        return A.data_ptr(), max(A.stride(0), 1) if n > 1 else 1, n
    if A.stride(0) == 1:
        return A.data_ptr(), A.stride(1), n
    raise ValueError("A must be contiguous (row- or column-major)")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, SpdOpts):
        return C.byref(opts)
    o = spd_opts_default()
    for k, v in dict(opts).items():
        if k == "crit" and isinstance(v, str):
            v = CRIT[v]
        if k == "resid" and isinstance(v, str):
            v = RESID[v]
        if k == "matvec_cores" and isinstance(v, str):
            v = MV_CORES[v]
        setattr(o, k, v)
    return C.byref(o)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


# ---------------------------------------------------------------------------
# the C ABI, one function each
# ---------------------------------------------------------------------------
def spd_create(stream=None):
    h = C.c_void_p()
    st = lib().spd_create(C.byref(h), _stream_ptr(stream))
    if st != SPD_OK:
        raise SpdError(st, "spd_create failed")
    return h


def spd_destroy(h):
    return lib().spd_destroy(h)


def spd_last_error_string(h):
    s = lib().spd_last_error_string(h)
    return s.decode() if s else ""


def spd_opts_default():
    o = SpdOpts()
    lib().spd_opts_default(C.byref(o))
    return o


def spd_factor(h, A, prec="fp32", flags=SPD_SCALE_DIAG):
    """Returns (status, factor handle or None, SpdReport)."""
    pA, lda, n = _sym(A)
    F = C.c_void_p()
    rep = SpdReport()
    st = lib().spd_factor(h, n, pA, lda, _prec(prec), flags, C.byref(F), C.byref(rep))
    return st, (F if st == SPD_OK else None), rep


def spd_factor_destroy(F):
    return lib().spd_factor_destroy(F)


def spd_factor_info(F):
    """(n, precision code) of a factor."""
    n, prec = C.c_int(), C.c_int()
    st = lib().spd_factor_info(F, C.byref(n), C.byref(prec))
    if st != SPD_OK:
        raise SpdError(st, "spd_factor_info failed")
    return n.value, prec.value


def spd_factor_copy(F, L=None, d=None):
    """Copy the factor's rows (row-major, ld = L.shape[1]) and scaling into
    numpy arrays or torch tensors (host or device)."""
    def ptr(a):
        if a is None:
            return None
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    ldl = L.shape[1] if L is not None else 0
    return lib().spd_factor_copy(F, ptr(L), ldl, ptr(d))


def spd_solve_ir(h, F, A, B, X, opts=None):
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    rep = SpdReport()
    st = lib().spd_solve_ir(h, F, n, m, pA, lda, pB, ldb, pX, ldx, _opts(opts), C.byref(rep))
    return st, rep


def spd_solve_ir_host(h, A, B, X, prec="fp32", opts=None):
    """Host numpy buffers: A (n, n) symmetric, B and X (n, m) Fortran-ordered."""
    import numpy as np
    n = A.shape[0]
    B2 = B if B.ndim == 2 else B[:, None]
    X2 = X if X.ndim == 2 else X[:, None]
    if A.dtype != np.float64 or not (A.flags.c_contiguous or A.flags.f_contiguous):
        raise ValueError("A must be a contiguous float64 array")
    for t in (B2, X2):
        if t.dtype != np.float64 or not (t.flags.f_contiguous or (t.flags.c_contiguous and t.shape[1] == 1)):
            raise ValueError("host buffers must be float64 and column-major")
    m = B2.shape[1]
    rep = SpdReport()
    st = lib().spd_solve_ir_host(h, n, m, A.ctypes.data, n, B2.ctypes.data, B2.shape[0], X2.ctypes.data,
                                 X2.shape[0], _prec(prec), _opts(opts), C.byref(rep))
    return st, rep


def spd_factor_solve(h, F, R, Z):
    n_f, _ = spd_factor_info(F)
    pR, ldr, n, m = _cols(R, "R", n_f)
    pZ, ldz, _, _ = _cols(Z, "Z", n, m)
    return lib().spd_factor_solve(h, F, n, m, pR, ldr, pZ, ldz)


def spd_residual(h, A, B, X, R, colnorms=None):
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    pR, ldr, _, _ = _cols(R, "R", n, m)
    pc = _norms(colnorms, m)
    return lib().spd_residual(h, n, m, pA, lda, pB, ldb, pX, ldx, pR, ldr, pc)


def spd_residual_df32(h, A, B, X, R, colnorms=None):
    """R = B - A X on the float32 units with error-free transformations."""
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    pR, ldr, _, _ = _cols(R, "R", n, m)
    pc = _norms(colnorms, m)
    return lib().spd_residual_df32(h, n, m, pA, lda, pB, ldb, pX, ldx, pR, ldr, pc)


def spd_residual_tc(h, A, B, X, R, colnorms=None):
    """R = B - A X from exact bf16 digit products on the tensor cores."""
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    pR, ldr, _, _ = _cols(R, "R", n, m)
    pc = _norms(colnorms, m)
    return lib().spd_residual_tc(h, n, m, pA, lda, pB, ldb, pX, ldx, pR, ldr, pc)


def spd_cg(h, A, B, X, matvec_prec="fp32", pc="none", pc_data=None, opts=None):
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    rep = SpdReport()
    pcv = PC[pc] if isinstance(pc, str) else int(pc)
    st = lib().spd_cg(h, n, m, pA, lda, _prec(matvec_prec), pcv, pc_data, pB, ldb, pX, ldx, _opts(opts),
                      C.byref(rep))
    return st, rep


PHASES = ["convert", "leaf", "trailing", "solve", "resid", "matvec", "vector", "panel", "batch", "trailing_x3",
          "resid_df32", "resid_tc", "trailing_last", "inverses", "estimate"]


def spd_profile_enable(h, on=True):
    return lib().spd_profile_enable(h, 1 if on else 0)


def spd_profile_read(h, phase):
    """dict(launches, ms, flops, bytes) of one phase (name or spd_phase code)."""
    ph = PHASES.index(phase) if isinstance(phase, str) else int(phase)
    n = C.c_int()
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    st = lib().spd_profile_read(h, ph, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by))
    if st != SPD_OK:
        raise SpdError(st, "spd_profile_read failed")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def spd_launch_count(h):
    c = C.c_longlong()
    st = lib().spd_launch_count(h, C.byref(c))
    if st != SPD_OK:
        raise SpdError(st, "spd_launch_count failed")
    return c.value


SPD_GEMM_LOWER, SPD_GEMM_STREAM_K, SPD_GEMM_NARROW = 1, 2, 4


def spd_gemm_update(h, prec, A, B, C, lower=False, stream_k=False, narrow=False):
    """C -= round(A) round(B)^T on the tensor cores; float32 row-major device
    tensors A (M, K), B (N, K), C (M, N)."""
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        _need_dev(t, nm, "float32")
        if t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(f"{nm} must be a row-major 2-D float32 tensor")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (M, N):
        raise ValueError(f"shapes A {tuple(A.shape)}, B {tuple(B.shape)}, C {tuple(C.shape)} do not match")
    return lib().spd_gemm_update(h, _prec(prec), M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                 C.data_ptr(), C.stride(0),
                                 (SPD_GEMM_LOWER if lower else 0) | (SPD_GEMM_STREAM_K if stream_k else 0) |
                                 (SPD_GEMM_NARROW if narrow else 0))


def spd_residual_static(stream, A, B, X, R, colnorms=None):
    """R = B - A X through the allocation-free entry point (fixed scratch)."""
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    pR, ldr, _, _ = _cols(R, "R", n, m)
    pc = _norms(colnorms, m)
    return lib().spd_residual_static(_stream_ptr(stream), n, m, pA, lda, pB, ldb, pX, ldx, pR, ldr, pc)


def spd_batch_create(h, As, Bs, Xs):
    """Plan for len(As) systems: As[i] (n_i, n_i) float64 device tensors
    (symmetric), Bs[i] and Xs[i] (n_i,) float64 device tensors."""
    import numpy as np
    cnt = len(As)
    n = np.array([a.shape[0] for a in As], dtype=np.int32)
    lda = np.array([a.stride(0) if a.is_contiguous() and a.shape[0] > 1 else max(a.shape[0], 1) for a in As],
                   dtype=np.int32)
    pa = np.array([a.data_ptr() for a in As], dtype=np.uint64)
    pb = np.array([b.data_ptr() for b in Bs], dtype=np.uint64)
    px = np.array([x.data_ptr() for x in Xs], dtype=np.uint64)
    plan = C.c_void_p()
    st = lib().spd_batch_create(h, cnt, n.ctypes.data, pa.ctypes.data, lda.ctypes.data, pb.ctypes.data,
                                px.ctypes.data, C.byref(plan))
    return st, (plan if st == SPD_OK else None)


def spd_batch_solve(plan, method="chol_ir", prec="fp32", opts=None, count=None):
    """Returns (status, summary SpdReport, per-system status, berr, iters)."""
    import numpy as np
    m = BATCH[method] if isinstance(method, str) else int(method)
    rep = SpdReport()
    cnt = int(count) if count is not None else 0
    sts = np.zeros(max(cnt, 1), dtype=np.int32)
    be = np.zeros(max(cnt, 1))
    it = np.zeros(max(cnt, 1), dtype=np.int32)
    args = (sts.ctypes.data, be.ctypes.data, it.ctypes.data) if cnt else (None, None, None)
    st = lib().spd_batch_solve(plan, m, _prec(prec), _opts(opts), C.byref(rep), *args)
    return st, rep, sts[:cnt], be[:cnt], it[:cnt]


def spd_batch_info(plan, method="chol_ir"):
    m = BATCH[method] if isinstance(method, str) else int(method)
    t, c = C.c_int(), C.c_int()
    ms = (C.c_float * 2)()
    st = lib().spd_batch_info(plan, m, C.byref(t), C.byref(c), ms)
    if st != SPD_OK:
        raise SpdError(st, "spd_batch_info failed")
    return {"threads_per_cta": t.value, "ctas": c.value, "tune_ms": [ms[0], ms[1]]}


def spd_batch_destroy(plan):
    return lib().spd_batch_destroy(plan)


def _ptr(a):
    if a is None:
        return None
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


def spd_mlp_create(h, hidden=256, seed=0, bf16=True):
    net = C.c_void_p()
    st = lib().spd_mlp_create(h, int(hidden), int(seed), 1 if bf16 else 0, C.byref(net))
    return st, (net if st == SPD_OK else None)


def spd_mlp_destroy(net):
    return lib().spd_mlp_destroy(net)


def spd_mlp_params(net, out=None, inp=None, grad=None):
    """Copy parameters out/in and the last gradient out; returns the count."""
    cnt = C.c_long()
    st = lib().spd_mlp_params(net, _ptr(out), _ptr(inp), _ptr(grad), C.byref(cnt))
    if st != SPD_OK:
        raise SpdError(st, "spd_mlp_params failed")
    return cnt.value


def spd_learned_features(h, A, coords, ell, nugget, F):
    pA, lda, n = _sym(A)
    _need_dev(coords, "coords")
    _need_dev(F, "F", "float32")
    if not coords.is_contiguous() or coords.numel() < 2 * n or not F.is_contiguous() or F.numel() < 16 * n:
        raise ValueError("coords must hold n x 2 float64 and F n x 16 float32 values, both contiguous")
    return lib().spd_learned_features(h, n, pA, lda, coords.data_ptr(), float(ell), float(nugget), F.data_ptr())


def spd_mlp_loss_grad(net, A, F, Z, T=None, wsup=0.0):
    pA, lda, n = _sym(A)
    pZ, ldz, _, p = _cols(Z, "Z", n)
    _need_dev(F, "F", "float32")
    if not F.is_contiguous() or F.numel() < 16 * n:
        raise ValueError("F must hold n x 16 contiguous float32 features")
    if T is not None:
        _need_dev(T, "T")
        if not T.is_contiguous() or T.numel() < n:
            raise ValueError("T must hold n contiguous float64 values")
    if ldz != n:
        raise ValueError("probe block must have leading dimension n")
    loss = C.c_double()
    st = lib().spd_mlp_loss_grad(net, n, pA, lda, F.data_ptr(), p, pZ, _ptr(T), float(wsup), C.byref(loss))
    return st, loss.value


def spd_mlp_adam(net, lr):
    return lib().spd_mlp_adam(net, float(lr))


def spd_lowrank_build(net, A, F):
    pA, lda, n = _sym(A)
    _need_dev(F, "F", "float32")
    if not F.is_contiguous() or F.numel() < 16 * n:
        raise ValueError("F must hold n x 16 contiguous float32 features")
    P = C.c_void_p()
    st = lib().spd_lowrank_build(net, n, pA, lda, F.data_ptr(), C.byref(P))
    return st, (P if st == SPD_OK else None)


def spd_lowrank_apply(P, R, Z):
    _need_dev(R, "R")
    pR, ldr, n, m = colmajor(R)
    pZ, ldz, _, _ = _cols(Z, "Z", n, m)
    return lib().spd_lowrank_apply(P, m, pR, ldr, pZ, ldz)


def spd_lowrank_destroy(P):
    return lib().spd_lowrank_destroy(P)


def spd_solve_learned(h, P, A, B, X, opts=None):
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    rep = SpdReport()
    st = lib().spd_solve_learned(h, P, n, m, pA, lda, pB, ldb, pX, ldx, _opts(opts), C.byref(rep))
    return st, rep


def spd_set_wait_limit(h, seconds):
    """Bound of every spin-wait of h's kernels on another CTA's flag."""
    return lib().spd_set_wait_limit(h, float(seconds))


def spd_set_memory_cap(h, nbytes):
    """Cap on the device memory one call on h may request (0: none)."""
    return lib().spd_set_memory_cap(h, int(nbytes))


def spd_wait_probe(h):
    """One bounded wait on a flag nothing sets: SPD_ERR_TIMEOUT after the limit."""
    return lib().spd_wait_probe(h)


def spd_batch_graph(plan, method="chol_ir", prec="fp32", opts=None):
    """(status, graph exec handle owned by the plan) of the batched solve."""
    m = BATCH[method] if isinstance(method, str) else int(method)
    gx = C.c_void_p()
    st = lib().spd_batch_graph(plan, m, _prec(prec), _opts(opts), C.byref(gx))
    return st, (gx if st == SPD_OK else None)


def spd_batch_results(plan, method="chol_ir", prec="fp32", count=0):
    """Per-system results of the plan's last launch (after the caller synchronised)."""
    import numpy as np
    m = BATCH[method] if isinstance(method, str) else int(method)
    rep = SpdReport()
    cnt = int(count)
    sts = np.zeros(max(cnt, 1), dtype=np.int32)
    be = np.zeros(max(cnt, 1))
    it = np.zeros(max(cnt, 1), dtype=np.int32)
    args = (sts.ctypes.data, be.ctypes.data, it.ctypes.data) if cnt else (None, None, None)
    st = lib().spd_batch_results(plan, m, _prec(prec), C.byref(rep), *args)
    return st, rep, sts[:cnt], be[:cnt], it[:cnt]


def spd_graph_launch(graph_exec, stream=None):
    return lib().spd_graph_launch(graph_exec, _stream_ptr(stream))


def spd_learned_save(net, path):
    return lib().spd_learned_save(net, str(path).encode())


def spd_learned_load(h, path):
    """(status, network or None)."""
    net = C.c_void_p()
    st = lib().spd_learned_load(h, str(path).encode(), C.byref(net))
    return st, (net if st == SPD_OK else None)


def spd_report_dev_buffer(device="cuda"):
    """A device buffer for spd_solve_ir_async's report (torch uint8 tensor)."""
    import torch
    return torch.zeros(C.sizeof(SpdReportDev), dtype=torch.uint8, device=device)


def spd_report_dev_read(buf):
    """Copy a device report to the host (synchronises with the device)."""
    raw = bytes(buf.cpu().numpy().tobytes())
    return SpdReportDev.from_buffer_copy(raw)


def spd_solve_ir_async(h, F, A, B, X, rep_buf, opts=None):
    """Enqueue Algorithm 1 with its stop decision on the device (capturable);
    rep_buf from spd_report_dev_buffer()."""
    pA, lda, n = _sym(A)
    pB, ldb, _, m = _cols(B, "B", n)
    pX, ldx, _, _ = _cols(X, "X", n, m)
    _need_dev(rep_buf, "rep_buf", "uint8")
    if rep_buf.numel() < C.sizeof(SpdReportDev):
        raise ValueError("rep_buf is too small for spd_report_dev")
    return lib().spd_solve_ir_async(h, F, n, m, pA, lda, pB, ldb, pX, ldx, _opts(opts), rep_buf.data_ptr())
