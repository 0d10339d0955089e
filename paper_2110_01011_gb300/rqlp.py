"""Thin ctypes binding of librqlp.so (the C ABI declared in include/rqlp.h).

The functions named ``rqlp_*`` mirror the C entry points one to one and only
marshal arguments: torch CUDA tensors are passed as raw device pointers, the
current torch stream as the cudaStream_t. Every step of the factorisation
runs in the library's CUDA kernels; there is no CPU fallback, and loading
fails loudly when the library has not been built.

``factor`` is the convenience call: it allocates the outputs and the workspace
with torch and returns (Q, L, P, info, diag).
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

__all__ = ["load", "RqlpError", "rqlp_default_opts", "rqlp_workspace_bytes", "rqlp_factor",
           "rqlp_host_workspace_bytes", "rqlp_factor_host", "rqlp_status_string", "rqlp_version",
           "factor", "factor_host", "Opts", "PREC_FP32", "PREC_BF16X3", "STATUS", "EXPORTED"]

PREC_FP32 = 0
PREC_BF16X3 = 1
MAX_D = 256
MLP_FEATURES = 12
MLP_HIDDEN = 64
MLP_OUTPUTS = 15
MLP_PARAMS = 5968
Q_CHOICES = (0, 1, 2, 3, 4)
P_CHOICES = (5, 10, 20)
STATUS = {0: "RQLP_OK", 1: "RQLP_ERR_ARG", 2: "RQLP_ERR_CUDA", 3: "RQLP_ERR_BREAKDOWN",
          4: "RQLP_ERR_NONFINITE", 5: "RQLP_ERR_TIMEOUT", 6: "RQLP_ERR_WORKSPACE",
          7: "RQLP_ERR_UNSUPPORTED"}

# Every symbol include/rqlp.h declares (checked by the ABI test).
EXPORTED = ["rqlp_default_opts", "rqlp_workspace_bytes", "rqlp_factor", "rqlp_host_workspace_bytes",
            "rqlp_factor_host", "rqlp_factor_noalloc", "rqlp_sketch_workspace_bytes", "rqlp_sketch",
            "rqlp_orth_workspace_bytes", "rqlp_orth", "rqlp_mlp_forward", "rqlp_mlp_workspace_bytes",
            "rqlp_mlp_grad", "rqlp_mlp_adam", "rqlp_learned_workspace_bytes", "rqlp_probe_features",
            "rqlp_predict_qp", "rqlp_factor_learned", "rqlp_learned_host_workspace_bytes",
            "rqlp_factor_learned_host", "rqlp_sparse_workspace_bytes", "rqlp_factor_sparse",
            "rqlp_rank_errors", "rqlp_rank_residual_workspace_bytes",
            "rqlp_rank_residual", "rqlp_subspace_workspace_bytes", "rqlp_subspace_angles",
            "rqlp_batch_workspace_bytes", "rqlp_batch_create",
            "rqlp_batch_autotune", "rqlp_batch_tuning", "rqlp_batch_run", "rqlp_batch_launch",
            "rqlp_batch_destroy", "rqlp_factor_batched", "rqlp_kernel_launches", "rqlp_profile_enable",
            "rqlp_profile_read", "rqlp_status_string", "rqlp_version"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("small_fp64", ctypes.c_int),
                ("test_stall", ctypes.c_int), ("bf16_parts", ctypes.c_int),
                ("literal_step5", ctypes.c_int), ("fused_power", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class Problem(ctypes.Structure):
    """rqlp_problem: one problem of a batch (device pointers, row-major)."""
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("Omega", ctypes.c_void_p), ("ldo", ctypes.c_int64), ("k", ctypes.c_int), ("p", ctypes.c_int),
                ("Q", ctypes.c_void_p), ("ldq", ctypes.c_int64), ("L", ctypes.c_void_p), ("ldl", ctypes.c_int64),
                ("P", ctypes.c_void_p), ("ldp", ctypes.c_int64)]


class Csr(ctypes.Structure):
    """rqlp_csr: a sparse A in CSR form (device arrays)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class RqlpError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({rqlp_status_string(status)})")
        self.status = status


_lib = None
_i64, _int, _vp, _sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t


def _declare(lib):
    lib.rqlp_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.rqlp_default_opts.restype = None
    lib.rqlp_workspace_bytes.argtypes = [_i64, _i64, _int, _int, _int, ctypes.POINTER(Opts)]
    lib.rqlp_workspace_bytes.restype = _sz
    lib.rqlp_host_workspace_bytes.argtypes = [_i64, _i64, _int, _int, _int, ctypes.POINTER(Opts)]
    lib.rqlp_host_workspace_bytes.restype = _sz
    sig = [_vp, _i64, _i64, _i64, _int, _int, _int, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
           _vp, _sz, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor.argtypes = sig
    lib.rqlp_factor.restype = _int
    lib.rqlp_factor_host.argtypes = sig
    lib.rqlp_factor_host.restype = _int
    lib.rqlp_factor_noalloc.argtypes = [_vp, _i64, _i64, _i64, _int, _int, _int, _vp, _i64, _vp, _i64,
                                         _vp, _i64, _vp, _i64, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor_noalloc.restype = _int
    lib.rqlp_sketch_workspace_bytes.argtypes = [_int, _i64, _i64, _int, ctypes.POINTER(Opts)]
    lib.rqlp_sketch_workspace_bytes.restype = _sz
    lib.rqlp_sketch.argtypes = [_int, _vp, _i64, _i64, _i64, _vp, _i64, _int, _vp, _i64, _vp, _sz,
                                ctypes.POINTER(Opts), _vp]
    lib.rqlp_sketch.restype = _int
    lib.rqlp_orth_workspace_bytes.argtypes = [_i64, _int, ctypes.POINTER(Opts)]
    lib.rqlp_orth_workspace_bytes.restype = _sz
    lib.rqlp_orth.argtypes = [_vp, _i64, _int, _i64, _vp, _i64, _vp, _sz, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_orth.restype = _int
    _f = ctypes.c_float
    lib.rqlp_mlp_forward.argtypes = [_vp, _vp, _int, _vp, _vp]
    lib.rqlp_mlp_forward.restype = _int
    lib.rqlp_mlp_workspace_bytes.argtypes = [_int]
    lib.rqlp_mlp_workspace_bytes.restype = _sz
    lib.rqlp_mlp_grad.argtypes = [_vp, _vp, _vp, _int, _vp, _vp, _vp, _sz, _vp]
    lib.rqlp_mlp_grad.restype = _int
    lib.rqlp_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _int, _f, _f, _f, _f, _int, _vp]
    lib.rqlp_mlp_adam.restype = _int
    lib.rqlp_learned_workspace_bytes.argtypes = [_i64, _i64, _int, ctypes.POINTER(Opts)]
    lib.rqlp_learned_workspace_bytes.restype = _sz
    _d = ctypes.c_double
    lib.rqlp_probe_features.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _i64, _vp, _vp, _sz, _vp,
                                        ctypes.POINTER(Opts), _vp]
    lib.rqlp_probe_features.restype = _int
    lib.rqlp_predict_qp.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _i64, _d, _vp, _vp, _vp, _sz, _vp,
                                    ctypes.POINTER(Opts), _vp]
    lib.rqlp_predict_qp.restype = _int
    lib.rqlp_factor_learned.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _i64, _d, _vp, _vp, _i64, _vp, _i64,
                                        _vp, _i64, _vp, _sz, _vp, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor_learned.restype = _int
    lib.rqlp_learned_host_workspace_bytes.argtypes = [_i64, _i64, _int, ctypes.POINTER(Opts)]
    lib.rqlp_learned_host_workspace_bytes.restype = _sz
    lib.rqlp_factor_learned_host.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _i64, _d, _vp, _vp, _i64, _vp,
                                             _i64, _vp, _i64, _vp, _sz, _vp, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor_learned_host.restype = _int
    lib.rqlp_sparse_workspace_bytes.argtypes = [ctypes.POINTER(Csr), _int, _int, _int, ctypes.POINTER(Opts)]
    lib.rqlp_sparse_workspace_bytes.restype = _sz
    lib.rqlp_factor_sparse.argtypes = [ctypes.POINTER(Csr), _int, _int, _int, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                                       _i64, _vp, _sz, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor_sparse.restype = _int
    lib.rqlp_rank_errors.argtypes = [_vp, _i64, _int, _vp, _vp, _vp]
    lib.rqlp_rank_errors.restype = _int
    lib.rqlp_rank_residual_workspace_bytes.argtypes = [_i64, _int]
    lib.rqlp_rank_residual_workspace_bytes.restype = _sz
    lib.rqlp_rank_residual.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _int, _vp, _i64, _int, _vp,
                                       _vp, _sz, _vp]
    lib.rqlp_rank_residual.restype = _int
    lib.rqlp_subspace_workspace_bytes.argtypes = [_i64, _int, _int]
    lib.rqlp_subspace_workspace_bytes.restype = _sz
    lib.rqlp_subspace_angles.argtypes = [_vp, _i64, _int, _i64, _vp, _int, _i64, _int, _vp, _vp, _sz, _vp]
    lib.rqlp_subspace_angles.restype = _int
    _pp = ctypes.POINTER(Problem)
    lib.rqlp_batch_workspace_bytes.argtypes = [_int, _pp, _int, ctypes.POINTER(Opts)]
    lib.rqlp_batch_workspace_bytes.restype = _sz
    lib.rqlp_batch_create.argtypes = [_int, _pp, _int, _vp, _sz, _vp, _vp, ctypes.POINTER(Opts), _vp,
                                      ctypes.POINTER(_vp)]
    lib.rqlp_batch_create.restype = _int
    lib.rqlp_batch_autotune.argtypes = [_vp, _int, _vp]
    lib.rqlp_batch_autotune.restype = _int
    lib.rqlp_batch_tuning.argtypes = [_vp, ctypes.POINTER(_int), _int]
    lib.rqlp_batch_tuning.restype = _int
    lib.rqlp_batch_run.argtypes = [_vp, _vp]
    lib.rqlp_batch_run.restype = _int
    lib.rqlp_batch_launch.argtypes = [_vp, _vp]
    lib.rqlp_batch_launch.restype = _int
    lib.rqlp_batch_destroy.argtypes = [_vp]
    lib.rqlp_batch_destroy.restype = _int
    lib.rqlp_factor_batched.argtypes = [_int, _pp, _int, _vp, _sz, _vp, _vp, ctypes.POINTER(Opts), _vp]
    lib.rqlp_factor_batched.restype = _int
    lib.rqlp_kernel_launches.argtypes = []
    lib.rqlp_kernel_launches.restype = ctypes.c_ulonglong
    lib.rqlp_profile_enable.argtypes = [_int]
    lib.rqlp_profile_enable.restype = _int
    lib.rqlp_profile_read.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_int), _int]
    lib.rqlp_profile_read.restype = _int
    lib.rqlp_status_string.argtypes = [_int]
    lib.rqlp_status_string.restype = ctypes.c_char_p
    lib.rqlp_version.argtypes = []
    lib.rqlp_version.restype = _int


def load(build_if_missing: bool = True):
    """Load librqlp.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_2110_01011_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    _declare(lib)
    _lib = lib
    return lib


def _opts(precision=PREC_FP32, small_fp64=False, parts=0, literal=False, fused=False):
    o = Opts()
    load().rqlp_default_opts(ctypes.byref(o))
    o.precision = int(precision)
    o.small_fp64 = 1 if small_fp64 else 0
    o.bf16_parts = int(parts)
    o.literal_step5 = 1 if literal else 0
    o.fused_power = 1 if fused else 0
    return o


# ------------------------------------------------------------------ 1:1 entry points

def rqlp_default_opts():
    return _opts()


def rqlp_workspace_bytes(m, n, k, p, q, opts=None):
    return int(load().rqlp_workspace_bytes(m, n, k, p, q, ctypes.byref(opts or _opts())))


def rqlp_host_workspace_bytes(m, n, k, p, q, opts=None):
    return int(load().rqlp_host_workspace_bytes(m, n, k, p, q, ctypes.byref(opts or _opts())))


def rqlp_factor(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp, workspace, ws_bytes,
                d_info, d_diag, opts, stream):
    """Raw call: pointer arguments are ints (device addresses) or None."""
    return int(load().rqlp_factor(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp,
                                  workspace, ws_bytes, d_info, d_diag,
                                  ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_factor_host(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp, workspace,
                     ws_bytes, h_info, h_diag, opts, stream):
    """Raw call: A, Omega, Q, L, P, h_info, h_diag are host addresses."""
    return int(load().rqlp_factor_host(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp,
                                       workspace, ws_bytes, h_info, h_diag,
                                       ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_factor_noalloc(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp, d_info, d_diag,
                        opts, stream):
    """Raw call of the allocation-free factorisation (library-owned scratch)."""
    return int(load().rqlp_factor_noalloc(A, m, n, lda, k, p, q, Omega, ldo, Q, ldq, L, ldl, P, ldp,
                                          d_info, d_diag,
                                          ctypes.byref(opts) if opts is not None else None, stream))


def header_define(name: str) -> int:
    """Integer value of a ``#define`` in include/rqlp.h (a decimal literal, or
    ``(a << b)`` with an optional ``u`` suffix), read from the header itself so
    that the binding carries no second copy of the library's limits."""
    hdr = os.path.join(_build.ROOT, "include", "rqlp.h")
    with open(hdr) as f:
        text = f.read()
    mt = re.search(r"^#define\s+" + re.escape(name) + r"\s+(.+?)\s*$", text, re.M)
    if mt is None:
        raise KeyError(f"{name} is not defined in {hdr}")
    expr = mt.group(1).replace("u", "").replace("(", "").replace(")", "").strip()
    parts = [x.strip() for x in expr.split("<<")]
    if not 1 <= len(parts) <= 2 or not all(x.isdigit() for x in parts):
        raise ValueError(f"{name}: unsupported expression {mt.group(1)!r}")
    return int(parts[0]) << (int(parts[1]) if len(parts) == 2 else 0)


NOALLOC_SCRATCH_BYTES = header_define("RQLP_NOALLOC_SCRATCH_BYTES")


def rqlp_sketch_workspace_bytes(trans, m, n, d, opts=None):
    return int(load().rqlp_sketch_workspace_bytes(trans, m, n, d, ctypes.byref(opts or _opts())))


def rqlp_sketch(trans, A, m, n, lda, X, ldx, d, Y, ldy, workspace, ws_bytes, opts, stream):
    return int(load().rqlp_sketch(trans, A, m, n, lda, X, ldx, d, Y, ldy, workspace, ws_bytes,
                                  ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_orth_workspace_bytes(rows, d, opts=None):
    return int(load().rqlp_orth_workspace_bytes(rows, d, ctypes.byref(opts or _opts())))


def rqlp_orth(X, rows, d, ldx, R, ldr, workspace, ws_bytes, d_info, opts, stream):
    return int(load().rqlp_orth(X, rows, d, ldx, R, ldr, workspace, ws_bytes, d_info,
                                ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_mlp_forward(params, X, batch, est, stream):
    return int(load().rqlp_mlp_forward(params, X, batch, est, stream))


def rqlp_mlp_workspace_bytes(batch):
    return int(load().rqlp_mlp_workspace_bytes(batch))


def rqlp_mlp_grad(params, X, Y, batch, grad, loss, workspace, ws_bytes, stream):
    return int(load().rqlp_mlp_grad(params, X, Y, batch, grad, loss, workspace, ws_bytes, stream))


def rqlp_mlp_adam(params, grad, m1, m2, n, lr, beta1, beta2, eps, step, stream):
    return int(load().rqlp_mlp_adam(params, grad, m1, m2, n, lr, beta1, beta2, eps, step, stream))


def rqlp_learned_workspace_bytes(m, n, k, opts=None):
    return int(load().rqlp_learned_workspace_bytes(m, n, k, ctypes.byref(opts or _opts())))


def rqlp_probe_features(A, m, n, lda, k, Omega, ldo, feat, workspace, ws_bytes, d_info, opts, stream):
    return int(load().rqlp_probe_features(A, m, n, lda, k, Omega, ldo, feat, workspace, ws_bytes, d_info,
                                          ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_predict_qp(A, m, n, lda, k, Omega, ldo, target, params, d_qp, workspace, ws_bytes, d_info, opts, stream):
    return int(load().rqlp_predict_qp(A, m, n, lda, k, Omega, ldo, target, params, d_qp, workspace, ws_bytes,
                                      d_info, ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_factor_learned(A, m, n, lda, k, Omega, ldo, target, params, Q, ldq, L, ldl, P, ldp, workspace, ws_bytes,
                        d_info, d_diag, h_qp, opts, stream):
    return int(load().rqlp_factor_learned(A, m, n, lda, k, Omega, ldo, target, params, Q, ldq, L, ldl, P, ldp,
                                          workspace, ws_bytes, d_info, d_diag, h_qp,
                                          ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_batch_workspace_bytes(count, probs, q, opts=None):
    return int(load().rqlp_batch_workspace_bytes(count, probs, q, ctypes.byref(opts or _opts())))


def rqlp_batch_create(count, probs, q, workspace, ws_bytes, d_info, d_diag, opts, stream):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = int(load().rqlp_batch_create(count, probs, q, workspace, ws_bytes, d_info, d_diag,
                                      ctypes.byref(opts) if opts is not None else None, stream, ctypes.byref(h)))
    return st, h


def rqlp_batch_autotune(batch, reps, stream):
    return int(load().rqlp_batch_autotune(batch, reps, stream))


def rqlp_batch_tuning(batch):
    n = int(load().rqlp_batch_tuning(batch, None, 0))
    buf = (_int * max(n, 1))()
    load().rqlp_batch_tuning(batch, buf, n)
    return [int(buf[i]) for i in range(n)]


def rqlp_batch_run(batch, stream):
    return int(load().rqlp_batch_run(batch, stream))


def rqlp_batch_launch(batch, stream):
    return int(load().rqlp_batch_launch(batch, stream))


def rqlp_batch_destroy(batch):
    return int(load().rqlp_batch_destroy(batch))


def rqlp_factor_batched(count, probs, q, workspace, ws_bytes, d_info, d_diag, opts, stream):
    return int(load().rqlp_factor_batched(count, probs, q, workspace, ws_bytes, d_info, d_diag,
                                          ctypes.byref(opts) if opts is not None else None, stream))


def rqlp_kernel_launches():
    return int(load().rqlp_kernel_launches())


def rqlp_profile_enable(on):
    return int(load().rqlp_profile_enable(1 if on else 0))


def rqlp_profile_read(cap=4096):
    """Returns a list of (ms, tag) for the recorded passes over A."""
    ms = (ctypes.c_float * cap)()
    tags = (_int * cap)()
    n = int(load().rqlp_profile_read(ms, tags, cap))
    return [(float(ms[i]), int(tags[i])) for i in range(n)]


def rqlp_status_string(status):
    return load().rqlp_status_string(int(status)).decode()


def rqlp_version():
    return int(load().rqlp_version())


# ------------------------------------------------------------------ torch conveniences

def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def factor(A, k, p, q, Omega, precision=PREC_FP32, small_fp64=False, workspace=None, out=None, parts=0,
           literal=False, fused=False):
    """Factor a CUDA FP32 row-major A (m x n) with Omega (m x (k+p)).

    Returns (Q, L, P, info, diag) as CUDA tensors; info (int32[2]) and diag
    (float64[4]) are filled asynchronously on the current stream. parts:
    BF16 parts per pass operand in the BF16X3 form (0 = automatic, 2, 3).
    literal: step 5 as Algorithm 1 prints it (QR of A^T Q, a third pass).
    fused: each power pass as A^T (A P~) over L2-sized row panels.
    """
    import torch
    m, n = A.shape
    d = k + p
    if A.dtype != torch.float32 or Omega.dtype != torch.float32 or not A.is_cuda:
        raise TypeError("A and Omega must be CUDA float32 tensors")
    if A.stride(1) != 1 or Omega.stride(1) != 1:
        raise ValueError("A and Omega must be row-major (unit column stride)")
    opts = _opts(precision, small_fp64, parts, literal, fused)
    ws_bytes = rqlp_workspace_bytes(m, n, k, p, q, opts)
    if ws_bytes == 0:
        raise RqlpError(1, "rqlp_workspace_bytes")
    dev = A.device
    if workspace is None or workspace.numel() < ws_bytes + 256:
        workspace = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    if out is None:
        Q = torch.empty(m, d, dtype=torch.float32, device=dev)
        L = torch.empty(d, d, dtype=torch.float32, device=dev)
        P = torch.empty(n, d, dtype=torch.float32, device=dev)
        info = torch.empty(2, dtype=torch.int32, device=dev)
        diag = torch.empty(4, dtype=torch.float64, device=dev)
    else:
        Q, L, P, info, diag = out
    base = workspace.data_ptr()
    aligned = (base + 255) // 256 * 256
    st = rqlp_factor(A.data_ptr(), m, n, A.stride(0), k, p, q, Omega.data_ptr(), Omega.stride(0),
                     Q.data_ptr(), Q.stride(0), L.data_ptr(), L.stride(0), P.data_ptr(), P.stride(0),
                     aligned, ws_bytes, info.data_ptr(), diag.data_ptr(), opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_factor")
    return Q, L, P, info, diag


def _workspace(nbytes, device):
    import torch
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return buf, (buf.data_ptr() + 255) // 256 * 256


def sketch(A, X, trans, precision=PREC_FP32, parts=0):
    """Y = A^T X (trans=1) or A X (trans=0) for CUDA float32 row-major A, X."""
    import torch
    m, n = A.shape
    d = X.shape[1]
    opts = _opts(precision, parts=parts)
    nb = rqlp_sketch_workspace_bytes(trans, m, n, d, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_sketch_workspace_bytes")
    buf, ws = _workspace(nb, A.device)
    Y = torch.empty(n if trans else m, d, dtype=torch.float32, device=A.device)
    st = rqlp_sketch(trans, A.data_ptr(), m, n, A.stride(0), X.data_ptr(), X.stride(0), d,
                     Y.data_ptr(), Y.stride(0), ws, nb, opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_sketch")
    return Y, buf


def orth(X, small_fp64=False):
    """In-place X = qf(X) for a CUDA float32 row-major X; returns (X, R, info)."""
    import torch
    rows, d = X.shape
    opts = _opts(PREC_FP32, small_fp64)
    nb = rqlp_orth_workspace_bytes(rows, d, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_orth_workspace_bytes")
    buf, ws = _workspace(nb, X.device)
    R = torch.empty(d, d, dtype=torch.float32, device=X.device)
    info = torch.empty(2, dtype=torch.int32, device=X.device)
    st = rqlp_orth(X.data_ptr(), rows, d, X.stride(0), R.data_ptr(), R.stride(0), ws, nb,
                   info.data_ptr(), opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_orth")
    return X, R, info, buf


def probe_features(A, k, Omega, precision=PREC_BF16X3, workspace=None):
    """Probe features (12 floats, CUDA tensor) of A with Omega (m x (k+20))."""
    import torch
    m, n = A.shape
    opts = _opts(precision)
    nb = rqlp_learned_workspace_bytes(m, n, k, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_learned_workspace_bytes")
    if workspace is None or workspace.numel() < nb + 256:
        workspace = torch.empty(nb + 256, dtype=torch.uint8, device=A.device)
    ws = (workspace.data_ptr() + 255) // 256 * 256
    feat = torch.empty(MLP_FEATURES, dtype=torch.float32, device=A.device)
    info = torch.empty(2, dtype=torch.int32, device=A.device)
    st = rqlp_probe_features(A.data_ptr(), m, n, A.stride(0), k, Omega.data_ptr(), Omega.stride(0),
                             feat.data_ptr(), ws, nb, info.data_ptr(), opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_probe_features")
    return feat, info


def factor_learned(A, k, Omega, params, target, precision=PREC_BF16X3, workspace=None, out=None, parts=0):
    """Rand-QLP with the (q, p) predicted for the requested excess rank-k
    error ``target``. Returns (Q, L, P, info, diag, (q, p)); Q, L, P are views
    of k + p columns of buffers sized for k + 20."""
    import torch
    m, n = A.shape
    dmax = k + 20
    opts = _opts(precision, parts=parts)
    nb = rqlp_learned_workspace_bytes(m, n, k, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_learned_workspace_bytes")
    dev = A.device
    if workspace is None or workspace.numel() < nb + 256:
        workspace = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    ws = (workspace.data_ptr() + 255) // 256 * 256
    if out is None:
        out = (torch.empty(m, dmax, device=dev), torch.empty(dmax, dmax, device=dev),
               torch.empty(n, dmax, device=dev), torch.empty(2, dtype=torch.int32, device=dev),
               torch.empty(4, dtype=torch.float64, device=dev))
    Q, L, P, info, diag = out
    qp = (ctypes.c_int * 2)()
    st = rqlp_factor_learned(A.data_ptr(), m, n, A.stride(0), k, Omega.data_ptr(), Omega.stride(0), float(target),
                             params.data_ptr(), Q.data_ptr(), Q.stride(0), L.data_ptr(), L.stride(0),
                             P.data_ptr(), P.stride(0), ws, nb, info.data_ptr(), diag.data_ptr(),
                             ctypes.addressof(qp), opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_factor_learned")
    d = k + qp[1]
    return Q[:, :d], L[:d, :d], P[:, :d], info, diag, (qp[0], qp[1])


def rqlp_learned_host_workspace_bytes(m, n, k, opts=None):
    return int(load().rqlp_learned_host_workspace_bytes(m, n, k, ctypes.byref(opts or _opts())))


def factor_learned_host(A, k, Omega, params, target, precision=PREC_BF16X3, workspace=None, out=None, parts=0):
    """Host-buffer learned form: CPU float32 A (m x n) and Omega (m x (k+20))
    (pinned for full bandwidth), params on the device. Returns host
    (Q, L, P, info, diag, (q, p)) with Q, L, P views of k + p columns;
    synchronous."""
    import torch
    A_t, O_t = torch.as_tensor(A), torch.as_tensor(Omega)
    m, n = A_t.shape
    w = k + 20
    opts = _opts(precision, parts=parts)
    nb = rqlp_learned_host_workspace_bytes(m, n, k, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_learned_host_workspace_bytes")
    if workspace is None or workspace.numel() < nb + 256:
        workspace = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    if out is None:
        pin = torch.cuda.is_available()
        out = (torch.empty(m, w, pin_memory=pin), torch.empty(w, w, pin_memory=pin), torch.empty(n, w, pin_memory=pin),
               torch.zeros(2, dtype=torch.int32), torch.zeros(4, dtype=torch.float64))
    Q, L, P, info, diag = out
    qp = (ctypes.c_int * 2)()
    ws = (workspace.data_ptr() + 255) // 256 * 256
    st = int(load().rqlp_factor_learned_host(A_t.data_ptr(), m, n, A_t.stride(0), k, O_t.data_ptr(), O_t.stride(0),
                                             float(target), params.data_ptr(), Q.data_ptr(), Q.stride(0),
                                             L.data_ptr(), L.stride(0), P.data_ptr(), P.stride(0), ws, nb,
                                             info.data_ptr(), diag.data_ptr(), ctypes.addressof(qp),
                                             ctypes.byref(opts), _stream()))
    if st != 0:
        raise RqlpError(st, "rqlp_factor_learned_host")
    d = k + qp[1]
    return Q[:, :d], L[:d, :d], P[:, :d], info, diag, (qp[0], qp[1])


def rqlp_sparse_workspace_bytes(csr, k, p, q, opts=None):
    return int(load().rqlp_sparse_workspace_bytes(ctypes.byref(csr), k, p, q, ctypes.byref(opts or _opts())))


def factor_sparse(row_ptr, col_idx, vals, m, n, k, p, q, Omega, workspace=None):
    """Rand-QLP of a sparse A in CSR form (CUDA int64 row_ptr, int32 col_idx,
    float32 vals) with Omega (CUDA float32, m x (k+p)). Returns (Q, L, P,
    info, diag) as CUDA tensors (asynchronous)."""
    import torch
    d = k + p
    csr = Csr(m, n, int(col_idx.numel()), row_ptr.data_ptr(), col_idx.data_ptr(), vals.data_ptr())
    opts = _opts(PREC_FP32)
    nb = rqlp_sparse_workspace_bytes(csr, k, p, q, opts)
    if nb == 0:
        raise RqlpError(1, "rqlp_sparse_workspace_bytes")
    dev = Omega.device
    if workspace is None or workspace.numel() < nb + 256:
        workspace = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    ws = (workspace.data_ptr() + 255) // 256 * 256
    Q = torch.empty(m, d, device=dev)
    L = torch.empty(d, d, device=dev)
    P = torch.empty(n, d, device=dev)
    info = torch.empty(2, dtype=torch.int32, device=dev)
    diag = torch.empty(4, dtype=torch.float64, device=dev)
    st = int(load().rqlp_factor_sparse(ctypes.byref(csr), k, p, q, Omega.data_ptr(), Omega.stride(0), Q.data_ptr(),
                                       Q.stride(0), L.data_ptr(), L.stride(0), P.data_ptr(), P.stride(0), ws, nb,
                                       info.data_ptr(), diag.data_ptr(), ctypes.byref(opts), _stream()))
    if st != 0:
        raise RqlpError(st, "rqlp_factor_sparse")
    return Q, L, P, info, diag


def rank_errors(L, diag):
    """||A - A_r||_F for r = 1..d (CUDA float64 tensor) from L and d_diag."""
    import torch
    d = L.shape[0]
    errs = torch.empty(d, dtype=torch.float64, device=L.device)
    st = int(load().rqlp_rank_errors(L.data_ptr(), L.stride(0), d, diag.data_ptr(), errs.data_ptr(), _stream()))
    if st != 0:
        raise RqlpError(st, "rqlp_rank_errors")
    return errs


def rank_residual(A, Q, L, P, r):
    """||A - Q L(:, 1:r) P(:, 1:r)^T||_F computed explicitly (CUDA float64 scalar tensor)."""
    import torch
    m, n = A.shape
    d = L.shape[0]
    nb = int(load().rqlp_rank_residual_workspace_bytes(m, r))
    if nb == 0:
        raise RqlpError(1, "rqlp_rank_residual_workspace_bytes")
    buf, ws = _workspace(nb, A.device)
    out = torch.empty(1, dtype=torch.float64, device=A.device)
    st = int(load().rqlp_rank_residual(A.data_ptr(), m, n, A.stride(0), Q.data_ptr(), Q.stride(0), L.data_ptr(),
                                       L.stride(0), d, P.data_ptr(), P.stride(0), r, out.data_ptr(), ws, nb,
                                       _stream()))
    if st != 0:
        raise RqlpError(st, "rqlp_rank_residual")
    return out


def subspace_angles(X, Y, cosines=False):
    """Sines (or cosines) of the canonical angles between R(Y) and R(X), for
    orthonormal CUDA float32 X (rows x a) and Y (rows x b); largest first."""
    import torch
    rows, a = X.shape
    b = Y.shape[1]
    nb = int(load().rqlp_subspace_workspace_bytes(rows, a, b))
    if nb == 0:
        raise RqlpError(1, "rqlp_subspace_workspace_bytes")
    buf, ws = _workspace(nb, X.device)
    out = torch.empty(b, dtype=torch.float64, device=X.device)
    st = int(load().rqlp_subspace_angles(X.data_ptr(), rows, a, X.stride(0), Y.data_ptr(), b, Y.stride(0),
                                         1 if cosines else 0, out.data_ptr(), ws, nb, _stream()))
    if st != 0:
        raise RqlpError(st, "rqlp_subspace_angles")
    return out


def factor_host(A, k, p, q, Omega, precision=PREC_FP32, workspace=None, out=None, parts=0):
    """Host-buffer form: numpy/torch CPU float32 A and Omega (pinned for full
    bandwidth). Returns host (Q, L, P, info, diag); synchronous."""
    import torch
    A_t = torch.as_tensor(A)
    O_t = torch.as_tensor(Omega)
    m, n = A_t.shape
    d = k + p
    opts = _opts(precision, parts=parts)
    ws_bytes = rqlp_host_workspace_bytes(m, n, k, p, q, opts)
    if ws_bytes == 0:
        raise RqlpError(1, "rqlp_host_workspace_bytes")
    if workspace is None or workspace.numel() < ws_bytes + 256:
        workspace = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
    if out is None:
        pin = torch.cuda.is_available()
        Q = torch.empty(m, d, dtype=torch.float32, pin_memory=pin)
        L = torch.empty(d, d, dtype=torch.float32, pin_memory=pin)
        P = torch.empty(n, d, dtype=torch.float32, pin_memory=pin)
        info = torch.zeros(2, dtype=torch.int32)
        diag = torch.zeros(4, dtype=torch.float64)
    else:
        Q, L, P, info, diag = out
    aligned = (workspace.data_ptr() + 255) // 256 * 256
    st = rqlp_factor_host(A_t.data_ptr(), m, n, A_t.stride(0), k, p, q, O_t.data_ptr(),
                          O_t.stride(0), Q.data_ptr(), Q.stride(0), L.data_ptr(), L.stride(0),
                          P.data_ptr(), P.stride(0), aligned, ws_bytes, info.data_ptr(),
                          diag.data_ptr(), opts, _stream())
    if st != 0:
        raise RqlpError(st, "rqlp_factor_host")
    return Q, L, P, info, diag


class Batch:
    """A batch plan over CUDA FP32 row-major matrices: As[i] (m_i x n_i),
    Omegas[i] (m_i x (k_i + p_i)), one q. Allocates the outputs, the
    per-problem info/diag rows and the workspace with torch; ``launch()``
    replays the captured graph, ``run()`` launches the kernels one by one.
    precision: PREC_FP32, or PREC_BF16X3 (the passes over A as grouped
    tensor-core passes over BF16 parts; parts: 0 = three, 2, 3)."""

    def __init__(self, As, Omegas, ks, ps, q, small_fp64=False, precision=PREC_FP32, test_stall=False, parts=0):
        import torch
        self.count = len(As)
        dev = As[0].device
        self.As, self.Omegas = list(As), list(Omegas)
        self.Q, self.L, self.P = [], [], []
        arr = (Problem * self.count)()
        for i, (A, O, k, p) in enumerate(zip(As, Omegas, ks, ps)):
            m, n = A.shape
            d = k + p
            Q = torch.empty(m, d, device=dev)
            L = torch.empty(d, d, device=dev)
            P = torch.empty(n, d, device=dev)
            self.Q.append(Q)
            self.L.append(L)
            self.P.append(P)
            arr[i] = Problem(A.data_ptr(), m, n, A.stride(0), O.data_ptr(), O.stride(0), k, p, Q.data_ptr(),
                             Q.stride(0), L.data_ptr(), L.stride(0), P.data_ptr(), P.stride(0))
        self.probs = arr
        self.opts = _opts(precision, small_fp64, parts)
        self.opts.test_stall = 1 if test_stall else 0
        nb = rqlp_batch_workspace_bytes(self.count, arr, q, self.opts)
        if nb == 0:
            raise RqlpError(1, "rqlp_batch_workspace_bytes")
        self.ws_bytes = nb
        self.ws_buf, self.ws = _workspace(nb, dev)
        self.info = torch.empty(self.count, 2, dtype=torch.int32, device=dev)
        self.diag = torch.empty(self.count, 4, dtype=torch.float64, device=dev)
        st, h = rqlp_batch_create(self.count, arr, q, self.ws, nb, self.info.data_ptr(), self.diag.data_ptr(),
                                  self.opts, _stream())
        if st != 0:
            raise RqlpError(st, "rqlp_batch_create")
        self.handle = h

    def autotune(self, reps=3):
        st = rqlp_batch_autotune(self.handle, reps, _stream())
        if st != 0:
            raise RqlpError(st, "rqlp_batch_autotune")
        return rqlp_batch_tuning(self.handle)

    def run(self):
        st = rqlp_batch_run(self.handle, _stream())
        if st != 0:
            raise RqlpError(st, "rqlp_batch_run")

    def launch(self):
        st = rqlp_batch_launch(self.handle, _stream())
        if st != 0:
            raise RqlpError(st, "rqlp_batch_launch")

    def close(self):
        if getattr(self, "handle", None):
            rqlp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
