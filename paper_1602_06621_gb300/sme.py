"""Thin Python binding of libsme (include/sme.h): same names, argument marshalling only.

Vectors are torch CUDA tensors (float64 for an SME_F64 operator, float32 otherwise);
CSR input may be host NumPy arrays or CUDA tensors.  Every function raises
SmeError on a non-OK status.  There is no fallback: if the CUDA library cannot be
built or loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build_library

__all__ = [
    "SmeError", "load", "SME_F64", "SME_F32", "SME_BF16", "SME_FP8E4M3", "SME_EQ_ASYNC", "SME_EQ_NO_GRAPH", "SME_EQ_TIMED",
    "SME_EQ_EXPIRE_PIPELINE_WAITS",
    "sme_op_create_csr", "sme_op_create_dense", "sme_op_destroy", "sme_op_get_info", "sme_draw_probes",
    "sme_equilibrate", "sme_op_check", "sme_estimate", "sme_evaluate", "sme_lsqr", "sme_status_string",
    "sme_estimate_rows_static", "SME_STATIC_MAX_COLS", "sme_op_create_csr_shard", "sme_shard_get_info",
    "sme_shard_begin", "sme_shard_step", "sme_shard_end", "sme_batch_create", "sme_batch_destroy",
    "sme_batch_get_info", "sme_batch_equilibrate", "sme_batch_estimate", "sme_batch_op", "sme_op_autotune", "sme_batch_lsqr",
    "sme_equilibrate_targets", "sme_equilibrate_symmetric", "sme_equilibrate_block", "sme_mlp_create",
    "sme_mlp_destroy", "sme_mlp_param_count", "sme_mlp_get_params", "sme_mlp_set_params", "sme_mlp_forward",
    "sme_mlp_gradient", "sme_mlp_train_step", "sme_op_features", "sme_warm_start", "sme_batch_evaluate",
    "sme_batch_features", "sme_batch_warm_start", "sme_op_norm2", "sme_ccp_lasso", "sme_release_cached_memory",
]
SME_STATIC_MAX_COLS = 1 << 20

SME_F64, SME_F32, SME_BF16, SME_FP8E4M3 = 0, 1, 2, 3
SME_EQ_ASYNC, SME_EQ_NO_GRAPH, SME_EQ_TIMED, SME_EQ_EXPIRE_PIPELINE_WAITS = 1, 2, 4, 8
_STATUS = {0: "SME_OK", -1: "SME_ERR_ARG", -2: "SME_ERR_INVALID_CSR", -3: "SME_ERR_OOM", -4: "SME_ERR_CUDA",
           -5: "SME_ERR_NONFINITE", -6: "SME_ERR_TIMEOUT", -7: "SME_ERR_NOT_CONVERGED", -8: "SME_ERR_UNSUPPORTED"}


class SmeError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)} ({detail})")
        self.status = status
        self.name = _STATUS.get(status, str(status))


class sme_equil_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("M", ctypes.c_double), ("T", ctypes.c_int32), ("k", ctypes.c_int32), ("t_begin", ctypes.c_int32),
                ("t0", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stream_base", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class sme_op_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("state_is_double", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("padded_entries_fwd", ctypes.c_int64), ("padded_entries_bwd", ctypes.c_int64),
                ("last_loop_ms", ctypes.c_double), ("last_loop_iters", ctypes.c_int64)]


class sme_eval_result(ctypes.Structure):
    _fields_ = [("row_spread", ctypes.c_double), ("col_spread", ctypes.c_double), ("rms", ctypes.c_double),
                ("objective", ctypes.c_double), ("empty_rows", ctypes.c_int64), ("empty_cols", ctypes.c_int64)]


class sme_ccp_params(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("tau", ctypes.c_double), ("sigma", ctypes.c_double),
                ("theta", ctypes.c_double), ("max_iters", ctypes.c_int64), ("check_every", ctypes.c_int32),
                ("norm_iters", ctypes.c_int32), ("p_star", ctypes.c_double), ("tol", ctypes.c_double)]


class sme_ccp_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("objective", ctypes.c_double), ("objective0", ctypes.c_double),
                ("rel_gap", ctypes.c_double), ("op_norm", ctypes.c_double), ("tau", ctypes.c_double),
                ("sigma", ctypes.c_double), ("converged", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("history_count", ctypes.c_int64)]


class sme_shard_info(ctypes.Structure):
    _fields_ = [("parts", ctypes.c_int32), ("part", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64), ("col_begin", ctypes.c_int64),
                ("col_end", ctypes.c_int64), ("row_chunk", ctypes.c_int64), ("col_chunk", ctypes.c_int64),
                ("entry_bytes", ctypes.c_int32)]


class sme_lsqr_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int64), ("check_every", ctypes.c_int32),
                ("stop_rule", ctypes.c_int32), ("history", ctypes.c_void_p), ("history_cap", ctypes.c_int64),
                ("predict_check", ctypes.c_int32)]


class sme_lsqr_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("rel_residual", ctypes.c_double), ("normal_residual", ctypes.c_double),
                ("converged", ctypes.c_int32), ("kernel_launches", ctypes.c_int64), ("history_count", ctypes.c_int64)]


_lib = None
_vp, _i64, _i32, _u64, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double

# Exported symbols and their argument types (kept in step with include/sme.h).
SIGNATURES = {
    "sme_status_string": ([_i32], ctypes.c_char_p),
    "sme_last_error": ([], ctypes.c_char_p),
    "sme_release_cached_memory": ([], _i32),
    "sme_op_create_csr": ([ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, _i32, _i32, _vp], _i32),
    "sme_op_create_dense": ([ctypes.POINTER(_vp), _i64, _i64, _vp, _i64, _i32, _vp, _i32, _vp], _i32),
    "sme_op_destroy": ([_vp], _i32),
    "sme_op_get_info": ([_vp, ctypes.POINTER(sme_op_info)], _i32),
    "sme_draw_probes": ([_u64, _i32, _i32, _i64, _i32, _vp, _vp], _i32),
    "sme_equilibrate": ([_vp, ctypes.POINTER(sme_equil_params), _vp, _vp, _vp, _vp, _vp], _i32),
    "sme_op_check": ([_vp, _vp], _i32),
    "sme_estimate": ([_vp, _vp, _vp, _i32, _i32, _u64, _i32, _vp, _vp, _vp], _i32),
    "sme_evaluate": ([_vp, _vp, _vp, _d, _d, _d, _vp, _vp, ctypes.POINTER(sme_eval_result), _vp], _i32),
    "sme_lsqr": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(sme_lsqr_params), ctypes.POINTER(sme_lsqr_result), _vp],
                 _i32),
    "sme_estimate_rows_static": ([_i64, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _u64, _i32, _vp, _vp], _i32),
    "sme_batch_create": ([ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp], _i32),
    "sme_batch_destroy": ([_vp], _i32),
    "sme_batch_get_info": ([_vp, ctypes.POINTER(_i32), _vp, _vp], _i32),
    "sme_batch_equilibrate": ([_vp, ctypes.POINTER(sme_equil_params), _vp, _vp, _vp, _vp, _vp], _i32),
    "sme_batch_estimate": ([_vp, _vp, _vp, _i32, _i32, _u64, _i32, _vp, _vp, _vp], _i32),
    "sme_batch_op": ([_vp, ctypes.POINTER(_vp)], _i32),
    "sme_op_autotune": ([_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float), _vp],
                        _i32),
    "sme_batch_lsqr": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(sme_lsqr_params), _vp, _vp], _i32),
    "sme_equilibrate_targets": ([_vp, ctypes.POINTER(sme_equil_params), _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sme_equilibrate_symmetric": ([_vp, ctypes.POINTER(sme_equil_params), _vp, _vp, _vp], _i32),
    "sme_equilibrate_block": ([_vp, ctypes.POINTER(sme_equil_params), _i64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp],
                              _i32),
    "sme_mlp_create": ([ctypes.POINTER(_vp), _u64], _i32),
    "sme_mlp_destroy": ([_vp], _i32),
    "sme_mlp_param_count": ([], _i64),
    "sme_mlp_get_params": ([_vp, _vp, _vp], _i32),
    "sme_mlp_set_params": ([_vp, _vp, _vp], _i32),
    "sme_mlp_forward": ([_vp, _vp, _i64, _vp, _vp], _i32),
    "sme_mlp_gradient": ([_vp, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "sme_mlp_train_step": ([_vp, _vp, _vp, _i64, ctypes.c_float, _vp, _vp], _i32),
    "sme_op_features": ([_vp, _u64, _vp, _vp, _vp], _i32),
    "sme_warm_start": ([_vp, _vp, _u64, _vp, _vp, _vp], _i32),
    "sme_batch_evaluate": ([_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp, _vp], _i32),
    "sme_batch_features": ([_vp, _u64, _vp, _vp, _vp], _i32),
    "sme_batch_warm_start": ([_vp, _vp, _u64, _vp, _vp, _vp], _i32),
    "sme_op_norm2": ([_vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_double), _vp], _i32),
    "sme_ccp_lasso": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp], _i32),
    "sme_mlp_fit_normalisation": ([_vp, _vp, _i64, _vp], _i32),
    "sme_mlp_draw_batch": ([_vp, _vp, _i64, _i64, _u64, _i64, _vp, _vp, _vp], _i32),
    "sme_op_create_csr_shard": ([ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp],
                                _i32),
    "sme_shard_get_info": ([_vp, _i32, ctypes.POINTER(sme_shard_info)], _i32),
    "sme_shard_begin": ([_vp, ctypes.POINTER(sme_equil_params), _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sme_shard_step": ([_vp, ctypes.POINTER(sme_equil_params), _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "sme_shard_end": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
}


def load(build: bool = True):
    """Load libsme.so, building it first when sources are newer.  Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = build_library() if build else LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsme.so not found at {path}; run paper_1602_06621_gb300.build")
        L = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise SmeError(st, where, load().sme_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def sme_status_string(status: int) -> str:
    """Short name of a status code (`sme_status_string` in include/sme.h)."""
    return load().sme_status_string(status).decode()


def sme_release_cached_memory() -> None:
    """Return the library's idle device memory (blocks of destroyed operators, pool scratch) to the device."""
    _check(load().sme_release_cached_memory(), "sme_release_cached_memory")


def sme_op_create_csr(m, n, row_ptr, col_idx, vals, dtype=None, stream=None):
    """Create a sparse operator.  Host NumPy arrays are copied; CUDA tensors are read in place."""
    on_device = not isinstance(row_ptr, np.ndarray)
    if on_device:
        import torch
        if dtype is None:
            dtype = SME_F64 if vals.dtype == torch.float64 else SME_F32
        nnz = int(col_idx.numel())
    else:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        if dtype is None:
            dtype = SME_F64 if vals.dtype == np.float64 else SME_F32
        vals = np.ascontiguousarray(vals, dtype=np.float64 if dtype == SME_F64 else np.float32)
        nnz = int(col_idx.size)
    op = ctypes.c_void_p()
    st = load().sme_op_create_csr(ctypes.byref(op), int(m), int(n), nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                  int(dtype), int(on_device), _stream(stream))
    _check(st, "sme_op_create_csr")
    return op


def sme_op_create_csr_shard(m, n, row_ptr, col_idx, vals, parts, part, dtype=None, stream=None):
    """Create part `part` of `parts` of a sparse matrix split over several devices (arguments as
    sme_op_create_csr, the whole matrix is passed)."""
    on_device = not isinstance(row_ptr, np.ndarray)
    if on_device:
        import torch
        if dtype is None:
            dtype = SME_F64 if vals.dtype == torch.float64 else SME_F32
        nnz = int(col_idx.numel())
    else:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        if dtype is None:
            dtype = SME_F64 if vals.dtype == np.float64 else SME_F32
        vals = np.ascontiguousarray(vals, dtype=np.float64 if dtype == SME_F64 else np.float32)
        nnz = int(col_idx.size)
    op = ctypes.c_void_p()
    st = load().sme_op_create_csr_shard(ctypes.byref(op), int(m), int(n), nnz, _ptr(row_ptr), _ptr(col_idx),
                                        _ptr(vals), int(dtype), int(on_device), int(parts), int(part), _stream(stream))
    _check(st, "sme_op_create_csr_shard")
    return op


def sme_shard_get_info(op, k) -> dict:
    """Blocks, table chunks and table entry size of a part of a split matrix."""
    info = sme_shard_info()
    _check(load().sme_shard_get_info(op, int(k), ctypes.byref(info)), "sme_shard_get_info")
    return {f: getattr(info, f) for f, _ in sme_shard_info._fields_}


def sme_shard_begin(op, u, v, u_bar, v_bar, row_table, col_table, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0,
                    alpha=0.0, beta=0.0, gamma=0.0, M=0.0, stream=None):
    """Load this part's start state and write its chunks of the tables of iteration t_begin."""
    p = sme_equil_params(alpha, beta, gamma, M, int(T), int(k), int(t_begin), int(t0), int(seed), int(stream_base), 0)
    _check(load().sme_shard_begin(op, ctypes.byref(p), _ptr(u), _ptr(v), _ptr(u_bar), _ptr(v_bar), _ptr(row_table),
                                  _ptr(col_table), _stream(stream)), "sme_shard_begin")


def sme_shard_step(op, t, row_in, col_in, row_out, col_out, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0,
                   alpha=0.0, beta=0.0, gamma=0.0, M=0.0, stream=None):
    """Iteration t of this part: whole current tables in, this part's chunks of the next tables out."""
    p = sme_equil_params(alpha, beta, gamma, M, int(T), int(k), int(t_begin), int(t0), int(seed), int(stream_base), 0)
    _check(load().sme_shard_step(op, ctypes.byref(p), int(t), _ptr(row_in), _ptr(col_in), _ptr(row_out), _ptr(col_out),
                                 _stream(stream)), "sme_shard_step")


def sme_shard_end(op, u, v, u_bar, v_bar, stream=None):
    """This part's u, v, u_bar, v_bar after the last step."""
    _check(load().sme_shard_end(op, _ptr(u), _ptr(v), _ptr(u_bar), _ptr(v_bar), _stream(stream)), "sme_shard_end")


def sme_op_create_dense(m, n, A, lda=None, dtype=SME_BF16, row_scales=None, stream=None):
    """Create a dense operator (BF16, or FP8-E4M3 with per-row scales); m and n multiples of 128."""
    on_device = not isinstance(A, np.ndarray)
    op = ctypes.c_void_p()
    st = load().sme_op_create_dense(ctypes.byref(op), int(m), int(n), _ptr(A), int(lda if lda else n), int(dtype),
                                    _ptr(row_scales), int(on_device), _stream(stream))
    _check(st, "sme_op_create_dense")
    return op


def sme_op_destroy(op):
    """Destroy an operator; its device blocks are kept for reuse by later operators of the same sizes."""
    if op:
        _check(load().sme_op_destroy(op), "sme_op_destroy")


def sme_op_get_info(op) -> dict:
    """Sizes, dtype, device bytes and the last timed iteration loop of an operator, as a dict."""
    info = sme_op_info()
    _check(load().sme_op_get_info(op, ctypes.byref(info)), "sme_op_get_info")
    return {f: getattr(info, f) for f, _ in sme_op_info._fields_}


def sme_draw_probes(seed, t, stream_id, length, k, words, stream=None):
    """Write the bit-packed +-1 probes of iteration t (Philox4x32-10 contract) into `words`."""
    _check(load().sme_draw_probes(int(seed), int(t), int(stream_id), int(length), int(k), _ptr(words),
                                  _stream(stream)), "sme_draw_probes")


def sme_equilibrate(op, u, v, u_bar, v_bar, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0, alpha=0.0,
                    beta=0.0, gamma=0.0, M=0.0, flags=0, stream=None):
    """Algorithm 1: T iterations with k probes from the given (u, v, u_bar, v_bar), updated in place."""
    p = sme_equil_params(alpha, beta, gamma, M, int(T), int(k), int(t_begin), int(t0), int(seed), int(stream_base),
                         int(flags))
    _check(load().sme_equilibrate(op, ctypes.byref(p), _ptr(u), _ptr(v), _ptr(u_bar), _ptr(v_bar), _stream(stream)),
           "sme_equilibrate")


def sme_op_check(op, stream=None):
    """Raise the error recorded in the operator's device status word, if any."""
    _check(load().sme_op_check(op, _stream(stream)), "sme_op_check")


def sme_estimate(op, u, v, t, k, seed, stream_base, z_u, z_v, stream=None):
    """One Section 3.1 estimate of the squared row / column norms of D A E at (u, v) into z_u, z_v."""
    _check(load().sme_estimate(op, _ptr(u), _ptr(v), int(t), int(k), int(seed), int(stream_base), _ptr(z_u),
                               _ptr(z_v), _stream(stream)), "sme_estimate")


def sme_evaluate(op, u, v, alpha=0.0, beta=0.0, gamma=0.0, r2=None, c2=None, stream=None) -> dict:
    """Exact squared row / column norms of D A E (FP64) and the spread, RMS error and objective, as a dict."""
    res = sme_eval_result()
    _check(load().sme_evaluate(op, _ptr(u), _ptr(v), float(alpha), float(beta), float(gamma), _ptr(r2), _ptr(c2),
                               ctypes.byref(res), _stream(stream)), "sme_evaluate")
    return {f: getattr(res, f) for f, _ in sme_eval_result._fields_}


def sme_lsqr(op, u_bar, v_bar, b, x, *, tol=1e-6, max_iters=100000, check_every=10, stop_rule=0, stream=None,
             raise_on_not_converged=False, history=False, predict_check=False) -> dict:
    """LSQR on D A E (Section 5.1).  With history=True the result's "history" lists the checked residual
    at every check (every check_every iterations, or earlier ones with predict_check)."""
    cap = (int(max_iters) + 1) if history and predict_check else \
        ((int(max_iters) // max(1, int(check_every)) + 1) if history else 0)
    hist = np.zeros(max(cap, 1))
    p = sme_lsqr_params(float(tol), int(max_iters), int(check_every), int(stop_rule),
                        ctypes.c_void_p(hist.ctypes.data) if cap else None, cap, 1 if predict_check else 0)
    res = sme_lsqr_result()
    st = load().sme_lsqr(op, _ptr(u_bar), _ptr(v_bar), _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(res),
                         _stream(stream))
    if st != -7 or raise_on_not_converged:
        _check(st, "sme_lsqr")
    out = {f: getattr(res, f) for f, _ in sme_lsqr_result._fields_}
    if history:
        out["history"] = list(hist[:res.history_count])
    return out


def _check_static_args(m, n, row_ptr, col_idx, vals, u, v, z_u):
    """The C side sees raw pointers only: check dtypes, device, contiguity and lengths here."""
    import torch

    named = dict(row_ptr=(row_ptr, torch.int32, m + 1), col_idx=(col_idx, torch.int32, None),
                 vals=(vals, torch.float32, None), u=(u, torch.float32, m), v=(v, torch.float32, n),
                 z_u=(z_u, torch.float32, m))
    devices = set()
    for name, (x, dt, length) in named.items():
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise SmeError(-1, "sme_estimate_rows_static", f"{name} must be a CUDA tensor")
        if x.dtype != dt:
            raise SmeError(-1, "sme_estimate_rows_static", f"{name} must be {dt}, got {x.dtype}")
        if not x.is_contiguous():
            raise SmeError(-1, "sme_estimate_rows_static", f"{name} must be contiguous")
        if length is not None and x.numel() != length:
            raise SmeError(-1, "sme_estimate_rows_static", f"{name} has {x.numel()} elements, expected {length}")
        devices.add(x.device)
    if col_idx.numel() != vals.numel():
        raise SmeError(-1, "sme_estimate_rows_static", "col_idx and vals differ in length")
    if len(devices) != 1:
        raise SmeError(-1, "sme_estimate_rows_static", "arguments on more than one device")


def sme_estimate_rows_static(m, n, row_ptr, col_idx, vals, u, v, t, k, seed, stream_base, z_u, stream=None):
    """Row estimate without any device allocation (see include/sme.h); all arguments are CUDA tensors."""
    _check_static_args(int(m), int(n), row_ptr, col_idx, vals, u, v, z_u)
    _check(load().sme_estimate_rows_static(int(m), int(n), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(u), _ptr(v),
                                           int(t), int(k), int(seed), int(stream_base), _ptr(z_u), _stream(stream)),
           "sme_estimate_rows_static")


def sme_batch_create(mats, dtype=None, stream=None):
    """Create a batch from a list of CSR matrices (objects with m, n, row_ptr, col_idx, vals; host NumPy)."""
    if dtype is None:
        dtype = SME_F64 if mats[0].vals.dtype == np.float64 else SME_F32
    vt = np.float64 if dtype == SME_F64 else np.float32
    keep = []
    B = len(mats)
    ms = np.array([A.m for A in mats], np.int64)
    ns = np.array([A.n for A in mats], np.int64)
    rps = (ctypes.c_void_p * B)()
    cis = (ctypes.c_void_p * B)()
    vas = (ctypes.c_void_p * B)()
    for i, A in enumerate(mats):
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
        va = np.ascontiguousarray(A.vals, dtype=vt)
        keep += [rp, ci, va]
        rps[i], cis[i], vas[i] = rp.ctypes.data, ci.ctypes.data, va.ctypes.data
    b = ctypes.c_void_p()
    st = load().sme_batch_create(ctypes.byref(b), B, _ptr(ms), _ptr(ns), ctypes.cast(rps, ctypes.c_void_p),
                                 ctypes.cast(cis, ctypes.c_void_p), ctypes.cast(vas, ctypes.c_void_p), int(dtype),
                                 _stream(stream))
    _check(st, "sme_batch_create")
    return b


def sme_batch_destroy(b):
    """Destroy a batch and its block-diagonal operator."""
    if b:
        _check(load().sme_batch_destroy(b), "sme_batch_destroy")


def sme_batch_get_info(b):
    """(count, row offsets, column offsets) of the matrices in a batch."""
    count = ctypes.c_int32()
    _check(load().sme_batch_get_info(b, ctypes.byref(count), None, None), "sme_batch_get_info")
    ro = np.zeros(count.value + 1, np.int64)
    co = np.zeros(count.value + 1, np.int64)
    _check(load().sme_batch_get_info(b, None, _ptr(ro), _ptr(co)), "sme_batch_get_info")
    return count.value, ro, co


def sme_batch_equilibrate(b, u, v, u_bar, v_bar, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0, alpha=0.0,
                          beta=0.0, gamma=0.0, M=0.0, flags=0, stream=None):
    """Algorithm 1 for every matrix of a batch at once (per-matrix targets and probe streams)."""
    p = sme_equil_params(alpha, beta, gamma, M, int(T), int(k), int(t_begin), int(t0), int(seed), int(stream_base),
                         int(flags))
    _check(load().sme_batch_equilibrate(b, ctypes.byref(p), _ptr(u), _ptr(v), _ptr(u_bar), _ptr(v_bar),
                                        _stream(stream)), "sme_batch_equilibrate")


def sme_batch_estimate(b, u, v, t, k, seed, stream_base, z_u, z_v, stream=None):
    """One estimate for every matrix of a batch (probe streams stream_base + 2b, + 2b + 1)."""
    _check(load().sme_batch_estimate(b, _ptr(u), _ptr(v), int(t), int(k), int(seed), int(stream_base), _ptr(z_u),
                                     _ptr(z_v), _stream(stream)), "sme_batch_estimate")


def sme_batch_op(b):
    """The batch's block-diagonal operator (owned by the batch), for calls that take an operator."""
    op = ctypes.c_void_p()
    _check(load().sme_batch_op(b, ctypes.byref(op)), "sme_batch_op")
    return op


def sme_op_autotune(op, k, stream=None) -> dict:
    """Time the launch shapes of the iteration kernel for k on this operator and keep the fastest."""
    spc, cf, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().sme_op_autotune(op, int(k), ctypes.byref(spc), ctypes.byref(cf), ctypes.byref(ms), _stream(stream)),
           "sme_op_autotune")
    return {"slices_per_cta": spc.value, "cols_first": cf.value, "ms_per_iteration": ms.value}


def sme_batch_lsqr(b, u_bar, v_bar, bvec, x, *, tol=1e-6, max_iters=100000, check_every=10, stop_rule=0, stream=None,
                   raise_on_not_converged=False):
    """Per-matrix LSQR over a batch; returns a list of per-matrix result dicts."""
    count = sme_batch_get_info(b)[0]
    p = sme_lsqr_params(float(tol), int(max_iters), int(check_every), int(stop_rule), None, 0)
    res = (sme_lsqr_result * count)()
    st = load().sme_batch_lsqr(b, _ptr(u_bar), _ptr(v_bar), _ptr(bvec), _ptr(x), ctypes.byref(p),
                               ctypes.cast(res, ctypes.c_void_p), _stream(stream))
    if st != -7 or raise_on_not_converged:
        _check(st, "sme_batch_lsqr")
    return [{f: getattr(r, f) for f, _ in sme_lsqr_result._fields_} for r in res]


def _params(T, k, t_begin, t0, seed, stream_base, alpha, beta, gamma, M, flags):
    return sme_equil_params(alpha, beta, gamma, M, int(T), int(k), int(t_begin), int(t0), int(seed), int(stream_base),
                            int(flags))


def sme_equilibrate_targets(op, row_targets_sq, col_targets_sq, u, v, u_bar, v_bar, *, T, k, t_begin=1, t0=0, seed=0,
                            stream_base=0, gamma=0.0, M=0.0, flags=0, stream=None):
    """Section 6 varying norms: squared row / column targets in place of alpha^2, beta^2."""
    p = _params(T, k, t_begin, t0, seed, stream_base, 0.0, 0.0, gamma, M, flags)
    _check(load().sme_equilibrate_targets(op, ctypes.byref(p), _ptr(row_targets_sq), _ptr(col_targets_sq), _ptr(u),
                                          _ptr(v), _ptr(u_bar), _ptr(v_bar), _stream(stream)),
           "sme_equilibrate_targets")


def sme_equilibrate_symmetric(op, u, u_bar, *, T, k, t_begin=1, t0=0, seed=0, stream_base=0, alpha=0.0, gamma=0.0,
                              M=0.0, flags=0, stream=None):
    """Algorithm 2: one scaling u for a symmetric operator."""
    p = _params(T, k, t_begin, t0, seed, stream_base, alpha, alpha, gamma, M, flags)
    _check(load().sme_equilibrate_symmetric(op, ctypes.byref(p), _ptr(u), _ptr(u_bar), _stream(stream)),
           "sme_equilibrate_symmetric")


def sme_equilibrate_block(op, row_block_ptr, col_block_ptr, u, v, u_bar, v_bar, *, T, k, t_begin=1, t0=0, seed=0,
                          stream_base=0, alpha=0.0, beta=0.0, gamma=0.0, M=0.0, flags=0, stream=None):
    """Section 6 block equilibration: one log-scaling per contiguous row block and column block."""
    rb = np.ascontiguousarray(row_block_ptr, dtype=np.int64)
    cb = np.ascontiguousarray(col_block_ptr, dtype=np.int64)
    p = _params(T, k, t_begin, t0, seed, stream_base, alpha, beta, gamma, M, flags)
    _check(load().sme_equilibrate_block(op, ctypes.byref(p), rb.size - 1, _ptr(rb), cb.size - 1, _ptr(cb), _ptr(u),
                                        _ptr(v), _ptr(u_bar), _ptr(v_bar), _stream(stream)), "sme_equilibrate_block")


def sme_mlp_create(seed=0):
    """Create the warm-start network (8 -> 128 -> 128 -> 1) with seeded initial weights."""
    h = ctypes.c_void_p()
    _check(load().sme_mlp_create(ctypes.byref(h), int(seed)), "sme_mlp_create")
    return h


def sme_mlp_destroy(mlp):
    """Destroy a warm-start network."""
    if mlp:
        _check(load().sme_mlp_destroy(mlp), "sme_mlp_destroy")


def sme_mlp_param_count() -> int:
    """Number of FP32 parameters of the warm-start network."""
    return int(load().sme_mlp_param_count())


def sme_mlp_get_params(mlp):
    """(parameters, input normalisation) of a network as NumPy arrays."""
    p = np.zeros(sme_mlp_param_count(), np.float32)
    nrm = np.zeros(16, np.float32)
    _check(load().sme_mlp_get_params(mlp, _ptr(p), _ptr(nrm)), "sme_mlp_get_params")
    return p, nrm


def sme_mlp_set_params(mlp, params=None, norm=None):
    """Set a network's parameters and / or its input normalisation."""
    p = None if params is None else np.ascontiguousarray(params, np.float32)
    nrm = None if norm is None else np.ascontiguousarray(norm, np.float32)
    _check(load().sme_mlp_set_params(mlp, _ptr(p), _ptr(nrm)), "sme_mlp_set_params")


def sme_mlp_forward(mlp, X, y, stream=None):
    """Network outputs y for the feature rows X (CUDA tensors)."""
    _check(load().sme_mlp_forward(mlp, _ptr(X), int(X.shape[0]), _ptr(y), _stream(stream)), "sme_mlp_forward")


def sme_mlp_gradient(mlp, X, target, grad=None, stream=None):
    """Mean squared-error loss and its gradient for (X, target); returns the loss."""
    loss = ctypes.c_float()
    _check(load().sme_mlp_gradient(mlp, _ptr(X), _ptr(target), int(X.shape[0]), _ptr(grad), ctypes.byref(loss),
                                   _stream(stream)), "sme_mlp_gradient")
    return loss.value


def sme_mlp_train_step(mlp, X, target, lr, stream=None, want_loss=False):
    """One Adam step on (X, target) with learning rate lr; optionally returns the loss."""
    loss = ctypes.c_float()
    _check(load().sme_mlp_train_step(mlp, _ptr(X), _ptr(target), int(X.shape[0]), float(lr),
                                     ctypes.byref(loss) if want_loss else None, _stream(stream)), "sme_mlp_train_step")
    return loss.value if want_loss else None


def sme_mlp_fit_normalisation(mlp, X, stream=None):
    """Set a network's input normalisation to the mean and deviation of the feature rows X (CUDA tensor)."""
    _check(load().sme_mlp_fit_normalisation(mlp, _ptr(X), int(X.shape[0]), _stream(stream)),
           "sme_mlp_fit_normalisation")


def sme_mlp_draw_batch(X, target, batch, seed, step, X_batch, target_batch, stream=None):
    """Fill (X_batch, target_batch) with `batch` rows of (X, target) drawn with replacement (library kernel)."""
    _check(load().sme_mlp_draw_batch(_ptr(X), _ptr(target), int(X.shape[0]), int(batch), int(seed), int(step),
                                     _ptr(X_batch), _ptr(target_batch), _stream(stream)), "sme_mlp_draw_batch")


def sme_op_features(op, seed, row_features, col_features, stream=None):
    """The 8 warm-start features of every row and column of an operator."""
    _check(load().sme_op_features(op, int(seed), _ptr(row_features), _ptr(col_features), _stream(stream)),
           "sme_op_features")


def sme_warm_start(op, mlp, seed, u0, v0, stream=None):
    """u0, v0 = network(features) for an operator."""
    _check(load().sme_warm_start(op, mlp, int(seed), _ptr(u0), _ptr(v0), _stream(stream)), "sme_warm_start")


def sme_batch_evaluate(b, u, v, alpha=0.0, beta=0.0, gamma=0.0, stream=None):
    """Per-matrix evaluation of a batch; returns a list of dicts like sme_evaluate's."""
    count = sme_batch_get_info(b)[0]
    res = (sme_eval_result * count)()
    _check(load().sme_batch_evaluate(b, _ptr(u), _ptr(v), float(alpha), float(beta), float(gamma),
                                     ctypes.cast(res, ctypes.c_void_p), _stream(stream)), "sme_batch_evaluate")
    return [{f: getattr(r, f) for f, _ in sme_eval_result._fields_} for r in res]


def sme_batch_features(b, seed, row_features, col_features, stream=None):
    """The warm-start features of every matrix of a batch."""
    _check(load().sme_batch_features(b, int(seed), _ptr(row_features), _ptr(col_features), _stream(stream)),
           "sme_batch_features")


def sme_batch_warm_start(b, mlp, seed, u0, v0, stream=None):
    """u0, v0 = network(features) for every matrix of a batch."""
    _check(load().sme_batch_warm_start(b, mlp, int(seed), _ptr(u0), _ptr(v0), _stream(stream)),
           "sme_batch_warm_start")


def sme_op_norm2(op, u_bar=None, v_bar=None, iters=100, stream=None) -> float:
    """||D A E||_2 by power iteration (the CCP step sizes of Section 5.2)."""
    out = ctypes.c_double()
    _check(load().sme_op_norm2(op, _ptr(u_bar), _ptr(v_bar), int(iters), ctypes.byref(out), _stream(stream)),
           "sme_op_norm2")
    return out.value


def sme_ccp_lasso(op, u_bar, v_bar, b, x, *, lam, max_iters, check_every=10, tau=0.0, sigma=0.0, theta=0.0,
                  norm_iters=0, p_star=0.0, tol=0.0, history=True, stream=None):
    """Section 5.2's Lasso by Chambolle-Cremers-Pock; returns (result dict, objective history list)."""
    p = sme_ccp_params(float(lam), float(tau), float(sigma), float(theta), int(max_iters), int(check_every),
                       int(norm_iters), float(p_star), float(tol))
    res = sme_ccp_result()
    cap = (int(max_iters) // max(1, int(check_every)) + 2) if history else 0
    hist = np.zeros(max(cap, 1))
    _check(load().sme_ccp_lasso(op, _ptr(u_bar), _ptr(v_bar), _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(res),
                                _ptr(hist) if cap else None, cap, _stream(stream)), "sme_ccp_lasso")
    out = {f: getattr(res, f) for f, _ in sme_ccp_result._fields_}
    return out, list(hist[:res.history_count])
