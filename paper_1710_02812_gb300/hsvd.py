"""Thin ctypes binding of libhsvd (include/hsvd.h).

Only argument marshalling lives here: every step of the path runs in the
CUDA kernels of the shared library.  PyTorch supplies device memory and
streams.  If the library has not been built the first call raises; there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhsvd.so")

HSVD_OK, HSVD_EINVAL, HSVD_ENOMEM, HSVD_ECUDA, HSVD_ENOTREADY, HSVD_EUNSUPPORTED = range(6)
TRUNC = {"fixed_k": 0, "gamma": 1, "energy": 2}
TREE = {"col_then_row": 0, "row_then_col": 1}
PREC = {"f64": 0, "f32": 1, "bf16_mixed": 2}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2}
WHERE = {"host": 0, "device": 1}

EXPORTED = ("hsvd_plan", "hsvd_run", "hsvd_run_host", "hsvd_status_query", "hsvd_factors",
            "hsvd_workspace_bytes", "hsvd_launches_per_run", "hsvd_destroy", "hsvd_error_string",
            "hsvd_tree_levels", "hsvd_jacobi_pair", "hsvd_step_count", "hsvd_step_info",
            "hsvd_set_timing", "hsvd_step_times", "hsvd_block_svd_noalloc", "hsvd_last_error",
            "hsvd_refine", "hsvd_gram", "hsvd_tree_root", "hsvd_merge_plan", "hsvd_merge_run",
            "hsvd_recover_begin", "hsvd_recover_orth", "hsvd_recover_core", "hsvd_recover_signs",
            "hsvd_recover_finish", "hsvd_step_variant", "hsvd_jacobi_block_order")
STEP_KIND = {1: "gemm_nn", 2: "gemm_tn", 3: "gemm_reduce", 4: "chol", 5: "jacobi", 6: "energy", 7: "signs",
             8: "gemm_tc", 9: "convert"}


class HsvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (status {code})")


class Options(ctypes.Structure):
    _fields_ = [("oversample", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("rank_tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("max_sweeps", ctypes.c_int32), ("host_staging", ctypes.c_int32),
                ("stop_after_rows", ctypes.c_int32), ("autotune", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("not_converged", ctypes.c_int32), ("chol_dropped", ctypes.c_int32),
                ("nonfinite", ctypes.c_int32), ("min_rank", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32),
                ("jacobi_cores", ctypes.c_int32), ("tensor_timeouts", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib_handle = None


def lib():
    """Load libhsvd.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.hsvd_plan.argtypes = [ctypes.POINTER(P), i32, ctypes.POINTER(i64), ctypes.POINTER(i64), i64, i64,
                                ctypes.c_int, dbl, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(Options)]
        L.hsvd_plan.restype = ctypes.c_int
        L.hsvd_run.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(i64), P]
        L.hsvd_run.restype = ctypes.c_int
        L.hsvd_run_host.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(i64), P]
        L.hsvd_run_host.restype = ctypes.c_int
        L.hsvd_status_query.argtypes = [P, i32, ctypes.POINTER(Report)]
        L.hsvd_status_query.restype = ctypes.c_int
        L.hsvd_factors.argtypes = [P, i32, ctypes.POINTER(i32), P, i64, P, P, i64, ctypes.c_int, P]
        L.hsvd_factors.restype = ctypes.c_int
        L.hsvd_workspace_bytes.argtypes = [P]
        L.hsvd_workspace_bytes.restype = i64
        L.hsvd_launches_per_run.argtypes = [P]
        L.hsvd_launches_per_run.restype = i32
        L.hsvd_destroy.argtypes = [P]
        L.hsvd_destroy.restype = None
        L.hsvd_error_string.argtypes = [ctypes.c_int]
        L.hsvd_error_string.restype = ctypes.c_char_p
        L.hsvd_tree_levels.argtypes = [i64]
        L.hsvd_tree_levels.restype = i32
        L.hsvd_jacobi_pair.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.hsvd_jacobi_pair.restype = ctypes.c_int
        L.hsvd_jacobi_block_order.argtypes = [i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.hsvd_jacobi_block_order.restype = ctypes.c_int
        L.hsvd_step_count.argtypes = [P]
        L.hsvd_step_count.restype = i32
        L.hsvd_step_info.argtypes = [P, i32, ctypes.c_char_p, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        L.hsvd_step_info.restype = ctypes.c_int
        L.hsvd_set_timing.argtypes = [P, i32]
        L.hsvd_set_timing.restype = ctypes.c_int
        L.hsvd_step_times.argtypes = [P, ctypes.POINTER(dbl), i32, ctypes.POINTER(i32)]
        L.hsvd_step_times.restype = ctypes.c_int
        L.hsvd_block_svd_noalloc.argtypes = [P, i64, i32, i32, i32, i32, P, i64, P, P, P, P]
        L.hsvd_block_svd_noalloc.restype = ctypes.c_int
        L.hsvd_last_error.argtypes = [P]
        L.hsvd_last_error.restype = ctypes.c_char_p
        L.hsvd_refine.argtypes = [P, i32, ctypes.c_double, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), P]
        L.hsvd_refine.restype = ctypes.c_int
        L.hsvd_gram.argtypes = [P, i64, i64, i64, ctypes.c_int, P, i64, P]
        L.hsvd_gram.restype = ctypes.c_int
        L.hsvd_tree_root.argtypes = [P, i32, ctypes.POINTER(i32), P, i64, P, P]
        L.hsvd_merge_plan.argtypes = [ctypes.POINTER(P), i64, i32, ctypes.c_int, dbl, ctypes.c_int,
                                      ctypes.POINTER(Options)]
        L.hsvd_merge_run.argtypes = [P, P, i64, P, i32, P, i64, P, i32, P]
        L.hsvd_recover_begin.argtypes = [P, P, i64, i32, P, P]
        L.hsvd_recover_orth.argtypes = [P, P, P, P]
        L.hsvd_recover_core.argtypes = [P, P, P, P]
        L.hsvd_recover_signs.argtypes = [P, P, i64, P, P]
        L.hsvd_recover_finish.argtypes = [P, P, P]
        L.hsvd_step_variant.argtypes = [P, i32, ctypes.c_char_p, i32, ctypes.POINTER(i32)]
        L.hsvd_step_variant.restype = ctypes.c_int
        for f in ("hsvd_tree_root", "hsvd_merge_plan", "hsvd_merge_run", "hsvd_recover_begin",
                  "hsvd_recover_orth", "hsvd_recover_core", "hsvd_recover_signs", "hsvd_recover_finish"):
            getattr(L, f).restype = ctypes.c_int
        _lib_handle = L
    return _lib_handle


def error_string(code: int) -> str:
    return lib().hsvd_error_string(code).decode()


def _check(code: int, where: str):
    if code != HSVD_OK:
        raise HsvdError(code, where)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ argument checks
# The C ABI receives raw pointers: the kernels read m x n elements of the
# planned type from each input and write kcap-column factors, so a buffer of
# the wrong size or element type would be read or written past its end.  The
# binding checks what the C side cannot see before any call.

def _torch_dtype(name: str):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[name]


def check_inputs(mats, ms, ns, in_dtype: str, device: bool) -> None:
    """Inputs of hsvd_run (device=True: CUDA tensors) or hsvd_run_host
    (device=False: numpy arrays or CPU tensors): one 2-D matrix per planned
    matrix, of the planned shape and element type, with contiguous rows."""
    import torch
    if len(mats) != len(ms):
        raise ValueError(f"{len(mats)} matrices given, the plan holds {len(ms)}")
    want = _torch_dtype(in_dtype)
    for i, (t, m, n) in enumerate(zip(mats, ms, ns)):
        if isinstance(t, np.ndarray):
            if device:
                raise TypeError(f"matrix {i}: hsvd_run reads device memory; pass a CUDA tensor")
            if t.ndim != 2 or t.shape != (m, n):
                raise ValueError(f"matrix {i}: shape {t.shape}, the plan expects {(m, n)}")
            if in_dtype == "bf16" or t.dtype != np.dtype(np.float64 if in_dtype == "f64" else np.float32):
                raise TypeError(f"matrix {i}: dtype {t.dtype}, the plan expects {want}")
            if (n > 1 and t.strides[1] != t.itemsize) or (m > 1 and t.strides[0] < n * t.itemsize):
                raise ValueError(f"matrix {i}: rows must be contiguous (strides {t.strides})")
            continue
        if not isinstance(t, torch.Tensor) or t.dim() != 2:
            raise TypeError(f"matrix {i}: a 2-D tensor is required")
        if tuple(t.shape) != (m, n):
            raise ValueError(f"matrix {i}: shape {tuple(t.shape)}, the plan expects {(m, n)}")
        if t.dtype != want:
            raise TypeError(f"matrix {i}: dtype {t.dtype}, the plan expects {want}")
        if (n > 1 and t.stride(1) != 1) or (m > 1 and t.stride(0) < n):
            raise ValueError(f"matrix {i}: rows must be contiguous (strides {t.stride()})")
        if t.is_cuda != device:
            raise ValueError(f"matrix {i}: " + ("hsvd_run reads device memory; pass a CUDA tensor" if device
                                                else "hsvd_run_host reads host memory; pass a CPU array"))


def check_factor_outputs(U, S, V, kcap: int, m: int, n: int, factor_dtype: str) -> None:
    """Device outputs of hsvd_factors: contiguous CUDA tensors of the factor
    type holding at least kcap x m (U), kcap (S) and kcap x n (V) elements."""
    import torch
    want = _torch_dtype(factor_dtype)
    for name, t, need in (("U", U, kcap * m), ("S", S, kcap), ("V", V, kcap * n)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name}: a CUDA tensor is required")
        if t.dtype != want:
            raise TypeError(f"{name}: dtype {t.dtype}, the plan's factors are {want}")
        if not t.is_contiguous() or t.numel() < need:
            raise ValueError(f"{name}: a contiguous tensor of at least {need} elements is required")


# ------------------------------------------------------------------ C names

def hsvd_plan(m: Sequence[int], n: Sequence[int], block_rows: int, block_cols: int, mode: str = "fixed_k",
              param: float = 10, rank_cap: int = 256, tree: str = "col_then_row", prec: str = "f32",
              in_dtype: Optional[str] = None, options: Optional[Options] = None) -> ctypes.c_void_p:
    """hsvd_plan(): returns the plan handle; raises HsvdError on failure."""
    m = [int(v) for v in m]
    n = [int(v) for v in n]
    if len(m) != len(n):
        raise ValueError("m and n must have the same length")
    if in_dtype is None:
        in_dtype = {"f64": "f64", "f32": "f32", "bf16_mixed": "f32"}[prec]
    h = ctypes.c_void_p()
    ma = (ctypes.c_int64 * max(1, len(m)))(*m)
    na = (ctypes.c_int64 * max(1, len(n)))(*n)
    code = lib().hsvd_plan(ctypes.byref(h), len(m), ma, na, int(block_rows), int(block_cols), TRUNC[mode],
                           float(param), int(rank_cap), TREE[tree], PREC[prec], DTYPE[in_dtype],
                           ctypes.byref(options) if options is not None else None)
    _check(code, "hsvd_plan")
    return h


def hsvd_run(plan, ptrs: Sequence[int], lda: Sequence[int], stream=None):
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    ld = (ctypes.c_int64 * len(lda))(*[int(v) for v in lda])
    code = lib().hsvd_run(plan, arr, ld, _stream_ptr(stream))
    if code != HSVD_OK:
        raise HsvdError(code, "hsvd_run" + _detail(plan))


def hsvd_run_host(plan, ptrs: Sequence[int], lda: Sequence[int], stream=None):
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    ld = (ctypes.c_int64 * len(lda))(*[int(v) for v in lda])
    code = lib().hsvd_run_host(plan, arr, ld, _stream_ptr(stream))
    if code != HSVD_OK:
        raise HsvdError(code, "hsvd_run_host" + _detail(plan))


def hsvd_refine(plan, max_iters: int, eps: float, stream=None):
    it, err = ctypes.c_int32(), ctypes.c_double()
    code = lib().hsvd_refine(plan, int(max_iters), float(eps), ctypes.byref(it), ctypes.byref(err),
                             _stream_ptr(stream))
    if code != HSVD_OK:
        raise HsvdError(code, "hsvd_refine" + _detail(plan))
    return it.value, err.value


def hsvd_gram(X, G, stream=None):
    """G = X^T X on the device (torch tensors: X m x n, G n x n, both float32 or
    both float64, row-major with unit column stride)."""
    import torch
    if X.dim() != 2 or G.dim() != 2:
        raise TypeError("X and G must be 2-D tensors")
    if X.dtype != G.dtype or X.dtype not in (torch.float32, torch.float64):
        raise TypeError("X and G must both be float32 or both float64")
    m, n = X.shape
    if tuple(G.shape) != (n, n):
        raise ValueError(f"G must be {n} x {n} for X of {m} x {n}, got {tuple(G.shape)}")
    if X.stride(1) != 1 or G.stride(1) != 1 or X.stride(0) < n or G.stride(0) < n:
        raise ValueError("rows must be contiguous")
    if not (X.is_cuda and G.is_cuda):
        raise ValueError("X and G must be CUDA tensors")
    prec = PREC["f64"] if X.dtype == torch.float64 else PREC["f32"]
    _check(lib().hsvd_gram(X.data_ptr(), X.stride(0), m, n, prec, G.data_ptr(), G.stride(0), _stream_ptr(stream)),
           "hsvd_gram")


def hsvd_last_error(plan) -> str:
    return (lib().hsvd_last_error(plan) or b"").decode()


def _detail(plan) -> str:
    d = hsvd_last_error(plan)
    return f" [{d}]" if d else ""


def hsvd_status_query(plan, sync: bool = True) -> dict:
    r = Report()
    _check(lib().hsvd_status_query(plan, 1 if sync else 0, ctypes.byref(r)), "hsvd_status_query")
    return r.as_dict()


def hsvd_factors(plan, idx, rank_p, U, ldu, S, V, ldv, where, stream):
    return lib().hsvd_factors(plan, idx, rank_p, U, ldu, S, V, ldv, where, stream)


def hsvd_workspace_bytes(plan) -> int:
    return int(lib().hsvd_workspace_bytes(plan))


def hsvd_launches_per_run(plan) -> int:
    return int(lib().hsvd_launches_per_run(plan))


def hsvd_destroy(plan):
    lib().hsvd_destroy(plan)


def hsvd_step_count(plan) -> int:
    return int(lib().hsvd_step_count(plan))


def hsvd_step_info(plan, i: int) -> dict:
    name = ctypes.create_string_buffer(96)
    kind, tasks, dim = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(lib().hsvd_step_info(plan, i, name, 96, ctypes.byref(kind), ctypes.byref(tasks), ctypes.byref(dim),
                                ctypes.byref(fl), ctypes.byref(by)), "hsvd_step_info")
    return {"name": name.value.decode(), "kind": STEP_KIND.get(kind.value, "other"), "tasks": tasks.value,
            "dim": dim.value, "flops": fl.value, "bytes": by.value}


def hsvd_set_timing(plan, on):
    """on: False/0 off, True/1 every step, 2 core-SVD steps only."""
    mode = on if (isinstance(on, int) and not isinstance(on, bool)) else (1 if on else 0)
    _check(lib().hsvd_set_timing(plan, mode), "hsvd_set_timing")


def hsvd_step_times(plan):
    n = hsvd_step_count(plan)
    arr = (ctypes.c_double * max(1, n))()
    runs = ctypes.c_int32()
    _check(lib().hsvd_step_times(plan, arr, n, ctypes.byref(runs)), "hsvd_step_times")
    return [arr[i] for i in range(n)], runs.value


def hsvd_tree_levels(count: int) -> int:
    return int(lib().hsvd_tree_levels(int(count)))


def hsvd_jacobi_pair(n: int, rnd: int, slot: int):
    p, q = ctypes.c_int32(), ctypes.c_int32()
    code = lib().hsvd_jacobi_pair(n, rnd, slot, ctypes.byref(p), ctypes.byref(q))
    if code != HSVD_OK:
        raise HsvdError(code, "hsvd_jacobi_pair")
    return p.value, q.value


def hsvd_jacobi_block_order(what: int, phase: int, i: int, j: int):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    code = lib().hsvd_jacobi_block_order(what, phase, i, j, ctypes.byref(a), ctypes.byref(b))
    if code != HSVD_OK:
        raise HsvdError(code, "hsvd_jacobi_block_order")
    return a.value, b.value


def check_noalloc_args(A, m, n, k, U, S, rank, flags=None, lda=None, ldu=None, require_cuda=True) -> None:
    """Arguments of hsvd_block_svd_noalloc, checked before the call: the C
    side sees raw pointers and would read past A or write past U, S, rank or
    flags if they were too small or of the wrong type.  A is a 2-D float32
    (m, n) tensor with unit column stride and row stride >= n (or lda); U a
    contiguous float32 tensor of at least k * ldu elements (column-major
    m x k, ldu >= m); S float32 with at least k elements; rank and flags
    int32 with at least one element.  require_cuda=False skips the device
    check (the shape and type checks run without a GPU)."""
    import torch
    for name, t in (("A", A), ("U", U), ("S", S), ("rank", rank), ("flags", flags)):
        if t is None and name == "flags":
            continue
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: a torch tensor is required")
        if require_cuda and not t.is_cuda:
            raise ValueError(f"{name}: a CUDA tensor is required (the entry point reads and writes device memory)")
    m, n, k = int(m), int(n), int(k)
    if A.dim() != 2 or tuple(A.shape) != (m, n):
        raise ValueError(f"A: shape {tuple(A.shape)}, expected {(m, n)}")
    if A.dtype != torch.float32:
        raise TypeError(f"A: dtype {A.dtype}, float32 required")
    lda = A.stride(0) if lda is None else int(lda)
    if (n > 1 and A.stride(1) != 1) or (m > 1 and A.stride(0) < n) or lda < n or (m > 1 and lda != A.stride(0)):
        raise ValueError(f"A: rows must be contiguous with leading dimension >= n (strides {A.stride()}, lda {lda})")
    ldu = m if ldu is None else int(ldu)
    if ldu < m:
        raise ValueError(f"ldu {ldu} < m {m}")
    for name, t, dt, need in (("U", U, torch.float32, k * ldu), ("S", S, torch.float32, k),
                              ("rank", rank, torch.int32, 1), ("flags", flags, torch.int32, 1)):
        if t is None:
            continue
        if t.dtype != dt:
            raise TypeError(f"{name}: dtype {t.dtype}, {dt} required")
        if not t.is_contiguous() or t.numel() < need:
            raise ValueError(f"{name}: a contiguous tensor of at least {need} elements is required")


def hsvd_block_svd_noalloc(A, m, n, k, power_iters, U, S, rank, stream=None, lda=None, ldu=None, flags=None):
    """Rank-k SVD of one block with no device allocation: A (m x n, row
    major), U (column-major m x k storage, e.g. a k x m row-major tensor),
    S (k), rank (one int32) and, optionally, flags (one int32: 1 Jacobi not
    converged, 2 CholeskyQR dropped directions, 4 non-finite values) are CUDA
    tensors; returns the status code."""
    check_noalloc_args(A, m, n, k, U, S, rank, flags, lda, ldu)
    return lib().hsvd_block_svd_noalloc(A.data_ptr(), lda if lda is not None else A.stride(0), m, n, k,
                                        power_iters, U.data_ptr(), ldu if ldu is not None else m, S.data_ptr(),
                                        rank.data_ptr(), flags.data_ptr() if flags is not None else None,
                                        _stream_ptr(stream))


# ------------------------------------------------------------------ wrapper

class Plan:
    """Owning wrapper around an hsvd plan."""

    def __init__(self, m, n, block_rows, block_cols, mode="fixed_k", param=10, rank_cap=None,
                 tree="col_then_row", prec="f32", in_dtype=None, oversample=0, power_iters=0,
                 rank_tol=0.0, seed=0, max_sweeps=0, host_staging=False, stop_after_rows=False,
                 autotune=False):
        if isinstance(m, int):
            m, n = [m], [n]
        if rank_cap is None:
            rank_cap = int(param) if mode == "fixed_k" else 128
        self.m, self.n = list(m), list(n)
        self.prec = prec
        self.in_dtype = in_dtype or {"f64": "f64", "f32": "f32", "bf16_mixed": "f32"}[prec]
        self.rank_cap = int(rank_cap)
        self.kcap = min(self.rank_cap, int(param) if mode == "fixed_k" else self.rank_cap)
        opts = Options(int(oversample), int(power_iters), float(rank_tol), int(seed), int(max_sweeps),
                       1 if host_staging else 0, 1 if stop_after_rows else 0, 1 if autotune else 0)
        self._h = hsvd_plan(self.m, self.n, block_rows, block_cols, mode, param, self.rank_cap, tree, prec,
                            self.in_dtype, opts)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            hsvd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def factor_dtype(self):
        return np.float64 if self.prec == "f64" else np.float32

    def run(self, mats, stream=None):
        """mats: list of CUDA tensors (row-major, contiguous rows)."""
        check_inputs(mats, self.m, self.n, self.in_dtype, device=True)
        ptrs = [t.data_ptr() for t in mats]
        lda = [t.stride(0) for t in mats]
        hsvd_run(self._h, ptrs, lda, stream)

    def run_host(self, arrays, stream=None):
        """arrays: list of host arrays (numpy or CPU tensors)."""
        check_inputs(arrays, self.m, self.n, self.in_dtype, device=False)
        ptrs, lda = [], []
        for a in arrays:
            if isinstance(a, np.ndarray):
                ptrs.append(a.ctypes.data)
                lda.append(a.strides[0] // a.itemsize)
            else:
                ptrs.append(a.data_ptr())
                lda.append(a.stride(0))
        hsvd_run_host(self._h, ptrs, lda, stream)

    def factors(self, idx=0, stream=None):
        """Copy (U, S, V) of matrix idx to host numpy arrays: U is m x r and V
        n x r, returned as views with column-major strides (the library's
        layout; no host-side transposing copy), S has r entries."""
        dt = self.factor_dtype
        m, n, kc = self.m[idx], self.n[idx], self.kcap
        U = np.empty((kc, m), dtype=dt)  # column-major m x kc == row-major kc x m
        V = np.empty((kc, n), dtype=dt)
        S = np.empty(kc, dtype=dt)
        r = ctypes.c_int32()
        code = hsvd_factors(self._h, idx, ctypes.byref(r), U.ctypes.data, m, S.ctypes.data, V.ctypes.data, n,
                            WHERE["host"], _stream_ptr(stream))
        _check(code, "hsvd_factors")
        k = r.value
        return U[:k].T, S[:k], V[:k].T

    def factors_device(self, U, S, V, idx=0, stream=None) -> int:
        """Write column-major factors into device tensors U (kcap x m storage),
        S (kcap), V (kcap x n storage); returns the rank."""
        check_factor_outputs(U, S, V, self.kcap, self.m[idx], self.n[idx], "f64" if self.prec == "f64" else "f32")
        r = ctypes.c_int32()
        code = hsvd_factors(self._h, idx, ctypes.byref(r), U.data_ptr() if U is not None else None, self.m[idx],
                            S.data_ptr() if S is not None else None, V.data_ptr() if V is not None else None,
                            self.n[idx], WHERE["device"], _stream_ptr(stream))
        _check(code, "hsvd_factors")
        return r.value

    # ---- one matrix split over ranks by row bands (a plan made with
    # stop_after_rows=True factors one band up to its row tree)

    def _ftype(self):
        import torch
        return torch.float64 if self.prec == "f64" else torch.float32

    def tree_root(self, V, S, idx=0, stream=None) -> int:
        """Row-tree result of matrix idx into device V (n x kcap column-major:
        a kcap x n row-major tensor) and S (kcap); returns the rank."""
        n = self.n[idx]
        _check_dev(V, self._ftype(), self.kcap * n, "V")
        _check_dev(S, self._ftype(), self.kcap, "S")
        r = ctypes.c_int32()
        _check(lib().hsvd_tree_root(self._h, idx, ctypes.byref(r), V.data_ptr(), n, S.data_ptr(),
                                    _stream_ptr(stream)), "hsvd_tree_root")
        return r.value

    def recover_begin(self, Vhat, r, G, stream=None):
        n, kc = self.n[0], self.kcap
        _check_dev(Vhat, self._ftype(), kc * n, "Vhat")
        _check_dev(G, self._ftype(), kc * kc, "G")
        _check(lib().hsvd_recover_begin(self._h, Vhat.data_ptr(), n, int(r), G.data_ptr(), _stream_ptr(stream)),
               "hsvd_recover_begin" + _detail(self._h))

    def recover_orth(self, Gsum, G2, stream=None):
        kc = self.kcap
        _check_dev(Gsum, self._ftype(), kc * kc, "Gsum")
        _check_dev(G2, self._ftype(), kc * kc, "G2")
        _check(lib().hsvd_recover_orth(self._h, Gsum.data_ptr(), G2.data_ptr(), _stream_ptr(stream)),
               "hsvd_recover_orth" + _detail(self._h))

    def recover_core(self, G2sum, absmax, stream=None):
        kc = self.kcap
        _check_dev(G2sum, self._ftype(), kc * kc, "G2sum")
        _check_dev(absmax, self._ftype(), kc, "absmax")
        _check(lib().hsvd_recover_core(self._h, G2sum.data_ptr(), absmax.data_ptr(), _stream_ptr(stream)),
               "hsvd_recover_core" + _detail(self._h))

    def recover_signs(self, absmax_all, row0, key, stream=None):
        import torch
        kc = self.kcap
        _check_dev(absmax_all, self._ftype(), kc, "absmax_all")
        _check_dev(key, torch.int64, kc, "key")
        _check(lib().hsvd_recover_signs(self._h, absmax_all.data_ptr(), int(row0), key.data_ptr(),
                                        _stream_ptr(stream)), "hsvd_recover_signs" + _detail(self._h))

    def recover_finish(self, key_min, stream=None):
        import torch
        _check_dev(key_min, torch.int64, self.kcap, "key_min")
        _check(lib().hsvd_recover_finish(self._h, key_min.data_ptr(), _stream_ptr(stream)),
               "hsvd_recover_finish" + _detail(self._h))

    def refine(self, max_iters=3, eps=1e-3, stream=None):
        """Alg. 2 on the last run's factors, in place; returns (passes, Error)."""
        return hsvd_refine(self._h, max_iters, eps, stream)

    def status(self, sync=True):
        return hsvd_status_query(self._h, sync)

    @property
    def workspace_bytes(self):
        return hsvd_workspace_bytes(self._h)

    @property
    def launches_per_run(self):
        return hsvd_launches_per_run(self._h)

    def steps(self):
        return [hsvd_step_info(self._h, i) for i in range(hsvd_step_count(self._h))]

    def variants(self):
        """Per step: (name, chosen variant, number of candidates)."""
        out = []
        for i in range(hsvd_step_count(self._h)):
            buf = ctypes.create_string_buffer(96)
            cnt = ctypes.c_int32()
            _check(lib().hsvd_step_variant(self._h, i, buf, 96, ctypes.byref(cnt)), "hsvd_step_variant")
            out.append((hsvd_step_info(self._h, i)["name"], buf.value.decode(), cnt.value))
        return out

    def set_timing(self, on=True):
        hsvd_set_timing(self._h, on)

    def step_times(self):
        return hsvd_step_times(self._h)


def _check_dev(t, dtype, need, name):
    """A contiguous CUDA tensor of the given type holding at least `need`
    elements (the C side reads or writes that many)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: a CUDA tensor is required")
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, {dtype} required")
    if not t.is_contiguous() or t.numel() < need:
        raise ValueError(f"{name}: a contiguous tensor of at least {need} elements is required")


class MergePlan:
    """hsvd_merge_plan: one MAT merge of two factor pairs of height h."""

    def __init__(self, h, mode="fixed_k", param=10, rank_cap=None, prec="f32", rank_tol=0.0, max_sweeps=0):
        if rank_cap is None:
            rank_cap = int(param) if mode == "fixed_k" else 128
        self.h, self.prec = int(h), prec
        self.kcap = min(int(rank_cap), int(param) if mode == "fixed_k" else int(rank_cap))
        opts = Options(0, 0, float(rank_tol), 0, int(max_sweeps), 0, 0, 0)
        hnd = ctypes.c_void_p()
        _check(lib().hsvd_merge_plan(ctypes.byref(hnd), self.h, int(rank_cap), TRUNC[mode], float(param),
                                     PREC[prec], ctypes.byref(opts)), "hsvd_merge_plan")
        self._h = hnd

    def _ftype(self):
        import torch
        return torch.float64 if self.prec == "f64" else torch.float32

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            hsvd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, V1, S1, r1, V2, S2, r2, stream=None):
        """V1, V2: device h x kcap column-major (kcap x h row-major tensors)."""
        for name, t, need in (("V1", V1, self.kcap * self.h), ("V2", V2, self.kcap * self.h),
                              ("S1", S1, max(1, int(r1))), ("S2", S2, max(1, int(r2)))):
            _check_dev(t, self._ftype(), need, name)
        _check(lib().hsvd_merge_run(self._h, V1.data_ptr(), self.h, S1.data_ptr(), int(r1), V2.data_ptr(), self.h,
                                    S2.data_ptr(), int(r2), _stream_ptr(stream)), "hsvd_merge_run" + _detail(self._h))

    def root(self, V, S, stream=None) -> int:
        _check_dev(V, self._ftype(), self.kcap * self.h, "V")
        _check_dev(S, self._ftype(), self.kcap, "S")
        r = ctypes.c_int32()
        _check(lib().hsvd_tree_root(self._h, 0, ctypes.byref(r), V.data_ptr(), self.h, S.data_ptr(),
                                    _stream_ptr(stream)), "hsvd_tree_root")
        return r.value

    def status(self, sync=True):
        return hsvd_status_query(self._h, sync)
