"""GB300-native Gauss-Jordan inversion (arXiv:1401.7962) -- Python binding of the C-ABI library.

The library (``_lib/libgj.so``, built from ``csrc/*.cu`` for sm_103a) does every step of
the inversion in its own CUDA kernels; this module only marshals arguments (pointers,
sizes, strides, streams) into the C entry points declared in ``include/gj.h``.  There
is no CPU fallback: if the library is not built, every call raises ``RuntimeError``.

Matrices are column-major.  A torch tensor or numpy array ``A`` of shape (n, n) is
accepted when its column stride is its leading dimension and its row stride is 1
(``A.t().contiguous().t()`` for torch, ``numpy.asfortranarray`` for numpy).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = ["lib", "invert", "invert_mixed", "invert_batched", "invert_batched_noalloc", "BatchedPlan", "GJError", "colmajor", "status_string",
           "PIVOT_NONE", "PIVOT_PARTIAL", "PIVOT_FULL"]

OK, SINGULAR, ZERO_PIVOT, NONFINITE, NOT_CONVERGED = 0, 1, 2, 3, 4
ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
PIVOT_NONE, PIVOT_PARTIAL, PIVOT_FULL = 0, 1, 2
PATH_AUTO, PATH_CTA, PATH_BLOCKED, PATH_UNBLOCKED, PATH_CLUSTER = 0, 1, 2, 3, 4
BATCHED_WARP4, BATCHED_WARP8, BATCHED_CTA64, BATCHED_CTA128, BATCHED_CTA256, BATCHED_CTA512 = range(6)
BATCHED_NAMES = ["warp4", "warp8", "cta64", "cta128", "cta256", "cta512"]
UPDATE_AUTO, UPDATE_DFMA, UPDATE_TC_OZAKI = 0, 1, 2
PREC_FP64, PREC_BF16, PREC_FP16, PREC_SPLIT_BF16_3, PREC_TF32x3 = 0, 1, 2, 3, 4
PREC_SLICES = {PREC_FP64: 7, PREC_BF16: 1, PREC_FP16: 2, PREC_SPLIT_BF16_3: 2, PREC_TF32x3: 3}


class GJError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {last_error()}".rstrip())


class _Opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("tau", ctypes.c_double), ("panel", ctypes.c_int32),
                ("path", ctypes.c_int32), ("update", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("piv_rows", ctypes.c_void_p), ("piv_cols", ctypes.c_void_p), ("pivots", ctypes.c_void_p),
                ("fail_step", ctypes.c_void_p), ("lookahead", ctypes.c_int32), ("update_sms", ctypes.c_int32)]


class _Peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_gflops", ctypes.c_double), ("fp64_mma_gflops", ctypes.c_double),
                ("fp32_fma_gflops", ctypes.c_double), ("sm_count", ctypes.c_int32), ("max_clock_mhz", ctypes.c_double)]


_LIB = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raises RuntimeError when it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run paper_1401_7962_gb300._build.build()")
    L = ctypes.CDLL(path)
    P, I64, I32, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    L.gj_invert.restype = I
    L.gj_invert.argtypes = [I64, P, I64, P, I, P, P]
    L.gj_invert_ex.restype = I
    L.gj_invert_ex.argtypes = [ctypes.POINTER(_Opts), I64, P, I64, P, I, P, P]
    L.gj_solve.restype = I
    L.gj_solve.argtypes = [I64, I64, P, I64, P, I64, P, I64, I, P, P]
    L.gj_solve_ex.restype = I
    L.gj_solve_ex.argtypes = [ctypes.POINTER(_Opts), I64, I64, P, I64, P, I64, P, I64, I, P, P]
    L.gj_invert_batched.restype = I
    L.gj_invert_batched.argtypes = [I64, I32, P, P, P, I, P, P, P, P]
    L.gj_invert_batched_noalloc.restype = I
    L.gj_invert_batched_noalloc.argtypes = [I64, I32, P, P, P, I, P, P, P, P]
    L.gj_gemm_update_emulated.restype = I
    L.gj_gemm_update_emulated.argtypes = [I64, I64, I64, P, I64, P, I64, P, I64, I, P]
    L.gj_invert_mixed.restype = I
    L.gj_invert_mixed.argtypes = [I64, P, I64, P, I, I, D, I, P, P, P, P, P, P]
    L.gj_invert_mixed_prec.restype = I
    L.gj_invert_mixed_prec.argtypes = [I64, P, I64, P, I, D, I, P, P, P, P, P, P]
    L.gj_invert_mixed_batched.restype = I
    L.gj_invert_mixed_batched.argtypes = [I64, P, P, P, P, I, I, D, I, I, P, P, P, P, P, P, P]
    L.gj_batched_plan_create.restype = I
    L.gj_batched_plan_create.argtypes = [ctypes.POINTER(P), I64, P, I]
    L.gj_batched_plan_create_ex.restype = I
    L.gj_batched_plan_create_ex.argtypes = [ctypes.POINTER(P), I64, P, I, ctypes.c_char_p, I32]
    L.gj_batched_plan_bins.restype = I32
    L.gj_batched_plan_bins.argtypes = [P, P, P, P, P, P, I32]
    L.gj_batched_plan_execute.restype = I
    L.gj_batched_plan_execute.argtypes = [P, P, P, P, P, P, P, I]
    L.gj_batched_plan_destroy.restype = None
    L.gj_batched_plan_destroy.argtypes = [P]
    L.gj_status_string.restype = ctypes.c_char_p
    L.gj_status_string.argtypes = [I]
    L.gj_last_error.restype = ctypes.c_char_p
    L.gj_last_error.argtypes = []
    L.gj_version.restype = ctypes.c_char_p
    L.gj_version.argtypes = []
    L.gj_trim_memory.restype = I
    L.gj_trim_memory.argtypes = []
    L.gj_measure_peaks.restype = I
    L.gj_measure_peaks.argtypes = [ctypes.POINTER(_Peaks)]
    L.gj_set_wait_limit_ns.restype = I
    L.gj_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
    _LIB = L
    return L


def status_string(status: int) -> str:
    return lib().gj_status_string(int(status)).decode()


def last_error() -> str:
    return lib().gj_last_error().decode()


def measure_peaks() -> dict:
    """``gj_measure_peaks``: measured FP64 FMA, FP64 mma.sync and FP32 FMA rates of the current GPU."""
    p = _Peaks()
    st = lib().gj_measure_peaks(ctypes.byref(p))
    if st != OK:
        raise GJError(st, "gj_measure_peaks")
    return {"fp64_fma_gflops": p.fp64_fma_gflops, "fp64_mma_gflops": p.fp64_mma_gflops,
            "fp32_fma_gflops": p.fp32_fma_gflops, "sm_count": p.sm_count, "max_clock_mhz": p.max_clock_mhz}


def set_wait_limit_ns(ns: int) -> None:
    """``gj_set_wait_limit_ns``: limit of the tensor-core update's pipeline waits (0 = 2 s)."""
    lib().gj_set_wait_limit_ns(int(ns))


# ----------------------------------------------------------------- marshalling helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int:
    if x is None:
        return 0
    if _is_torch(x):
        return int(x.data_ptr())
    return int(x.ctypes.data)


def _colmajor_ld(A) -> tuple[int, int]:
    """(n, lda) of a square column-major matrix, or ValueError."""
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square 2-D matrix expected")
    n = int(A.shape[0])
    if _is_torch(A):
        if A.dtype.__repr__() != "torch.float64":
            raise TypeError("float64 matrix expected")
        s0, s1 = A.stride()
    else:
        if str(A.dtype) != "float64":
            raise TypeError("float64 matrix expected")
        s0, s1 = (A.strides[0] // 8, A.strides[1] // 8)
    if n <= 1:
        return n, max(n, 1)
    if s0 != 1 or s1 < n:
        raise ValueError("matrix must be column-major (row stride 1, column stride >= n)")
    return n, int(s1)


def colmajor(A):
    """Column-major copy of a square torch tensor or numpy array (same device)."""
    if _is_torch(A):
        return A.t().contiguous().t()
    import numpy as np
    return np.asfortranarray(A)


def _empty_like_colmajor(A, n):
    if _is_torch(A):
        import torch
        return torch.empty((n, n), dtype=torch.float64, device=A.device).t().contiguous().t() if n else \
            torch.empty((0, 0), dtype=torch.float64, device=A.device)
    import numpy as np
    return np.empty((n, n), dtype=np.float64, order="F")


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def invert(A, pivot_mode: int = PIVOT_PARTIAL, out=None, *, tau: float = 0.0, path: int = PATH_AUTO,
           panel: int = 0, update: int = UPDATE_AUTO, slices: int = 0, stream=None, record: bool = False,
           lookahead: int = 0, update_sms: int = 0):
    """Invert one square matrix with ``gj_invert_ex``.

    ``A`` and ``out`` may live on the host or on the device (the library stages host
    buffers).  Returns a dict: ``X`` (the output array), ``status``, ``det_sign``,
    ``det_log2`` and, with ``record=True``, ``piv_rows``, ``piv_cols``, ``pivots``
    (host numpy arrays) and ``fail_step``.
    """
    import numpy as np
    L = lib()
    n, lda = _colmajor_ld(A)
    if out is None:
        out = _empty_like_colmajor(A, n)
    else:
        no, ldo = _colmajor_ld(out)
        if no != n or (n > 1 and ldo != n):
            raise ValueError("out must be n x n column-major with leading dimension n")
    o = _Opts()
    o.stream = _stream_handle(stream)
    o.tau = float(tau)
    o.panel = int(panel)
    o.path = int(path)
    o.update = int(update)
    o.slices = int(slices)
    o.lookahead = int(lookahead)
    o.update_sms = int(update_sms)
    rec = {}
    fs = ctypes.c_int64(-1)
    if record:
        rec["piv_rows"] = np.full(max(n, 1), -1, dtype=np.int32)
        rec["piv_cols"] = np.full(max(n, 1), -1, dtype=np.int32)
        rec["pivots"] = np.zeros(max(n, 1), dtype=np.float64)
        o.piv_rows = rec["piv_rows"].ctypes.data
        o.piv_cols = rec["piv_cols"].ctypes.data
        o.pivots = rec["pivots"].ctypes.data
    o.fail_step = ctypes.addressof(fs)
    sgn = ctypes.c_int(0)
    lg = ctypes.c_double(0.0)
    st = L.gj_invert_ex(ctypes.byref(o), n, _ptr(A), lda, _ptr(out), int(pivot_mode), ctypes.addressof(sgn),
                        ctypes.addressof(lg))
    if st < 0:
        raise GJError(st, "gj_invert_ex")
    res = {"X": out, "status": st, "det_sign": sgn.value, "det_log2": lg.value, "fail_step": fs.value}
    if record:
        for k in ("piv_rows", "piv_cols", "pivots"):
            res[k] = rec[k][:n].copy()
    return res


def _rhs_ld(B, n) -> tuple[int, int]:
    """(m, ldb) of an n x m column-major float64 array."""
    if B.ndim != 2 or int(B.shape[0]) != n:
        raise ValueError("right-hand sides must be a 2-D array with n rows")
    m = int(B.shape[1])
    if _is_torch(B):
        if B.dtype.__repr__() != "torch.float64":
            raise TypeError("float64 right-hand sides expected")
        s0, s1 = B.stride()
    else:
        if str(B.dtype) != "float64":
            raise TypeError("float64 right-hand sides expected")
        s0, s1 = (B.strides[0] // 8, B.strides[1] // 8)
    ld = max(n, 1)
    if m > 1 and n > 0:
        if (n > 1 and s0 != 1) or s1 < n:
            raise ValueError("right-hand sides must be column-major (row stride 1, column stride >= n)")
        ld = int(s1)
    return m, ld


def solve(A, B, pivot_mode: int = PIVOT_PARTIAL, out=None, *, tau: float = 0.0, path: int = PATH_AUTO,
          panel: int = 0, update: int = UPDATE_AUTO, slices: int = 0, stream=None, record: bool = False,
          lookahead: int = 0):
    """Solve ``A X = B`` with ``gj_solve_ex`` (one Gauss-Jordan sweep of ``[A | B]``).

    ``A`` (n x n) and ``B`` (n x m) column-major float64, host or device; ``out`` (n x m,
    column-major) is allocated like ``B`` when omitted (``out is B`` solves in place).
    Returns a dict: ``X``, ``status``, ``det_sign``, ``det_log2``, ``fail_step`` and, with
    ``record=True``, ``piv_rows``, ``piv_cols``, ``pivots``.
    """
    import numpy as np
    L = lib()
    n, lda = _colmajor_ld(A)
    m, ldb = _rhs_ld(B, n)
    if out is None:
        if _is_torch(B):
            import torch
            out = torch.empty((m, n), dtype=torch.float64, device=B.device).t()
        else:
            out = np.empty((n, m), dtype=np.float64, order="F")
    mo, ldx = _rhs_ld(out, n)
    if mo != m:
        raise ValueError("out must be n x m")
    o = _Opts()
    o.stream = _stream_handle(stream)
    o.tau = float(tau)
    o.panel = int(panel)
    o.path = int(path)
    o.update = int(update)
    o.slices = int(slices)
    o.lookahead = int(lookahead)
    rec = {}
    fs = ctypes.c_int64(-1)
    if record:
        rec["piv_rows"] = np.full(max(n, 1), -1, dtype=np.int32)
        rec["piv_cols"] = np.full(max(n, 1), -1, dtype=np.int32)
        rec["pivots"] = np.zeros(max(n, 1), dtype=np.float64)
        o.piv_rows = rec["piv_rows"].ctypes.data
        o.piv_cols = rec["piv_cols"].ctypes.data
        o.pivots = rec["pivots"].ctypes.data
    o.fail_step = ctypes.addressof(fs)
    sgn = ctypes.c_int(0)
    lg = ctypes.c_double(0.0)
    st = L.gj_solve_ex(ctypes.byref(o), n, m, _ptr(A), lda, _ptr(B) if m else None, ldb, _ptr(out) if m else None,
                       ldx, int(pivot_mode), ctypes.addressof(sgn), ctypes.addressof(lg))
    if st < 0:
        raise GJError(st, "gj_solve_ex")
    res = {"X": out, "status": st, "det_sign": sgn.value, "det_log2": lg.value, "fail_step": fs.value}
    if record:
        for k in ("piv_rows", "piv_cols", "pivots"):
            res[k] = rec[k][:n].copy()
    return res


def invert_mixed(A32, out=None, *, x0_slices: int = 3, corr_slices: int = 4, tol: float = 1e-12,
                 max_iter: int = 10, stream=None) -> dict:
    """``gj_invert_mixed``: FP32 device matrix (column-major) -> FP64 inverse by reduced-precision
    Gauss-Jordan plus Newton-Schulz refinement.  Returns a dict with ``X``, ``status``,
    ``resid``, ``iters``, ``rung``, ``det_sign``, ``det_log2``."""
    L = lib()
    if A32.ndim != 2 or A32.shape[0] != A32.shape[1] or str(A32.dtype) != "torch.float32":
        raise ValueError("square float32 torch tensor expected")
    n = int(A32.shape[0])
    s0, s1 = A32.stride()
    if n > 1 and (s0 != 1 or s1 < n):
        raise ValueError("matrix must be column-major")
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.float64, device=A32.device).t().contiguous().t()
    r, it, rg, sg, lg = ctypes.c_double(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    st = L.gj_invert_mixed(n, _ptr(A32), max(1, int(s1) if n > 1 else 1), _ptr(out), int(x0_slices), int(corr_slices),
                           float(tol), int(max_iter), ctypes.addressof(r), ctypes.addressof(it), ctypes.addressof(rg),
                           ctypes.addressof(sg), ctypes.addressof(lg), _stream_handle(stream))
    if st < 0:
        raise GJError(st, "gj_invert_mixed")
    return {"X": out, "status": st, "resid": r.value, "iters": it.value, "rung": rg.value, "det_sign": sg.value,
            "det_log2": lg.value}


def invert_mixed_prec(A32, prec: int, out=None, *, tol: float = 1e-12, max_iter: int = 10, stream=None) -> dict:
    """``gj_invert_mixed_prec``: as ``invert_mixed`` with the first inverse's arithmetic named by
    a ``PREC_*`` value.  Returns the same dict."""
    L = lib()
    if A32.ndim != 2 or A32.shape[0] != A32.shape[1] or str(A32.dtype) != "torch.float32":
        raise ValueError("square float32 torch tensor expected")
    n = int(A32.shape[0])
    s0, s1 = A32.stride()
    if n > 1 and (s0 != 1 or s1 < n):
        raise ValueError("matrix must be column-major")
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.float64, device=A32.device).t().contiguous().t()
    r, it, rg, sg, lg = ctypes.c_double(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    st = L.gj_invert_mixed_prec(n, _ptr(A32), max(1, int(s1) if n > 1 else 1), _ptr(out), int(prec), float(tol),
                                int(max_iter), ctypes.addressof(r), ctypes.addressof(it), ctypes.addressof(rg),
                                ctypes.addressof(sg), ctypes.addressof(lg), _stream_handle(stream))
    if st < 0:
        raise GJError(st, "gj_invert_mixed_prec")
    return {"X": out, "status": st, "resid": r.value, "iters": it.value, "rung": rg.value, "det_sign": sg.value,
            "det_log2": lg.value}


def invert_mixed_batched(As, Xs=None, *, x0_slices: int = 3, corr_slices: int = 4, tol: float = 1e-12,
                         max_iter: int = 10, workers: int = 0, stream=None) -> dict:
    """``gj_invert_mixed_batched``: a list of square FP32 column-major device matrices -> their FP64
    inverses (``Xs``, allocated when not given).  Returns a dict with ``X`` (the list), the call's
    ``status`` and per-matrix numpy arrays ``statuses``, ``resid``, ``iters``, ``rung``,
    ``det_sign``, ``det_log2``."""
    import numpy as np
    import torch
    L = lib()
    count = len(As)
    ns = np.zeros(max(1, count), dtype=np.int32)
    lds = np.ones(max(1, count), dtype=np.int32)
    if Xs is None:
        Xs = [torch.empty((int(a.shape[0]), int(a.shape[0])), dtype=torch.float64, device=a.device).t().contiguous().t()
              for a in As]
    if len(Xs) != count:
        raise ValueError("As and Xs differ in length")
    for m, (a, x) in enumerate(zip(As, Xs)):
        if a.ndim != 2 or a.shape[0] != a.shape[1] or str(a.dtype) != "torch.float32":
            raise ValueError("square float32 torch tensors expected")
        n = int(a.shape[0])
        if n > 1 and (a.stride(0) != 1 or a.stride(1) < n):
            raise ValueError("matrices must be column-major")
        if tuple(x.shape) != (n, n) or str(x.dtype) != "torch.float64" or (n > 1 and x.stride() != (1, n)):
            raise ValueError("outputs must be column-major float64 (n, n) with leading dimension n")
        ns[m] = n
        lds[m] = max(1, int(a.stride(1)) if n > 1 else 1)
    pa = np.array([_ptr(a) for a in As] or [0], dtype=np.uint64)
    px = np.array([_ptr(x) for x in Xs] or [0], dtype=np.uint64)
    st = np.zeros(max(1, count), dtype=np.int32)
    rs = np.zeros(max(1, count), dtype=np.float64)
    it = np.zeros(max(1, count), dtype=np.int32)
    rg = np.zeros(max(1, count), dtype=np.int32)
    sg = np.zeros(max(1, count), dtype=np.int8)
    lg = np.zeros(max(1, count), dtype=np.float64)
    r = L.gj_invert_mixed_batched(count, ns.ctypes.data, lds.ctypes.data, pa.ctypes.data, px.ctypes.data,
                                  int(x0_slices), int(corr_slices), float(tol), int(max_iter), int(workers),
                                  st.ctypes.data, rs.ctypes.data, it.ctypes.data, rg.ctypes.data, sg.ctypes.data,
                                  lg.ctypes.data, _stream_handle(stream))
    if r < 0:
        raise GJError(r, "gj_invert_mixed_batched")
    return {"X": Xs, "status": r, "statuses": st[:count], "resid": rs[:count], "iters": it[:count],
            "rung": rg[:count], "det_sign": sg[:count], "det_log2": lg[:count]}


def invert_batched(n_dev, A_ptrs, X_ptrs, status, det_sign=None, det_log2=None, *, pivot_mode: int = PIVOT_PARTIAL,
                   nmax: int = 0, stream=None) -> None:
    """Stream-ordered batched inversion (``gj_invert_batched``); all arrays are device tensors.

    ``n_dev`` int32 [count]; ``A_ptrs`` / ``X_ptrs`` int64 [count] device pointers;
    ``status`` int32 [count]; ``det_sign`` int8 [count]; ``det_log2`` float64 [count].
    """
    L = lib()
    count = int(n_dev.shape[0])
    st = L.gj_invert_batched(count, int(nmax), _ptr(n_dev), _ptr(A_ptrs), _ptr(X_ptrs), int(pivot_mode),
                             _ptr(status), _ptr(det_sign), _ptr(det_log2), _stream_handle(stream))
    if st != OK:
        raise GJError(st, "gj_invert_batched")


NOALLOC_MAX_COUNT = 1048576


def invert_batched_noalloc(n_dev, A_ptrs, X_ptrs, status, det_sign=None, det_log2=None, *,
                           pivot_mode: int = PIVOT_PARTIAL, nmax: int = 0, stream=None) -> None:
    """``gj_invert_batched_noalloc``: as ``invert_batched`` but with no device allocation
    (scratch in a static device array; at most ``NOALLOC_MAX_COUNT`` matrices; calls that
    overlap on the GPU race and must be serialised by the caller)."""
    L = lib()
    count = int(n_dev.shape[0])
    st = L.gj_invert_batched_noalloc(count, int(nmax), _ptr(n_dev), _ptr(A_ptrs), _ptr(X_ptrs), int(pivot_mode),
                                     _ptr(status), _ptr(det_sign), _ptr(det_log2), _stream_handle(stream))
    if st != OK:
        raise GJError(st, "gj_invert_batched_noalloc")


class BatchedPlan:
    """A planned batch (``gj_batched_plan_*``): fixed orders, largest-first order, one
    autotuned kernel variant per order bin, graph replay.

    ``variant=-1`` autotunes (``BATCHED_*`` forces one variant); ``tune_cache`` is an
    optional text file path for the tuner's choices."""

    def __init__(self, n_host, pivot_mode: int = PIVOT_PARTIAL, *, variant: int = -1, tune_cache=None):
        import numpy as np
        L = lib()
        self._n = np.ascontiguousarray(n_host, dtype=np.int32)
        self.count = int(self._n.shape[0])
        self._plan = ctypes.c_void_p()
        cache = None if tune_cache is None else os.fsencode(tune_cache)
        st = L.gj_batched_plan_create_ex(ctypes.byref(self._plan), self.count, self._n.ctypes.data, int(pivot_mode),
                                         cache, int(variant))
        if st != OK:
            raise GJError(st, "gj_batched_plan_create_ex")

    def bins(self) -> list[dict]:
        """Order bins of the plan: ``lo``, ``hi``, ``count``, ``variant`` (name), ``tuned_us``."""
        import numpy as np
        lo = np.zeros(16, dtype=np.int32)
        hi = np.zeros(16, dtype=np.int32)
        cnt = np.zeros(16, dtype=np.int64)
        var = np.zeros(16, dtype=np.int32)
        us = np.zeros(16, dtype=np.float32)
        nb = lib().gj_batched_plan_bins(self._plan, lo.ctypes.data, hi.ctypes.data, cnt.ctypes.data, var.ctypes.data,
                                        us.ctypes.data, 16)
        return [{"lo": int(lo[b]), "hi": int(hi[b]), "count": int(cnt[b]), "variant": BATCHED_NAMES[int(var[b])],
                 "tuned_us": float(us[b])} for b in range(nb)]

    def execute(self, A_ptrs, X_ptrs, status, det_sign=None, det_log2=None, *, stream=None,
                use_graph: bool = True) -> None:
        st = lib().gj_batched_plan_execute(self._plan, _ptr(A_ptrs), _ptr(X_ptrs), _ptr(status), _ptr(det_sign),
                                           _ptr(det_log2), _stream_handle(stream), int(bool(use_graph)))
        if st != OK:
            raise GJError(st, "gj_batched_plan_execute")

    def close(self) -> None:
        if getattr(self, "_plan", None) is not None and self._plan.value:
            lib().gj_batched_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
