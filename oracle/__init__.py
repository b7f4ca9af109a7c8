"""CPU oracle for Gauss-Jordan inversion (arXiv:1401.7962, Section 2, eqs. 1-15).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library (``paper_1401_7962_gb300``) never imports, links or executes it,
and the two share no code: the oracle is a plain C file compiled with gcc and
loaded through ctypes.

``build()`` compiles ``gj_oracle.c`` into ``oracle/_build/libgj_oracle.so``
(``-O2 -ffp-contract=off``: every operation of eq. 15 rounded separately).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgj_oracle.so")

# Status codes of the oracle (same numbering the C library documents).
OK, SINGULAR, ZERO_PIVOT, NONFINITE, ERR_ARG, ERR_NOMEM = 0, 1, 2, 3, -1, -3
PIVOT_NONE, PIVOT_PARTIAL, PIVOT_FULL, PIVOT_PAPER_SIGNED = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False, cflags: tuple[str, ...] = ()) -> str:
    """Compile the oracle; returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               *cflags, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(src_text: str, out_path: str) -> ctypes.CDLL:
    """Compile a modified copy of the oracle source (used by the mutation tests)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-shared", "-fPIC", src, "-o", out_path,
                    "-lm"], check=True)
    return _bind(ctypes.CDLL(out_path))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    P = ctypes.c_void_p
    lib.gjo_invert.restype = ctypes.c_int
    lib.gjo_invert.argtypes = [ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_double,
                               P, P, P, P, P, P, P]
    lib.gjo_solve.restype = ctypes.c_int
    lib.gjo_solve.argtypes = [ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P,
                              ctypes.c_int64, ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
    lib.gjo_invert_range.restype = None
    lib.gjo_invert_range.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, ctypes.c_int, P, P, P]
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def invert(A: np.ndarray, pivot_mode: int = PIVOT_PARTIAL, tau: float = 0.0, _lib=None) -> dict:
    """Invert one square matrix with the oracle.

    ``A`` is any 2-D float array; it is passed column-major.  Returns a dict with
    ``X`` (n x n inverse, or the partially reduced array on failure), ``status``,
    ``det_sign``, ``det_log2``, ``piv_rows``, ``piv_cols``, ``pivots``, ``gaps``,
    ``fail_step``.
    """
    L = _lib if _lib is not None else lib()
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    n = A.shape[0]
    Af = np.asfortranarray(A)
    X = np.zeros((n, n), dtype=np.float64, order="F")
    sgn = ctypes.c_int(0)
    lg = ctypes.c_double(0.0)
    pr = np.full(max(n, 1), -1, dtype=np.int32)
    pc = np.full(max(n, 1), -1, dtype=np.int32)
    pv = np.zeros(max(n, 1), dtype=np.float64)
    gp = np.zeros(max(n, 1), dtype=np.float64)
    fs = ctypes.c_int64(-1)
    st = L.gjo_invert(n, _ptr(Af), max(n, 1), _ptr(X), pivot_mode, tau, ctypes.addressof(sgn),
                      ctypes.addressof(lg), _ptr(pr), _ptr(pc), _ptr(pv), _ptr(gp), ctypes.addressof(fs))
    return {"X": X, "status": st, "det_sign": sgn.value, "det_log2": lg.value, "piv_rows": pr[:n].copy(),
            "piv_cols": pc[:n].copy(), "pivots": pv[:n].copy(), "gaps": gp[:n].copy(), "fail_step": fs.value}


def solve(A: np.ndarray, B: np.ndarray, pivot_mode: int = PIVOT_PARTIAL, tau: float = 0.0, _lib=None) -> dict:
    """Solve A X = B with the oracle's Gauss-Jordan sweep of [A | B] (eqs. 3-10, B in the
    place of D).  ``B`` is n x m (a 1-D vector is taken as one column).  Returns a dict with
    ``X`` (n x m), ``status``, ``det_sign``, ``det_log2``, ``piv_rows``, ``piv_cols``,
    ``pivots``, ``fail_step``."""
    L = _lib if _lib is not None else lib()
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    if A.ndim != 2 or A.shape[0] != A.shape[1] or B.ndim != 2 or B.shape[0] != A.shape[0]:
        raise ValueError("A square, B with as many rows as A")
    n, m = A.shape[0], B.shape[1]
    Af = np.asfortranarray(A)
    Bf = np.asfortranarray(B)
    X = np.zeros((n, m), dtype=np.float64, order="F")
    sgn = ctypes.c_int(0)
    lg = ctypes.c_double(0.0)
    pr = np.full(max(n, 1), -1, dtype=np.int32)
    pc = np.full(max(n, 1), -1, dtype=np.int32)
    pv = np.zeros(max(n, 1), dtype=np.float64)
    fs = ctypes.c_int64(-1)
    st = L.gjo_solve(n, m, _ptr(Af), max(n, 1), _ptr(Bf) if m else None, max(n, 1), _ptr(X) if m else None,
                     max(n, 1), pivot_mode, tau, ctypes.addressof(sgn), ctypes.addressof(lg), _ptr(pr), _ptr(pc),
                     _ptr(pv), ctypes.addressof(fs))
    return {"X": X, "status": st, "det_sign": sgn.value, "det_log2": lg.value, "piv_rows": pr[:n].copy(),
            "piv_cols": pc[:n].copy(), "pivots": pv[:n].copy(), "fail_step": fs.value}


def invert_many(sizes: np.ndarray, packed: np.ndarray, offsets: np.ndarray, pivot_mode: int = PIVOT_PARTIAL,
                threads: int = 1) -> dict:
    """Invert a packed batch: matrix m is ``packed[offsets[m]: offsets[m] + n_m**2]`` (column-major).

    ``threads`` > 1 splits the matrices across Python threads; the ctypes call
    releases the GIL, so the threads run on separate cores.  Returns ``X`` (packed
    like the input), ``status``, ``det_sign``, ``det_log2``.
    """
    L = lib()
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    packed = np.ascontiguousarray(packed, dtype=np.float64)
    count = sizes.shape[0]
    X = np.zeros_like(packed)
    status = np.zeros(count, dtype=np.int32)
    dsign = np.zeros(count, dtype=np.int32)
    dlog = np.zeros(count, dtype=np.float64)

    def run(m0: int, m1: int) -> None:
        L.gjo_invert_range(m0, m1, _ptr(sizes), _ptr(packed), _ptr(offsets), _ptr(X), _ptr(offsets), pivot_mode,
                           _ptr(status), _ptr(dsign), _ptr(dlog))

    threads = max(1, int(threads))
    if threads == 1 or count < 2:
        run(0, count)
    else:
        # split by cumulative n^3 so each thread gets a similar amount of work
        w = np.cumsum(sizes.astype(np.float64) ** 3)
        cuts = [0] + [int(np.searchsorted(w, w[-1] * t / threads)) for t in range(1, threads)] + [count]
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda t: run(cuts[t], cuts[t + 1]), range(threads)))
    return {"X": X, "status": status, "det_sign": dsign, "det_log2": dlog}
