"""The C-ABI library: builds, loads, exports every symbol its header declares, and rejects
bad arguments before touching the GPU (these checks run without a GPU)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gj_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gj.lib()


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("gj_invert", "gj_invert_ex", "gj_solve", "gj_solve_ex", "gj_invert_batched", "gj_invert_batched_noalloc",
                 "gj_invert_mixed", "gj_invert_mixed_batched", "gj_batched_plan_create",
                 "gj_batched_plan_execute", "gj_batched_plan_destroy", "gj_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(lib):
    for code in (0, 1, 2, 3, 4, -1, -2, -3, -4, -5):
        assert gj.status_string(code)
    assert gj.status_string(12345) == "unknown status"


def test_argument_errors_need_no_gpu(lib):
    L = lib
    sgn, lg = ctypes.c_int(7), ctypes.c_double(1.0)
    buf = np.zeros(16)
    p = buf.ctypes.data
    # negative order, lda < n, bad pivot mode, null pointers, in-place with lda != n
    assert L.gj_invert(-1, p, 1, p, 1, None, None) == gj.ERR_ARG
    assert L.gj_invert(4, p, 3, p + 8, 1, None, None) == gj.ERR_ARG
    assert L.gj_invert(2, p, 2, p + 64, 5, None, None) == gj.ERR_ARG
    assert L.gj_invert(2, None, 2, p, 1, None, None) == gj.ERR_ARG
    assert L.gj_invert(2, p, 3, p, 1, None, None) == gj.ERR_ARG
    # empty matrix: det is the empty product
    assert L.gj_invert(0, None, 1, None, 1, ctypes.byref(sgn), ctypes.byref(lg)) == gj.OK
    assert sgn.value == 1 and lg.value == 0.0
    # failed calls leave det_sign = 0, det_log2 = -inf
    assert L.gj_invert(-3, p, 1, p, 1, ctypes.byref(sgn), ctypes.byref(lg)) == gj.ERR_ARG
    assert sgn.value == 0 and math.isinf(lg.value) and lg.value < 0
    # options: negative tau, unknown path / update, bad panel width
    for field, val in (("tau", -1.0), ("path", 9), ("update", 7), ("panel", 48), ("lookahead", 3)):
        o = gj._Opts()
        setattr(o, field, val)
        assert L.gj_invert_ex(ctypes.byref(o), 2, p, 2, p + 64, 1, None, None) == gj.ERR_ARG
    # batched: negative count, bad mode, order bound above 128
    assert L.gj_invert_batched(-1, 0, None, None, None, 1, None, None, None, None) == gj.ERR_ARG
    assert L.gj_invert_batched(3, 0, p, p, p, 9, p, None, None, None) == gj.ERR_ARG
    assert L.gj_invert_batched(3, 129, p, p, p, 1, p, None, None, None) == gj.ERR_UNSUPPORTED
    assert L.gj_invert_batched(0, 0, None, None, None, 1, None, None, None, None) == gj.OK
    # mixed: bad slices / tol / lda
    assert L.gj_invert_mixed(4, p, 4, p, 0, 4, 1e-12, 5, None, None, None, None, None, None) == gj.ERR_ARG
    assert L.gj_invert_mixed(4, p, 4, p, 3, 4, 0.0, 5, None, None, None, None, None, None) == gj.ERR_ARG
    assert L.gj_invert_mixed(4, p, 3, p, 3, 4, 1e-12, 5, None, None, None, None, None, None) == gj.ERR_ARG
    assert L.gj_invert_mixed(0, None, 1, None, 3, 4, 1e-12, 5, None, None, None, None, None, None) == gj.OK
    # batched mixed: every argument is checked before the device is touched
    ns = np.array([4, 0, 5], dtype=np.int32)
    lds = np.array([4, 1, 5], dtype=np.int32)
    ptrs = np.array([p, 0, p], dtype=np.uint64)
    nul = np.array([p, 0, 0], dtype=np.uint64)

    def mb(count=3, n=ns, ld=lds, a=ptrs, x=ptrs, x0=3, corr=4, tol=1e-12, it=5, workers=0):
        return L.gj_invert_mixed_batched(count, n.ctypes.data if n is not None else None,
                                         ld.ctypes.data if ld is not None else None,
                                         a.ctypes.data if a is not None else None,
                                         x.ctypes.data if x is not None else None, x0, corr, tol, it, workers,
                                         None, None, None, None, None, None, None)
    assert mb(count=-1) == gj.ERR_ARG
    assert mb(x0=0) == gj.ERR_ARG and mb(corr=9) == gj.ERR_ARG
    assert mb(tol=0.0) == gj.ERR_ARG and mb(it=-1) == gj.ERR_ARG
    assert mb(workers=65) == gj.ERR_ARG and mb(workers=-1) == gj.ERR_ARG
    assert mb(n=None) == gj.ERR_ARG and mb(a=None) == gj.ERR_ARG
    assert mb(ld=np.array([3, 1, 5], dtype=np.int32)) == gj.ERR_ARG          # lda < n
    assert mb(ld=np.array([4, 0, 5], dtype=np.int32)) == gj.ERR_ARG          # lda < 1 for n == 0
    assert mb(n=np.array([4, -1, 5], dtype=np.int32)) == gj.ERR_ARG
    assert mb(x=nul) == gj.ERR_ARG                                           # null X of a non-empty matrix
    assert mb(count=0, n=None, ld=None, a=None, x=None) == gj.OK
    # solve: negative sizes, leading dimensions below n, bad mode, null pointers, the
    # single-CTA path (no right-hand sides there); n == 0 is the empty product
    assert L.gj_solve(-1, 1, p, 1, p, 1, p, 1, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, -1, p, 4, p, 4, p, 4, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 1, p, 3, p, 4, p, 4, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 1, p, 4, p, 3, p, 4, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 1, p, 4, p, 4, p, 3, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 1, p, 4, p, 4, p, 4, 7, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 1, None, 4, p, 4, p, 4, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(4, 2, p, 4, p, 4, p, 5, 1, None, None) == gj.ERR_ARG   # X == B with ldx != ldb
    o = gj._Opts()
    o.path = gj.PATH_CTA
    assert L.gj_solve_ex(ctypes.byref(o), 4, 1, p, 4, p, 4, p, 4, 1, None, None) == gj.ERR_ARG
    assert L.gj_solve(0, 3, None, 1, None, 1, None, 1, 1, ctypes.byref(sgn), ctypes.byref(lg)) == gj.OK
    assert sgn.value == 1 and lg.value == 0.0
    plan = ctypes.c_void_p()
    nh = np.array([4, 200], dtype=np.int32)
    assert L.gj_batched_plan_create(ctypes.byref(plan), 2, nh.ctypes.data, 1) == gj.ERR_UNSUPPORTED
    assert L.gj_batched_plan_create(ctypes.byref(plan), -2, nh.ctypes.data, 1) == gj.ERR_ARG
    assert L.gj_batched_plan_create(None, 2, nh.ctypes.data, 1) == gj.ERR_ARG
    L.gj_batched_plan_destroy(None)


def test_binding_checks_layout(lib):
    A = np.zeros((3, 3))  # C-ordered: not column-major
    with pytest.raises(ValueError):
        gj.invert(A[:, :2])
    with pytest.raises(ValueError):
        gj.invert(np.ascontiguousarray(np.arange(9.0).reshape(3, 3))[:, ::-1])
    with pytest.raises(TypeError):
        gj.invert(np.asfortranarray(np.eye(3, dtype=np.float32)))
