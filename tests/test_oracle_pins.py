"""The CPU oracle against its pins (values fixed by the paper and by mathematics)."""
import pytest

import oracle
from tests import pins


def _inv(A, mode, tau=0.0):
    return oracle.invert(A, mode, tau)


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    pin(_inv)


def _sol(A, B, mode, tau=0.0):
    return oracle.solve(A, B, mode, tau)


@pytest.mark.parametrize("pin", pins.ALL_SOLVE_PINS, ids=lambda p: p.__name__)
def test_oracle_solve_pin(pin):
    pin(_sol)


def test_oracle_batched_matches_single():
    """The batched oracle entry runs the same per-matrix inversion."""
    import numpy as np
    from paper_1401_7962_gb300 import workloads as wl
    sizes, packed, offsets = wl.diag_dominant_batch(40, seed=5)
    r = oracle.invert_many(sizes, packed, offsets, oracle.PIVOT_PARTIAL, threads=3)
    for m in range(len(sizes)):
        A = wl.unpack(sizes, packed, offsets, m)
        one = oracle.invert(A, oracle.PIVOT_PARTIAL)
        Xm = r["X"][offsets[m]: offsets[m] + sizes[m] ** 2].reshape(sizes[m], sizes[m], order="F")
        assert np.array_equal(Xm, one["X"])
        assert r["det_sign"][m] == one["det_sign"] and r["det_log2"][m] == one["det_log2"]
        assert r["status"][m] == 0


def test_oracle_arg_errors():
    import ctypes
    import numpy as np
    L = oracle.lib()
    A = np.eye(3, order="F")
    X = np.zeros((3, 3), order="F")
    # lda < n
    assert L.gjo_invert(3, A.ctypes.data, 2, X.ctypes.data, 1, 0.0, None, None, None, None, None, None,
                        None) == oracle.ERR_ARG
    # negative n, bad mode, negative tau
    assert L.gjo_invert(-1, A.ctypes.data, 3, X.ctypes.data, 1, 0.0, *([None] * 7)) == oracle.ERR_ARG
    assert L.gjo_invert(3, A.ctypes.data, 3, X.ctypes.data, 7, 0.0, *([None] * 7)) == oracle.ERR_ARG
    assert L.gjo_invert(3, A.ctypes.data, 3, X.ctypes.data, 1, -1.0, *([None] * 7)) == oracle.ERR_ARG
    # null pointers
    assert L.gjo_invert(3, None, 3, X.ctypes.data, 1, 0.0, *([None] * 7)) == oracle.ERR_ARG
