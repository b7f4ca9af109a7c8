"""gj_invert_batched_noalloc, the batched entry point that allocates no device memory.

It serves callers that cannot allocate when they invert: real-time loops that must not take
the allocator's locks or risk its latency or an out-of-memory failure, programs that handed
all device memory to their own pool, and code that allocates only during initialisation.
Its scratch lives in a static device array shared by every call, so the test makes two calls
in a row on two different batches (different counts, orders and contents) and checks each
against the allocating entry point, gj_invert_batched, on the same input: scratch left over
from the first call would show up in the second.  Both calls go through the C ABI.

This file is named to be collected last; it passes alone in a fresh process (the first
call on the device does the array's set-up) and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl
from tests.parity import EPS

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()


def ragged_batch(seed):
    rng = np.random.default_rng(seed)
    sizes = np.concatenate([rng.integers(4, 65, size=4500), [0, 1, 2, 128, 127, 65, 3]]).astype(np.int32)
    offsets = np.zeros(len(sizes), dtype=np.int64)
    offsets[1:] = np.cumsum(sizes.astype(np.int64) ** 2)[:-1]
    packed = np.zeros(int((sizes.astype(np.int64) ** 2).sum()))
    for m, n in enumerate(sizes):
        M = rng.uniform(-1, 1, size=(n, n)) + (n + 1) * np.eye(n)
        packed[offsets[m]: offsets[m] + n * n] = M.reshape(-1, order="F")
    packed[offsets[10]: offsets[10] + sizes[10]] = 0.0      # singular: zero first column
    packed[offsets[20] + 5] = np.nan                        # non-finite entry
    return sizes, packed, offsets


def run(entry, sizes, packed, offsets, mode):
    count = len(sizes)
    dA = torch.from_numpy(packed).cuda()
    dX = torch.full_like(dA, float("nan"))
    ap = torch.from_numpy(dA.data_ptr() + 8 * offsets).cuda()
    xp = torch.from_numpy(dX.data_ptr() + 8 * offsets).cuda()
    nd = torch.from_numpy(sizes).cuda()
    st = torch.full((count,), -99, dtype=torch.int32, device="cuda")
    sg = torch.zeros((count,), dtype=torch.int8, device="cuda")
    lg = torch.zeros((count,), dtype=torch.float64, device="cuda")
    rc = entry(count, 0, nd.data_ptr(), ap.data_ptr(), xp.data_ptr(), mode, st.data_ptr(), sg.data_ptr(),
               lg.data_ptr(), None)
    assert rc == gj.OK, (rc, gj.last_error())
    torch.cuda.synchronize()
    return dX.cpu().numpy(), st.cpu().numpy(), sg.cpu().numpy(), lg.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    L = gj.lib()
    batches = [wl.diag_dominant_batch(3000, seed=91), ragged_batch(92)]
    for (sizes, packed, offsets), mode in zip(batches, (gj.PIVOT_PARTIAL, gj.PIVOT_FULL)):
        Xr, sr, gr, lr = run(L.gj_invert_batched, sizes, packed, offsets, mode)
        Xn, sn, gn, ln = run(L.gj_invert_batched_noalloc, sizes, packed, offsets, mode)
        assert np.array_equal(sr, sn)
        assert np.array_equal(gr, gn)
        ok = sr == 0
        assert ok.sum() >= len(sizes) - 2
        assert np.all(np.abs(ln[ok] - lr[ok]) <= 1e-12 * np.maximum(1.0, np.abs(lr[ok])))
        for m in np.nonzero(ok)[0]:
            n = int(sizes[m])
            a, b = offsets[m], offsets[m] + n * n
            A = packed[a:b].reshape(n, n, order="F")
            if n == 0:
                continue
            kappa = np.linalg.cond(A, 1)
            tol = 64 * n * kappa * EPS * np.max(np.abs(Xr[a:b]))
            assert np.max(np.abs(Xn[a:b] - Xr[a:b])) <= tol, m


def test_noalloc_rejects_batches_above_its_limit():
    L = gj.lib()
    rc = L.gj_invert_batched_noalloc(gj.NOALLOC_MAX_COUNT + 1, 0, None, None, None, gj.PIVOT_PARTIAL, None,
                                     None, None, None)
    assert rc == gj.ERR_UNSUPPORTED
    assert "GJ_NOALLOC_MAX_COUNT" in gj.last_error()
