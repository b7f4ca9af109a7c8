"""Expiry of a bounded device wait in the tensor-core update kernel, and what follows it.

Every wait of the update's producer / MMA / epilogue pipeline is bounded in time.  The
limit is a process-wide setting (gj_set_wait_limit_ns); at 1 ns the first wait of every
CTA that is not satisfied at once gives up.  The kernel must then stop issuing work, wait
(with the full 2 s limit) for the tile loads and MMAs it already issued, free its tensor
memory and exit, and the call must report GJ_ERR_TIMEOUT.  Nothing is left hanging: a
normal call on the same GPU right after must give the right result.  No wait is left
without a limit and nothing faults on purpose: the expiry is caused by the limit alone.
"""
import numpy as np
import pytest

import oracle
import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl
from tests.parity import assert_matches_oracle, tie_free_seed
from tests.test_gpu_ozaki import run as run_update

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()
    yield
    gj.set_wait_limit_ns(0)


def test_update_wait_expiry_returns_timeout_then_device_is_usable():
    L = gj.lib()
    rng = np.random.default_rng(5)
    M, N, K = 512, 512, 128
    dL = torch.from_numpy(np.asfortranarray(rng.standard_normal((M, K)))).cuda()
    dU = torch.from_numpy(np.asfortranarray(rng.standard_normal((K, N)))).cuda()
    dC = torch.zeros((N, M), dtype=torch.float64, device="cuda").t()
    try:
        gj.set_wait_limit_ns(1)
        st = L.gj_gemm_update_emulated(M, N, K, dL.data_ptr(), M, dU.data_ptr(), K, dC.data_ptr(), M, 8, None)
    finally:
        gj.set_wait_limit_ns(0)
    assert st == gj.ERR_TIMEOUT, (st, gj.last_error())
    torch.cuda.synchronize()  # the context is intact: no sticky error
    # the same kernel right after, with the default limit, is within its error bound
    got, ref, bound = run_update(1000, 1000, 128, 8, np.random.default_rng(6))
    assert np.all(np.abs(got - ref) <= bound)


def test_blocked_inversion_reports_update_expiry_then_matches_oracle():
    n = 700
    seed, A, o = tie_free_seed(lambda s: wl.gaussian(n, s, shift=0.1 * n), 77, gj.PIVOT_PARTIAL)
    dA = torch.from_numpy(A).cuda()
    try:
        gj.set_wait_limit_ns(1)
        with pytest.raises(gj.GJError) as ei:
            gj.invert(dA, gj.PIVOT_PARTIAL, path=gj.PATH_BLOCKED, update=gj.UPDATE_TC_OZAKI)
    finally:
        gj.set_wait_limit_ns(0)
    assert ei.value.status == gj.ERR_TIMEOUT
    r = gj.invert(dA, gj.PIVOT_PARTIAL, path=gj.PATH_BLOCKED, update=gj.UPDATE_TC_OZAKI, record=True)
    r["X"] = r["X"].cpu().numpy()
    assert_matches_oracle(A, r, o, gj.PIVOT_PARTIAL)
