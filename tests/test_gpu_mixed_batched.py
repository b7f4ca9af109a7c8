"""Batched reduced-precision Gauss-Jordan + Newton-Schulz refinement (gj_invert_mixed_batched)
against the FP64 oracle, on ragged batches of A = U diag(sigma) V^T (Haar U, V; sigma
log-spaced from 1 to kappa; kappa log-uniform) stored as FP32.

Per matrix the gates of the single-matrix path hold: the normalised residual
||A X - I||_F / (||A||_F ||X||_F) reaches the tolerance (recomputed on the host); X agrees
with the oracle's inverse of the same FP32 matrix (converted exactly to FP64) within
64 n kappa eps relative in the Frobenius norm; the determinant sign is the oracle's.  The
workers run the single-matrix kernels on their own streams, so every matrix's result is
also bitwise the single-matrix call's."""
import numpy as np
import pytest

import oracle
import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = float(np.finfo(np.float64).eps)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()


def _batch(sizes, kappas, seed):
    """Host FP32 matrices of the batch recipe and their column-major device copies."""
    sizes = np.asarray(sizes, dtype=np.int32)
    off = np.zeros(len(sizes), dtype=np.int64)
    off[1:] = np.cumsum(sizes.astype(np.int64) ** 2)[:-1]
    packed = wl.mixed_batch_host(sizes, np.asarray(kappas, dtype=np.float64), off, seed)
    flat = torch.from_numpy(packed).cuda()
    host = [wl.unpack(sizes, packed, off, m) for m in range(len(sizes))]
    dev = [wl.matrix_view(flat, int(n), int(o)) for n, o in zip(sizes, off)]
    return host, dev, flat


def _check_against_oracle(A32, X, r_m, tol):
    n = A32.shape[0]
    if n == 0:
        return
    A = A32.astype(np.float64)
    o = oracle.invert(A, oracle.PIVOT_PARTIAL)
    R = A @ X - np.eye(n)
    assert np.linalg.norm(R) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 2 * tol
    kap = np.linalg.cond(A, 2)
    rel = np.linalg.norm(X - o["X"]) / np.linalg.norm(o["X"])
    assert rel <= 64 * n * kap * EPS, (n, rel, kap)
    assert r_m["det_sign"] == o["det_sign"]


@pytest.mark.parametrize("workers", [1, 3, 8])
def test_ragged_batch_matches_oracle(workers):
    sizes = [0, 1, 2, 100, 128, 129, 200, 257, 300, 140, 5]
    g = np.random.default_rng(11)
    kappas = 10.0 ** g.uniform(2, 6, size=len(sizes))
    host, dev, _ = _batch(sizes, kappas, seed=4100)
    r = gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-12, max_iter=10, workers=workers)
    assert r["status"] == gj.OK, r["statuses"]
    assert np.all(r["statuses"] == 0)
    assert np.all(r["resid"] <= 1e-12)
    for m, n in enumerate(sizes):
        X = r["X"][m].cpu().numpy()
        _check_against_oracle(host[m], X, {"det_sign": int(r["det_sign"][m])}, 1e-12)


def test_batch_equals_single_matrix_calls():
    """Each worker runs gj_invert_mixed on its own stream: results are bitwise the single
    calls', whatever the number of workers."""
    sizes = [300, 131, 257, 64, 200]
    kappas = [1e3, 1e5, 1e2, 1e4, 1e6]
    host, dev, _ = _batch(sizes, kappas, seed=4200)
    r = gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-12, max_iter=10, workers=4)
    for m in range(len(sizes)):
        s = gj.invert_mixed(dev[m].clone().t().contiguous().t(), x0_slices=3, corr_slices=4, tol=1e-12, max_iter=10)
        assert torch.equal(s["X"], r["X"][m])
        assert s["resid"] == r["resid"][m] and s["iters"] == r["iters"][m] and s["rung"] == r["rung"][m]
        assert s["det_sign"] == r["det_sign"][m] and s["det_log2"] == r["det_log2"][m]


def test_each_matrix_climbs_its_own_ladder():
    """3-slice X0 (update truncation about 5 128 2^-21 of the scales per panel): the
    kappa = 1e2 matrix contracts on the first rung, the kappa = 1e6 one cannot and climbs,
    in the same batch."""
    host, dev, _ = _batch([400, 400], [1e2, 1e6], seed=4300)
    r = gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-12, workers=2)
    assert r["status"] == gj.OK
    assert r["rung"][0] == 0 and r["rung"][1] >= 1
    for m in range(2):
        _check_against_oracle(host[m], r["X"][m].cpu().numpy(), {"det_sign": int(r["det_sign"][m])}, 1e-12)


def test_kappa_1e8_reaches_the_fp64_rung():
    """The top of the recipe's condition range: the 3- and 5-slice rungs cannot contract
    (2^-21 kappa, 2^-35 kappa n are not small), the FP64-level rung does."""
    host, dev, _ = _batch([520], [1e8], seed=4400)
    r = gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-12, workers=1)
    assert r["status"] == gj.OK and r["resid"][0] <= 1e-12
    _check_against_oracle(host[0], r["X"][0].cpu().numpy(), {"det_sign": int(r["det_sign"][0])}, 1e-12)


def _panel_launches(fn):
    """Launches of the cluster panel kernel made by fn(), from the library's profiling hooks."""
    import ctypes

    class Entry(ctypes.Structure):
        _fields_ = [("kernel", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                    ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]
    L = gj.lib()
    entries = (Entry * 16)()
    total = ctypes.c_int64(0)
    L.gj_profile_begin()
    out = fn()
    cnt = L.gj_profile_end(entries, 16, ctypes.byref(total))
    return out, sum(entries[i].launches for i in range(cnt) if entries[i].kernel == b"panel_cluster")


def test_ladder_skips_the_middle_rung_when_it_cannot_contract():
    """kappa = 1e8 from a 3-slice X0: the first residual norm is far above 2^14 / 4, so the
    5-slice X0 is skipped: two X0 sweeps (3 and 7 slices) of 17 sub-panels of 32 columns
    each, not three."""
    host, dev, _ = _batch([520], [1e8], seed=4400)
    r, panels = _panel_launches(lambda: gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-12,
                                                                 workers=1))
    assert r["status"] == gj.OK and r["rung"][0] == 2
    assert panels == 2 * 17, panels


def test_nonconvergence_is_per_matrix():
    """tol below what FP64 can reach: every matrix reports GJ_NOT_CONVERGED with its
    residual, and the call returns that status."""
    host, dev, _ = _batch([150, 0, 90], [1e2, 1e2, 1e3], seed=4500)
    r = gj.invert_mixed_batched(dev, x0_slices=3, corr_slices=4, tol=1e-30, max_iter=3, workers=2)
    assert r["status"] == gj.NOT_CONVERGED
    assert r["statuses"][0] == gj.NOT_CONVERGED and r["statuses"][2] == gj.NOT_CONVERGED
    assert r["statuses"][1] == gj.OK and r["resid"][1] == 0.0
    assert r["resid"][0] < 1e-13 and r["resid"][2] < 1e-13


@pytest.mark.parametrize("x0,workers", [(3, 8), (7, 16)])
def test_full_recipe_sampled(x0, workers):
    """The batch recipe, 256 matrices of orders 128..1024 and kappa 1e2..1e8 generated on
    the GPU, with the 3-slice ladder and in the benchmark's launch configuration (16
    workers, 7-slice FP64-level first inverse): every matrix meets the residual gate; three sampled
    matrices are recomputed on the host, one of them against the oracle."""
    sizes, kappas, off = wl.mixed_batch_params(256, wl.SEED_BASE + 5)
    flat = wl.mixed_batch_device(sizes, kappas, off, wl.SEED_BASE + 5, device="cuda")
    dev = [wl.matrix_view(flat, int(n), int(o)) for n, o in zip(sizes, off)]
    r = gj.invert_mixed_batched(dev, x0_slices=x0, corr_slices=4, tol=1e-12, max_iter=10, workers=workers)
    assert r["status"] == gj.OK, np.unique(r["statuses"], return_counts=True)
    assert np.all(r["resid"] <= 1e-12)
    if x0 == 3:
        # the 3-slice and the FP64-level rungs are both used by this recipe's kappa range
        assert set(np.unique(r["rung"]).tolist()) >= {0, 2}
    order = np.argsort(sizes)
    for m in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        A = dev[m].double().cpu().numpy()
        X = r["X"][m].cpu().numpy()
        n = A.shape[0]
        assert np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 2e-12
    m = int(order[0])
    _check_against_oracle(dev[m].cpu().numpy(), r["X"][m].cpu().numpy(), {"det_sign": int(r["det_sign"][m])}, 1e-12)
