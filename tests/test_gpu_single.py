"""CUDA single-matrix paths against the CPU oracle (same seeded inputs).

Paths: the single-CTA shared-memory kernel (n <= 128), the blocked cluster-panel path
(partial / no pivoting) and the unblocked multi-launch path (any pivoting).  Every
call goes through the C ABI (gj_invert_ex) via the ctypes binding.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl
from tests.parity import EPS, assert_matches_oracle, norm_resid, tie_free_seed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()


def dev(A):
    return torch.from_numpy(np.asfortranarray(A)).cuda()


def run(A, mode, **kw):
    r = gj.invert(dev(A), mode, record=True, **kw)
    r["X"] = r["X"].cpu().numpy()
    return r


def make_input(n, mode, seed):
    # no pivoting needs nonzero leading minors: diagonally shifted input
    shift = float(n) if mode == gj.PIVOT_NONE else 0.0
    return lambda s: wl.gaussian(n, s, shift=shift)


@pytest.mark.parametrize("path", [gj.PATH_CTA, gj.PATH_UNBLOCKED, gj.PATH_CLUSTER])
def test_paper_example(path):
    g = json.load(open(os.path.join(GOLDEN, "paper_example_3x3.json")))
    A = np.array(g["A"], dtype=np.float64)
    Xe = np.array(g["inverse"], dtype=np.float64)
    for name, mode in (("none", 0), ("partial", 1), ("full", 2)):
        r = run(A, mode, path=path)
        exp = g["modes"][name]
        assert r["status"] == 0
        assert list(r["piv_rows"]) == exp["piv_rows"] and list(r["piv_cols"]) == exp["piv_cols"]
        assert np.max(np.abs(r["X"] - Xe)) <= 1e-13
        assert r["det_sign"] == 1 and abs(r["det_log2"]) <= 1e-14


def test_paper_example_blocked():
    g = json.load(open(os.path.join(GOLDEN, "paper_example_3x3.json")))
    A = np.array(g["A"], dtype=np.float64)
    for name, mode in (("none", 0), ("partial", 1)):
        r = run(A, mode, path=gj.PATH_BLOCKED)
        assert r["status"] == 0 and list(r["piv_rows"]) == g["modes"][name]["piv_rows"]
        assert np.max(np.abs(r["X"] - np.array(g["inverse"]))) <= 1e-13
        assert r["det_sign"] == 1 and abs(r["det_log2"]) <= 1e-14


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 31, 32, 33, 63, 64, 65, 100, 127, 128])
def test_cta_random(n, mode):
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 1000 + n, mode)
    r = run(A, mode, path=gj.PATH_CTA)
    assert_matches_oracle(A, r, o, mode)


@pytest.mark.parametrize("update", [gj.UPDATE_DFMA, gj.UPDATE_TC_OZAKI])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,panel", [(2, 16), (129, 16), (200, 32), (257, 64), (300, 0), (700, 32), (1031, 16)])
def test_blocked_random(n, panel, mode, update):
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 2000 + n, mode)
    r = run(A, mode, path=gj.PATH_BLOCKED, panel=panel, update=update)
    assert_matches_oracle(A, r, o, mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 47, 48, 64, 95, 96, 127, 128])
def test_cluster_path_matches_oracle_and_cta_kernel(n, mode):
    """The cluster kernel (rows spread over 4-16 CTAs) runs the single-CTA kernel's arithmetic:
    bitwise equal results, pivots identical to the oracle on tie-free inputs."""
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 3000 + n, mode)
    r = run(A, mode, path=gj.PATH_CLUSTER)
    c = run(A, mode, path=gj.PATH_CTA)
    assert np.array_equal(r["X"], c["X"])
    assert r["det_log2"] == c["det_log2"] and r["det_sign"] == c["det_sign"]
    assert np.array_equal(r["piv_rows"], c["piv_rows"]) and np.array_equal(r["piv_cols"], c["piv_cols"])
    assert_matches_oracle(A, r, o, mode)


def test_cluster_path_failures():
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert run(S, 0, path=gj.PATH_CLUSTER)["status"] == gj.ZERO_PIVOT
    Z = wl.gaussian(100, 3100)
    Z[:, 60] = 0.0
    for mode in (1, 2):
        r = run(Z, mode, path=gj.PATH_CLUSTER)
        c = run(Z, mode, path=gj.PATH_CTA)
        assert r["status"] == gj.SINGULAR and r["status"] == c["status"] and r["fail_step"] == c["fail_step"]
    N = np.eye(64)
    N[5, 3] = np.inf
    assert run(N, 2, path=gj.PATH_CLUSTER)["status"] == gj.NONFINITE


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,panel", [(300, 32), (1031, 16), (2100, 0)])
def test_lookahead_matches_oracle_and_sequential_schedule(n, panel, mode):
    """The look-ahead schedule (next outer panel reduced on a second stream during the wide
    update) runs the same kernels on the same operands: results bitwise equal to the
    sequential schedule, and parity with the oracle."""
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 2700 + n, mode)
    on = run(A, mode, path=gj.PATH_BLOCKED, panel=panel, update=gj.UPDATE_TC_OZAKI, lookahead=2)
    off = run(A, mode, path=gj.PATH_BLOCKED, panel=panel, update=gj.UPDATE_TC_OZAKI, lookahead=1)
    assert np.array_equal(on["X"], off["X"])
    assert on["det_log2"] == off["det_log2"] and on["det_sign"] == off["det_sign"]
    assert np.array_equal(on["piv_rows"], off["piv_rows"])
    assert_matches_oracle(A, on, o, mode)


def test_lookahead_failure_is_reported():
    """A singular input stops both streams: the status, failing step and det come back."""
    n = 700
    A = wl.gaussian(n, 2800)
    A[:, 400] = 0.0
    r = run(A, 1, path=gj.PATH_BLOCKED, update=gj.UPDATE_TC_OZAKI, lookahead=2)
    assert r["status"] == gj.SINGULAR and r["fail_step"] == 400 and r["det_sign"] == 0


@pytest.mark.parametrize("slices", [7, 8])
def test_blocked_tensor_update_slices(slices):
    """7 digit slices (49 bits) still meet the parity bar on a well-conditioned input; 6 (42
    bits) do not reach the 1e-14 residual gate and are not offered as an FP64 setting."""
    n, mode = 520, 1
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 2600, mode)
    r = run(A, mode, path=gj.PATH_BLOCKED, update=gj.UPDATE_TC_OZAKI, slices=slices)
    assert_matches_oracle(A, r, o, mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 5, 129, 300])
def test_unblocked_random(n, mode):
    seed, A, o = tie_free_seed(make_input(n, mode, 0), 3000 + n, mode)
    r = run(A, mode, path=gj.PATH_UNBLOCKED)
    assert_matches_oracle(A, r, o, mode)


@pytest.mark.parametrize("path,n", [(gj.PATH_CTA, 40), (gj.PATH_BLOCKED, 150), (gj.PATH_BLOCKED, 600),
                                    (gj.PATH_UNBLOCKED, 140)])
def test_lda_inplace_and_host_buffers(path, n):
    mode = 1
    _, A, o = tie_free_seed(make_input(n, mode, 0), 4000 + n, mode)
    # lda > n: the matrix is the top n rows of a taller column-major buffer
    big = np.zeros((n + 7, n), order="F")
    big[:n] = A
    Bd = torch.from_numpy(big).cuda()
    r = gj.invert(Bd[:n], mode, path=path, record=True)
    r["X"] = r["X"].cpu().numpy()
    assert_matches_oracle(A, r, o, mode)
    # in place: Ainv == A
    Ad = dev(A)
    r = gj.invert(Ad, mode, out=Ad, path=path, record=True)
    r["X"] = Ad.cpu().numpy()
    assert_matches_oracle(A, r, o, mode)
    # host buffers in and out (the library stages them)
    Xh = np.empty((n, n), order="F")
    r = gj.invert(np.asfortranarray(A), mode, out=Xh, path=path, record=True)
    assert r["X"] is Xh
    assert_matches_oracle(A, r, o, mode)


@pytest.mark.parametrize("path", [gj.PATH_CTA, gj.PATH_BLOCKED, gj.PATH_UNBLOCKED])
def test_failure_statuses(path):
    def check(A, mode, tau=0.0):
        o = oracle.invert(A, mode, tau)
        r = run(A, mode, path=path, tau=tau)
        assert r["status"] == o["status"], (r["status"], o["status"])
        if o["status"] != 0:
            assert r["fail_step"] == o["fail_step"]
            assert r["det_sign"] == 0 and r["det_log2"] == -math.inf
    Z = np.array([[1.0, 2.0, 0.0], [3.0, 4.0, 0.0], [5.0, 6.0, 0.0]])
    check(Z, 1)
    D = np.array([[2.0, 1.0, 1.0], [4.0, 3.0, 3.0], [2.0, 1.0, 1.0]])
    check(D, 1)
    check(np.zeros((5, 5)), 1)
    N = np.eye(4)
    N[2, 0] = np.nan
    check(N, 1)
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    check(S, 0)
    check(S, 1)
    check(np.diag([1.0, 1e-3, 1.0]), 1, tau=1e-2)
    if path != gj.PATH_BLOCKED:
        check(Z, 2)
        I = np.eye(3)
        I[2, 2] = np.inf
        check(I, 2)


def test_full_pivoting_rejected_by_blocked_path():
    with pytest.raises(gj.GJError):
        gj.invert(dev(np.eye(4)), gj.PIVOT_FULL, path=gj.PATH_BLOCKED)


def test_workload_128_full_pivoting():
    """The 128 x 128 N(0,1) full-pivoting workload, auto path (single CTA), against the oracle."""
    seed, A, o = tie_free_seed(lambda s: wl.gaussian(128, s), wl.SEED_BASE + 1, gj.PIVOT_FULL)
    r = run(A, gj.PIVOT_FULL)
    assert_matches_oracle(A, r, o, gj.PIVOT_FULL)


def test_workload_8192_partial_blocked():
    """The 8192 x 8192 N(0,1) + 0.1 n I workload in the launch configuration the benchmark
    times (blocked, partial pivoting, auto panel and update engine: tensor cores, look-ahead)
    against the oracle's result for the same input, computed once by
    tests/golden/make_inv8192_golden.py (eqs. 13-15, obs. 2-3): the whole pivot sequence
    identical (the smallest relative gap between best and second-best candidate is 0.99, far
    from a tie), the pivot values, det sign and log2|det| (eq. 13) as in tests/parity.py,
    16 whole columns, 16 whole rows and 4096 scattered entries of A^-1 element by element
    within 64 n kappa_1 eps max|x| (kappa_1 = ||A||_1 ||A^-1||_1 with the oracle's
    inverse), and sampled columns and rows of A X = I and X A = I at the normalised-residual
    gate."""
    meta = json.load(open(os.path.join(GOLDEN, "inv8192_partial_oracle.json")))
    ref = np.load(os.path.join(GOLDEN, "inv8192_partial_oracle.npz"))
    n = meta["n"]
    A = wl.gaussian(n, meta["seed"], shift=meta["shift"])
    import hashlib
    assert hashlib.sha256(np.asfortranarray(A).tobytes(order="F")).hexdigest() == meta["input_sha256"], \
        "the seeded generator did not reproduce the golden input"
    r = gj.invert(dev(A), gj.PIVOT_PARTIAL, record=True)
    assert r["status"] == meta["status"] == 0
    assert ref["gaps"].min() > 1e-9
    assert np.array_equal(r["piv_rows"], ref["piv_rows"]), "row pivot sequence differs"
    assert np.array_equal(r["piv_cols"], np.arange(n))
    kappa1 = np.max(np.sum(np.abs(A), axis=0)) * float(ref["X_norm1"][0])
    assert np.allclose(r["pivots"], ref["pivots"], rtol=64 * n * EPS * max(1.0, kappa1), atol=0)
    assert r["det_sign"] == meta["det_sign"]
    assert abs(r["det_log2"] - meta["det_log2"]) <= 1e-12 * max(1.0, abs(meta["det_log2"]))
    X = r["X"].cpu().numpy()
    tol = 64 * n * kappa1 * EPS * float(ref["X_absmax"][0])
    cols, rows, pairs = ref["cols"], ref["rows"], ref["pairs"]
    d_cols = np.max(np.abs(X[:, cols] - ref["X_cols"]))
    d_rows = np.max(np.abs(X[rows, :] - ref["X_rows"]))
    d_pairs = np.max(np.abs(X[pairs[:, 0], pairs[:, 1]] - ref["X_pairs"]))
    assert max(d_cols, d_rows, d_pairs) <= tol, (d_cols, d_rows, d_pairs, tol)
    nA, nX = np.linalg.norm(A), np.linalg.norm(X)
    Rc = A @ X[:, cols]
    Rc[cols, np.arange(len(cols))] -= 1.0
    assert np.linalg.norm(Rc) / (n * nA * nX) <= 1e-14
    Rr = X[rows, :] @ A
    Rr[np.arange(len(rows)), rows] -= 1.0
    assert np.linalg.norm(Rr) / (n * nA * nX) <= 1e-14
