"""gj_solve (A X = B by the Gauss-Jordan sweep of [A | B]) against the CPU oracle's gjo_solve.

Same seeded inputs on both sides; the blocked path (none / partial pivoting, FP64-FMA and
tensor-core updates) and the unblocked path (full pivoting).  Tolerances as for the
inversion: status, det sign and (on tie-free inputs) the pivot sequence equal; the
normalised residual ||A X - B||_F / (||A||_F ||X||_F + ||B||_F) <= n * 1e-15; element by
element |X_gpu - X_oracle| <= 64 n kappa_1(A) eps max|X_oracle| (both are eliminations
whose forward error is bounded by a small multiple of n kappa eps ||X||).
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl
from tests.parity import EPS, tie_free_seed

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


def rhs(n, m, seed):
    g = wl.rng(seed)
    return np.asfortranarray(g.standard_normal((n, m)))


def check(A, B, r, o, mode, check_pivots=True):
    n = A.shape[0]
    assert r["status"] == o["status"], (r["status"], o["status"])
    if o["status"] != 0:
        assert r["det_sign"] == 0 and r["fail_step"] == o["fail_step"]
        return
    X = r["X"] if isinstance(r["X"], np.ndarray) else r["X"].cpu().numpy()
    assert r["det_sign"] == o["det_sign"]
    assert abs(r["det_log2"] - o["det_log2"]) <= 1e-12 * max(1.0, abs(o["det_log2"]))
    if check_pivots and "piv_rows" in r:
        assert np.array_equal(r["piv_rows"], o["piv_rows"]), "row pivot sequence differs"
        if mode == 2:
            assert np.array_equal(r["piv_cols"], o["piv_cols"]), "column pivot sequence differs"
    res = np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X) + np.linalg.norm(B))
    assert res <= max(n, 1) * 1e-15, res
    kappa = np.linalg.cond(A, 1)
    tol = 64 * n * kappa * EPS * max(np.max(np.abs(o["X"])), 1e-300)
    diff = np.max(np.abs(X - o["X"]))
    assert diff <= tol, (diff, tol)


def test_paper_example_solution():
    g = json.load(open(os.path.join(GOLDEN, "paper_example_3x3.json")))
    A = np.array(g["A"], dtype=np.float64)
    b = A @ np.array([[1.0], [2.0], [3.0]])
    for name, mode in (("none", 0), ("partial", 1), ("full", 2)):
        r = gj.solve(dev(A), dev(b), mode, record=True)
        exp = g["modes"][name]
        assert r["status"] == 0
        assert list(r["piv_rows"]) == exp["piv_rows"] and list(r["piv_cols"]) == exp["piv_cols"]
        assert np.max(np.abs(r["X"].cpu().numpy()[:, 0] - [1.0, 2.0, 3.0])) <= 1e-13
        assert r["det_sign"] == 1 and abs(r["det_log2"]) <= 1e-14


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64, 129, 300, 520, 700])
@pytest.mark.parametrize("m", [1, 5, 64])
@pytest.mark.parametrize("mode", [gj.PIVOT_PARTIAL, gj.PIVOT_NONE])
def test_blocked_solve_matches_oracle(n, m, mode):
    shift = float(n) if mode == gj.PIVOT_NONE else 0.0
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s, shift=shift), 9000 + n + m, mode)
    B = rhs(n, m, seed + 1)
    o = oracle.solve(A, B, mode)
    r = gj.solve(dev(A), dev(B), mode, record=True)
    check(A, B, r, o, mode)


@pytest.mark.parametrize("n", [520, 700])
@pytest.mark.parametrize("update", [gj.UPDATE_DFMA, gj.UPDATE_TC_OZAKI])
def test_blocked_solve_update_engines(n, update):
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s), 9100 + n, 1)
    B = rhs(n, 37, seed + 2)
    o = oracle.solve(A, B, 1)
    r = gj.solve(dev(A), dev(B), 1, update=update, record=True)
    check(A, B, r, o, 1)


@pytest.mark.parametrize("lookahead", [1, 2])
def test_solve_lookahead(lookahead):
    n, m = 1100, 7
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s), 9500, 1)
    B = rhs(n, m, seed)
    o = oracle.solve(A, B, 1)
    r = gj.solve(dev(A), dev(B), 1, update=gj.UPDATE_TC_OZAKI, lookahead=lookahead, record=True)
    check(A, B, r, o, 1)


@pytest.mark.parametrize("n", [1, 5, 64, 130, 257])
@pytest.mark.parametrize("m", [1, 9])
def test_full_pivoting_solve_matches_oracle(n, m):
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s), 9200 + n, 2)
    B = rhs(n, m, seed + 3)
    o = oracle.solve(A, B, 2)
    r = gj.solve(dev(A), dev(B), 2, record=True)
    check(A, B, r, o, 2)


def test_partial_pivoting_on_unblocked_path():
    n = 150
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s), 9300, 1)
    B = rhs(n, 4, seed)
    o = oracle.solve(A, B, 1)
    r = gj.solve(dev(A), dev(B), 1, path=gj.PATH_UNBLOCKED, record=True)
    check(A, B, r, o, 1)


def test_host_buffers_padding_and_in_place():
    n, m = 200, 6
    seed, A, _ = tie_free_seed(lambda s: wl.gaussian(n, s), 9400, 1)
    B = rhs(n, m, seed)
    o = oracle.solve(A, B, 1)
    # host A and B with leading dimensions larger than n, host output
    Ap = np.zeros((n + 5, n), order="F")
    Ap[:n] = A
    Bp = np.zeros((n + 3, m), order="F")
    Bp[:n] = B
    r = gj.solve(Ap[:n], Bp[:n], 1)
    check(A, B, r, o, 1, check_pivots=False)
    # device, solution written over B
    dB = dev(B)
    r = gj.solve(dev(A), dB, 1, out=dB)
    assert r["X"] is dB
    check(A, B, r, o, 1, check_pivots=False)


def test_solve_failures_and_edges():
    # zero pivot without pivoting vs a swap with partial pivoting
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    b = np.array([[2.0], [3.0]])
    assert gj.solve(dev(S), dev(b), gj.PIVOT_NONE)["status"] == gj.ZERO_PIVOT
    r = gj.solve(dev(S), dev(b), gj.PIVOT_PARTIAL)
    assert r["status"] == 0 and np.array_equal(r["X"].cpu().numpy(), [[3.0], [2.0]]) and r["det_sign"] == -1
    # an exactly singular matrix on each path
    Z = np.array([[1.0, 2.0, 0.0], [3.0, 4.0, 0.0], [5.0, 6.0, 0.0]])
    for mode in (1, 2):
        r = gj.solve(dev(Z), dev(np.ones((3, 1))), mode)
        assert r["status"] == gj.SINGULAR and r["fail_step"] == 2 and r["det_sign"] == 0
    # non-finite input
    N = np.eye(4)
    N[2, 0] = np.nan
    assert gj.solve(dev(N), dev(np.ones((4, 2))), 1)["status"] == gj.NONFINITE
    # no right-hand sides: det only
    D = np.diag([2.0, 4.0, 8.0])
    r = gj.solve(dev(D), dev(np.zeros((3, 0))), 1)
    assert r["status"] == 0 and r["det_sign"] == 1 and abs(r["det_log2"] - 6.0) <= 1e-15
    # n == 0
    r = gj.solve(dev(np.zeros((0, 0))), dev(np.zeros((0, 2))), 1)
    assert r["status"] == 0 and r["det_sign"] == 1


def test_solve_8192_workload_properties():
    """The 8192 workload of the inversion benchmark with 16 right-hand sides: the identity
    pivot sequence the recipe produces, the residual gate, and sampled rows against a direct
    FP64 computation with the oracle-independent LAPACK solution."""
    n, m = 8192, 16
    A = wl.gaussian(n, wl.SEED_BASE + 2, shift=0.1 * n)
    B = rhs(n, m, 77)
    dA, dB = dev(A), dev(B)
    r = gj.solve(dA, dB, 1, record=True)
    assert r["status"] == 0
    assert np.array_equal(r["piv_rows"], np.arange(n))
    X = r["X"]
    R = torch.from_numpy(A).cuda() @ X - dB
    res = float(torch.linalg.norm(R) / (torch.linalg.norm(dA) * torch.linalg.norm(X) + torch.linalg.norm(dB)))
    assert res <= n * 1e-15, res  # the gate of the smaller cases (n x 4.5 eps)
    ref = np.linalg.solve(A, B)
    Xh = X.cpu().numpy()
    # kappa_2(A) <= (0.1 n + 2 sqrt(n)) / (0.1 n - 2 sqrt(n)) < 2 for N(0,1) + 0.1 n I at this n
    assert np.max(np.abs(Xh - ref)) <= 64 * n * 2.0 * EPS * np.max(np.abs(ref))
