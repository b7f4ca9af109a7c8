"""Reduced-precision Gauss-Jordan + Newton-Schulz refinement (gj_invert_mixed) against the
FP64 oracle, on A = U diag(sigma) V^T with Haar U, V and log-spaced sigma, stored as FP32.

What is checked: the normalised residual ||A X - I||_F / (||A||_F ||X||_F) reaches the
requested tolerance (1e-12); the refined X agrees with the oracle's inverse of the same
FP32 matrix (converted exactly to FP64) element by element, to the forward-error level of a
backward-stable inverse (64 n kappa_1 eps max|X|, the tolerance of the FP64 paths), and in
the Frobenius norm; the determinant sign equals the oracle's.  log2|det| comes from the
pivots of the last X0 sweep, whose updates carry an error of about 2^-8S of the scales:
it must match the oracle to n kappa 2^-(8 S) relative (at least 1e-12, the FP64 paths'
tolerance, which the 7-slice rung meets for small kappa), capped at 1/4 so that the
assertion can always fail.  One case (n = 2304) is large enough for the look-ahead
schedule of the blocked sweep (n >= 2048)."""
import math

import numpy as np
import pytest

import oracle
import paper_1401_7962_gb300 as gj
from paper_1401_7962_gb300 import workloads as wl
from tests.parity import norm_resid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = float(np.finfo(np.float64).eps)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()


@pytest.mark.parametrize("n,kappa,x0", [(300, 1e2, 1), (520, 1e4, 2), (700, 1e6, 5), (1000, 1e6, 3),
                                        (640, 1e6, 7), (400, 1e2, 7), (2304, 1e6, 3)])
def test_mixed_refined_inverse(n, kappa, x0):
    A32 = wl.svd_conditioned(n, kappa, seed=5000 + n, dtype=np.float32)
    A = A32.astype(np.float64)
    o = oracle.invert(A, oracle.PIVOT_PARTIAL)
    dA = torch.from_numpy(np.asfortranarray(A32)).cuda()
    r = gj.invert_mixed(dA, x0_slices=x0, corr_slices=4, tol=1e-12, max_iter=10)
    X = r["X"].cpu().numpy()
    assert r["status"] == 0, r
    assert r["resid"] <= 1e-12
    # independent recomputation of the gate on the host
    R = A @ X - np.eye(n)
    assert np.linalg.norm(R) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 2e-12
    kap = np.linalg.cond(A, 2)
    rel = np.linalg.norm(X - o["X"]) / np.linalg.norm(o["X"])
    assert rel <= 64 * n * kap * EPS, (rel, kap)
    kap1 = np.linalg.cond(A, 1)
    diff = np.max(np.abs(X - o["X"]))
    assert diff <= 64 * n * kap1 * EPS * np.max(np.abs(o["X"])), (diff, kap1)
    assert r["det_sign"] == o["det_sign"]
    S_used = [min(x0, 7), min(max(x0, 5), 7), 7][r["rung"]]
    rel_tol = min(0.25, max(1e-12, n * kap * 2.0 ** (-8 * S_used)))
    assert abs(r["det_log2"] - o["det_log2"]) <= rel_tol * max(1.0, abs(o["det_log2"])), \
        (r["det_log2"], o["det_log2"], S_used)


def test_mixed_ladder_climbs_when_x0_too_coarse():
    """kappa = 1e6 with 1-slice X0 cannot contract (2^-8 kappa >> 1): the ladder moves up."""
    n = 400
    A32 = wl.svd_conditioned(n, 1e6, seed=77, dtype=np.float32)
    r = gj.invert_mixed(torch.from_numpy(np.asfortranarray(A32)).cuda(), x0_slices=1, tol=1e-12)
    assert r["status"] == 0 and r["rung"] >= 1


def test_mixed_reports_nonconvergence():
    n = 200
    A32 = wl.svd_conditioned(n, 1e2, seed=78, dtype=np.float32)
    r = gj.invert_mixed(torch.from_numpy(np.asfortranarray(A32)).cuda(), x0_slices=3, tol=1e-30, max_iter=3)
    assert r["status"] == gj.NOT_CONVERGED and r["resid"] < 1e-13


@pytest.mark.parametrize("prec", [gj.PREC_FP64, gj.PREC_BF16, gj.PREC_FP16, gj.PREC_SPLIT_BF16_3, gj.PREC_TF32x3])
def test_mixed_prec_names_the_slice_counts(prec):
    """gj_invert_mixed_prec is gj_invert_mixed with the documented slice count of each gj_prec
    value: bitwise the same X, residual, rung and determinant."""
    n = 260
    A32 = wl.svd_conditioned(n, 1e3, seed=90, dtype=np.float32)
    dA = torch.from_numpy(np.asfortranarray(A32)).cuda()
    a = gj.invert_mixed_prec(dA, prec, tol=1e-12)
    b = gj.invert_mixed(dA, x0_slices=gj.PREC_SLICES[prec], corr_slices=4, tol=1e-12)
    assert a["status"] == b["status"] == 0
    assert torch.equal(a["X"], b["X"])
    for k in ("resid", "iters", "rung", "det_sign", "det_log2"):
        assert a[k] == b[k], k


def test_mixed_prec_rejects_unknown_value():
    dA = torch.zeros((4, 4), dtype=torch.float32, device="cuda").t()  # column-major
    with pytest.raises(gj.GJError):
        gj.invert_mixed_prec(dA, 5)
