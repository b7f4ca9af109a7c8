"""Comparison of a CUDA result with the CPU oracle on the same seeded input.

Tolerances (derived from binary64 arithmetic):
  * status, det sign: equal;
  * pivot sequence: identical when the oracle's smallest relative gap between the best
    and second-best candidate exceeds 1e-9 (the two sides round differently -- FMA
    contraction, reciprocal-multiply for eq. 14, reduction order -- so only a gap far
    above the rounding noise fixes the choice); else the sequence is not compared and
    the result is checked for validity only;
  * normalised residual ||A X - I||_F / (n ||A||_F ||X||_F) <= 1e-14;
  * |log2|det|_gpu - log2|det|_oracle| <= 1e-12 * max(1, |log2|det||);
  * element by element |X_gpu - X_oracle| <= 64 n kappa_1(A) eps max|X_oracle|: both are
    computed by eliminations whose forward error is bounded by a small multiple of
    n kappa eps ||X||, so their difference is too.
"""
from __future__ import annotations

import numpy as np

import oracle

EPS = float(np.finfo(np.float64).eps)


def tie_free_seed(make, seed: int, mode: int, max_tries: int = 20, gap: float = 1e-9):
    """First seed >= `seed` whose matrix has all oracle pivot gaps > `gap` (seed + 1 on failure)."""
    for s in range(seed, seed + max_tries):
        A = make(s)
        o = oracle.invert(A, mode)
        if o["status"] == 0 and (A.shape[0] == 0 or o["gaps"].min() > gap):
            return s, A, o
    raise AssertionError("no tie-free seed found")


def norm_resid(A: np.ndarray, X: np.ndarray) -> float:
    n = A.shape[0]
    if n == 0:
        return 0.0
    R = A @ X - np.eye(n)
    return float(np.linalg.norm(R) / (n * np.linalg.norm(A) * np.linalg.norm(X)))


def assert_matches_oracle(A: np.ndarray, r: dict, o: dict, mode: int, check_pivots: bool = True,
                          X: np.ndarray | None = None):
    n = A.shape[0]
    assert r["status"] == o["status"], (r["status"], o["status"])
    if o["status"] != 0:
        assert r["det_sign"] == 0
        assert r["fail_step"] == o["fail_step"], (r["fail_step"], o["fail_step"])
        return
    X = np.asarray(X if X is not None else r["X"])
    assert r["det_sign"] == o["det_sign"], (r["det_sign"], o["det_sign"])
    assert abs(r["det_log2"] - o["det_log2"]) <= 1e-12 * max(1.0, abs(o["det_log2"])), (r["det_log2"], o["det_log2"])
    tie_free = n == 0 or o["gaps"].min() > 1e-9
    if check_pivots and tie_free and "piv_rows" in r:
        assert np.array_equal(r["piv_rows"], o["piv_rows"]), "row pivot sequence differs"
        if mode == 2:
            assert np.array_equal(r["piv_cols"], o["piv_cols"]), "column pivot sequence differs"
        assert np.allclose(r["pivots"], o["pivots"], rtol=64 * n * EPS * max(1.0, np.linalg.cond(A, 1)), atol=0)
    res = norm_resid(A, X)
    assert res <= 1e-14, res
    if n:
        kappa = np.linalg.cond(A, 1)
        tol = 64 * n * kappa * EPS * np.max(np.abs(o["X"]))
        diff = np.max(np.abs(X - o["X"]))
        assert diff <= tol, (diff, tol)
