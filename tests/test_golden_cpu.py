"""The stored oracle result of the 8192 x 8192 workload (tests/golden/inv8192_partial_oracle.*)
checked on the CPU against what it must equal, independently of the oracle that wrote it:

  * the seeded generator reproduces the input the golden was computed from (fingerprint);
  * the pivot sequence is the identity: every column of N(0,1) + 0.1 n I is dominated by its
    diagonal entry (|0.1 n + z| against max |z| of ~4.5), and the recorded gaps are large;
  * the 16 stored columns of A^-1 solve A x = e_j, and the 16 stored rows solve x A = e_i, as
    LAPACK's LU solver (a different elimination) computes them, to the forward-error level
    of the well-conditioned input;
  * det A: positive, and log2|det| equals the sum of log2|u_ii| of LAPACK's LU factors, and
    the product of the stored pivots (eq. 13);
  * the scattered entries agree with the stored columns and rows where they overlap.
"""
import json
import os

import numpy as np
import pytest

from paper_1401_7962_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
scipy_linalg = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module")
def golden():
    meta = json.load(open(os.path.join(GOLDEN, "inv8192_partial_oracle.json")))
    ref = np.load(os.path.join(GOLDEN, "inv8192_partial_oracle.npz"))
    A = wl.gaussian(meta["n"], meta["seed"], shift=meta["shift"])
    return meta, ref, A


def test_input_fingerprint(golden):
    import hashlib
    meta, _, A = golden
    assert hashlib.sha256(np.asfortranarray(A).tobytes(order="F")).hexdigest() == meta["input_sha256"]


def test_pivots_are_the_diagonal(golden):
    meta, ref, _ = golden
    n = meta["n"]
    assert np.array_equal(ref["piv_rows"], np.arange(n))
    assert ref["gaps"].min() > 0.5 and meta["min_gap"] == pytest.approx(float(ref["gaps"].min()))


def test_columns_rows_and_det_against_lapack(golden):
    meta, ref, A = golden
    n = meta["n"]
    lu, piv = scipy_linalg.lu_factor(A)
    cols, rows = ref["cols"], ref["rows"]
    E = np.zeros((n, len(cols)))
    E[cols, np.arange(len(cols))] = 1.0
    Xc = scipy_linalg.lu_solve((lu, piv), E)
    Er = np.zeros((n, len(rows)))
    Er[rows, np.arange(len(rows))] = 1.0
    Xr = scipy_linalg.lu_solve((lu, piv), Er, trans=1).T  # rows of A^-1: x^T A = e_i^T
    kappa1 = np.max(np.sum(np.abs(A), axis=0)) * float(ref["X_norm1"][0])
    tol = 64 * n * kappa1 * np.finfo(float).eps * float(ref["X_absmax"][0])
    assert np.max(np.abs(Xc - ref["X_cols"])) <= tol
    assert np.max(np.abs(Xr - ref["X_rows"])) <= tol
    d = np.diag(lu)
    sign = np.prod(np.sign(d)) * (-1) ** int(np.sum(piv != np.arange(n)))
    assert sign == meta["det_sign"] == 1
    lg = float(np.sum(np.log2(np.abs(d))))
    assert abs(lg - meta["det_log2"]) <= 1e-12 * abs(lg)
    assert abs(float(np.sum(np.log2(np.abs(ref["pivots"])))) - meta["det_log2"]) <= 1e-12 * abs(lg)


def test_scattered_entries_consistent(golden):
    meta, ref, _ = golden
    pairs = ref["pairs"]
    cols = {int(c): k for k, c in enumerate(ref["cols"])}
    rows = {int(r): k for k, r in enumerate(ref["rows"])}
    hits = 0
    for (i, j), v in zip(pairs, ref["X_pairs"]):
        if int(j) in cols:
            assert v == ref["X_cols"][i, cols[int(j)]]
            hits += 1
        if int(i) in rows:
            assert v == ref["X_rows"][rows[int(i)], j]
            hits += 1
    assert np.all(np.isfinite(ref["X_pairs"]))
