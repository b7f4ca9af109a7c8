"""Write the oracle's result for the 8192 x 8192 partial-pivoting workload to tests/golden/.

The workload is one 8192 x 8192 matrix with i.i.d. N(0,1) entries plus 0.1 n on the
diagonal (seed 1403), inverted with partial pivoting (largest |a| in the pivot column,
observations 2-3 of Section 2).  The plain FP64 oracle (eqs. 13-15, one thread) takes a
few minutes for it, too long for a test, so this script runs it once and stores:

  * a fingerprint of the input (SHA-256 of its column-major bytes), so that a test can
    confirm it regenerated the same matrix;
  * the whole pivot record: the row position chosen at every step, the pivot values
    (the eq. 13 factors) and the relative gap between the best and second-best candidate;
  * det A as sign and log2|det| (eq. 13);
  * 16 whole columns and 16 whole rows of A^-1 at seeded random indices, and 4096
    single entries at seeded random (row, column) pairs;
  * max |x_ij|, the 1-norm and the Frobenius norm of A^-1 (for the tolerances).

Only the oracle and the seeded input generator are called.  Run from the repository root:

    python tests/golden/make_inv8192_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1401_7962_gb300 import workloads as wl  # noqa: E402

N = 8192
SEED = wl.SEED_BASE + 2
SHIFT = 0.1 * N
OUT_NPZ = os.path.join(HERE, "inv8192_partial_oracle.npz")
OUT_JSON = os.path.join(HERE, "inv8192_partial_oracle.json")


def input_matrix() -> np.ndarray:
    return wl.gaussian(N, SEED, shift=SHIFT)


def fingerprint(A: np.ndarray) -> str:
    return hashlib.sha256(np.asfortranarray(A).tobytes(order="F")).hexdigest()


def sample_indices():
    """Seeded sample positions shared by the script and the test."""
    g = np.random.default_rng(81920)
    cols = np.sort(g.choice(N, 16, replace=False))
    rows = np.sort(g.choice(N, 16, replace=False))
    pairs = g.integers(0, N, size=(4096, 2))
    return cols, rows, pairs


def main() -> None:
    A = input_matrix()
    fp = fingerprint(A)
    t0 = time.time()
    o = oracle.invert(A, oracle.PIVOT_PARTIAL)
    dt = time.time() - t0
    assert o["status"] == oracle.OK, o["status"]
    X = o["X"]
    cols, rows, pairs = sample_indices()
    np.savez_compressed(
        OUT_NPZ,
        piv_rows=o["piv_rows"].astype(np.int32),
        pivots=o["pivots"],
        gaps=o["gaps"],
        cols=cols,
        rows=rows,
        X_cols=np.ascontiguousarray(X[:, cols]),
        X_rows=np.ascontiguousarray(X[rows, :]),
        pairs=pairs,
        X_pairs=X[pairs[:, 0], pairs[:, 1]],
        X_absmax=np.array([np.max(np.abs(X))]),
        X_norm1=np.array([np.max(np.sum(np.abs(X), axis=0))]),
        X_normF=np.array([np.linalg.norm(X)]),
    )
    meta = {
        "_source": "Written by tests/golden/make_inv8192_golden.py with the FP64 CPU oracle (oracle/gj_oracle.c: "
                   "eqs. 13-15 and observations 2-3 of Section 2 of arXiv:1401.7962, partial pivoting). "
                   "Input: 8192 x 8192 i.i.d. N(0,1) + 0.1 n I, seed 1403, column-major float64.",
        "n": N,
        "seed": SEED,
        "shift": SHIFT,
        "input_sha256": fp,
        "status": int(o["status"]),
        "det_sign": int(o["det_sign"]),
        "det_log2": float(o["det_log2"]),
        "min_gap": float(o["gaps"].min()),
        "oracle_seconds": round(dt, 1),
    }
    with open(OUT_JSON, "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
