"""Pins of a Gauss-Jordan inverter against values that the paper and mathematics fix.

Every pin takes ``inv(A, mode, tau=0.0) -> dict`` (the oracle's result dict:
X, status, det_sign, det_log2, piv_rows, piv_cols, pivots, fail_step) and raises
AssertionError when the inverter disagrees.  The solve pins (``ALL_SOLVE_PINS``) take
``sol(A, B, mode, tau=0.0) -> dict`` with the same keys, X being A^-1 B.  The expected values never come from
the inverter under test: they are closed forms (symmetric Pascal and Hilbert
inverses and determinants), exact integer arithmetic (cofactor expansion,
Fraction forward substitution), special matrices (permutations, diagonal,
orthogonal), invariants (A X = I, X A = I, det A det X = 1), LAPACK through
numpy, or the hand-run of the paper's 3x3 example stored under tests/golden.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np

EPS = float(np.finfo(np.float64).eps)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MODES = {"none": 0, "partial": 1, "full": 2, "paper_signed": 3}
OK, SINGULAR, ZERO_PIVOT, NONFINITE, ERR_ARG = 0, 1, 2, 3, -1


# ---------------------------------------------------------------- exact helpers

def pascal_sym(n: int) -> list[list[int]]:
    """Symmetric Pascal matrix P[i][j] = C(i+j, i) (0-based)."""
    return [[math.comb(i + j, i) for j in range(n)] for i in range(n)]


def pascal_sym_inverse(n: int) -> list[list[int]]:
    """P = L L^T with L[i][j] = C(i, j); L^-1[i][j] = (-1)^(i-j) C(i, j); P^-1 = L^-T L^-1."""
    Li = [[(-1) ** (i - j) * math.comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)]
    return [[sum(Li[k][i] * Li[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def hilbert_inverse(n: int) -> list[list[int]]:
    """Closed-form inverse of the n x n Hilbert matrix (1-based formula)."""
    out = [[0] * n for _ in range(n)]
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            out[i - 1][j - 1] = ((-1) ** (i + j) * (i + j - 1) * math.comb(n + i - 1, n - j)
                                 * math.comb(n + j - 1, n - i) * math.comb(i + j - 2, i - 1) ** 2)
    return out


def hilbert_det(n: int) -> Fraction:
    """det H_n = c_n^4 / c_{2n} with c_n = prod_{i=1}^{n-1} i!."""
    def c(m):
        p = 1
        for i in range(1, m):
            p *= math.factorial(i)
        return p
    return Fraction(c(n) ** 4, c(2 * n))


def det_cofactor(M) -> Fraction:
    """Laplace expansion along the first row, exact over Fractions."""
    M = [[Fraction(v) for v in row] for row in M]
    n = len(M)
    if n == 0:
        return Fraction(1)
    if n == 1:
        return M[0][0]
    total = Fraction(0)
    for j in range(n):
        if M[0][j] == 0:
            continue
        minor = [row[:j] + row[j + 1:] for row in M[1:]]
        total += (-1) ** j * M[0][j] * det_cofactor(minor)
    return total


def inverse_fraction(M) -> list[list[Fraction]]:
    """Exact inverse by Fraction Gaussian elimination with a nonzero-pivot search.

    Independent of the inverter under test: exact rational arithmetic, no
    magnitude pivoting, returns the mathematically exact inverse."""
    n = len(M)
    a = [[Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        pv = a[c][c]
        a[c] = [v / pv for v in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [row[n:] for row in a]


def perm_sign(p) -> int:
    p = list(p)
    s, seen = 1, [False] * len(p)
    for i in range(len(p)):
        if seen[i]:
            continue
        j, L = i, 0
        while not seen[j]:
            seen[j] = True
            j = p[j]
            L += 1
        if L % 2 == 0:
            s = -s
    return s


def rel_resid(A: np.ndarray, X: np.ndarray) -> float:
    """||A X - I||_F / (n ||A||_F ||X||_F), the normalised residual gate."""
    n = A.shape[0]
    R = A @ X - np.eye(n)
    return float(np.linalg.norm(R) / (n * np.linalg.norm(A) * np.linalg.norm(X)))


def log2_close(got: float, want: float, rtol: float = 1e-12) -> bool:
    return abs(got - want) <= rtol * max(1.0, abs(want))


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- pins

def pin_paper_example(inv):
    """Section 3 default matrix: det 1, integer inverse, hand-run pivot sequences."""
    with open(os.path.join(GOLDEN, "paper_example_3x3.json")) as f:
        g = json.load(f)
    A = np.array(g["A"], dtype=np.float64)
    Xe = np.array(g["inverse"], dtype=np.float64)
    for name, exp in g["modes"].items():
        r = inv(A, MODES[name])
        assert r["status"] == OK, (name, r["status"])
        if exp["exact"]:
            assert np.array_equal(r["X"], Xe), (name, r["X"])
        else:
            assert np.max(np.abs(r["X"] - Xe)) <= 16 * EPS * 6, (name, r["X"])
        assert r["det_sign"] == 1, (name, r["det_sign"])
        assert abs(r["det_log2"]) <= 8 * EPS, (name, r["det_log2"])
        assert list(r["piv_rows"]) == exp["piv_rows"], (name, r["piv_rows"])
        assert list(r["piv_cols"]) == exp["piv_cols"], (name, r["piv_cols"])
        pv = [float(Fraction(s)) for s in exp["pivots"]]
        assert np.allclose(r["pivots"], pv, rtol=16 * EPS, atol=0), (name, r["pivots"])


def pin_pascal(inv):
    """Symmetric Pascal P_n: det 1 and the integer inverse L^-T L^-1."""
    for n in range(1, 13):
        P = np.array(pascal_sym(n), dtype=np.float64)
        Pi = np.array(pascal_sym_inverse(n), dtype=np.float64)
        kappa = np.linalg.norm(P, 1) * np.linalg.norm(Pi, 1)
        for mode in (1, 2):
            r = inv(P, mode)
            assert r["status"] == OK
            err = np.linalg.norm(r["X"] - Pi, 1) / np.linalg.norm(Pi, 1)
            assert err <= max(50 * n * kappa * EPS, 4 * EPS), (n, mode, err)
            assert r["det_sign"] == 1
            assert abs(r["det_log2"]) <= max(1e-12, 50 * n * kappa * EPS), (n, r["det_log2"])


def pin_hilbert(inv):
    """Hilbert H_n: closed-form integer inverse and det = c_n^4 / c_2n."""
    for n in range(1, 11):
        H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
        Hi = np.array(hilbert_inverse(n), dtype=np.float64)
        kappa = np.linalg.norm(H, 1) * np.linalg.norm(Hi, 1)
        lg = math.log2(hilbert_det(n).numerator) - math.log2(hilbert_det(n).denominator)
        for mode in (1, 2):
            r = inv(H, mode)
            assert r["status"] == OK
            err = np.linalg.norm(r["X"] - Hi, 1) / np.linalg.norm(Hi, 1)
            assert err <= 50 * n * kappa * EPS, (n, mode, err)
            assert r["det_sign"] == 1
            assert abs(r["det_log2"] - lg) <= max(1e-12 * abs(lg), 50 * n * kappa * EPS), (n, r["det_log2"], lg)


def pin_cofactor_det(inv):
    """Integer matrices n <= 7: det by cofactor expansion (exact), also as the eq. 13 pivot product."""
    g = _rng(7)
    for n in range(1, 8):
        for _ in range(6):
            M = g.integers(-9, 10, size=(n, n))
            d = det_cofactor(M.tolist())
            if d == 0:
                continue
            for mode in (1, 2):
                r = inv(M.astype(np.float64), mode)
                assert r["status"] == OK
                assert r["det_sign"] == (1 if d > 0 else -1), (M, d, r["det_sign"])
                want = math.log2(abs(d))
                assert log2_close(r["det_log2"], want, 1e-12), (n, r["det_log2"], want)
                # eq. 13 with one sign change per interchange
                nsw = sum(int(a != k) for k, a in enumerate(r["piv_rows"])) + \
                    sum(int(a != k) for k, a in enumerate(r["piv_cols"]))
                prod = (-1) ** nsw * np.prod(r["pivots"])
                assert abs(prod - float(d)) <= 1e-10 * abs(float(d)), (prod, d)
                Xe = np.array([[float(v) for v in row] for row in inverse_fraction(M.tolist())])
                assert np.max(np.abs(r["X"] - Xe)) <= 1e-9 * max(1.0, np.max(np.abs(Xe))), (M, r["X"], Xe)


def pin_permutation(inv):
    """Permutation matrices: inverse is the transpose, det is the permutation sign, all exact."""
    g = _rng(11)
    for n in range(1, 13):
        for _ in range(4):
            p = g.permutation(n)
            P = np.zeros((n, n))
            P[np.arange(n), p] = 1.0
            for mode in (1, 2, 3):
                r = inv(P, mode)
                assert r["status"] == OK, (p, mode)
                assert np.array_equal(r["X"], P.T), (p, mode, r["X"])
                assert r["det_sign"] == perm_sign(p), (p, mode, r["det_sign"])
                assert r["det_log2"] == 0.0
            r = inv(P, 0)
            if p[0] != 0:
                assert r["status"] == ZERO_PIVOT and r["fail_step"] == 0


def pin_diagonal(inv):
    """Diagonal with power-of-two entries: exact reciprocal inverse and det."""
    g = _rng(13)
    for n in range(1, 20):
        e = g.integers(-20, 21, size=n)
        s = g.choice([-1.0, 1.0], size=n)
        d = s * np.ldexp(1.0, e)
        D = np.diag(d)
        for mode in (0, 1, 2):
            r = inv(D, mode)
            assert r["status"] == OK
            assert np.array_equal(r["X"], np.diag(1.0 / d)), (mode, r["X"])
            assert r["det_sign"] == int(np.prod(s)), mode
            assert r["det_log2"] == float(np.sum(e)), (r["det_log2"], np.sum(e))


def pin_triangular(inv):
    """Unit lower / upper triangular integer matrices: exact integer inverse, det 1."""
    g = _rng(17)
    for n in range(2, 12):
        L = np.tril(g.integers(-3, 4, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
        Li = np.array([[float(v) for v in row] for row in inverse_fraction(L.tolist())])
        # no pivoting: every step divides by 1, all arithmetic is on integers -> exact
        r = inv(L.astype(np.float64), 0)
        assert r["status"] == OK and np.array_equal(r["X"], Li), r["X"]
        r = inv(L.T.astype(np.float64), 0)
        assert r["status"] == OK and np.array_equal(r["X"], Li.T)
        for mode in (1, 2):
            for M, Mi in ((L, Li), (L.T, Li.T)):
                r = inv(M.astype(np.float64), mode)
                assert r["status"] == OK
                assert np.max(np.abs(r["X"] - Mi)) <= 1e-9 * max(1.0, np.max(np.abs(Mi))), (mode, r["X"], Mi)
                assert r["det_sign"] == 1 and abs(r["det_log2"]) <= 1e-9


def pin_orthogonal(inv):
    """Orthogonal Q (QR of a Gaussian matrix): inverse is Q^T, |det| = 1."""
    g = _rng(19)
    for n in (1, 2, 5, 16, 40):
        Q, _ = np.linalg.qr(g.standard_normal((n, n)))
        sgn = 1 if np.linalg.det(Q) > 0 else -1
        for mode in (1, 2):
            r = inv(Q, mode)
            assert r["status"] == OK
            assert np.max(np.abs(r["X"] - Q.T)) <= 64 * n * EPS, (n, mode)
            assert r["det_sign"] == sgn
            assert abs(r["det_log2"]) <= 64 * n * EPS


def pin_invariants_random(inv):
    """Random N(0,1): A X = I and X A = I (normalised), det A det X = 1, inv(inv A) = A."""
    g = _rng(23)
    for n in (1, 2, 3, 5, 17, 64, 100):
        A = g.standard_normal((n, n))
        for mode in (1, 2):
            r = inv(A, mode)
            assert r["status"] == OK
            X = r["X"]
            assert rel_resid(A, X) <= 1e-15, (n, mode, rel_resid(A, X))
            assert rel_resid(X, A) <= 1e-15, (n, mode)
            r2 = inv(X, mode)
            assert r2["status"] == OK
            assert r2["det_sign"] == r["det_sign"]
            assert abs(r2["det_log2"] + r["det_log2"]) <= 1e-10 * max(1.0, abs(r["det_log2"]))
            kappa = np.linalg.cond(A)
            assert np.max(np.abs(r2["X"] - A)) <= 100 * n * kappa * EPS * np.max(np.abs(A))


def pin_numpy_crosscheck(inv):
    """LAPACK getrf/getri (numpy) for values: inverse and slogdet."""
    g = _rng(29)
    for n in (4, 33, 128, 200):
        A = g.standard_normal((n, n))
        Xn = np.linalg.inv(A)
        s, ld = np.linalg.slogdet(A)
        kappa = np.linalg.cond(A)
        for mode in (1, 2):
            r = inv(A, mode)
            assert r["status"] == OK
            assert np.linalg.norm(r["X"] - Xn) / np.linalg.norm(Xn) <= 20 * n * kappa * EPS
            assert r["det_sign"] == int(s)
            assert log2_close(r["det_log2"], ld / math.log(2.0), 1e-12)


def pin_pivot_rule(inv):
    """Observation 3: the largest |a| is chosen, not the largest signed value."""
    A = np.array([[1.0, 2.0, 0.5], [0.5, 1.0, 3.0], [-4.0, 1.0, 1.0]])
    r = inv(A, 1)
    assert r["piv_rows"][0] == 2, r["piv_rows"]       # |-4| is the largest magnitude in column 0
    r = inv(A, 3)
    assert r["piv_rows"][0] == 0, r["piv_rows"]       # the program's signed search keeps +1 (row 0)
    B = np.array([[1.0, 0.0, 2.0], [0.0, -9.0, 1.0], [3.0, 1.0, 1.0]])
    r = inv(B, 2)
    assert (r["piv_rows"][0], r["piv_cols"][0]) == (1, 1), (r["piv_rows"], r["piv_cols"])
    assert r["pivots"][0] == -9.0


def pin_tie_rule(inv):
    """Ties: smallest row position (partial); smallest column, then row position (full)."""
    A = np.array([[2.0, 1.0, 0.0], [-2.0, 0.0, 1.0], [2.0, 5.0, 1.0]])
    r = inv(A, 1)
    assert r["piv_rows"][0] == 0
    B = np.array([[1.0, 7.0, 0.0], [7.0, 1.0, -7.0], [0.0, 7.0, 1.0]])
    r = inv(B, 2)
    # candidates equal to 7 at (1,0), (0,1), (2,1), (1,2): column 0 comes first
    assert (r["piv_rows"][0], r["piv_cols"][0]) == (1, 0), (r["piv_rows"], r["piv_cols"])


def pin_diag_dominant_identity(inv):
    """Columns dominated by the diagonal (N(0,1) + 0.1 n I with n large enough): no interchange."""
    g = _rng(31)
    n = 256
    A = g.standard_normal((n, n)) + 0.1 * n * np.eye(n)
    r = inv(A, 1)
    assert r["status"] == OK
    assert np.array_equal(r["piv_rows"], np.arange(n))


def pin_row_swap_flips_det(inv):
    """det(P A) = -det(A) for one row interchange P; inverse columns interchange."""
    g = _rng(37)
    n = 9
    A = g.standard_normal((n, n))
    B = A.copy()
    B[[2, 6]] = B[[6, 2]]
    ra, rb = inv(A, 1), inv(B, 1)
    assert rb["det_sign"] == -ra["det_sign"]
    assert abs(rb["det_log2"] - ra["det_log2"]) <= 1e-12 * max(1.0, abs(ra["det_log2"]))
    Xs = ra["X"].copy()
    Xs[:, [2, 6]] = Xs[:, [6, 2]]
    assert np.max(np.abs(rb["X"] - Xs)) <= 1e-12 * np.max(np.abs(Xs))


def pin_failures(inv):
    """Observation 2: zero pivots, singular matrices, non-finite input, empty input."""
    # zero pivot without pivoting is not singularity: [[0,1],[1,0]]
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert inv(S, 0)["status"] == ZERO_PIVOT
    r = inv(S, 1)
    assert r["status"] == OK and np.array_equal(r["X"], S) and r["det_sign"] == -1
    # exactly singular: zero column 2 -> partial pivoting fails when it reaches column 2
    Z = np.array([[1.0, 2.0, 0.0], [3.0, 4.0, 0.0], [5.0, 6.0, 0.0]])
    r = inv(Z, 1)
    assert r["status"] == SINGULAR and r["fail_step"] == 2 and r["det_sign"] == 0 and r["det_log2"] == -math.inf
    r = inv(Z, 2)
    assert r["status"] == SINGULAR and r["fail_step"] == 2
    # duplicate rows, integer entries (exact elimination) -> singular at the last step
    D = np.array([[2.0, 1.0, 1.0], [4.0, 3.0, 3.0], [2.0, 1.0, 1.0]])
    assert inv(D, 1)["status"] == SINGULAR
    assert inv(D, 2)["status"] == SINGULAR
    # the zero matrix fails at step 0
    assert inv(np.zeros((4, 4)), 2)["fail_step"] == 0
    # non-finite candidates
    N = np.eye(3)
    N[1, 0] = np.nan
    assert inv(N, 1)["status"] == NONFINITE
    N = np.eye(3)
    N[2, 2] = np.inf
    assert inv(N, 2)["status"] == NONFINITE
    # empty matrix: empty product
    r = inv(np.zeros((0, 0)), 1)
    assert r["status"] == OK and r["det_sign"] == 1 and r["det_log2"] == 0.0
    # zero threshold tau (observation 2)
    E = np.diag([1.0, 1e-3, 1.0])
    assert inv(E, 1, tau=1e-2)["status"] == SINGULAR
    assert inv(E, 1, tau=1e-4)["status"] == OK


ALL_PINS = [pin_paper_example, pin_pascal, pin_hilbert, pin_cofactor_det, pin_permutation, pin_diagonal,
            pin_triangular, pin_orthogonal, pin_invariants_random, pin_numpy_crosscheck, pin_pivot_rule,
            pin_tie_rule, pin_diag_dominant_identity, pin_row_swap_flips_det, pin_failures]


# ---------------------------------------------------------------- solve pins (A X = B)

def _int_rhs(n: int, m: int, seed: int) -> list[list[int]]:
    g = _rng(seed)
    return [[int(v) for v in row] for row in g.integers(-9, 10, size=(n, m))]


def _matmul_int(P, Q):
    return [[sum(P[i][t] * Q[t][j] for t in range(len(Q))) for j in range(len(Q[0]))] for i in range(len(P))]


def pin_solve_paper_example(sol):
    """Section 3 matrix: b = A (1, 2, 3)^T gives x = (1, 2, 3) (exactly where the pivots are dyadic); with
    B = I the sweep returns the integer inverse; pivot sequences are the hand-run ones."""
    with open(os.path.join(GOLDEN, "paper_example_3x3.json")) as f:
        g = json.load(f)
    A = np.array(g["A"], dtype=np.float64)
    b = A @ np.array([1.0, 2.0, 3.0])
    for name, exp in g["modes"].items():
        r = sol(A, b[:, None], MODES[name])
        assert r["status"] == OK, (name, r["status"])
        if exp["exact"]:  # dyadic pivots: every intermediate is exact
            assert np.array_equal(r["X"][:, 0], [1.0, 2.0, 3.0]), (name, r["X"])
        else:
            assert np.max(np.abs(r["X"][:, 0] - [1.0, 2.0, 3.0])) <= 16 * EPS * 25, (name, r["X"])
        assert r["det_sign"] == 1 and abs(r["det_log2"]) <= 8 * EPS, name
        assert list(r["piv_rows"]) == exp["piv_rows"], (name, r["piv_rows"])
        assert list(r["piv_cols"]) == exp["piv_cols"], (name, r["piv_cols"])
        r = sol(A, np.eye(3), MODES[name])
        assert np.max(np.abs(r["X"] - np.array(g["inverse"]))) <= 16 * EPS * 6, (name, r["X"])


def pin_solve_pascal(sol):
    """Symmetric Pascal P_n with integer right-hand sides: X = P^-1 B exactly in integers."""
    for n in range(1, 13):
        P = pascal_sym(n)
        Bi = _int_rhs(n, 3, 100 + n)
        Xe = np.array(_matmul_int(pascal_sym_inverse(n), Bi), dtype=np.float64)
        Pf = np.array(P, dtype=np.float64)
        kappa = np.linalg.norm(Pf, 1) * np.linalg.norm(np.array(pascal_sym_inverse(n), dtype=np.float64), 1)
        for mode in (1, 2):
            r = sol(Pf, np.array(Bi, dtype=np.float64), mode)
            assert r["status"] == OK
            scale = np.linalg.norm(np.array(pascal_sym_inverse(n), dtype=np.float64), 1) * \
                np.max(np.abs(np.array(Bi, dtype=np.float64))) * 3
            err = np.max(np.abs(r["X"] - Xe)) / max(scale, 1.0)
            assert err <= max(50 * n * kappa * EPS, 4 * EPS), (n, mode, err)


def pin_solve_hilbert(sol):
    """Hilbert H_n: X = H^-1 B with the closed-form integer inverse; det c_n^4 / c_2n."""
    for n in range(1, 9):
        H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
        Hi = hilbert_inverse(n)
        Bi = _int_rhs(n, 2, 200 + n)
        Xe = np.array(_matmul_int(Hi, Bi), dtype=np.float64)
        Hif = np.array(Hi, dtype=np.float64)
        kappa = np.linalg.norm(H, 1) * np.linalg.norm(Hif, 1)
        for mode in (1, 2):
            r = sol(H, np.array(Bi, dtype=np.float64), mode)
            assert r["status"] == OK
            err = np.max(np.abs(r["X"] - Xe)) / max(np.max(np.abs(Xe)), 1.0)
            assert err <= 100 * n * kappa * EPS, (n, mode, err)
            want = math.log2(hilbert_det(n))
            assert abs(r["det_log2"] - want) <= 1e-9 * max(1.0, abs(want)), (n, mode)


def pin_solve_exact_fraction(sol):
    """Integer matrices n <= 6: X = A^-1 B from exact Fraction elimination; det by cofactors."""
    g = _rng(31)
    for n in range(1, 7):
        for _ in range(3):
            M = [[int(v) for v in row] for row in g.integers(-9, 10, size=(n, n))]
            d = det_cofactor(M)
            if d == 0:
                continue
            Bi = _int_rhs(n, 2, 300 + n)
            Mi = inverse_fraction(M)
            Xe = np.array([[float(sum(Mi[i][t] * Bi[t][j] for t in range(n))) for j in range(2)]
                           for i in range(n)])
            A = np.array(M, dtype=np.float64)
            kappa = np.linalg.norm(A, 1) * np.linalg.norm(np.array([[float(v) for v in row] for row in Mi]), 1)
            for mode in (1, 2):
                r = sol(A, np.array(Bi, dtype=np.float64), mode)
                assert r["status"] == OK
                err = np.max(np.abs(r["X"] - Xe)) / max(np.max(np.abs(Xe)), 1.0)
                assert err <= 50 * n * kappa * EPS, (n, mode, err)
                assert r["det_sign"] == (1 if d > 0 else -1)
                assert log2_close(r["det_log2"], math.log2(abs(d)), 1e-12)


def pin_solve_permutation(sol):
    """A permutation matrix: X = P^T B exactly, det = sign of the permutation."""
    g = _rng(41)
    for n in (1, 2, 5, 9):
        p = g.permutation(n)
        P = np.zeros((n, n))
        P[np.arange(n), p] = 1.0
        B = g.standard_normal((n, 3))
        for mode in (1, 2):
            r = sol(P, B, mode)
            assert r["status"] == OK and np.array_equal(r["X"], P.T @ B), (n, mode)
            assert r["det_sign"] == perm_sign(list(p))


def pin_solve_invariants(sol):
    """Random inputs: A X = B at the residual level, solve(A, A) = I, and the pivot sequence
    of the sweep does not depend on the right-hand sides."""
    g = _rng(51)
    for n in (2, 9, 40):
        A = g.standard_normal((n, n)) + 0.5 * np.eye(n)
        B = g.standard_normal((n, 4))
        for mode in (1, 2):
            r = sol(A, B, mode)
            assert r["status"] == OK
            res = np.linalg.norm(A @ r["X"] - B) / (np.linalg.norm(A) * np.linalg.norm(r["X"]) + np.linalg.norm(B))
            assert res <= 50 * n * EPS, (n, mode, res)
            r2 = sol(A, A, mode)
            assert np.max(np.abs(r2["X"] - np.eye(n))) <= 1e-10, (n, mode)
            r3 = sol(A, B[:, :1], mode)
            assert list(r3["piv_rows"]) == list(r["piv_rows"]) and list(r3["piv_cols"]) == list(r["piv_cols"])
            ref = np.linalg.solve(A, B)
            assert np.max(np.abs(r["X"] - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), (n, mode)


def pin_solve_failures(sol):
    """Observation 2 for the solve: zero pivot vs singular, non-finite input, no right-hand side."""
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    b = np.array([[2.0], [3.0]])
    assert sol(S, b, 0)["status"] == ZERO_PIVOT
    r = sol(S, b, 1)
    assert r["status"] == OK and np.array_equal(r["X"], np.array([[3.0], [2.0]])) and r["det_sign"] == -1
    Z = np.array([[1.0, 2.0, 0.0], [3.0, 4.0, 0.0], [5.0, 6.0, 0.0]])
    r = sol(Z, np.ones((3, 1)), 1)
    assert r["status"] == SINGULAR and r["fail_step"] == 2 and r["det_sign"] == 0 and r["det_log2"] == -math.inf
    N = np.eye(3)
    N[1, 0] = np.nan
    assert sol(N, np.ones((3, 1)), 1)["status"] == NONFINITE
    r = sol(np.array([[2.0, 0.0], [0.0, 4.0]]), np.zeros((2, 0)), 1)
    assert r["status"] == OK and r["det_sign"] == 1 and r["det_log2"] == 3.0


ALL_SOLVE_PINS = [pin_solve_paper_example, pin_solve_pascal, pin_solve_hilbert, pin_solve_exact_fraction,
                  pin_solve_permutation, pin_solve_invariants, pin_solve_failures]
