/*
 * gj_oracle.c -- plain, slow, double-precision CPU reference of the Gauss-Jordan
 * inversion in "Numerical application and Turbo C program using the Gauss-Jordan
 * method" (arXiv:1401.7962).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or call
 * this file; only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Section 2 of the paper):
 * (gjo_invert; gjo_solve applies the same steps to [A | B] for right-hand sides B, below)
 *   - initialisation A^0 = A, D^0 = I (eqs. 1-2);
 *   - n steps, each: pivot selection (observations 2-3), pivot-row scaling by the
 *     pivot (eq. 14), and elimination of the pivot column from every other row
 *     (eq. 15).  The pair [A | D] is held in ONE n x n array: at step k the column
 *     of A that becomes a unit column is replaced by the column of D that stops
 *     being one (the compact form equivalent to eqs. 3-10, which is also what the
 *     paper's program does when it sets the diagonal to 1 before dividing);
 *   - at the end the row and column interchanges are undone in reverse order
 *     (observation 3 and the conclusions): a row interchange of A becomes a column
 *     interchange of the inverse, a column interchange of A a row interchange;
 *   - det A is the product of the pivots (eq. 13), with one sign change per
 *     nontrivial interchange, returned as a sign and log2|det|.
 *
 * Readings of the paper taken here (each listed in the design notes):
 *   - eq. 15's second line is read with d_kj, not a_kj (eq. 8 has it right);
 *   - pivoting uses the largest absolute value (observation 3); ties go to the
 *     first candidate in scan order: smallest row position for partial pivoting
 *     (the strict '>' of the paper's program), smallest column position and then
 *     smallest row position for full pivoting;
 *   - the "zero threshold" of observation 2 is a parameter tau (default 0): a step
 *     fails when the largest candidate magnitude is <= tau;
 *   - a NaN or infinite candidate makes the step fail with status NONFINITE;
 *   - mode PAPER_SIGNED reproduces the program's signed search (largest value,
 *     not magnitude, starting from q = 0, no interchange when no candidate is
 *     positive).
 *
 * Arithmetic: binary64, round to nearest, compiled with -ffp-contract=off so that
 * every multiply and subtract of eq. 15 is rounded separately.  Division is a true
 * division per element, as in eq. 14.  log2|det| is summed in step order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  GJO_OK = 0,
  GJO_SINGULAR = 1,
  GJO_ZERO_PIVOT = 2,
  GJO_NONFINITE = 3,
  GJO_ERR_ARG = -1,
  GJO_ERR_NOMEM = -3
};

enum { GJO_PIVOT_NONE = 0, GJO_PIVOT_PARTIAL = 1, GJO_PIVOT_FULL = 2, GJO_PIVOT_PAPER_SIGNED = 3 };

/* Row-major working array x[i][j] -> x[i * n + j]; the elimination loop of
 * eq. 15 then runs along contiguous memory. */
#define X_(i, j) x[(size_t)(i) * (size_t)n + (size_t)(j)]

static void swap_rows(double* x, int64_t n, int64_t a, int64_t b) {
  for (int64_t l = 0; l < n; ++l) {
    double t = X_(a, l);
    X_(a, l) = X_(b, l);
    X_(b, l) = t;
  }
}

static void swap_cols(double* x, int64_t n, int64_t a, int64_t b) {
  for (int64_t l = 0; l < n; ++l) {
    double t = X_(l, a);
    X_(l, a) = X_(l, b);
    X_(l, b) = t;
  }
}

/*
 * gjo_invert: invert the n x n column-major matrix A (leading dimension lda) into
 * the column-major n x n array X (leading dimension n).
 *
 * Outputs (each optional, may be NULL):
 *   det_sign  : +1 / -1, 0 when the inversion failed
 *   det_log2  : sum over steps of log2|pivot|, -inf when the inversion failed
 *   piv_rows  : [n] row position interchanged with position k at step k
 *   piv_cols  : [n] column position interchanged with position k at step k
 *   pivots    : [n] pivot value a_kk^{k-1} used at step k (eq. 13 factors)
 *   gaps      : [n] (best - second best)/best over the candidate magnitudes at step k
 *               (1 when there is a single candidate; 0 when best == 0)
 *   fail_step : step at which the inversion failed, -1 on success
 * Returns a status code (GJO_*).  On failure X holds the partially reduced array.
 */
int gjo_invert(int64_t n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
               int* det_sign, double* det_log2, int32_t* piv_rows, int32_t* piv_cols,
               double* pivots, double* gaps, int64_t* fail_step) {
  if (det_sign) *det_sign = 0;
  if (det_log2) *det_log2 = -INFINITY;
  if (fail_step) *fail_step = -1;
  if (n < 0 || lda < (n > 0 ? n : 1) || pivot_mode < 0 || pivot_mode > 3 || !(tau >= 0.0))
    return GJO_ERR_ARG;
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    if (det_log2) *det_log2 = 0.0;
    return GJO_OK;
  }
  if (!A || !X) return GJO_ERR_ARG;

  double* x = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  int64_t* prow = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* pcol = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!x || !prow || !pcol) {
    free(x); free(prow); free(pcol);
    return GJO_ERR_NOMEM;
  }

  /* eqs. 1-2: A^0 = A; D^0 = I is implicit in the compact array. */
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) X_(i, j) = A[(size_t)i + (size_t)j * (size_t)lda];

  int sign = 1;
  double lg = 0.0;
  int status = GJO_OK;

  for (int64_t k = 0; k < n; ++k) {
    /* ---- pivot selection: observations 2-3 ---- */
    int64_t r = k, c = k;
    double best = -1.0, second = -1.0;
    int ncand = 0, nonfinite = 0;
    if (pivot_mode == GJO_PIVOT_NONE) {
      best = fabs(X_(k, k));
      ncand = 1;
      if (!isfinite(X_(k, k))) nonfinite = 1;
    } else if (pivot_mode == GJO_PIVOT_PARTIAL) {
      for (int64_t i = k; i < n; ++i) {
        double v = fabs(X_(i, k));
        ++ncand;
        if (!isfinite(X_(i, k))) nonfinite = 1;
        if (v > best) { second = best; best = v; r = i; }
        else if (v > second) second = v;
      }
    } else if (pivot_mode == GJO_PIVOT_FULL) {
      /* scan column by column, each column top to bottom */
      for (int64_t j = k; j < n; ++j)
        for (int64_t i = k; i < n; ++i) {
          double v = fabs(X_(i, j));
          ++ncand;
          if (!isfinite(X_(i, j))) nonfinite = 1;
          if (v > best) { second = best; best = v; r = i; c = j; }
          else if (v > second) second = v;
        }
    } else { /* GJO_PIVOT_PAPER_SIGNED: the program's signed search */
      double q = 0.0;
      for (int64_t i = k; i < n; ++i) {
        ++ncand;
        if (!isfinite(X_(i, k))) nonfinite = 1;
        if (X_(i, k) > q) { q = X_(i, k); r = i; }
      }
      best = fabs(X_(r, k));
      second = -1.0;
    }
    if (gaps) {
      if (ncand <= 1 || second < 0.0) gaps[k] = 1.0;
      else if (best > 0.0 && isfinite(best)) gaps[k] = (best - second) / best;
      else gaps[k] = 0.0;
    }
    if (nonfinite || !isfinite(best)) { status = GJO_NONFINITE; if (fail_step) *fail_step = k; break; }
    if (best <= tau) {
      status = (pivot_mode == GJO_PIVOT_NONE || pivot_mode == GJO_PIVOT_PAPER_SIGNED) ? GJO_ZERO_PIVOT
                                                                                   : GJO_SINGULAR;
      if (fail_step) *fail_step = k;
      break;
    }

    /* ---- interchanges (observation 2) ---- */
    if (r != k) { swap_rows(x, n, k, r); sign = -sign; }
    if (c != k) { swap_cols(x, n, k, c); sign = -sign; }
    prow[k] = r;
    pcol[k] = c;
    if (piv_rows) piv_rows[k] = (int32_t)r;
    if (piv_cols) piv_cols[k] = (int32_t)c;

    /* ---- eq. 13 factor ---- */
    double q = X_(k, k);
    if (pivots) pivots[k] = q;
    if (q < 0.0) sign = -sign;
    lg += log2(fabs(q));

    /* ---- eq. 14: pivot row of A and of D divided by the pivot.  The A column k
     * becomes the unit column and its slot takes D's column k, whose pivot-row
     * entry is 1 before the division. ---- */
    X_(k, k) = 1.0;
    for (int64_t j = 0; j < n; ++j) X_(k, j) = X_(k, j) / q;

    /* ---- eq. 15: every other row minus a_ik times the new pivot row.  Before the
     * update the slot (i,k) is set to D's entry, 0, so it ends at -a_ik/a_kk. ---- */
    for (int64_t i = 0; i < n; ++i) {
      if (i == k) continue;
      double a_ik = X_(i, k);
      X_(i, k) = 0.0;
      for (int64_t j = 0; j < n; ++j) X_(i, j) = X_(i, j) - X_(k, j) * a_ik;
    }
  }

  if (status == GJO_OK) {
    /* ---- undo the interchanges in reverse order (observation 3) ---- */
    for (int64_t k = n - 1; k >= 0; --k) {
      if (prow[k] != k) swap_cols(x, n, k, prow[k]);
      if (pcol[k] != k) swap_rows(x, n, k, pcol[k]);
    }
    if (det_sign) *det_sign = sign;
    if (det_log2) *det_log2 = lg;
  }

  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) X[(size_t)i + (size_t)j * (size_t)n] = X_(i, j);

  free(x);
  free(prow);
  free(pcol);
  return status;
}

/*
 * gjo_invert_many: the same inversion applied to `count` independent matrices
 * (the batched workload).  Matrix m has order n[m], column-major input at
 * A + a_off[m] with leading dimension n[m], output at X + x_off[m].  Results per
 * matrix go to status[m], det_sign[m], det_log2[m].  Plain loop; a caller that
 * wants several cores splits the range [m0, m1) across threads.
 */
void gjo_invert_range(int64_t m0, int64_t m1, const int32_t* n, const double* A, const int64_t* a_off,
                      double* X, const int64_t* x_off, int pivot_mode, int32_t* status,
                      int32_t* det_sign, double* det_log2) {
  for (int64_t m = m0; m < m1; ++m) {
    int s = 0;
    double l = 0.0;
    int st = gjo_invert(n[m], A + a_off[m], n[m] > 0 ? n[m] : 1, X + x_off[m], pivot_mode, 0.0, &s, &l,
                        NULL, NULL, NULL, NULL, NULL);
    status[m] = st;
    det_sign[m] = s;
    det_log2[m] = l;
  }
}

/*
 * gjo_solve: solve A X = B for the n x n column-major A (leading dimension lda) and the
 * n x m column-major right-hand sides B (leading dimension ldb) by the Gauss-Jordan sweep
 * of Section 2 with B in the place of D: eqs. 3-10 with d replaced by the columns of B.
 * At step k (after the pivot selection and interchanges of observations 2-3, chosen
 * exactly as in gjo_invert, on the columns of A only):
 *   eq. 3:  a_kj <- a_kj / a_kk                 for the columns j of A after k
 *   eq. 4:  b_kj <- b_kj / a_kk                 for every column j of B
 *   eq. 7:  a_ij <- a_ij - a_ik a_kj            for i != k, the columns j of A after k
 *   eq. 8:  b_ij <- b_ij - a_ik b_kj            for i != k, every column j of B
 * (column k of A becomes the unit column and is not needed again).  Row interchanges move
 * whole rows of [A | B] and need no undoing; a column interchange of A exchanges two
 * unknowns, so at the end the rows of the solution are exchanged back in reverse order.
 * X (n x m, leading dimension ldx) receives A^-1 B.  Outputs and statuses as for
 * gjo_invert.  The working array is row-major n x (n + m).
 */
int gjo_solve(int64_t n, int64_t m, const double* A, int64_t lda, const double* B, int64_t ldb, double* X,
              int64_t ldx, int pivot_mode, double tau, int* det_sign, double* det_log2, int32_t* piv_rows,
              int32_t* piv_cols, double* pivots, int64_t* fail_step) {
  if (det_sign) *det_sign = 0;
  if (det_log2) *det_log2 = -INFINITY;
  if (fail_step) *fail_step = -1;
  if (n < 0 || m < 0 || lda < (n > 0 ? n : 1) || ldb < (n > 0 ? n : 1) || ldx < (n > 0 ? n : 1) ||
      pivot_mode < 0 || pivot_mode > 3 || !(tau >= 0.0))
    return GJO_ERR_ARG;
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    if (det_log2) *det_log2 = 0.0;
    return GJO_OK;
  }
  if (!A || (m > 0 && (!B || !X))) return GJO_ERR_ARG;

  const int64_t w = n + m; /* row length of the working array [A | B] */
  double* y = (double*)malloc(sizeof(double) * (size_t)n * (size_t)w);
  int64_t* pcol = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!y || !pcol) {
    free(y); free(pcol);
    return GJO_ERR_NOMEM;
  }
#define Y_(i, j) y[(size_t)(i) * (size_t)w + (size_t)(j)]
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) Y_(i, j) = A[(size_t)i + (size_t)j * (size_t)lda];
    for (int64_t j = 0; j < m; ++j) Y_(i, n + j) = B[(size_t)i + (size_t)j * (size_t)ldb];
  }

  int sign = 1;
  double lg = 0.0;
  int status = GJO_OK;
  for (int64_t k = 0; k < n; ++k) {
    /* ---- pivot selection over the columns of A (observations 2-3) ---- */
    int64_t r = k, c = k;
    double best = -1.0;
    int nonfinite = 0;
    if (pivot_mode == GJO_PIVOT_NONE) {
      best = fabs(Y_(k, k));
      if (!isfinite(Y_(k, k))) nonfinite = 1;
    } else if (pivot_mode == GJO_PIVOT_PARTIAL) {
      for (int64_t i = k; i < n; ++i) {
        if (!isfinite(Y_(i, k))) nonfinite = 1;
        if (fabs(Y_(i, k)) > best) { best = fabs(Y_(i, k)); r = i; }
      }
    } else if (pivot_mode == GJO_PIVOT_FULL) {
      for (int64_t j = k; j < n; ++j) { /* column by column, each top to bottom */
        for (int64_t i = k; i < n; ++i) {
          if (!isfinite(Y_(i, j))) nonfinite = 1;
          if (fabs(Y_(i, j)) > best) { best = fabs(Y_(i, j)); r = i; c = j; }
        }
      }
    } else {
      double q = 0.0;
      for (int64_t i = k; i < n; ++i) {
        if (!isfinite(Y_(i, k))) nonfinite = 1;
        if (Y_(i, k) > q) { q = Y_(i, k); r = i; }
      }
      best = fabs(Y_(r, k));
    }
    if (nonfinite || !isfinite(best)) { status = GJO_NONFINITE; if (fail_step) *fail_step = k; break; }
    if (!(best > tau)) { /* observation 2: no usable pivot */
      status = (pivot_mode == GJO_PIVOT_NONE || pivot_mode == GJO_PIVOT_PAPER_SIGNED) ? GJO_ZERO_PIVOT
                                                                                   : GJO_SINGULAR;
      if (fail_step) *fail_step = k;
      break;
    }
    /* ---- interchanges: whole rows of [A | B]; columns of A only ---- */
    if (r != k) {
      for (int64_t j = 0; j < w; ++j) { double t = Y_(k, j); Y_(k, j) = Y_(r, j); Y_(r, j) = t; }
      sign = -sign;
    }
    if (c != k) {
      for (int64_t i = 0; i < n; ++i) { double t = Y_(i, k); Y_(i, k) = Y_(i, c); Y_(i, c) = t; }
      sign = -sign;
    }
    pcol[k] = c;
    if (piv_rows) piv_rows[k] = (int32_t)r;
    if (piv_cols) piv_cols[k] = (int32_t)c;
    const double q = Y_(k, k);
    if (pivots) pivots[k] = q;
    if (q < 0.0) { sign = -sign; } /* eq. 13 */
    lg = lg + log2(fabs(q));
    /* ---- eqs. 3-4: the pivot row after column k, divided by the pivot ---- */
    for (int64_t j = k + 1; j < w; ++j) Y_(k, j) = Y_(k, j) / q;
    Y_(k, k) = 1.0;
    /* ---- eqs. 7-8: every other row ---- */
    for (int64_t i = 0; i < n; ++i) {
      if (i == k) continue;
      const double a_ik = Y_(i, k);
      for (int64_t j = k + 1; j < w; ++j) Y_(i, j) = Y_(i, j) - a_ik * Y_(k, j);
      Y_(i, k) = 0.0;
    }
  }
  if (status == GJO_OK) {
    /* ---- exchanged unknowns back, in reverse order ---- */
    for (int64_t k = n - 1; k >= 0; --k)
      if (pcol[k] != k)
        for (int64_t j = n; j < w; ++j) { double t = Y_(k, j); Y_(k, j) = Y_(pcol[k], j); Y_(pcol[k], j) = t; }
    for (int64_t j = 0; j < m; ++j)
      for (int64_t i = 0; i < n; ++i) X[(size_t)i + (size_t)j * (size_t)ldx] = Y_(i, n + j);
    if (det_sign) *det_sign = sign;
    if (det_log2) *det_log2 = lg;
  }
#undef Y_
  free(y);
  free(pcol);
  return status;
}
