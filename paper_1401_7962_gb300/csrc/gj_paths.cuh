// gj_paths.cuh -- multi-kernel single-matrix paths (large n).
#pragma once

#include "gj_internal.cuh"

namespace gj {

// Right-hand sides for A X = B (m == 0: inversion).  B (n x m, ld ldb) is appended to the
// working array as extra columns that every step updates like the columns of A (eqs. 3-10
// with B in the place of D); X (n x m, ld ldx) receives A^-1 B.  In this mode the inverse
// itself is not formed: column updates left of the current panel, which only carry the
// inverse, are skipped.
struct Rhs {
  int64_t m = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  double* X = nullptr;
  int64_t ldx = 0;
};

// Blocked Gauss-Jordan (partial or no pivoting): panels of width b eliminated by one
// thread-block cluster, then a rank-b update of all other columns.  A (ld lda) -> X (ld n).
// update: 0 = automatic (tensor-core update from kTensorUpdateMinN), 1 = FP64 FMA, 2 = tensor
// cores with `slices` digit slices (0 = 7, the FP64 level).
constexpr int kTensorUpdateMinN = 512;
// lookahead: 0 = automatic (on for the tensor-core update from kLookaheadMinN), 1 = off, 2 = on.
// update_sms: SMs of the wide update's grid under look-ahead (0 = automatic).
constexpr int kLookaheadMinN = 2048;
gj_status run_blocked(int64_t n, const double* A, int64_t lda, double* X, int pivot_mode, double tau, int panel,
                      int update, int slices, const CtaOut& out, cudaStream_t s, const Rhs* rhs = nullptr,
                      int lookahead = 0, int update_sms = 0);

// Rows per CTA that the calling host thread's blocked calls aim at when they size the panel
// cluster (default 256; at most 16 CTAs per cluster).  The batched mixed path's workers use
// 128: more CTAs per cluster halve each CTA's FP64 work per pivot step.
void set_thread_panel_rows(int rows);

// Unblocked Gauss-Jordan over the whole grid, one rank-1 step per launch (any pivoting).
gj_status run_unblocked(int64_t n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                        const CtaOut& out, cudaStream_t s, const Rhs* rhs = nullptr);

}  // namespace gj
