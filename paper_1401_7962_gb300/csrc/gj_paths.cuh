// gj_paths.cuh -- multi-kernel single-matrix paths (large n).
#pragma once

#include "gj_internal.cuh"

namespace gj {

// Blocked Gauss-Jordan (partial or no pivoting): panels of width b eliminated by one
// thread-block cluster, then a rank-b update of all other columns.  A (ld lda) -> X (ld n).
// update: 0 = automatic (tensor-core update from kTensorUpdateMinN), 1 = FP64 FMA, 2 = tensor
// cores with `slices` digit slices (0 = 8).
constexpr int kTensorUpdateMinN = 512;
gj_status run_blocked(int64_t n, const double* A, int64_t lda, double* X, int pivot_mode, double tau, int panel,
                      int update, int slices, const CtaOut& out, cudaStream_t s);

// Unblocked Gauss-Jordan over the whole grid, one rank-1 step per launch (any pivoting).
gj_status run_unblocked(int64_t n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                        const CtaOut& out, cudaStream_t s);

}  // namespace gj
