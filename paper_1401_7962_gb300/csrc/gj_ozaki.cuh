// gj_ozaki.cuh -- FP64-accurate rank-k update on BF16 tensor cores (k_ozaki.cu).
#pragma once

#include "gj_internal.cuh"

namespace gj {

// Device workspace bytes for ozaki_update with an M x N result and S digit slices.
size_t ozaki_workspace_bytes(int64_t M, int64_t N, int S);

// C[M x N] += L[M x K] U[K x N] (K <= 128), FP64 in and out, emulated on BF16 tcgen05 with
// S digit slices per operand.  L is column-major (ld ldl); with l_minus_one_at, 1 is
// subtracted from L[l_minus_one_at[k], k].  U[k, j] = U[k + j*ldu], or with u_row_ids
// U[u_row_ids[k] + j*ldu]; columns j in [zero_lo, zero_hi) of U are taken as zero and those
// columns of C are left untouched.  `ws` holds ozaki_workspace_bytes(M, N, S); `err`
// receives a nonzero code if a bounded device wait expired; kernels return at once when
// *status != GJ_OK (status may be null).  max_ctas > 0 caps the persistent grid (one CTA
// per SM), leaving the other SMs to work on another stream.  prof_name labels the launch for
// the library's profiling hooks.
// Default cap of the calling host thread on the persistent grid of ozaki_update when the
// call passes max_ctas = 0 (0: no cap).  The batched mixed path sets it on its worker
// threads so that the updates of several matrices share the SMs with their panel clusters.
void set_thread_update_cap(int ctas);

// Row and column options of an update, keyed on row positions row_pos[i] (null: none):
//   - rows with row_pos[i] in [unit_lo, unit_hi) take the row -e_(row_pos[i] - unit_lo) as
//     their row of L (instead of L's own values);
//   - the epilogue stores the product into C, instead of adding it, on the rows with
//     row_pos[i] in [set_row_lo, set_row_hi) and on the columns in [set_col_lo, set_col_hi).
struct OzEpilogue {
  const int* row_pos = nullptr;
  int unit_lo = 0, unit_hi = 0;
  int set_row_lo = 0, set_row_hi = 0;
  int set_col_lo = 0, set_col_hi = 0;
};

gj_status ozaki_update(int64_t M, int64_t N, int K, const double* L, int64_t ldl, const int* l_minus_one_at,
                       const double* U, int64_t ldu, const int* u_row_ids, int zero_lo, int zero_hi, double* C,
                       int64_t ldc, int S, void* ws, int32_t* err, int32_t* status, cudaStream_t s,
                       int max_ctas = 0, const char* prof_name = "update_ozaki_tc", OzEpilogue epi = OzEpilogue());

}  // namespace gj
