// gj_internal.cuh -- shared declarations of the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gj.h"

namespace gj {

// ----------------------------------------------------------------- status plumbing

// Record a CUDA error in the thread-local last-error text; returns GJ_ERR_CUDA.
gj_status cuda_fail(cudaError_t e, const char* what);

// Set the thread-local text returned by gj_last_error().
void set_last_error(const char* msg);

#define GJ_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return gj::cuda_fail(e_, #call); \
  } while (0)

// Raise a kernel's dynamic shared memory cap to the device's opt-in maximum (less its
// static shared memory), once per kernel and device.  The cap is one value per function for
// the whole process: a call that lowered it to its own need could make a concurrent call's
// larger launch (on another host thread) fail, so every launch site sets the same, largest
// value.  The cap only bounds what a launch may request; occupancy follows the bytes each
// launch asks for.
cudaError_t allow_max_dynamic_smem(const void* func);

// ----------------------------------------------------------------- profiling

bool prof_enabled();
void prof_count(int launches);

// Records a CUDA event pair around the launches made during its lifetime when
// profiling is on; `flops` / `bytes` are the algorithmic counts of those launches.
class ProfScope {
 public:
  ProfScope(cudaStream_t s, const char* name, double flops, double bytes);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t s_;
  int rec_;
};

// ----------------------------------------------------------------- pivot keys
//
// Candidate magnitudes are compared as the bit patterns of |v|: for non-negative
// binary64 values the unsigned integer order of the bit patterns is the numeric order,
// +inf is 0x7ff0000000000000 and every NaN pattern is larger.  The comparison then
// runs on the integer pipe instead of the (narrow) FP64 pipe.  Ties are broken by a
// 32-bit position key: the smaller key wins.

constexpr uint64_t kAbsMask = 0x7fffffffffffffffull;
constexpr uint64_t kInfBits = 0x7ff0000000000000ull;

__device__ __forceinline__ uint64_t abs_bits(double v) {
  return static_cast<uint64_t>(__double_as_longlong(v)) & kAbsMask;
}

__device__ __forceinline__ bool key_better(uint64_t a, int ka, uint64_t b, int kb) {
  return a > b || (a == b && ka < kb);
}

__device__ __forceinline__ void warp_argmax(uint64_t& v, int& key) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint64_t ov = __shfl_xor_sync(0xffffffffu, v, off);
    int ok = __shfl_xor_sync(0xffffffffu, key, off);
    if (key_better(ov, ok, v, key)) {
      v = ov;
      key = ok;
    }
  }
}

constexpr int kNoKey = 0x7fffffff;

// ----------------------------------------------------------------- launchers

// Per-matrix outputs of the shared-memory kernel.  Any pointer may be null.
struct CtaOut {
  int32_t* status;     // [count] gj_status
  int8_t* det_sign;    // [count]
  double* det_log2;    // [count]
  int32_t* piv_rows;   // [n] (single-matrix launches only)
  int32_t* piv_cols;   // [n]
  double* pivots;      // [n]
  int64_t* fail_step;  // [count]
};

// Largest order handled by one CTA in shared memory.
// Stream-ordered allocation from the library's own memory pool on the current device.  The
// pool keeps freed memory for the next call (the default pool returns it to the driver at
// every synchronisation, which made each call pay for fresh allocations); gj_trim_memory
// releases it.
cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t s);

constexpr int kCtaMaxN = 128;

// Shared memory needed by the single-CTA kernel for orders up to nmax.
size_t cta_smem_bytes(int nmax);

// One matrix, one CTA.  A (ld lda) -> X (ld n); X may equal A when lda == n.
// One matrix (n <= 128) on a thread-block cluster (k_cluster.cu), rows spread over its CTAs.
gj_status launch_cluster_single(int n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                                const CtaOut& out, cudaStream_t s);
gj_status launch_cta_single(int n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                            const CtaOut& out, cudaStream_t s);

// Batched persistent launch.  order[q] (q < count) is the matrix processed q-th; the
// work counter is taken with atomicAdd on *counter (must be 0 at launch).
gj_status launch_cta_batched(int64_t count, int nmax, const int32_t* n, const double* const* A,
                             double* const* X, const int32_t* order, int32_t* counter, int pivot_mode,
                             double tau, const CtaOut& out, cudaStream_t s);

// Device-side work order: counting sort of the orders, largest first.  Writes
// Kernel variants of the batched inversion, chosen per order bin by the plan's autotuner:
// one warp per matrix (orders <= 32, partial / no pivoting; 4 or 8 warps per CTA) or one
// CTA of NT threads per matrix in shared memory.
enum BatchedVariant { kVarWarp4 = 0, kVarWarp8, kVarCta64, kVarCta128, kVarCta256, kVarCta512, kNumVariants };
bool batched_variant_applies(int variant, int nmax, int pivot_mode);
// Items q_begin .. q_end - 1 of `order` with one kernel variant; *counter must be 0.
gj_status launch_batched_variant(int variant, int64_t q_begin, int64_t q_end, int nmax, const int32_t* n,
                                 const double* const* A, double* const* X, const int32_t* order, int32_t* counter,
                                 int pivot_mode, double tau, const CtaOut& out, cudaStream_t s);

// order[count]; ws must hold (kCtaMaxN + 2) int32.  Also leaves *counter = 0.
gj_status launch_order_by_size(int64_t count, const int32_t* n, int32_t* order, int32_t* ws, int32_t* counter,
                               cudaStream_t s);

}  // namespace gj
