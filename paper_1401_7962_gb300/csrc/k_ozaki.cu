// k_ozaki.cu -- FP64-accurate rank-k update C += L U (k <= 128) on BF16 tcgen05 tensor cores.
//
// The blocked Gauss-Jordan update is a product with a short inner dimension (the panel
// width).  GB300's FP64 units deliver about 1.2 TFLOP/s, its BF16 tensor cores about
// 1.9 PFLOP/s, so the update is emulated (an error-free splitting in the manner of the
// Ozaki scheme):
//   * every row i of L gets the power of two 2^e_i with max_k |L_ik| < 2^e_i, and every
//     column j of U a 2^f_j.  The scaled entry L_ik 2^-(e_i+1), in (-1/2, 1/2), is rounded
//     to 8S - 1 fractional bits and written in balanced base 256: S signed digits
//     a_s in [-128, 128] (exactly representable in BF16) with
//         L_ik ~ 2^(e_i+1) sum_s a_s[i,k] 2^-8(s+1),   error <= 2^(e_i - 8S);
//   * the digit products with s + t <= S - 1 are accumulated by the tensor cores in FP32
//     in tensor memory, one accumulator per group g = s + t.  Each digit product is at
//     most 2^14, each pair's sum over k <= 128 terms at most 2^21 and each group (<= 8
//     pairs) at most 2^24, so every FP32 partial sum is an exact integer;
//   * the epilogue combines the groups exactly in a 64-bit integer (weights 2^(41 - 8g)),
//     converts once to FP64, scales by 2^(e_i + f_j - 55) and adds to C.
// The error per entry is below (S + 2) K 2^(e_i + f_j - 8S) plus the FP64 roundings (S = 7:
// 2^-56 of the scales, the level of an FP64 product's rounding, with 28 digit products per
// term; 7-bit truncated digits needed 8 slices and 36 products for the same level).
//
// Kernel shape: persistent, one CTA per SM walking 128 x 64 tiles of C.  Warp 0 issues the
// TMA loads (all S digit slices of the U tile stay resident; the L slices stream through a
// 2-stage ring), warp 1 and the last warp issue the MMAs (M = 128, N = 64, K = 16 per
// instruction), each for its own digit groups, sixteen warps run the epilogue (TMEM lane =
// row of the tile).  Every mbarrier wait is bounded in
// time; on expiry the kernel records an error, drains its own TMA loads and MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "gj_internal.cuh"
#include "gj_ozaki.cuh"
#include "tc_ptx.cuh"

namespace gj {
namespace {

constexpr int kTM = 128;          // tile rows (MMA M)
constexpr int kTN = 64;           // tile columns (MMA N)
constexpr int kKB = 128;          // slice row length in elements (max inner dimension)
constexpr int kKC = 64;           // elements per TMA box along k (128 bytes, one swizzle row)
constexpr int kStages = 2;        // ring of L slices: one stage = one digit slice, kKB wide
constexpr int kABox = kTM * kKC * 2;   // 16 KiB: one TMA box (128 rows x 64 k)
constexpr int kAStage = 2 * kABox;     // 32 KiB: the two boxes of a slice (k 0..63, 64..127)
constexpr int kBBox = kTN * kKC * 2;   // 8 KiB
#ifndef GJ_EPI_WARPS
#define GJ_EPI_WARPS 16
#endif
// Per TMEM lane quarter kEpiWarps / 4 warps, each with a column slice.  The epilogue is bound
// by latency (dependent integer and FP64 chains, TMEM and memory round trips), not by any one
// pipe: sixteen warps of 16 columns (92 registers) hide it where eight warps of 32 columns
// (166 registers, the most a 10-warp block gets) left it setting the tile period.
constexpr int kEpiWarps = GJ_EPI_WARPS;
constexpr int kEpiSlices = kEpiWarps / 4;
// Two threads issue the MMAs, each for its own digit groups (accumulators): the issue of one
// thread, sharing its SM sub-partition with four epilogue warps, set the MMA rate at this
// N = 64 shape.  Warp 1 and the last warp issue; they sit on different sub-partitions.
constexpr int kIssuers = 2;
constexpr int kIssuerWarp2 = 2 + kEpiWarps;
constexpr int kThreads = 64 + 32 * kEpiWarps + 32;  // producer warp, MMA warps, epilogue warps
// digit groups whose MMAs each issuer takes (bit g = group g) when S = 7: 13 and 15 of the 28
// digit products per term; for other S the groups alternate
constexpr uint32_t kOwnS7[kIssuers] = {0x47u, 0x38u};
static_assert((kOwnS7[0] & kOwnS7[1]) == 0u && (kOwnS7[0] | kOwnS7[1]) == 0x7Fu,
              "each of the 7 digit groups has exactly one issuer");
constexpr int kEpiCols = kTN / kEpiSlices;  // columns per epilogue thread
constexpr int kCSm = kEpiCols / 2; // of those, prefetched into shared memory (the rest load in the final pass)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s: default pipeline wait, and every teardown drain
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTM, kTN);

// ---------------------------------------------------------------- digit slicing

__device__ __forceinline__ int exp_of(double x) {
  // e with |x| < 2^e for normal x; -100000 for zero / subnormal (flushed)
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  return E == 0 ? -100000 : E - 1022;
}

// round(|x| 2^(8S - 1 - e)) for |x| < 2^e (at most 2^(8S - 1); subnormals flush to 0)
__device__ __forceinline__ unsigned long long magnitude_of(double x, int e, int S) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E == 0) return 0ull;
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int shift = (E - 1023) - 52 + 8 * S - 1 - e;
  if (shift >= 0) return M << shift;  // shift <= 8S - 54, so M << shift < 2^(8S - 1)
  if (shift <= -64) return 0ull;
  return (M + (1ull << (-shift - 1))) >> (-shift);  // round half up
}

// The S balanced base-256 digits of four entries (digit 0 the most significant), written to
// slices s = 0..S-1 at out + s * slice_stride + off.
__device__ __forceinline__ void write_digits(__nv_bfloat16* out, int S, int64_t slice_stride, int64_t off,
                                             const double (&x)[4], int e) {
  long long v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long m = static_cast<long long>(magnitude_of(x[q], e, S));
    v[q] = x[q] < 0.0 ? -m : m;
  }
  for (int s = S - 1; s >= 0; --s) {
    __align__(8) __nv_bfloat16 d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r;
      if (s > 0) {
        r = static_cast<int>(v[q] & 255);  // low 8 bits (two's complement)
        if (r > 128) r -= 256;             // balanced: r in [-127, 128]
        v[q] = (v[q] - r) >> 8;            // exact
      } else {
        r = static_cast<int>(v[q]);        // |r| <= 128 (see the header)
      }
      d[q] = __float2bfloat16_rn(static_cast<float>(r));
    }
    *reinterpret_cast<uint2*>(out + s * slice_stride + off) = *reinterpret_cast<const uint2*>(d);
  }
}

// Rows of L (M x K, column-major, ld ldl) -> slices [S][mpad][128] and row exponents.
// minus_one_at[k] (optional): subtract 1 from L[minus_one_at[k], k] (the blocked
// Gauss-Jordan L of the panel: pivot entries minus the identity).
__device__ __forceinline__ void slice_rows(int warp, int nwarps, int M, int K, const double* __restrict__ L,
                                           int64_t ldl, const int* __restrict__ minus_one_at,
                                           const int* __restrict__ row_pos, int unit_lo, int unit_hi, int S, int mpad,
                                           __nv_bfloat16* __restrict__ out, int* __restrict__ erow) {
  const int lane = threadIdx.x & 31;
  int mo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = lane * 4 + q;
    mo[q] = (minus_one_at && k < K) ? minus_one_at[k] : -1;
  }
  for (int i = warp; i < mpad; i += nwarps) {
    double x[4];
    int e = -100000;
    const int pos = (row_pos && i < M) ? row_pos[i] : -1;
    const bool unit = row_pos && pos >= unit_lo && pos < unit_hi;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = lane * 4 + q;
      double v = (i < M && k < K) ? L[(int64_t)i + (int64_t)k * ldl] : 0.0;
      if (mo[q] == i) v -= 1.0;
      if (unit) v = (k == pos - unit_lo) ? -1.0 : 0.0;
      x[q] = v;
      e = max(e, exp_of(v));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    // only the k the MMAs read: whole K16 steps up to K (the rest of the row is never read)
    if (lane * 4 < ((K + 15) & ~15)) write_digits(out, S, (int64_t)mpad * kKB, (int64_t)i * kKB + lane * 4, x, e);
    if (lane == 0) erow[i] = e;
  }
}

// Columns of U (K x N) -> slices [S][npad][128] and column exponents.  U[k, j] is
// U[k + j*ldu], or, with row_ids, W[row_ids[k] + j*ldu] (the pivot rows of a panel);
// columns in [zero_lo, zero_hi) are zero.
__device__ __forceinline__ void slice_cols(int warp, int nwarps, int N, int K, const double* __restrict__ U,
                                           int64_t ldu, const int* __restrict__ row_ids, int zero_lo, int zero_hi,
                                           int S, int npad, __nv_bfloat16* __restrict__ out,
                                           int* __restrict__ ecol) {
  const int lane = threadIdx.x & 31;
  int rid[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = lane * 4 + q;
    rid[q] = (k < K) ? (row_ids ? row_ids[k] : k) : -1;
  }
  for (int j = warp; j < npad; j += nwarps) {
    double x[4];
    int e = -100000;
    const bool live = j < N && !(j >= zero_lo && j < zero_hi);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double v = (live && rid[q] >= 0) ? U[(int64_t)rid[q] + (int64_t)j * ldu] : 0.0;
      x[q] = v;
      e = max(e, exp_of(v));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    if (lane * 4 < ((K + 15) & ~15)) write_digits(out, S, (int64_t)npad * kKB, (int64_t)j * kKB + lane * 4, x, e);
    if (lane == 0) ecol[j] = e;
  }
}

// One launch slices both operands: blocks [0, row_blocks) take the rows of L, the rest the
// columns of U.
__global__ void slice_kernel(int row_blocks, int M, int N, int K, const double* __restrict__ L, int64_t ldl,
                             const int* __restrict__ minus_one_at, const int* __restrict__ row_pos, int unit_lo,
                             int unit_hi, const double* __restrict__ U, int64_t ldu,
                             const int* __restrict__ row_ids, int zero_lo, int zero_hi, int S, int mpad, int npad,
                             __nv_bfloat16* __restrict__ As, __nv_bfloat16* __restrict__ Bs, int* __restrict__ erow,
                             int* __restrict__ ecol, const int32_t* status) {
  if (status && *status != GJ_OK) return;
  const int wpb = blockDim.x >> 5;
  if ((int)blockIdx.x < row_blocks) {
    slice_rows((int)blockIdx.x * wpb + (threadIdx.x >> 5), row_blocks * wpb, M, K, L, ldl, minus_one_at, row_pos,
               unit_lo, unit_hi, S, mpad,
               As, erow);
  } else {
    const int b = (int)blockIdx.x - row_blocks;
    slice_cols(b * wpb + (threadIdx.x >> 5), ((int)gridDim.x - row_blocks) * wpb, N, K, U, ldu, row_ids, zero_lo,
               zero_hi, S, npad, Bs, ecol);
  }
}

// ---------------------------------------------------------------- tensor-core update

// T * 2^e via the hardware conversion of T (correctly rounded) and an exponent add (exact
// for normal results).  One FP64-pipe conversion: an integer-only conversion (normalise,
// round, assemble the bits) measured slower here, its integer work slowing the MMA issue.
__device__ __forceinline__ double i64_to_double_pow2(long long T, int e) {
  const double d = __ll2double_rn(T);
  const long long bits = __double_as_longlong(d);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (d == 0.0 || E + e <= 0 || E + e >= 2047) return ldexp(d, e);
  return __longlong_as_double(bits + (static_cast<long long>(e) << 52));
}

// The MMAs of slice SL of a tile for the common case S = 7 digit slices, K = 128 (two TMA
// boxes per slice), fully unrolled: every accumulator address and descriptor is the slice's
// base plus a constant.  One thread issues all MMAs of the CTA, and the instructions between
// two MMAs bound their rate at this N = 64 shape (a loop with run-time bounds issued about
// one MMA per 80 clocks where the tensor pipe can take one per ~60).  Descriptors hold the
// shared-memory address in 16-byte units in their low bits, so adding (bytes >> 4) moves them.
template <int SL, uint32_t OWN>
__device__ __forceinline__ void mma_slice_s7k2(uint32_t tmem, uint64_t a_stage, uint64_t b_res) {
#pragma unroll
  for (int kc = 0; kc < 2; ++kc)
#pragma unroll
    for (int t = 0; t < 7 - SL; ++t)
#pragma unroll
      for (int k16 = 0; k16 < kKC / 16; ++k16)
        if ((OWN >> (SL + t)) & 1u)
          tc::mma_bf16(tmem + (uint32_t)(kTN * (SL + t)), a_stage + (uint64_t)((kc * kABox) >> 4) + 2u * k16,
                     b_res + (uint64_t)(((t * 2 + kc) * kBBox) >> 4) + 2u * k16, kIdesc,
                     (SL > 0 || kc > 0 || k16 > 0) ? 1u : 0u);
}

struct SmemLayout {
  static size_t bytes(int S) {
    return 1024 /*align slack*/ + (size_t)S * 2 * kBBox + (size_t)kStages * kAStage +
           (size_t)kEpiSlices * kCSm * kTM * 8;
  }
};

// Persistent kernel: CTA b takes the contiguous range [b T / G, (b + 1) T / G) of the T tiles
// in column-major order, so consecutive tiles of a CTA share their U slices, which are
// loaded again only when the tile column changes.
// Roles: warp 0 = TMA producer (U slices of a new tile column, then the L slices through the
// ring), warp 1 and warp kIssuerWarp2 = MMA issuers (each for its own digit groups, with the
// same waits and commits), warps 2 .. kEpiWarps + 1 = epilogue (warp w reads TMEM lanes
// 32 (w % 4) .. + 31 and the column slice (w - 2) / 4 of the tile).
// The L slices are consumed in ascending order, so digit group g is final once slice g has
// been consumed (its terms come from slices s <= g): both issuers commit to group g's barrier
// there (it counts both), and the epilogue drains the groups one by one while the MMAs of the
// higher groups run.  At the end of a tile each issuer waits once, on a shared-memory counter,
// for the epilogue to have read the last group; the epilogue then combines and stores the tile
// while the next tile's MMAs run.  (Waits of an issuer inside a tile's MMA stream, on
// epilogue-arrived mbarriers or on per-group counters, measured markedly slower MMA issue on
// GB300; this single end-of-tile wait, with the pipe about to drain anyway, did not.)
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_update_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                        int N, int mpad, int npad, int S, int nkc, int nk16_last, int tiles_m, int tiles_n, int ts_lo, int ts_hi,
                        int skip_lo, int skip_hi, double* __restrict__ C, int64_t ldc, const int* __restrict__ erow,
                        const int* __restrict__ ecol, int32_t* err, int32_t* status, uint64_t wait_ns,
                        OzEpilogue epi) {
  if (status && *status != GJ_OK) return;
  const int tiles_n_act = tiles_n - (ts_hi - ts_lo);
  const int ntiles = tiles_m * tiles_n_act;
  const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
  const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);
  if (t_begin >= t_end) return;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Bres = smem;                                   // [S][2] boxes of 8 KiB
  uint8_t* Aring = smem + (size_t)S * 2 * kBBox;          // [kStages] slices of 2 boxes of 16 KiB
  double* Cs = reinterpret_cast<double*>(Aring + (size_t)kStages * kAStage);  // [kEpiSlices][kCSm][kTM]
  __shared__ __align__(8) uint64_t bar_bfull, bar_bempty, bar_full[kStages], bar_empty[kStages], bar_gready[8],
      bar_fin;
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_drained;  // epilogue warps that have read the last group, summed over tiles
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&bar_bfull, 1);
    tc::mbar_init(&bar_bempty, kIssuers);
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&bar_full[i], 1);
      tc::mbar_init(&bar_empty[i], kIssuers);
    }
    for (int g = 0; g < 8; ++g) tc::mbar_init(&bar_gready[g], kIssuers);
    tc::mbar_init(&bar_fin, kIssuers);
    tc::fence_mbar_init();
    s_drained = 0;
    s_abort = 0;
    tc::tma_prefetch_desc(&mapA);
    tc::tma_prefetch_desc(&mapB);
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;

  auto tile_of = [&](int idx, int& m0, int& c0) {
    const int tna = idx / tiles_m, tm = idx - tna * tiles_m;
    const int tn = (tna < ts_lo) ? tna : tna + (ts_hi - ts_lo);
    m0 = tm * kTM;
    c0 = tn * kTN;
  };
  // the tile starts a new tile column (its U slices must be loaded)
  auto new_column = [&](int idx) { return idx == t_begin || (idx % tiles_m) == 0; };

  int issued_uses[kStages] = {};
  int b_issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer
      int it = 0, local = 0;
      for (int idx = t_begin; idx < t_end && !s_abort; ++idx, ++local) {
        int m0, c0;
        tile_of(idx, m0, c0);
        if (new_column(idx)) {
          // the MMAs of the previous tile column must have finished reading the resident U
          // slices (bar_bempty completes one phase per tile column that is followed by another)
          if (b_issued > 0 && !tc::mbar_wait_backoff(&bar_bempty, (uint32_t)((b_issued - 1) & 1), wait_ns)) {
            atomicExch(err, 10);
            s_abort = 1;
            break;
          }
          tc::mbar_arrive_expect_tx(&bar_bfull, (uint32_t)(S * nkc * kBBox));
          ++b_issued;
          for (int t = 0; t < S; ++t)
            for (int kc = 0; kc < nkc; ++kc)
              tc::tma_load_2d(Bres + (size_t)(t * 2 + kc) * kBBox, &mapB, kc * kKC, t * npad + c0, &bar_bfull);
        }
        bool ok = true;
        for (int sl = 0; sl < S; ++sl, ++it) {
          const int stage = it % kStages, use = it / kStages;
          // the stage's previous slice must be consumed: with S >= kStages that slice's
          // group barrier says so (slice sl - 2 of this tile, or slice S - 2 + sl of the
          // previous one); with fewer slices a per-stage barrier is committed instead
          bool free_ok = true;
          if (use > 0) {
            if (S >= kStages) {
              const int g = (sl >= kStages) ? sl - kStages : S - kStages + sl;
              const int tl = (sl >= kStages) ? local : local - 1;
              free_ok = tc::mbar_wait_backoff(&bar_gready[g], (uint32_t)(tl & 1), wait_ns);
            } else {
              free_ok = tc::mbar_wait_backoff(&bar_empty[stage], (uint32_t)((use - 1) & 1), wait_ns);
            }
          }
          if (!free_ok) {
            atomicExch(err, 11);
            s_abort = 1;
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&bar_full[stage], (uint32_t)(nkc * kABox));
          for (int kc = 0; kc < nkc; ++kc)
            tc::tma_load_2d(Aring + (size_t)stage * kAStage + (size_t)kc * kABox, &mapA, kc * kKC, sl * mpad + m0,
                            &bar_full[stage]);
          issued_uses[stage] = use + 1;
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1 || warp == kIssuerWarp2) {
    if (lane == 0) {
      // ---------------- MMA issuers: the same waits and commits, each its own MMAs
      const int me = (warp == 1) ? 0 : 1;
      int it = 0, local = 0, b_used = 0;
      for (int idx = t_begin; idx < t_end && !s_abort; ++idx, ++local) {
        bool ok = true;
        if (new_column(idx)) {
          ok = tc::mbar_wait(&bar_bfull, (uint32_t)(b_used & 1), wait_ns);
          ++b_used;
          if (!ok) {
            atomicExch(err, 20);
            s_abort = 1;
            break;
          }
          tc::tc_fence_after();
        }
        for (int sl = 0; sl < S && ok; ++sl, ++it) {
          const int stage = it % kStages, use = it / kStages;
          if (!tc::mbar_wait(&bar_full[stage], (uint32_t)(use & 1), wait_ns)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          // one wait and two commits per slice: all k of the slice against every U slice t
          if (S == 7 && nkc == 2 && nk16_last == kKC / 16) {
            const uint64_t as = tc::desc_k128_sw128(tc::smem_u32(Aring + (size_t)stage * kAStage));
            const uint64_t bs = tc::desc_k128_sw128(tc::smem_u32(Bres));
            if (me == 0) {
              switch (sl) {
                case 0: mma_slice_s7k2<0, kOwnS7[0]>(tmem, as, bs); break;
                case 1: mma_slice_s7k2<1, kOwnS7[0]>(tmem, as, bs); break;
                case 2: mma_slice_s7k2<2, kOwnS7[0]>(tmem, as, bs); break;
                case 3: mma_slice_s7k2<3, kOwnS7[0]>(tmem, as, bs); break;
                case 4: mma_slice_s7k2<4, kOwnS7[0]>(tmem, as, bs); break;
                case 5: mma_slice_s7k2<5, kOwnS7[0]>(tmem, as, bs); break;
                default: mma_slice_s7k2<6, kOwnS7[0]>(tmem, as, bs); break;
              }
            } else {
              switch (sl) {
                case 0: mma_slice_s7k2<0, kOwnS7[1]>(tmem, as, bs); break;
                case 1: mma_slice_s7k2<1, kOwnS7[1]>(tmem, as, bs); break;
                case 2: mma_slice_s7k2<2, kOwnS7[1]>(tmem, as, bs); break;
                case 3: mma_slice_s7k2<3, kOwnS7[1]>(tmem, as, bs); break;
                case 4: mma_slice_s7k2<4, kOwnS7[1]>(tmem, as, bs); break;
                case 5: mma_slice_s7k2<5, kOwnS7[1]>(tmem, as, bs); break;
                default: mma_slice_s7k2<6, kOwnS7[1]>(tmem, as, bs); break;
              }
            }
          } else {
            for (int kc = 0; kc < nkc; ++kc) {
              const uint64_t a0 =
                  tc::desc_k128_sw128(tc::smem_u32(Aring + (size_t)stage * kAStage + (size_t)kc * kABox));
              for (int t = 0; sl + t < S; ++t) {
                if (((sl + t) & 1) != me) continue;
                const uint32_t d = tmem + (uint32_t)(kTN * (sl + t));
                const uint64_t b0 = tc::desc_k128_sw128(tc::smem_u32(Bres + (size_t)(t * 2 + kc) * kBBox));
                // the last box holds K - 64 (nkc - 1) of its 64 k: nk16_last K16 steps
                const int nk16 = (kc == nkc - 1) ? nk16_last : kKC / 16;
#pragma unroll
                for (int k16 = 0; k16 < kKC / 16; ++k16)
                  if (k16 < nk16)
                    tc::mma_bf16(d, a0 + 2u * k16, b0 + 2u * k16, kIdesc, (sl > 0 || kc > 0 || k16 > 0) ? 1u : 0u);
              }
            }
          }
          if (S < kStages) tc::mma_commit(&bar_empty[stage]);
          // digit group sl has received all of its terms (and, with S >= kStages, the
          // stage of slice sl is free again)
          tc::mma_commit(&bar_gready[sl]);
        }
        if (!ok) {
          atomicExch(err, 21);
          s_abort = 1;
          break;
        }
        if (idx + 1 < t_end && new_column(idx + 1)) tc::mma_commit(&bar_bempty);
        // the epilogue must have read this tile's accumulators before the next tile's MMAs
        // overwrite them
        const uint32_t target = (uint32_t)(kEpiWarps * (local + 1));
        const uint64_t w0 = tc::global_timer_ns();
        while (tc::counter_load_acquire(&s_drained) < target) {
          if (s_abort || tc::global_timer_ns() - w0 > wait_ns) {
            ok = false;
            break;
          }
        }
        if (!ok) {
          atomicExch(err, 22);
          s_abort = 1;
          break;
        }
        tc::tc_fence_after();
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. kEpiWarps + 1)
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;   // column slice of the tile
    const int r = q * 32 + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(q * 32) << 16) + (uint32_t)(h * kEpiCols);
    double* Csh = Cs + (size_t)h * kCSm * kTM;
    int local = 0;
    for (int idx = t_begin; idx < t_end; ++idx, ++local) {
      int m0, c0;
      tile_of(idx, m0, c0);
      c0 += h * kEpiCols;
      const int gi = m0 + r;
      const bool row_ok = gi < M;
      // rows whose position is in the set range take the product instead of adding it
      const int gpos = (epi.row_pos && row_ok) ? epi.row_pos[gi] : -1;
      const bool set_row = epi.row_pos && gpos >= epi.set_row_lo && gpos < epi.set_row_hi;
      // kCSm of this row's C values into shared memory now (cp.async, overlapping the MMAs);
      // the column exponents of the warp's kEpiCols columns, one per lane
#pragma unroll
      for (int c = 0; c < kCSm; ++c) {
        const int gj = c0 + c;
        if (row_ok && gj < N) tc::cp_async8(&Csh[c * kTM + r], &C[(int64_t)gi + (int64_t)gj * ldc]);
      }
      tc::cp_async_commit();
      const int ec_lane = (c0 + lane < N) ? ecol[c0 + lane] : 0;
      const int er = row_ok ? erow[gi] : 0;
      // drain the groups in order as each becomes final
      long long T[kEpiCols];
#pragma unroll
      for (int c = 0; c < kEpiCols; ++c) T[c] = 0;
      bool ok = true;
#pragma unroll
      for (int g = 0; g < 8; ++g) {  // unrolled: each group's shift is a constant
        if (g >= S) break;
        // one lane polls, the warp follows; the last group gates the next tile's MMAs, so it
        // is polled without sleeping
        int ok0 = 0;
        if (lane == 0)
          ok0 = ((g == S - 1) ? tc::mbar_wait(&bar_gready[g], (uint32_t)(local & 1), wait_ns)
                              : tc::mbar_wait_backoff(&bar_gready[g], (uint32_t)(local & 1), wait_ns)) &&
                !s_abort;
        ok = __shfl_sync(0xffffffffu, ok0, 0) != 0;  // warp-uniform
        if (!ok) break;
        tc::tc_fence_after();
        const int sh = 57 - 8 * (g + 2);  // group weight 2^-8(g+2) of 2^(e_i+1+f_j+1), over 2^(e_i+f_j-55)
        // 16 columns at a time (keeps the live registers within one CTA per SM)
#pragma unroll
        for (int half = 0; half < kEpiCols / 16; ++half) {
          uint32_t v[2][8];
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
            tc::tmem_ld8(lane_base + (uint32_t)(kTN * g + 16 * half + 8 * cc), v[cc]);
          tc::tmem_ld_wait();
          if (g == S - 1 && half == kEpiCols / 16 - 1) {
            // all of this tile's accumulators read by this warp: release them to the MMA warp
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::counter_add_release(&s_drained, 1u);
          }
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const long long G = static_cast<long long>(__float2int_rn(__uint_as_float(v[cc][c])));
              T[16 * half + 8 * cc + c] += (sh >= 0) ? (G << sh) : (G >> (-sh));
            }
        }
      }
      if (!ok) {
        atomicExch(err, 30);
        s_abort = 1;
        tc::cp_async_wait_all();
        break;
      }
      tc::cp_async_wait_all();
      // combine and store in batches of 8 columns; each batch's old C values are loaded
      // (from shared memory, or from global memory for the second half) before the
      // previous batch is computed, so the loads' latency overlaps the arithmetic
      constexpr int kB = (kEpiSlices >= 4) ? 4 : 8;  // fewer live registers with more warps
      double cold[2][kB];
      auto load_batch = [&](int b, double (&dst)[kB]) {
#pragma unroll
        for (int c = 0; c < kB; ++c) {
          const int cl = b * kB + c, gj = c0 + cl;
          if (cl < kCSm)
            dst[c] = Csh[cl * kTM + r];
          else
            dst[c] = (row_ok && gj < N) ? C[(int64_t)gi + (int64_t)gj * ldc] : 0.0;
        }
      };
      load_batch(0, cold[0]);
#pragma unroll
      for (int b = 0; b < kEpiCols / kB; ++b) {
        if (b + 1 < kEpiCols / kB) load_batch(b + 1, cold[(b + 1) & 1]);
#pragma unroll
        for (int c = 0; c < kB; ++c) {
          const int cl = b * kB + c, gj = c0 + cl;
          const int ec = __shfl_sync(0xffffffffu, ec_lane, cl);
          const bool set = set_row || (gj >= epi.set_col_lo && gj < epi.set_col_hi);
          if (!row_ok || gj >= N || (gj >= skip_lo && gj < skip_hi) || (T[cl] == 0 && !set)) continue;
          const double prod = i64_to_double_pow2(T[cl], er + ec - 55);
          C[(int64_t)gi + (int64_t)gj * ldc] = set ? prod : cold[b & 1][c] + prod;
        }
      }
    }
  }

  // ---------------- teardown: drain own async work (bounded), then free tensor memory
  // After an abort the drains below wait with the full default limit whatever limit the
  // pipeline waits had: every TMA load this CTA issued lands in its own shared memory and
  // every MMA it issued writes its own tensor memory, so both must have completed before
  // the CTA frees that memory and exits.  A drain that still expires records its own code
  // (40: a U-slice load, 41: an L-slice load, 42: the MMAs); the CTA then exits with that
  // copy or MMA still outstanding, which only a broken device could cause.
  __syncthreads();
  if (s_abort) {
    if (warp == 0 && lane == 0) {
      if (b_issued > 0 && !tc::mbar_wait(&bar_bfull, (uint32_t)((b_issued - 1) & 1), kWaitNs)) atomicExch(err, 40);
      for (int st = 0; st < kStages; ++st)
        if (issued_uses[st] > 0 && !tc::mbar_wait(&bar_full[st], (uint32_t)((issued_uses[st] - 1) & 1), kWaitNs))
          atomicExch(err, 41);
    }
    if ((warp == 1 || warp == kIssuerWarp2) && lane == 0) {
      tc::mma_commit(&bar_fin);
      if (!tc::mbar_wait(&bar_fin, 0, kWaitNs)) atomicExch(err, 42);
    }
    // the caller's status (when it passes one) fails at once, so that the kernels queued
    // after this one skip their work instead of running on a partly updated array
    if (tid == 0 && status) atomicCAS(status, (int32_t)GJ_OK, (int32_t)GJ_ERR_TIMEOUT);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 tensor [rows][128] (row pitch 256 B), box {64, box_rows}, 128-byte swizzle.
gj_status make_slice_map(CUtensorMap* map, void* base, int64_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_last_error("cuTensorMapEncodeTiled is not available from the driver");
    return GJ_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)kKB, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kKB * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char msg[128];
    snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled failed (%d)", (int)r);
    set_last_error(msg);
    return GJ_ERR_CUDA;
  }
  return GJ_OK;
}

}  // namespace

namespace {
thread_local int t_update_cap = 0;
// Limit of the update kernel's pipeline waits in nanoseconds (0 = the 2 s default); set by
// gj_set_wait_limit_ns to exercise the expiry path.
std::atomic<uint64_t> g_wait_ns{0};
}  // namespace

void set_thread_update_cap(int ctas) { t_update_cap = ctas > 0 ? ctas : 0; }

size_t ozaki_workspace_bytes(int64_t M, int64_t N, int S) {
  const int64_t mpad = (M + kTM - 1) / kTM * kTM, npad = (N + kTM - 1) / kTM * kTM;
  return (size_t)S * (mpad + npad) * kKB * 2 + (size_t)(mpad + npad) * sizeof(int) + 256;
}

gj_status ozaki_update(int64_t M, int64_t N, int K, const double* L, int64_t ldl, const int* l_minus_one_at,
                       const double* U, int64_t ldu, const int* u_row_ids, int zero_lo, int zero_hi, double* C,
                       int64_t ldc, int S, void* ws, int32_t* err, int32_t* status, cudaStream_t s,
                       int max_ctas, const char* prof_name, OzEpilogue epi) {
  if (K < 1 || K > kKB || S < 1 || S > 8) return GJ_ERR_ARG;
  if (max_ctas <= 0) max_ctas = t_update_cap;
  const int64_t mpad = (M + kTM - 1) / kTM * kTM, npad = (N + kTM - 1) / kTM * kTM;
  uint8_t* p = static_cast<uint8_t*>(ws);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)S * mpad * kKB * 2;
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(p);
  p += (size_t)S * npad * kKB * 2;
  int* erow = reinterpret_cast<int*>(p);
  int* ecol = erow + mpad;

  int dev = 0, sms = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // 8 warps per block, one row (column) per warp per pass
  const int sb = (int)std::min<int64_t>((mpad + 7) / 8, (int64_t)sms * 16);
  const int sc = (int)std::min<int64_t>((npad + 7) / 8, (int64_t)sms * 16);
  slice_kernel<<<sb + sc, 256, 0, s>>>(sb, (int)M, (int)N, K, L, ldl, l_minus_one_at, epi.row_pos, epi.unit_lo,
                                       epi.unit_hi, U, ldu, u_row_ids, zero_lo,
                                       zero_hi, S, (int)mpad, (int)npad, As, Bs, erow, ecol, status);
  GJ_CUDA(cudaGetLastError());
  prof_count(1);

  CUtensorMap mapA, mapB;
  gj_status st = make_slice_map(&mapA, As, (int64_t)S * mpad, kTM);
  if (st != GJ_OK) return st;
  st = make_slice_map(&mapB, Bs, (int64_t)S * npad, kTN);
  if (st != GJ_OK) return st;
  const size_t smem = SmemLayout::bytes(S);
  GJ_CUDA(allow_max_dynamic_smem((const void*)ozaki_update_kernel));
  const int nkc = (K + kKC - 1) / kKC;
  const int nk16_last = (K - (nkc - 1) * kKC + 15) / 16;
  const int tiles_m = (int)((M + kTM - 1) / kTM), tiles_n = (int)((N + kTN - 1) / kTN);
  // column tiles lying wholly inside [zero_lo, zero_hi) receive nothing: not scheduled
  int ts_lo = 0, ts_hi = 0;
  if (zero_hi > zero_lo) {
    ts_lo = (zero_lo + kTN - 1) / kTN;
    ts_hi = (zero_hi >= N) ? tiles_n : zero_hi / kTN;
    if (ts_hi > tiles_n) ts_hi = tiles_n;
    if (ts_hi < ts_lo) ts_hi = ts_lo;
  }
  const int ntiles = tiles_m * (tiles_n - (ts_hi - ts_lo));
  if (ntiles <= 0) return GJ_OK;
  const int grid = std::min(ntiles, (max_ctas > 0 && max_ctas < sms) ? max_ctas : sms);
  const uint64_t lim = g_wait_ns.load(std::memory_order_relaxed);
  const uint64_t wait_ns = lim ? lim : kWaitNs;
  {
    // tensor FLOP: S (S + 1) / 2 digit-slice products per FP64 product term
    ProfScope ps(s, prof_name, 0.5 * S * (S + 1) * 2.0 * (double)M * (double)(N - (zero_hi - zero_lo)) * K,
                 16.0 * (double)M * (double)N);
    ozaki_update_kernel<<<grid, kThreads, smem, s>>>(mapA, mapB, (int)M, (int)N, (int)mpad, (int)npad, S, nkc,
                                                    nk16_last, tiles_m, tiles_n, ts_lo, ts_hi, zero_lo, zero_hi, C, ldc, erow,
                                                    ecol, err, status, wait_ns, epi);
  }
  GJ_CUDA(cudaGetLastError());
  prof_count(1);
  return GJ_OK;
}

}  // namespace gj

using namespace gj;

extern "C" gj_status gj_gemm_update_emulated(int64_t M, int64_t N, int64_t K, const double* L, int64_t ldl,
                                             const double* U, int64_t ldu, double* C, int64_t ldc, int slices,
                                             void* stream) {
  set_last_error("");
  if (M < 0 || N < 0 || K < 0 || K > 128 || slices < 1 || slices > 8) return GJ_ERR_ARG;
  if (M == 0 || N == 0 || K == 0) return GJ_OK;
  if (ldl < M || ldu < K || ldc < M || !L || !U || !C) return GJ_ERR_ARG;
  if (M > 0x3fffffff || N > 0x3fffffff) return GJ_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  const size_t bytes = ozaki_workspace_bytes(M, N, slices) + 16;
  cudaError_t e = lib_malloc_async(&ws, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GJ_ERR_NOMEM;
  }
  int32_t* err = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(ws) + bytes - 16);
  cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  gj_status st = ozaki_update(M, N, (int)K, L, ldl, nullptr, U, ldu, nullptr, 0, 0, C, ldc, slices, ws, err, nullptr,
                              s);
  int32_t herr = 0;
  if (st == GJ_OK) {
    e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "gj_gemm_update_emulated");
  }
  cudaFreeAsync(ws, s);
  if (st == GJ_OK && herr != 0) {
    set_last_error("tensor-core update: a bounded wait expired");
    st = GJ_ERR_TIMEOUT;
  }
  return st;
}

extern "C" gj_status gj_set_wait_limit_ns(uint64_t ns) {
  gj::g_wait_ns.store(ns, std::memory_order_relaxed);
  return GJ_OK;
}
