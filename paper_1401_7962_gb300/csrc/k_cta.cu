// k_cta.cu -- one CTA inverts one matrix held in shared memory (orders up to 128).
//
// The matrix lives in shared memory as the compact [A | D] array of the paper's
// Section 2: at step k the column of A that becomes a unit column is reused for the
// column of D that stops being one (eqs. 3-10 in the equivalent form of eqs. 14-15).
// Interchanges (observations 2-3) are implicit: rows and columns stay where they
// are and two position maps (rowat: position -> row, colat: position -> column) are
// permuted instead; ties are broken on positions, so the pivot sequence is the one
// of the physical-interchange algorithm.  At the end the inverse is gathered as
//   X[i, j] = W[rowat[poscol[i]], colat[posrow[j]]],
// which is the reverse-order un-permutation of observation 3 applied at once.
//
// Per step (all threads of the CTA):
//   B  thread 0 takes the winning candidate, applies the interchange to the maps,
//      records the eq. 13 factor and forms 1/pivot;
//   C  the scaled pivot row (eq. 14) and the pivot column are staged in shared memory;
//   D  every element is updated with one FMA (eq. 15); in the same pass each thread
//      scans the elements that are candidates of the next step, so the pivot search
//      costs no extra pass over the matrix.
// The FP64 pipe of GB300 issues about 2 lanes per clock per SM, so the FMA of phase D
// is the bound; candidate comparisons run on the integer pipe (pivot keys).
#include <math.h>

#include "gj_internal.cuh"

namespace gj {
namespace {

__host__ __device__ inline int cta_ldw(int n) { return (n % 2 == 0) ? n + 1 : (n > 0 ? n : 1); }

struct Carve {
  double* W;
  double* prow;
  double* lcol;
  double* pivs;
  uint64_t* red_v;
  int* rowat;
  int* colat;
  int* posrow;
  int* poscol;
  int* pr_rec;
  int* pc_rec;
  int* red_k;
};

__host__ __device__ inline size_t carve_bytes(int nmax, Carve* c, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) & ~size_t(15);
    return base ? base + o : nullptr;
  };
  const int ldw = cta_ldw(nmax);
  double* W = (double*)take(sizeof(double) * (size_t)nmax * ldw);
  double* prow = (double*)take(sizeof(double) * nmax);
  double* lcol = (double*)take(sizeof(double) * nmax);
  double* pivs = (double*)take(sizeof(double) * nmax);
  uint64_t* red_v = (uint64_t*)take(sizeof(uint64_t) * 32);
  int* rowat = (int*)take(sizeof(int) * nmax);
  int* colat = (int*)take(sizeof(int) * nmax);
  int* posrow = (int*)take(sizeof(int) * nmax);
  int* poscol = (int*)take(sizeof(int) * nmax);
  int* pr_rec = (int*)take(sizeof(int) * nmax);
  int* pc_rec = (int*)take(sizeof(int) * nmax);
  int* red_k = (int*)take(sizeof(int) * 32);
  if (c) *c = Carve{W, prow, lcol, pivs, red_v, rowat, colat, posrow, poscol, pr_rec, pc_rec, red_k};
  return off;
}

__device__ __forceinline__ void consider(double v, int key, uint64_t& bv, int& bk) {
  uint64_t a = abs_bits(v);
  if (key_better(a, key, bv, bk)) {
    bv = a;
    bk = key;
  }
}

template <int NT>
__device__ void solve_matrix(const int n, const double* __restrict__ A, const int64_t lda, double* X, const int mode,
                             const double tau, const CtaOut& out, const int64_t m, const bool single, char* smem,
                             const int nmax) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ double s_inv_q;
  __shared__ int s_R, s_C, s_status, s_fail;

  if (n == 0) {
    if (tid == 0) {
      if (out.status) out.status[m] = GJ_OK;
      if (out.det_sign) out.det_sign[m] = 1;
      if (out.det_log2) out.det_log2[m] = 0.0;
      if (out.fail_step) out.fail_step[m] = -1;
    }
    return;
  }

  Carve c;
  carve_bytes(nmax, &c, smem);
  const int ldw = cta_ldw(n);
  double* __restrict__ W = c.W;
  const int nn = n * n;

  for (int t = tid; t < n; t += NT) {
    c.rowat[t] = t;
    c.colat[t] = t;
    c.posrow[t] = t;
    c.poscol[t] = t;
  }
  if (tid == 0) {
    s_status = GJ_OK;
    s_fail = -1;
  }

  // eqs. 1-2: load A (D = I stays implicit) and scan the step-0 candidates.
  uint64_t bv = 0;
  int bk = kNoKey;
  for (int e = tid; e < nn; e += NT) {
    const int j = e / n, i = e - j * n;
    const double v = A[i + (int64_t)j * lda];
    W[i + j * ldw] = v;
    if (mode == GJ_PIVOT_PARTIAL) {
      if (j == 0) consider(v, i, bv, bk);
    } else if (mode == GJ_PIVOT_FULL) {
      consider(v, j * n + i, bv, bk);
    }
  }
  warp_argmax(bv, bk);
  if (lane == 0) {
    c.red_v[wid] = bv;
    c.red_k[wid] = bk;
  }
  __syncthreads();

  int sign = 1;  // meaningful in thread 0 only
  const int di = NT % n, dj = NT / n;
  for (int k = 0; k < n; ++k) {
    // ---- B: pivot decision (observations 2-3), interchange, eq. 13 factor
    if (tid == 0) {
      uint64_t v = 0;
      int key = kNoKey;
      int rp = k, cp = k;
      if (mode == GJ_PIVOT_NONE) {
        v = abs_bits(W[c.rowat[k] + c.colat[k] * ldw]);
      } else {
#pragma unroll
        for (int w = 0; w < NW; ++w)
          if (key_better(c.red_v[w], c.red_k[w], v, key)) {
            v = c.red_v[w];
            key = c.red_k[w];
          }
        if (mode == GJ_PIVOT_PARTIAL) {
          rp = key;
        } else {
          cp = key / n;
          rp = key - cp * n;
        }
      }
      int st = GJ_OK;
      if (v >= kInfBits) st = GJ_NONFINITE;
      else if (__longlong_as_double((long long)v) <= tau) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
      if (st != GJ_OK) {
        s_status = st;
        s_fail = k;
      } else {
        const int ra = c.rowat[k], rb = c.rowat[rp];
        c.rowat[k] = rb;
        c.rowat[rp] = ra;
        c.posrow[rb] = k;
        c.posrow[ra] = rp;
        const int ca = c.colat[k], cb = c.colat[cp];
        c.colat[k] = cb;
        c.colat[cp] = ca;
        c.poscol[cb] = k;
        c.poscol[ca] = cp;
        const int R = rb, C = cb;
        const double q = W[R + C * ldw];
        c.pivs[k] = q;
        c.pr_rec[k] = rp;
        c.pc_rec[k] = cp;
        if (rp != k) sign = -sign;
        if (cp != k) sign = -sign;
        if (q < 0.0) sign = -sign;
        s_R = R;
        s_C = C;
        s_inv_q = 1.0 / q;
      }
    }
    __syncthreads();
    if (s_status != GJ_OK) break;
    const int R = s_R, C = s_C;
    const double inv_q = s_inv_q;

    // ---- C: eq. 14 pivot row (the D entry of the pivot slot is 1 before the division)
    //         and the pivot column of eq. 15.
    for (int t = tid; t < 2 * n; t += NT) {
      if (t < n) {
        c.prow[t] = (t == C) ? inv_q : W[R + t * ldw] * inv_q;
      } else {
        const int i = t - n;
        c.lcol[i] = (i == R) ? 0.0 : W[i + C * ldw];
      }
    }
    __syncthreads();

    // ---- D: eq. 15 for every other row, fused with the next step's candidate scan.
    const int kn = k + 1;
    const bool search = (kn < n) && (mode != GJ_PIVOT_NONE);
    bv = 0;
    bk = kNoKey;
    int i = tid % n, j = tid / n;
    for (int e = tid; e < nn; e += NT) {
      double* wp = &W[i + j * ldw];
      double nv;
      if (i == R) {
        nv = c.prow[j];
      } else {
        const double base = (j == C) ? 0.0 : *wp;
        nv = fma(-c.lcol[i], c.prow[j], base);
      }
      *wp = nv;
      if (search) {
        if (mode == GJ_PIVOT_PARTIAL) {
          if (j == kn) {
            const int pr = c.posrow[i];
            if (pr >= kn) consider(nv, pr, bv, bk);
          }
        } else {
          const int pr = c.posrow[i], pc = c.poscol[j];
          if (pr >= kn && pc >= kn) consider(nv, pc * n + pr, bv, bk);
        }
      }
      i += di;
      j += dj;
      if (i >= n) {
        i -= n;
        ++j;
      }
    }
    if (search) {
      warp_argmax(bv, bk);
      if (lane == 0) {
        c.red_v[wid] = bv;
        c.red_k[wid] = bk;
      }
    }
    __syncthreads();
  }

  const int status = s_status;
  if (status == GJ_OK) {
    // reverse-order un-permutation (observation 3), as one gather
    for (int e = tid; e < nn; e += NT) {
      const int j = e / n, i = e - j * n;
      X[i + (int64_t)j * n] = W[c.rowat[c.poscol[i]] + c.colat[c.posrow[j]] * ldw];
    }
  }
  if (wid == 0) {
    double lg = 0.0;
    if (status == GJ_OK)
      for (int t = lane; t < n; t += 32) lg += log2(fabs(c.pivs[t]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, off);
    if (lane == 0) {
      if (out.status) out.status[m] = status;
      if (out.det_sign) out.det_sign[m] = (int8_t)(status == GJ_OK ? sign : 0);
      if (out.det_log2) out.det_log2[m] = (status == GJ_OK) ? lg : -INFINITY;
      if (out.fail_step) out.fail_step[m] = (status == GJ_OK) ? -1 : s_fail;
    }
  }
  if (single) {
    const int upto = (status == GJ_OK) ? n : s_fail;
    for (int t = tid; t < upto; t += NT) {
      if (out.piv_rows) out.piv_rows[t] = c.pr_rec[t];
      if (out.piv_cols) out.piv_cols[t] = c.pc_rec[t];
      if (out.pivots) out.pivots[t] = c.pivs[t];
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) cta_single_kernel(int n, const double* A, int64_t lda, double* X, int mode,
                                                        double tau, CtaOut out) {
  extern __shared__ __align__(16) char smem[];
  solve_matrix<NT>(n, A, lda, X, mode, tau, out, 0, true, smem, n);
}

// Persistent: the CTA takes work items q_begin, q_begin + 1, ... < q_end from a shared
// counter; item q is matrix order[q] (the work order lists the largest orders first).
template <int NT>
__global__ void __launch_bounds__(NT) cta_batched_kernel(int64_t q_begin, int64_t q_end, int nmax,
                                                         const int32_t* __restrict__ nv,
                                                         const double* const* __restrict__ A,
                                                         double* const* __restrict__ X,
                                                         const int32_t* __restrict__ order, int32_t* counter,
                                                         int mode, double tau, CtaOut out) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t q = q_begin + s_item;
    __syncthreads();
    if (q >= q_end) break;
    const int64_t m = order ? order[q] : q;
    const int n = nv[m];
    if (n < 0 || n > nmax) {
      if (threadIdx.x == 0) {
        if (out.status) out.status[m] = GJ_ERR_ARG;
        if (out.det_sign) out.det_sign[m] = 0;
        if (out.det_log2) out.det_log2[m] = -INFINITY;
        if (out.fail_step) out.fail_step[m] = -1;
      }
      continue;
    }
    solve_matrix<NT>(n, A[m], n > 0 ? n : 1, X[m], mode, tau, out, m, false, smem, nmax);
    __syncthreads();
  }
}

// One warp inverts one matrix of order n <= 32 held in registers: lane i keeps row i of
// the compact [A | D] array (w[j] = W[i, j]).  Interchanges stay implicit (each lane
// knows the position of its row); per step the candidates of eq. 14 are compared across
// the warp by shuffles, the pivot row is broadcast from its lane by shuffles and every
// lane applies eq. 15 to its own row.  No shared memory, no block barriers.  Partial or
// no pivoting (full pivoting needs column positions in every lane: the CTA kernel).
template <int WPC>
__global__ void __launch_bounds__(WPC * 32) warp_batched_kernel(int64_t q_begin, int64_t q_end,
                                                                const int32_t* __restrict__ nv,
                                                                const double* const* __restrict__ A,
                                                                double* const* __restrict__ X,
                                                                const int32_t* __restrict__ order,
                                                                int32_t* counter, int mode, double tau,
                                                                CtaOut out) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    const int64_t q = q_begin + __shfl_sync(0xffffffffu, item, 0);
    if (q >= q_end) break;
    const int64_t m = order ? order[q] : q;
    const int n = nv[m];
    if (n < 0 || n > 32) {
      if (lane == 0) {
        if (out.status) out.status[m] = GJ_ERR_ARG;
        if (out.det_sign) out.det_sign[m] = 0;
        if (out.det_log2) out.det_log2[m] = -INFINITY;
        if (out.fail_step) out.fail_step[m] = -1;
      }
      continue;
    }
    const double* __restrict__ Am = A[m];
    double w[32];
    const bool live = lane < n;
#pragma unroll
    for (int j = 0; j < 32; ++j) w[j] = (live && j < n) ? Am[lane + j * n] : 0.0;
    int pos = lane;       // position of this lane's row (rows of lanes >= n are never candidates)
    bool used = !live;    // row already chosen as a pivot row
    int sign = 1, status = GJ_OK, fail = -1;
    double lg = 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k >= n) break;
      // ---- pivot candidates of step k (observations 2-3), compared on the integer pipe
      uint64_t bv = 0;
      int bk = kNoKey;
      if (mode == GJ_PIVOT_NONE) {
        if (live && pos == k) {
          bv = abs_bits(w[k]);
          bk = k;
        }
      } else if (!used) {
        bv = abs_bits(w[k]);
        bk = pos;
      }
      warp_argmax(bv, bk);
      if (bk == kNoKey || __longlong_as_double((long long)bv) <= tau) {
        status = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
        fail = k;
        break;
      }
      if (bv >= kInfBits) {
        status = GJ_NONFINITE;
        fail = k;
        break;
      }
      const int rp = bk;  // position of the pivot row
      const int R = __ffs(__ballot_sync(0xffffffffu, live && pos == rp)) - 1;
      if (rp != k) {
        sign = -sign;
        pos = (pos == k) ? rp : (pos == rp ? k : pos);
      }
      const double qv = __shfl_sync(0xffffffffu, w[k], R);
      if (qv < 0.0) sign = -sign;
      lg += log2(fabs(qv));
      const double inv_q = 1.0 / qv;
      // ---- eq. 14 (pivot row, broadcast) and eq. 15 (own row); the slot of column k
      //      carries D's column from now on
      const bool isR = lane == R;
      const double l = w[k];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= n) break;
        const double pj = (j == k) ? inv_q : __shfl_sync(0xffffffffu, w[j], R) * inv_q;
        w[j] = isR ? pj : fma(-l, pj, (j == k) ? 0.0 : w[j]);
      }
      if (isR) used = true;
    }
    if (status == GJ_OK) {
      // reverse-order un-permutation (observation 3) as one gather: the row of position p
      // goes to output row p, column c of W to output column rowat[c]
      double* __restrict__ Xm = X[m];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c >= n) break;
        const int col = __ffs(__ballot_sync(0xffffffffu, live && pos == c)) - 1;
        if (live) Xm[pos + col * n] = w[c];
      }
    }
    if (lane == 0) {
      if (out.status) out.status[m] = status;
      if (out.det_sign) out.det_sign[m] = (int8_t)(status == GJ_OK ? sign : 0);
      if (out.det_log2) out.det_log2[m] = (status == GJ_OK) ? lg : -INFINITY;
      if (out.fail_step) out.fail_step[m] = (status == GJ_OK) ? -1 : fail;
    }
  }
}

// ---- largest-first work order: counting sort over the orders 0..kCtaMaxN
__global__ void order_hist_kernel(int64_t count, const int32_t* __restrict__ n, int32_t* hist) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < count; m += (int64_t)gridDim.x * blockDim.x) {
    int v = n[m];
    if (v < 0 || v > kCtaMaxN) v = 0;
    atomicAdd(&hist[v], 1);
  }
}

__global__ void order_scan_kernel(int32_t* hist, int32_t* counter) {
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int v = kCtaMaxN; v >= 0; --v) {
      const int32_t h = hist[v];
      hist[v] = run;
      run += h;
    }
    *counter = 0;
  }
}

__global__ void order_scatter_kernel(int64_t count, const int32_t* __restrict__ n, int32_t* start, int32_t* order) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < count; m += (int64_t)gridDim.x * blockDim.x) {
    int v = n[m];
    if (v < 0 || v > kCtaMaxN) v = 0;
    order[atomicAdd(&start[v], 1)] = (int32_t)m;
  }
}

template <int NT>
gj_status launch_batched_nt(int64_t q_begin, int64_t q_end, int nmax, const int32_t* n, const double* const* A,
                            double* const* X, const int32_t* order, int32_t* counter, int mode, double tau,
                            const CtaOut& out, cudaStream_t s) {
  const size_t smem = cta_smem_bytes(nmax);
  auto kern = cta_batched_kernel<NT>;
  GJ_CUDA(allow_max_dynamic_smem((const void*)kern));
  int dev = 0, sms = 0, per_sm = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) return GJ_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > q_end - q_begin) grid = q_end - q_begin;
  if (grid < 1) grid = 1;
  prof_count(1);
  ProfScope ps(s, "cta_batched", 0.0, 0.0);
  kern<<<(unsigned)grid, NT, smem, s>>>(q_begin, q_end, nmax, n, A, X, order, counter, mode, tau, out);
  GJ_CUDA(cudaGetLastError());
  return GJ_OK;
}

template <int WPC>
gj_status launch_batched_warp(int64_t q_begin, int64_t q_end, const int32_t* n, const double* const* A,
                              double* const* X, const int32_t* order, int32_t* counter, int mode, double tau,
                              const CtaOut& out, cudaStream_t s) {
  auto kern = warp_batched_kernel<WPC>;
  int dev = 0, sms = 0, per_sm = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPC * 32, 0));
  if (per_sm < 1) return GJ_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t need = (q_end - q_begin + WPC - 1) / WPC;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  prof_count(1);
  ProfScope ps(s, "warp_batched", 0.0, 0.0);
  kern<<<(unsigned)grid, WPC * 32, 0, s>>>(q_begin, q_end, n, A, X, order, counter, mode, tau, out);
  GJ_CUDA(cudaGetLastError());
  return GJ_OK;
}

}  // namespace

size_t cta_smem_bytes(int nmax) { return carve_bytes(nmax < 1 ? 1 : nmax, nullptr, nullptr); }

gj_status launch_cta_single(int n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                            const CtaOut& out, cudaStream_t s) {
  if (n < 0 || n > kCtaMaxN) return GJ_ERR_ARG;
  const size_t smem = cta_smem_bytes(n);
  prof_count(1);
  ProfScope ps(s, "cta_single", 2.0 * n * n * (double)n, 16.0 * n * n);
  if (n > 64) {
    GJ_CUDA(allow_max_dynamic_smem((const void*)cta_single_kernel<512>));
    cta_single_kernel<512><<<1, 512, smem, s>>>(n, A, lda, X, pivot_mode, tau, out);
  } else if (n > 32) {
    GJ_CUDA(allow_max_dynamic_smem((const void*)cta_single_kernel<256>));
    cta_single_kernel<256><<<1, 256, smem, s>>>(n, A, lda, X, pivot_mode, tau, out);
  } else {
    GJ_CUDA(allow_max_dynamic_smem((const void*)cta_single_kernel<128>));
    cta_single_kernel<128><<<1, 128, smem, s>>>(n, A, lda, X, pivot_mode, tau, out);
  }
  GJ_CUDA(cudaGetLastError());
  return GJ_OK;
}

gj_status launch_cta_batched(int64_t count, int nmax, const int32_t* n, const double* const* A, double* const* X,
                             const int32_t* order, int32_t* counter, int pivot_mode, double tau, const CtaOut& out,
                             cudaStream_t s) {
  if (count <= 0) return GJ_OK;
  if (nmax < 1) nmax = 1;
  if (nmax > kCtaMaxN) return GJ_ERR_ARG;
  if (nmax > 64) return launch_batched_nt<256>(0, count, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
  if (nmax > 16) return launch_batched_nt<128>(0, count, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
  return launch_batched_nt<64>(0, count, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
}

bool batched_variant_applies(int variant, int nmax, int pivot_mode) {
  switch (variant) {
    case kVarWarp4:
    case kVarWarp8:
      return nmax <= 32 && pivot_mode != GJ_PIVOT_FULL;
    case kVarCta64:
    case kVarCta128:
    case kVarCta256:
    case kVarCta512:
      return nmax <= kCtaMaxN;
    default:
      return false;
  }
}

gj_status launch_batched_variant(int variant, int64_t q_begin, int64_t q_end, int nmax, const int32_t* n,
                                 const double* const* A, double* const* X, const int32_t* order, int32_t* counter,
                                 int pivot_mode, double tau, const CtaOut& out, cudaStream_t s) {
  if (q_end <= q_begin) return GJ_OK;
  if (nmax < 1) nmax = 1;
  if (!batched_variant_applies(variant, nmax, pivot_mode)) return GJ_ERR_ARG;
  switch (variant) {
    case kVarWarp4:
      return launch_batched_warp<4>(q_begin, q_end, n, A, X, order, counter, pivot_mode, tau, out, s);
    case kVarWarp8:
      return launch_batched_warp<8>(q_begin, q_end, n, A, X, order, counter, pivot_mode, tau, out, s);
    case kVarCta64:
      return launch_batched_nt<64>(q_begin, q_end, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
    case kVarCta128:
      return launch_batched_nt<128>(q_begin, q_end, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
    case kVarCta256:
      return launch_batched_nt<256>(q_begin, q_end, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
    default:
      return launch_batched_nt<512>(q_begin, q_end, nmax, n, A, X, order, counter, pivot_mode, tau, out, s);
  }
}

gj_status launch_order_by_size(int64_t count, const int32_t* n, int32_t* order, int32_t* ws, int32_t* counter,
                               cudaStream_t s) {
  GJ_CUDA(cudaMemsetAsync(ws, 0, sizeof(int32_t) * (kCtaMaxN + 1), s));
  if (count > 0) {
    const int threads = 256;
    int64_t blocks = (count + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    prof_count(3);
    order_hist_kernel<<<(unsigned)blocks, threads, 0, s>>>(count, n, ws);
    GJ_CUDA(cudaGetLastError());
    order_scan_kernel<<<1, 32, 0, s>>>(ws, counter);
    GJ_CUDA(cudaGetLastError());
    order_scatter_kernel<<<(unsigned)blocks, threads, 0, s>>>(count, n, ws, order);
    GJ_CUDA(cudaGetLastError());
  } else {
    GJ_CUDA(cudaMemsetAsync(counter, 0, sizeof(int32_t), s));
  }
  return GJ_OK;
}

}  // namespace gj
