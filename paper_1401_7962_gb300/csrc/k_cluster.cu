// k_cluster.cu -- one matrix of order n <= 128 inverted by a thread-block cluster.
//
// A single CTA is bound by its SM's FP64 units (about 8 GFLOP/s on GB300), so for the
// latency of one small inversion the rows are spread over the CTAs of a cluster (row g to
// CTA g mod cs) and the FP64 work of eq. 15 runs on cs SMs.  Each step of Section 2:
//   * every CTA reduces its own best candidate (observations 2-3: max |a| over the unused
//     rows of the candidate columns; ties to the smallest column position, then row
//     position) during the previous step's eq. 15 pass;
//   * it pushes a record -- key, value, the candidate row (all n columns, unscaled) -- into
//     a slot of every CTA of the cluster with st.async, counted on the receiver's mbarrier;
//   * every CTA waits for the cs records, takes the same winner, applies the interchange to
//     its copy of the position maps, forms the eq. 14 row from the winner's record and
//     applies eq. 15 to its own rows.
// Three slots per CTA: a slot is rewritten (step t + 3) only after every CTA has read it
// (step t), because a CTA cannot push step t + 3's record before it has received all
// records of step t + 2, which every CTA pushes after finishing step t + 1.  Waits are
// bounded (2 s); on expiry the status becomes GJ_ERR_TIMEOUT.
#include <cooperative_groups.h>
#include <math.h>

#include "cluster_ptx.cuh"
#include "gj_internal.cuh"

namespace cg = cooperative_groups;

namespace gj {
namespace {

constexpr int kCluThreads = 256;
constexpr int kCluWarps = kCluThreads / 32;
constexpr int kCluSlots = 3;

struct __align__(16) CluRecHead {
  uint64_t absv;  // |value| bits of the candidate (pivot key)
  int key;        // tie key: row position (partial), column position * n + row position (full)
  int row;        // physical row (-1: no candidate)
  int col;        // physical column
  int pad;
  double q;       // the candidate value
};

__host__ __device__ inline int clu_rec_bytes(int n) {  // multiple of 16 bytes
  return (int)sizeof(CluRecHead) + 8 * ((n + 1) & ~1);
}

__host__ __device__ inline size_t clu_smem_bytes(int n, int cs) {
  const int rpc = (n + cs - 1) / cs;
  size_t b = (size_t)clu_rec_bytes(n) * (kCluSlots * cs + 1);  // slots + staging record
  b += sizeof(double) * (size_t)rpc * (n + 1);                 // own rows, ld n + 1
  b += sizeof(double) * (size_t)(2 * 128 + 128);               // prow, lcol, pivots
  b += sizeof(int) * 6 * 128;                                  // maps and pivot record
  return (b + 15) & ~size_t(15);
}

__device__ __forceinline__ void clu_consider(double v, int key, int il, int j, uint64_t& bv, int& bk, int& bi,
                                             int& bj) {
  const uint64_t a = abs_bits(v);
  if (key_better(a, key, bv, bk)) {
    bv = a;
    bk = key;
    bi = il;
    bj = j;
  }
}

__global__ void __launch_bounds__(kCluThreads, 1)
    cluster_inv_kernel(int n, const double* __restrict__ A, int64_t lda, double* __restrict__ X, int mode,
                       double tau, CtaOut out) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cs = (int)cluster.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rpc = (n + cs - 1) / cs;           // rows per CTA (upper bound)
  const int ldr = n + 1;
  const int rec = clu_rec_bytes(n);
  extern __shared__ __align__(16) char smem[];
  char* slots = smem;                                            // [kCluSlots][cs] records
  char* stage = slots + (size_t)rec * kCluSlots * cs;            // own record being pushed
  double* Wl = reinterpret_cast<double*>(stage + rec);           // [rpc][ldr] own rows
  double* prow = Wl + (size_t)rpc * ldr;                         // eq. 14 row of the step
  double* lcol = prow + 128;                                     // eq. 15 multipliers of own rows
  double* pivs = lcol + 128;
  int* rowat = reinterpret_cast<int*>(pivs + 128);
  int* colat = rowat + 128;
  int* posrow = colat + 128;
  int* poscol = posrow + 128;
  int* pr_rec = poscol + 128;
  int* pc_rec = pr_rec + 128;
  __shared__ __align__(8) uint64_t slot_bar[kCluSlots];
  __shared__ uint64_t red_v[kCluWarps];
  __shared__ int red_k[kCluWarps], red_i[kCluWarps], red_j[kCluWarps];
  __shared__ int s_R, s_C, s_status, s_fail;
  __shared__ double s_inv;
  const uint32_t tx_bytes = (uint32_t)(cs * rec);
  const uint64_t tau_bits = static_cast<uint64_t>(__double_as_longlong(tau));
  const int nown = (rank < n) ? (n - 1 - rank) / cs + 1 : 0;  // rows g = rank + il cs < n

  if (tid == 0) {
    for (int q = 0; q < kCluSlots; ++q) bar_init(&slot_bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < kCluSlots; ++q) bar_expect(&slot_bar[q], tx_bytes);  // phase 0 of every slot
    s_status = GJ_OK;
    s_fail = -1;
  }
  for (int t = tid; t < n; t += kCluThreads) {
    rowat[t] = colat[t] = posrow[t] = poscol[t] = t;
  }
  // eqs. 1-2: own rows of A (D = I stays implicit in the compact array)
  for (int e = tid; e < nown * n; e += kCluThreads) {
    const int il = e / n, j = e - il * n;
    const int g = rank + il * cs;
    Wl[il * ldr + j] = A[(int64_t)g + (int64_t)j * lda];
  }
  __syncthreads();
  cluster.sync();  // every CTA has armed its slots before any remote store

  // Block-reduce the candidates, stage the record (candidate row unscaled) and push it into
  // slot `slot` of every CTA.
  auto push = [&](uint64_t bv, int bk, int bi, int bj, int slot) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
      if (key_better(ov, ok, bv, bk)) {
        bv = ov;
        bk = ok;
        bi = oi;
        bj = oj;
      }
    }
    if (lane == 0) {
      red_v[wid] = bv;
      red_k[wid] = bk;
      red_i[wid] = bi;
      red_j[wid] = bj;
    }
    __syncthreads();
    if (wid == 0) {
      uint64_t v = (lane < kCluWarps) ? red_v[lane] : 0ull;
      int key = (lane < kCluWarps) ? red_k[lane] : kNoKey;
      int il = (lane < kCluWarps) ? red_i[lane] : -1;
      int jj = (lane < kCluWarps) ? red_j[lane] : -1;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const uint64_t ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int oi = __shfl_xor_sync(0xffffffffu, il, off);
        const int oj = __shfl_xor_sync(0xffffffffu, jj, off);
        if (key_better(ov, ok, v, key)) {
          v = ov;
          key = ok;
          il = oi;
          jj = oj;
        }
      }
      CluRecHead* h = reinterpret_cast<CluRecHead*>(stage);
      double* vals = reinterpret_cast<double*>(stage + sizeof(CluRecHead));
      for (int j = lane; j < ((n + 1) & ~1); j += 32) vals[j] = (il >= 0 && j < n) ? Wl[il * ldr + j] : 0.0;
      if (lane == 0) {
        h->absv = v;
        h->key = key;
        h->row = (il >= 0) ? rank + il * cs : -1;
        h->col = jj;
        h->pad = 0;
        h->q = (il >= 0) ? Wl[il * ldr + jj] : 0.0;
      }
    }
    __syncthreads();
    // warp w stores the staged record into the slots of CTAs w, w + 8, ...
    for (int dr = wid; dr < cs; dr += kCluWarps) {
      const uint32_t dst = map_rank(smem_addr(slots + (size_t)rec * (slot * cs + rank)), dr);
      const uint32_t rbar = map_rank(smem_addr(&slot_bar[slot]), dr);
      const int4* src4 = reinterpret_cast<const int4*>(stage);
      for (int w = lane; w < rec / 16; w += 32) st_async16(dst + 16u * w, src4[w], rbar);
    }
  };

  {  // step 0 candidates
    uint64_t bv = 0;
    int bk = kNoKey, bi = -1, bj = -1;
    for (int e = tid; e < nown * n; e += kCluThreads) {
      const int il = e / n, j = e - il * n;
      const int g = rank + il * cs;
      const double v = Wl[il * ldr + j];
      if (mode == GJ_PIVOT_FULL) clu_consider(v, j * n + g, il, j, bv, bk, bi, bj);
      else if (mode == GJ_PIVOT_PARTIAL ? (j == 0) : (j == 0 && g == 0)) clu_consider(v, g, il, j, bv, bk, bi, bj);
    }
    push(bv, bk, bi, bj, 0);
  }

  int sign = 1;
  for (int k = 0; k < n; ++k) {
    const int sq = k % kCluSlots;
    const bool got = bar_wait(&slot_bar[sq], (uint32_t)((k / kCluSlots) & 1));
    if (__syncthreads_or(!got)) {
      if (tid == 0) {
        s_status = GJ_ERR_TIMEOUT;
        s_fail = k;
      }
      break;
    }
    // ---- the winner of step k (identical in every CTA): lane c of warp 0 reads record c
    if (wid == 0) {
      const char* base = slots + (size_t)rec * sq * cs;
      uint64_t wv = 0;
      int wk = kNoKey, ws = -1;
      if (lane < cs) {
        const CluRecHead* h = reinterpret_cast<const CluRecHead*>(base + (size_t)rec * lane);
        if (h->row >= 0) {
          wv = h->absv;
          wk = h->key;
          ws = lane;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const uint64_t ov = __shfl_xor_sync(0xffffffffu, wv, off);
        const int ok = __shfl_xor_sync(0xffffffffu, wk, off);
        const int os = __shfl_xor_sync(0xffffffffu, ws, off);
        if (os >= 0 && (ws < 0 || key_better(ov, ok, wv, wk))) {
          wv = ov;
          wk = ok;
          ws = os;
        }
      }
      if (lane == 0) {
        if (k + kCluSlots < n) bar_expect(&slot_bar[sq], tx_bytes);  // next use of this slot
        int st = GJ_OK;
        if (ws < 0) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
        else if (wv >= kInfBits) st = GJ_NONFINITE;
        else if (wv <= tau_bits) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
        if (st != GJ_OK) {
          s_status = st;
          s_fail = k;
        } else {
          const CluRecHead* h = reinterpret_cast<const CluRecHead*>(base + (size_t)rec * ws);
          const int R = h->row, C = h->col;
          const int rp = posrow[R], cp = poscol[C];
          const int ra = rowat[k], ca = colat[k];
          rowat[k] = R;
          rowat[rp] = ra;
          posrow[R] = k;
          posrow[ra] = rp;
          colat[k] = C;
          colat[cp] = ca;
          poscol[C] = k;
          poscol[ca] = cp;
          if (rp != k) sign = -sign;
          if (cp != k) sign = -sign;
          if (h->q < 0.0) sign = -sign;
          pivs[k] = h->q;
          pr_rec[k] = rp;
          pc_rec[k] = cp;
          s_R = R;
          s_C = C;
          s_inv = 1.0 / h->q;
          s_fail = ws;  // slot of the winner (reused below)
        }
      }
    }
    __syncthreads();
    if (s_status != GJ_OK) break;
    const int R = s_R, C = s_C;
    const double inv_q = s_inv;
    // ---- eq. 14 row from the winner's record; multipliers of own rows
    {
      const double* vals =
          reinterpret_cast<const double*>(slots + (size_t)rec * (sq * cs + s_fail) + sizeof(CluRecHead));
      for (int j = tid; j < n; j += kCluThreads) prow[j] = (j == C) ? inv_q : vals[j] * inv_q;
      for (int il = tid; il < nown; il += kCluThreads) {
        const int g = rank + il * cs;
        lcol[il] = (g == R) ? 0.0 : Wl[il * ldr + C];
      }
    }
    __syncthreads();
    // ---- eq. 15 on own rows, fused with the next step's candidate scan
    const int kn = k + 1;
    const bool search = kn < n;
    uint64_t bv = 0;
    int bk = kNoKey, bi = -1, bj = -1;
    const int cnext = search ? colat[kn] : -1;
    for (int e = tid; e < nown * n; e += kCluThreads) {
      const int il = e / n, j = e - il * n;
      const int g = rank + il * cs;
      double nv;
      if (g == R) {
        nv = prow[j];
      } else {
        const double base = (j == C) ? 0.0 : Wl[il * ldr + j];
        nv = fma(-lcol[il], prow[j], base);
      }
      Wl[il * ldr + j] = nv;
      if (search) {
        const int pr = posrow[g];
        if (mode == GJ_PIVOT_FULL) {
          const int pc = poscol[j];
          if (pr >= kn && pc >= kn) clu_consider(nv, pc * n + pr, il, j, bv, bk, bi, bj);
        } else if (mode == GJ_PIVOT_PARTIAL) {
          if (j == cnext && pr >= kn) clu_consider(nv, pr, il, j, bv, bk, bi, bj);
        } else if (j == cnext && pr == kn) {
          clu_consider(nv, kn, il, j, bv, bk, bi, bj);
        }
      }
    }
    if (search) push(bv, bk, bi, bj, kn % kCluSlots);
    else __syncthreads();
  }
  __syncthreads();
  const int status = s_status;
  if (status == GJ_OK) {
    // reverse-order un-permutation (observation 3) as one gather: W[g, c] goes to
    // X[colat[posrow[g]], rowat[poscol[c]]]
    for (int e = tid; e < nown * n; e += kCluThreads) {
      const int il = e / n, c = e - il * n;
      const int g = rank + il * cs;
      const int i = colat[posrow[g]], j = rowat[poscol[c]];
      X[(int64_t)i + (int64_t)j * n] = Wl[il * ldr + c];
    }
  }
  if (rank == 0) {
    if (wid == 0) {
      double lg = 0.0;
      if (status == GJ_OK)
        for (int t = lane; t < n; t += 32) lg += log2(fabs(pivs[t]));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) lg += __shfl_xor_sync(0xffffffffu, lg, off);
      if (lane == 0) {
        if (out.status) *out.status = status;
        if (out.det_sign) *out.det_sign = (int8_t)(status == GJ_OK ? sign : 0);
        if (out.det_log2) *out.det_log2 = (status == GJ_OK) ? lg : -INFINITY;
        if (out.fail_step) *out.fail_step = (status == GJ_OK) ? -1 : s_fail;
      }
    }
    const int upto = (status == GJ_OK) ? n : s_fail;
    for (int t = tid; t < upto; t += kCluThreads) {
      if (out.piv_rows) out.piv_rows[t] = pr_rec[t];
      if (out.piv_cols) out.piv_cols[t] = pc_rec[t];
      if (out.pivots) out.pivots[t] = pivs[t];
    }
  }
  cluster.sync();  // no CTA leaves while stores into its shared memory may be in flight
}

}  // namespace

gj_status launch_cluster_single(int n, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                                const CtaOut& out, cudaStream_t s) {
  if (n < 1 || n > kCtaMaxN) return GJ_ERR_ARG;
  int cs = (n >= 96) ? 16 : (n >= 48 ? 8 : 4);
  const size_t smem = clu_smem_bytes(n, cs);
  GJ_CUDA(allow_max_dynamic_smem((const void*)cluster_inv_kernel));
  if (cs > 8) GJ_CUDA(cudaFuncSetAttribute(cluster_inv_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kCluThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  GJ_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, cluster_inv_kernel, &cfg));
  if (nclusters < 1) return GJ_ERR_UNSUPPORTED;
  prof_count(1);
  ProfScope ps(s, "cluster_single", 2.0 * n * n * (double)n, 16.0 * n * n);
  GJ_CUDA(cudaLaunchKernelEx(&cfg, cluster_inv_kernel, n, A, lda, X, pivot_mode, tau, out));
  return GJ_OK;
}

}  // namespace gj
