// k_blocked.cu -- Gauss-Jordan for large n: blocked (panel + rank-b update) and unblocked.
//
// Blocked form (partial or no pivoting).  Applying eqs. 14-15 for the b steps of a
// panel P = columns k0..k0+b-1 only changes the panel columns among themselves, so
// the panel can be reduced first on its own (n x b, held in the shared memory of a
// thread-block cluster) and the b steps applied to every other column afterwards as
// one product.  With p the b pivot rows, M = W[p, P] and N = W[others, P] before the
// panel, the panel ends as W[p, P] = M^-1 and W[others, P] = -N M^-1 (compact storage
// of the D columns), and every other column R must become
//     W[p, R] <- M^-1 W[p, R],     W[others, R] <- W[others, R] - N M^-1 W[p, R].
// Both are one product L U with U = W[p, R] taken before the update and L = W[:, P] after
// the panel: stored on the pivot rows, added to the others.  U is zero on the columns of
// P, which the update leaves unchanged.
//
// Interchanges are implicit (positions, as in the single-CTA kernel); at the end the
// inverse is gathered as X[i, j] = W[rowat[i], posrow[j]] (reverse-order
// un-permutation of observation 3; no column interchanges in partial pivoting).
//
// Unblocked form (any pivoting, used for full pivoting at n > 128): one launch picks
// the pivot and stages the eq. 14 row and the eq. 15 column, a second launch updates
// the whole array and scans the next step's candidates.
#include <cooperative_groups.h>

#include <algorithm>
#include <functional>
#include <math.h>

#include "gj_ozaki.cuh"
#include "gj_paths.cuh"
#include "cluster_ptx.cuh"

namespace cg = cooperative_groups;

namespace gj {
namespace {

constexpr int kPanelMaxB = 64;
constexpr int kPanelThreads = 512;
constexpr int kPanelWarps = kPanelThreads / 32;

// One pivot candidate as pushed by a cluster CTA to every CTA of the cluster.
struct __align__(16) PanelCand {
  uint64_t absv;                // |value| bits (pivot key)
  int key;                      // position of the candidate row
  int row;                      // its row index
  double q;                     // the candidate value (the pivot if it wins)
  double inv_q;                 // 1 / q
  double prow[kPanelMaxB];      // eq. 14 row over the panel: row * inv_q, inv_q in the pivot slot
};

constexpr int kSlots = 3;        // candidate slots: pushes for step t+1 and reads of step t never collide
constexpr int kRowBlock = 32;    // rows are dealt to the cluster CTAs in blocks of 32, round robin

struct PanelSmem {
  static size_t bytes(int cs, int rp, int bb) {
    size_t s = sizeof(PanelCand) * (size_t)(kSlots * cs + 1);
    s += sizeof(double) * (size_t)(rp + 1) * bb;  // Wp, leading dimension rp + 1
    s += sizeof(double) * (size_t)rp * 2;         // lrow (two steps)
    s += sizeof(double) * (size_t)bb * bb;        // hist: the pivot block's LU factors, step by step
    s += sizeof(int) * (size_t)rp * 3;            // posl, act, pstep
    return (s + 15) & ~size_t(15);
  }
};

// Global row of local row il of cluster CTA `rank` (block-cyclic distribution).
__device__ __forceinline__ int panel_row(int il, int rank, int cs) {
  return ((il / kRowBlock) * cs + rank) * kRowBlock + (il % kRowBlock);
}

__device__ __forceinline__ void consider3(double v, int key, int il, uint64_t& bv, int& bk, int& bi) {
  const uint64_t a = abs_bits(v);
  if (key_better(a, key, bv, bk)) {
    bv = a;
    bk = key;
    bi = il;
  }
}

// As warp_argmax3, carrying the candidate's value and the reciprocal of it along.
__device__ __forceinline__ void warp_argmax5(uint64_t& v, int& key, int& il, double& q, double& inv_q) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int ok = __shfl_xor_sync(0xffffffffu, key, off);
    const int oi = __shfl_xor_sync(0xffffffffu, il, off);
    const double oq = __shfl_xor_sync(0xffffffffu, q, off);
    const double oinv = __shfl_xor_sync(0xffffffffu, inv_q, off);
    if (key_better(ov, ok, v, key)) {
      v = ov;
      key = ok;
      il = oi;
      q = oq;
      inv_q = oinv;
    }
  }
}

__device__ __forceinline__ void warp_argmax3(uint64_t& v, int& key, int& il) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int ok = __shfl_xor_sync(0xffffffffu, key, off);
    const int oi = __shfl_xor_sync(0xffffffffu, il, off);
    if (key_better(ov, ok, v, key)) {
      v = ov;
      key = ok;
      il = oi;
    }
  }
}

// Panel of columns [k0, k0+bb) searched for its pivots by one cluster of `cs` CTAs.  The
// cluster runs eqs. 14-15 only as far as the pivot search needs them: the rows not yet
// pivoted when the panel starts ("active" rows: position >= k0) are eliminated step by step
// on the panel columns right of the current one, their columns left of it keep their eq. 15
// multipliers, and a row leaves the elimination when it becomes a pivot row.  Each step's
// record carries the winner's multipliers and its eq. 14 row, so the panel's records are the
// LU factors of the pivot block M (the pivot rows' panel values at the start).  With them
// every CTA solves M y = r for some right-hand sides at the end, and the rest is one
// product on the whole GPU: the pivot rows end as M^-1 (and M^-1 U on the other columns),
// every other row, pivoted earlier or not, as -N M^-1 with N its panel values at the start
// (and its eq. 15 update on the other columns).  The cluster writes the pivot record, the
// positions and the right-hand factor of that product (on the FP64-FMA path: M^-1 into the
// pivot rows, for the FP64 fix-up); W is otherwise unchanged.
//
// Each CTA splits its warps in two groups.  The critical warps (C, warps 0-3) carry the
// chain that decides the pivots: step t waits on the CTA's own mbarrier for the candidates
// of all CTAs, takes the same winner everywhere, applies the eq. 15 update of steps t - 1
// and t to column t + 1 of the active rows, finds the CTA's candidate for step t + 1 and
// stores it with its eq. 14 row into every CTA's shared memory (st.async, counted on the
// receiver's mbarrier of that slot).  The bulk warps (B, warps 4-15) apply eq. 15 of step
// s to the columns right of s + 2 one step behind, while C runs the exchange of the next
// step (column s + 1 has steps s - 1 and s from C already, column s + 2 gets steps s and
// s + 1 from C in step s + 1).  Two shared-memory step counters (release / acquire) order
// the groups: B starts step s once C has finished column s + 1 of step s; C builds the
// record of its step-(t + 1) candidate only once B has finished step t - 1 (the record
// applies step t to the candidate row on the fly and writes it back).  There is no
// cluster-wide barrier per step: three slots guarantee that a slot is only rewritten after
// every CTA has finished the step that read it (B included: a CTA pushes its step-(t + 1)
// candidate only after its B has finished step t - 1).  Every wait is bounded.
__device__ __forceinline__ void group_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// arrive at named barrier `id` (of `count` threads) without waiting for it
__device__ __forceinline__ void bar_arrive_group(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// barrier over `count` threads of named barrier `id`, returns whether any of them passed pred != 0
__device__ __forceinline__ int group_any(int id, int count, int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(count)
      : "memory");
  return r;
}
__device__ __forceinline__ void step_release(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int step_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
// wait until *ctr >= target (bounded); false when the limit ran out
__device__ __forceinline__ bool step_wait(const int* ctr, int target) {
  if (step_acquire(ctr) >= target) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    __nanosleep(32);
    if (step_acquire(ctr) >= target) return true;
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (t1 - t0 > kClusterWaitNs) return false;
  }
}

constexpr int kPanelCWarps = 4;                                   // critical warps
constexpr int kPanelCThreads = 32 * kPanelCWarps;                 // 128
constexpr int kPanelBThreads = kPanelThreads - kPanelCThreads;    // 384 bulk threads
constexpr int kBarC = 1, kBarB = 2, kBarRec = 3;                  // named barriers of the groups
constexpr int kStepAbort = 1 << 30;                               // C's step counter after an abort

__global__ void __launch_bounds__(kPanelThreads, 1)
    panel_kernel(int n, int k0, int bb, int rp, int K0, int BB, double* __restrict__ W, int* __restrict__ posrow,
                 double* __restrict__ Mbuf, double* __restrict__ Ufix, int* __restrict__ prow_ids,
                 double* __restrict__ pivots, int* __restrict__ piv_rows, int32_t* status, int64_t* fail_step,
                 int mode, double tau) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cs = (int)cluster.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ldp = rp + 1;
  extern __shared__ __align__(16) char smem[];
  PanelCand* slots = reinterpret_cast<PanelCand*>(smem);  // [kSlots][cs]
  PanelCand* stage = slots + kSlots * cs;
  double* Wp = reinterpret_cast<double*>(stage + 1);       // [bb][ldp], column-major over own rows
  double* lrow = Wp + (size_t)ldp * bb;                    // [2][rp]: eq. 15 multipliers of steps t, t - 1
  double* hist = lrow + 2 * rp;                            // [bb][bb]: record row of step s at hist[s * bb]
  int* posl = reinterpret_cast<int*>(hist + (size_t)bb * bb);
  int* act = posl + rp;                                    // local indices of the active rows
  int* pstep = act + rp;                                   // step at which a row became a pivot (bb: not yet)
  __shared__ __align__(8) uint64_t slot_bar[kSlots];
  __shared__ uint64_t red_v[kPanelCWarps];
  __shared__ double red_q[kPanelCWarps], red_inv[kPanelCWarps];
  __shared__ int red_k[kPanelCWarps], red_i[kPanelCWarps], wcount[kPanelWarps];
  __shared__ int s_nact;
  __shared__ int s_cdone, s_bdone;   // steps whose column t + 1 (C) / bulk update (B) is done
  __shared__ volatile int s_abort;   // C gave up (timeout or failed step)
  __shared__ int s_bgo, s_cok;
  __shared__ int s_win[2];           // slot index (sq * cs + winner) of step t, at t & 1
  __shared__ int s_cand[2];          // local row of the CTA's step-(t + 1) candidate (-1: none), at t & 1
  __shared__ int s_prow_g[kPanelMaxB];  // pivot row of step t
  // a record carries its header and the bb entries of prow (rounded up to pairs)
  const uint32_t rec_bytes = (uint32_t)(cs * (32 + 16 * ((bb + 1) / 2)));
  // |v| <= tau  <=>  bits(|v|) <= bits(tau) for non-negative binary64 (tau >= 0)
  const uint64_t tau_bits = static_cast<uint64_t>(__double_as_longlong(tau));

  __shared__ int s_skip;  // rank 0's reading of the call's status (an earlier step failed)

  if (tid == 0) {
    for (int q = 0; q < kSlots; ++q) bar_init(&slot_bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < kSlots; ++q) bar_expect(&slot_bar[q], rec_bytes);  // phase 0 of every slot
    s_nact = 0;
    s_cdone = 0;
    s_bdone = 0;
    s_abort = 0;
    // the status can change while the cluster starts (an update on another stream may fail
    // it): rank 0 reads it once and every CTA follows rank 0's reading
    s_skip = (rank == 0) ? (*status != GJ_OK) : 0;
  }
  for (int il = tid; il < rp; il += kPanelThreads) {
    const int g = panel_row(il, rank, cs);
    posl[il] = (g < n) ? posrow[g] : -1;
    pstep[il] = bb;
  }
  for (int e = tid; e < rp * bb; e += kPanelThreads) {
    const int j = e / rp, il = e - j * rp;
    const int g = panel_row(il, rank, cs);
    Wp[il + j * ldp] = (g < n) ? W[(int64_t)g + (int64_t)(k0 + j) * n] : 0.0;
  }
  __syncthreads();
  // compact the active rows (order preserved) into act[0 .. s_nact)
  for (int base = 0; base < rp; base += kPanelThreads) {
    const int il = base + tid;
    const bool a = il < rp && posl[il] >= k0;
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    int off = s_nact;
    for (int w = 0; w < wid; ++w) off += wcount[w];
    if (a) act[off + __popc(m & ((1u << lane) - 1u))] = il;
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int w = 0; w < kPanelWarps; ++w) tot += wcount[w];
      s_nact += tot;
    }
    __syncthreads();
  }
  const int nact = s_nact;
  cluster.sync();  // every CTA has armed its slots before any remote store
  if (ld_cluster_s32(map_rank(smem_addr(&s_skip), 0))) {
    cluster.sync();  // rank 0 stays until every CTA has read its flag
    return;
  }

  if (tid < kPanelCThreads) {
    // ================================================================ critical warps
    // Reduce the C threads' candidates to the CTA's candidate for step (k0 + tt) (a row whose
    // column tt is current), build its record and store it into every CTA's slot `slot`.
    // For tt > 0 the candidate row still lacks the eq. 15 update of step tprev = tt - 1 on
    // its columns other than tt (multiplier lpend, row prow_prev); the record applies it on
    // the fly and writes the updated values back, except on columns tt and tt + 1, which C
    // handles itself -- so B's step tprev, released here, skips that row.  The record may
    // read the row only once B has finished step tprev - 1 (bulk_needed steps done).
    auto push_candidate = [&](uint64_t bv, int bk, int bi, int tt, int slot, const double* lpend,
                              const double* prow_prev, int bulk_needed) -> bool {
      const bool pend = tt > 0;
      const int tprev = tt - 1;
      warp_argmax3(bv, bk, bi);
      if (lane == 0) {
        red_v[wid] = bv;
        red_k[wid] = bk;
        red_i[wid] = bi;
        // the warp's candidate value (column tt of its row, written by a lane of this warp)
        // and its reciprocal, formed while the barrier below waits for the bulk warps
        const double q = (bi >= 0) ? Wp[bi + tt * ldp] : 0.0;
        red_q[wid] = q;
        red_inv[wid] = (bi >= 0) ? 1.0 / q : 0.0;
      }
      if (tid == 0) s_cok = (bulk_needed <= 0) ? 1 : (int)step_wait(&s_bdone, bulk_needed);
      group_sync(kBarC, kPanelCThreads);
      if (!s_cok) return false;  // uniform: read after the barrier
      // every C warp reduces the four warps' candidates: all C threads know the CTA's one
      uint64_t v = (lane < kPanelCWarps) ? red_v[lane] : 0ull;
      int key = (lane < kPanelCWarps) ? red_k[lane] : kNoKey;
      int il = (lane < kPanelCWarps) ? red_i[lane] : -1;
      double q = (lane < kPanelCWarps) ? red_q[lane] : 0.0;
      double inv_q = (lane < kPanelCWarps) ? red_inv[lane] : 0.0;
      warp_argmax5(v, key, il, q, inv_q);
      il = __shfl_sync(0xffffffffu, il, 0);
      v = __shfl_sync(0xffffffffu, v, 0);
      key = __shfl_sync(0xffffffffu, key, 0);
      q = __shfl_sync(0xffffffffu, q, 0);
      inv_q = __shfl_sync(0xffffffffu, inv_q, 0);
      if (pend && tid == 0) {
        s_cand[tprev & 1] = il;
        step_release(&s_cdone, tt);  // B may run step tprev (skipping row il)
      }
      // Every C warp forms the record in registers (lane j: entry j, and j + 32 of a 64-wide
      // panel) and stores it into the CTAs w, w + 4, ... (st.async of 16-byte pairs); warp 0
      // writes the candidate's step-tprev values back once all four warps have read the row
      // (named barrier kBarRec: warps 1-3 arrive without waiting, warp 0 waits).  Left of tt the candidate holds
      // its eq. 15 multipliers l_j (it is not a pivot row); the record carries them, so that
      // the records of the panel's steps together are the LU factors of the pivot block.
      double pv[2] = {0.0, 0.0}, wb[2] = {0.0, 0.0};
      if (il >= 0) {
        const double l = pend ? lpend[il] : 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = lane + 32 * h;
          if (j >= bb) continue;
          double x = Wp[il + j * ldp];
          if (j < tt) {
            pv[h] = x;
            continue;
          }
          if (pend && j > tt) x = fma(-l, prow_prev[j], x);
          wb[h] = x;
          pv[h] = (j == tt) ? inv_q : x * inv_q;
        }
      }
      if (wid != 0) {
        bar_arrive_group(kBarRec, kPanelCThreads);
      } else {
        group_sync(kBarRec, kPanelCThreads);
        if (il >= 0 && pend) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j < bb && j > tt + 1) Wp[il + j * ldp] = wb[h];  // B's step tprev for this row
          }
        }
      }
      // 16-byte words of the record: 0 = (absv, key, row), 1 = (q, inv_q), 2 + m = prow[2m..2m+1]
      const int npairs = (bb + 1) >> 1;
      const int nwords = 2 + npairs;
      int4 wrd[2];
      // entry j lives in lane j & 31, in pv[0] for j < 32 and pv[1] above (the receiving lane
      // picks the half: a shuffle returns the source lane's value of the variable it names)
      auto entry = [&](int j) -> double {
        const double lo = __shfl_sync(0xffffffffu, pv[0], j & 31);
        const double hi = (bb > 32) ? __shfl_sync(0xffffffffu, pv[1], j & 31) : 0.0;
        return (j >= 32) ? hi : lo;
      };
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = lane + 32 * h - 2;  // prow pair of word lane + 32 h
        const double e0 = entry(2 * m), e1 = entry(2 * m + 1);
        const long long b0 = __double_as_longlong(e0), b1 = __double_as_longlong(e1);
        wrd[h] = make_int4((int)b0, (int)(b0 >> 32), (int)b1, (int)(b1 >> 32));
      }
      if (lane == 0) {
        const long long av = (long long)v;
        wrd[0] = make_int4((int)av, (int)(av >> 32), key, (il >= 0) ? panel_row(il, rank, cs) : -1);
      } else if (lane == 1) {
        const long long bq = __double_as_longlong((il >= 0) ? q : 0.0);
        const long long bi2 = __double_as_longlong((il >= 0) ? inv_q : 0.0);
        wrd[0] = make_int4((int)bq, (int)(bq >> 32), (int)bi2, (int)(bi2 >> 32));
      }
      for (int dst_rank = wid; dst_rank < cs; dst_rank += kPanelCWarps) {
        const uint32_t dst = map_rank(smem_addr(&slots[slot * cs + rank]), dst_rank);
        const uint32_t rbar = map_rank(smem_addr(&slot_bar[slot]), dst_rank);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int w = lane + 32 * h;
          if (w < nwords) st_async16(dst + 16u * w, wrd[h], rbar);
        }
      }
      return true;
    };

    bool abort = false;
    {  // step 0 candidates from the panel as loaded
      uint64_t bv = 0;
      int bk = kNoKey, bi = -1;
      for (int a = tid; a < nact; a += kPanelCThreads) {
        const int il = act[a], p = posl[il];
        if (mode == GJ_PIVOT_NONE ? (p == k0) : (p >= k0)) consider3(Wp[il], p, il, bv, bk, bi);
      }
      push_candidate(bv, bk, bi, 0, 0, nullptr, nullptr, 0);
    }
    const double* prow_prev = nullptr;  // eq. 14 row of step t - 1
    for (int t = 0; t < bb; ++t) {
      const int k = k0 + t;
      const int sq = t % kSlots;
      // all candidates of step t are in slot sq once its phase t / kSlots completes
      const bool got = bar_wait(&slot_bar[sq], (uint32_t)((t / kSlots) & 1));
      if (group_any(kBarC, kPanelCThreads, !got)) {
        if (tid == 0) {
          atomicExch(status, GJ_ERR_TIMEOUT);
          *fail_step = k;
        }
        abort = true;
        break;
      }
      if (tid == 0 && t + kSlots < bb) bar_expect(&slot_bar[sq], rec_bytes);  // next use of this slot
      const PanelCand* sl = &slots[sq * cs];
      // lane c reads CTA c's candidate; a shuffle argmax gives every C warp the same winner
      uint64_t wv = (lane < cs) ? sl[lane].absv : 0ull;
      int wk = (lane < cs) ? sl[lane].key : kNoKey;
      int ws = lane;
      warp_argmax3(wv, wk, ws);
      // keys of real candidates are distinct; only empty ones tie, and lanes may then hold
      // different tied slots: every lane takes lane 0's (slot 0 when all are empty)
      wv = __shfl_sync(0xffffffffu, wv, 0);
      wk = __shfl_sync(0xffffffffu, wk, 0);
      ws = __shfl_sync(0xffffffffu, ws, 0);
      const PanelCand& win = sl[ws];
      int st = GJ_OK;
      if (win.row < 0) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
      else if (wv >= kInfBits) st = GJ_NONFINITE;
      else if (wv <= tau_bits) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
      if (st != GJ_OK) {
        if (rank == 0 && tid == 0) {
          *status = st;
          *fail_step = k;
        }
        abort = true;
        break;
      }
      const int rpos = wk, R = win.row;
      if (rank == 0 && tid == 0) {
        pivots[k] = win.q;
        piv_rows[k] = rpos;
        prow_ids[t] = R;
      }
      const bool next = t + 1 < bb;
      double* lcur = lrow + (t & 1) * rp;
      const double* lprev = lrow + ((t + 1) & 1) * rp;
      // interchange (positions), multipliers of step t, column t + 1 through step t, next
      // candidates
      uint64_t bv = 0;
      int bk = kNoKey, bi = -1;
      const double pr_t = win.prow[next ? t + 1 : t];
      const double pr_p = (t > 0 && next) ? prow_prev[t + 1] : 0.0;
      // four active rows per pass, their loads issued together
      for (int a0 = tid; a0 < nact; a0 += 4 * kPanelCThreads) {
        int il[4], g[4];
        double wt[4], wn[4], lp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = a0 + q * kPanelCThreads;
          il[q] = (a < nact) ? act[a] : -1;
          if (il[q] >= 0 && pstep[il[q]] < t) il[q] = -1;  // pivot rows of earlier steps are done
          g[q] = (il[q] >= 0) ? panel_row(il[q], rank, cs) : -1;
          wt[q] = (il[q] >= 0) ? Wp[il[q] + t * ldp] : 0.0;  // column t: current through step t - 1
          wn[q] = (il[q] >= 0 && next) ? Wp[il[q] + (t + 1) * ldp] : 0.0;  // column t + 1: through t - 2
          lp[q] = (il[q] >= 0 && t > 0) ? lprev[il[q]] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (il[q] < 0) continue;
          int p = posl[il[q]];
          if (g[q] == R) {
            p = k;
            pstep[il[q]] = t;  // the pivot row leaves the elimination
          } else {
            if (p == k) p = rpos;
            lcur[il[q]] = wt[q];
            if (next) {
              const double base = (t == 0) ? wn[q] : fma(-lp[q], pr_p, wn[q]);
              const double nv = fma(-wt[q], pr_t, base);
              Wp[il[q] + (t + 1) * ldp] = nv;
              if (mode == GJ_PIVOT_NONE ? (p == k + 1) : (p >= k + 1)) consider3(nv, p, il[q], bv, bk, bi);
            }
          }
          posl[il[q]] = p;
        }
      }
      if (tid == 0) {
        s_win[t & 1] = sq * cs + ws;
        s_prow_g[t] = R;
      }
      for (int j = tid; j < bb; j += kPanelCThreads) hist[t * bb + j] = win.prow[j];
      if (next) {
        // the barrier inside makes column t + 1, lcur and s_win visible before B is released
        if (!push_candidate(bv, bk, bi, t + 1, (t + 1) % kSlots, lcur, win.prow, t)) {
          if (tid == 0) {
            atomicExch(status, GJ_ERR_TIMEOUT);
            *fail_step = k;
          }
          abort = true;
          break;
        }
      } else {
        group_sync(kBarC, kPanelCThreads);
        if (tid == 0) {
          s_cand[t & 1] = -1;
          step_release(&s_cdone, t + 1);  // B may run the last step
        }
      }
      prow_prev = win.prow;
    }
    if (abort && tid == 0) {
      s_abort = 1;
      step_release(&s_cdone, kStepAbort);  // releases B from its wait
    }
  } else {
    // ================================================================ bulk warps
    const int btid = tid - kPanelCThreads;
    for (int s = 0; s < bb; ++s) {
      if (btid == 0) s_bgo = step_wait(&s_cdone, s + 1) && !s_abort;
      group_sync(kBarB, kPanelBThreads);
      if (!s_bgo) break;  // uniform
      const PanelCand& win = slots[s_win[s & 1]];
      const double* lcur = lrow + (s & 1) * rp;
      const int skip_il = s_cand[s & 1];  // the candidate row: C applied this step to it
      // local index of the pivot row of step s if this CTA owns it (block-cyclic rows)
      // one active row per thread and pass, four columns at a time with every load issued
      // before the dependent FMAs (shared-memory stores would otherwise serialise them)
      for (int a = btid; a < nact; a += kPanelBThreads) {
        const int il = act[a];
        if (il == skip_il || pstep[il] <= s) continue;  // pivot rows are done
        // only the columns right of s + 2 (the next pivot searches read them); the columns
        // left of those keep the row's multipliers
        const double l = lcur[il];
        double* wr = Wp + il;
        for (int j0 = s + 3; j0 < bb; j0 += 4) {
          double w[4], pj[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + q;
            pj[q] = (j < bb) ? win.prow[j] : 0.0;
            w[q] = (j < bb) ? wr[j * ldp] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + q;
            if (j < bb) wr[j * ldp] = fma(-l, pj[q], w[q]);
          }
        }
      }
      group_sync(kBarB, kPanelBThreads);
      if (btid == 0) step_release(&s_bdone, s + 1);
    }
  }
  __syncthreads();
  const bool failed = s_abort != 0;

  if (!failed) {
    for (int a = tid; a < nact; a += kPanelThreads) {
      const int il = act[a];
      posrow[panel_row(il, rank, cs)] = posl[il];
    }
    // The pivot block: M = Lt D U with (from the records) Lt[t][s] = l_s(t) / q_s unit lower,
    // D = diag(q_t) and U[t][j] = prow_t[j] unit upper.  M y = r is solved for a right-hand
    // side r by forward substitution with Lt, the scaling by 1 / q_t and back substitution
    // with U; warp w of CTA `rank` takes the right-hand sides c = rank + cs (w + 16 m), lane
    // t holds y_t (and y_{t + 32}).
    //   Ufix == null (FP64 update path): r = e_c, c < bb: the columns of M^-1, written to Mbuf
    //     and to the pivot rows' panel columns of W (the compact inverse of M).
    //   Ufix != null (tensor-core path): c runs over the outer panel [K0, K0 + BB); r = e_t for
    //     the panel's column k0 + t, else the pivot rows' values in column c (U_R), and
    //     Ufix[:, c] = -y: V = -M^-1 [I | U_R], the right-hand factor of the one product that
    //     ends the panel on the outer panel's columns.  Its left-hand factor is W[:, P] (the
    //     panel values at the start) with the pivot row of step t replaced by -e_t: the pivot
    //     rows are set to M^-1 [I | U_R], the other rows set to -N M^-1 on the panel's columns
    //     and given their eq. 15 update -N M^-1 U_R on the others.
    const int nrhs = Ufix ? BB : bb;
    const int cP = k0 - K0;  // first panel column within the outer panel
    for (int c = rank + cs * wid; c < nrhs; c += cs * kPanelWarps) {
      const int e_at = Ufix ? c - cP : c;  // unit right-hand side e_{e_at}, or none
      const bool unit = e_at >= 0 && e_at < bb;
      const int t0 = lane, t1 = lane + 32;
      double x0 = 0.0, x1 = 0.0;  // rows lane, lane + 32
      if (unit) {
        if (t0 == e_at) x0 = 1.0;
        if (t1 == e_at) x1 = 1.0;
      } else {
        if (t0 < bb) x0 = W[(int64_t)s_prow_g[t0] + (int64_t)(K0 + c) * n];
        if (t1 < bb) x1 = W[(int64_t)s_prow_g[t1] + (int64_t)(K0 + c) * n];
      }
      for (int s2 = unit ? e_at : 0; s2 < bb; ++s2) {  // forward: y_t -= Lt[t][s2] y_s2 for t > s2
        const double ys = __shfl_sync(0xffffffffu, s2 < 32 ? x0 : x1, s2 & 31);
        const double inv_qs = hist[s2 * bb + s2];
        if (t0 > s2 && t0 < bb) x0 = fma(-(hist[t0 * bb + s2] * inv_qs), ys, x0);
        if (t1 > s2 && t1 < bb) x1 = fma(-(hist[t1 * bb + s2] * inv_qs), ys, x1);
      }
      if (t0 < bb) x0 *= hist[t0 * bb + t0];
      if (t1 < bb) x1 *= hist[t1 * bb + t1];
      for (int s2 = bb - 1; s2 > 0; --s2) {  // back: z_t -= U[t][s2] x_s2 for t < s2
        const double xs = __shfl_sync(0xffffffffu, s2 < 32 ? x0 : x1, s2 & 31);
        if (t0 < s2) x0 = fma(-hist[t0 * bb + s2], xs, x0);
        if (t1 < s2) x1 = fma(-hist[t1 * bb + s2], xs, x1);
      }
      if (Ufix) {
        if (t0 < bb) Ufix[t0 + (int64_t)c * bb] = -x0;
        if (t1 < bb) Ufix[t1 + (int64_t)c * bb] = -x1;
      } else {
        if (t0 < bb) {
          W[(int64_t)s_prow_g[t0] + (int64_t)(k0 + c) * n] = x0;
          Mbuf[t0 * kPanelMaxB + c] = x0;
        }
        if (t1 < bb) {
          W[(int64_t)s_prow_g[t1] + (int64_t)(k0 + c) * n] = x1;
          Mbuf[t1 * kPanelMaxB + c] = x1;
        }
      }
    }
  }
  cluster.sync();  // no CTA leaves while stores into its shared memory may be in flight
}

// The rows that are not pivot rows of the panel (position outside [k0, k0 + bb)): the
// panel leaves them at L[i, :] = -W[i, P] M^-1, with W[i, P] their panel values at the start
// of the panel (the cluster kernel writes only the pivot rows back) and
// M^-1[s, t] = Mbuf[s * 64 + t] (the panel's pivot block, written by the panel).  FP64
// version (the FP64-FMA update path): block (x, y) takes 64 consecutive rows and the 8
// columns 8y .. 8y + 7 of the result, so that the FP64 work spreads over as many SMs as the
// rows allow; the rows' panel values are staged in shared memory with coalesced loads,
// thread (r, q) forms row r, columns 8y + 2q and 8y + 2q + 1.  Blocks of the same rows read
// W[i, P] while others write their results, so the results go to L only;
// fixup_store_kernel then copies them into W[i, P].
constexpr int kFixRows = 64, kFixCols = 8;
__device__ __forceinline__ bool panel_pivot_row(int pos, int k0, int bb) { return pos >= k0 && pos < k0 + bb; }

__global__ void __launch_bounds__(256) fixup_rows_kernel(int n, int k0, int bb, double* __restrict__ W,
                                                         const int* __restrict__ posrow,
                                                         const double* __restrict__ Mbuf,
                                                         double* __restrict__ Lbuf, const int32_t* status) {
  if (*status != GJ_OK) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = blockIdx.x * kFixRows, t0 = blockIdx.y * kFixCols;
  const int r = tid % kFixRows, q = tid / kFixRows;  // row in the block, column pair
  const int i = r0 + r;
  const bool other = i < n && !panel_pivot_row(posrow[i], k0, bb);
  __shared__ double Minv[kPanelMaxB][kFixCols];
  __shared__ double Nt[kPanelMaxB][kFixRows + 1];  // Nt[s][r] = W[r0 + r, k0 + s]
  for (int e = tid; e < bb * kFixCols; e += blockDim.x) {
    const int s2 = e / kFixCols, c = e % kFixCols;
    Minv[s2][c] = (t0 + c < bb) ? Mbuf[s2 * kPanelMaxB + t0 + c] : 0.0;
  }
  for (int s2 = w; s2 < bb; s2 += 8) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rr = lane + 32 * h, ii = r0 + rr;
      Nt[s2][rr] = (ii < n) ? W[(int64_t)ii + (int64_t)(k0 + s2) * n] : 0.0;
    }
  }
  __syncthreads();
  double acc0 = 0.0, acc1 = 0.0;
  for (int s2 = 0; s2 < bb; ++s2) {
    const double a = Nt[s2][r];
    acc0 = fma(a, Minv[s2][2 * q], acc0);
    acc1 = fma(a, Minv[s2][2 * q + 1], acc1);
  }
  if (!other) return;
  const int ta = t0 + 2 * q;
  if (ta < bb) Lbuf[(int64_t)i + (int64_t)ta * n] = -acc0;
  if (ta + 1 < bb) Lbuf[(int64_t)i + (int64_t)(ta + 1) * n] = -acc1;
}

// W[i, k0 + t] = L[i, t] for the rows that are not pivot rows of the panel (the FP64
// fix-up's results); the pivot rows' L is set to their panel values (M^-1, written by the
// cluster kernel).
__global__ void fixup_store_kernel(int n, int k0, int bb, double* __restrict__ W, const int* __restrict__ posrow,
                                   double* __restrict__ Lbuf, const int32_t* status) {
  if (*status != GJ_OK) return;
  const int64_t total = (int64_t)n * bb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), i = (int)(e - (int64_t)t * n);
    const int pos = posrow[i];
    double* w = &W[(int64_t)i + (int64_t)(k0 + t) * n];
    if (!panel_pivot_row(pos, k0, bb)) *w = Lbuf[e];
    else Lbuf[e] = *w;
  }
}

// U[t, j - c_lo] = W[prow_ids[t], j] for j in the column window [c_lo, c_hi) outside the
// panel [k0, k0 + bb), 0 inside it (bb x (c_hi - c_lo), column-major).
__global__ void gather_u_kernel(int n, int k0, int bb, int c_lo, int c_hi, const double* __restrict__ W,
                                const int* __restrict__ prow_ids, double* __restrict__ U, const int32_t* status) {
  if (*status != GJ_OK) return;
  const int64_t total = (int64_t)bb * (c_hi - c_lo);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int jj = (int)(e / bb), t = (int)(e - (int64_t)jj * bb);
    const int j = c_lo + jj;
    U[e] = (j >= k0 && j < k0 + bb) ? 0.0 : W[(int64_t)prow_ids[t] + (int64_t)j * n];
  }
}

// W[:, c_lo:c_hi] += L U in FP64 (one FMA per term).  64 x 64 tile per CTA, 4 x 4 per thread.
// The panel's pivot rows (position in [k0, k0 + bb)) take L U instead (their L is M^-1: eq. 14
// for them is W[p, R] = M^-1 W[p, R]), outside the panel's own columns.
constexpr int kTM = 64, kTN = 64, kTK = 32;
__global__ void __launch_bounds__(256) update_dfma_kernel(int n, int bb, int c_lo, int c_hi,
                                                          const double* __restrict__ L,
                                                          const double* __restrict__ U, double* __restrict__ W,
                                                          const int* __restrict__ posrow, int k0,
                                                          const int32_t* status) {
  if (*status != GJ_OK) return;
  __shared__ double Ls[kTK][kTM];
  __shared__ double Us[kTK][kTN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kTM, cw0 = blockIdx.y * kTN;  // cw: column within the window
  const int wn = c_hi - c_lo;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int t0 = 0; t0 < bb; t0 += kTK) {
    const int tk = min(kTK, bb - t0);
    for (int e = tid; e < kTK * kTM; e += 256) {
      const int t = e / kTM, r = e - t * kTM;
      Ls[t][r] = (t < tk && m0 + r < n) ? L[(int64_t)(m0 + r) + (int64_t)(t0 + t) * n] : 0.0;
    }
    for (int e = tid; e < kTK * kTN; e += 256) {
      const int c = e / kTK, t = e - c * kTK;
      Us[t][c] = (t < tk && cw0 + c < wn) ? U[(int64_t)(t0 + t) + (int64_t)(cw0 + c) * bb] : 0.0;
    }
    __syncthreads();
    for (int t = 0; t < tk; ++t) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ls[t][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Us[t][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cw = cw0 + ty + 16 * j;
    if (cw >= wn) continue;
    const int c = c_lo + cw;
    const bool in_panel = c >= k0 && c < k0 + bb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + tx + 16 * i;
      if (r < n) {
        double* p = &W[(int64_t)r + (int64_t)c * n];
        const int pos = posrow[r];
        if (pos >= k0 && pos < k0 + bb) {
          if (!in_panel) *p = acc[i][j];
        } else {
          *p = *p + acc[i][j];
        }
      }
    }
  }
}

// A bounded device wait of the tensor-core update expired: report it as the call's status.
__global__ void fold_error_kernel(const int32_t* err, int32_t* status) {
  if (*err != 0 && *status == GJ_OK) *status = GJ_ERR_TIMEOUT;
}

// ------------------------------------------------------------------ shared epilogues

__global__ void init_positions_kernel(int n, int* posrow, int* poscol, int* rowat, int* colat) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (posrow) posrow[i] = i;
    if (poscol) poscol[i] = i;
    if (rowat) rowat[i] = i;
    if (colat) colat[i] = i;
  }
}

__global__ void copy_in_kernel(int n, const double* __restrict__ A, int64_t lda, double* __restrict__ W) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    W[e] = A[i + j * lda];
  }
}

__global__ void rowat_from_posrow_kernel(int n, const int* __restrict__ posrow, int* __restrict__ rowat,
                                         const int32_t* status) {
  if (*status != GJ_OK) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) rowat[posrow[i]] = i;
}

// X[i, j] = W[rowat[poscol[i]], colat[posrow[j]]]  (colat / poscol null = identity)
__global__ void unpermute_kernel(int n, const double* __restrict__ W, const int* __restrict__ rowat,
                                 const int* __restrict__ posrow, const int* __restrict__ colat,
                                 const int* __restrict__ poscol, double* __restrict__ X, const int32_t* status) {
  if (*status != GJ_OK) return;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    const int src_r = rowat[poscol ? poscol[i] : i];
    const int src_c = colat ? colat[posrow[j]] : posrow[j];
    X[e] = W[(int64_t)src_r + (int64_t)src_c * n];
  }
}

// Right-hand sides appended to the working array: W[:, n + j] = B[:, j].
__global__ void copy_rhs_kernel(int n, int64_t m, const double* __restrict__ B, int64_t ldb,
                                double* __restrict__ Wb) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    Wb[e] = B[i + j * ldb];
  }
}

// Solution of A X = B after the sweep: unknown i was eliminated at position poscol[i]
// (identity without column pivoting) by the row that holds it, rowat[position], so
// X[i, j] = W[rowat[poscol[i]], n + j].
__global__ void gather_solution_kernel(int n, int64_t m, const double* __restrict__ Wb,
                                       const int* __restrict__ rowat, const int* __restrict__ poscol,
                                       double* __restrict__ X, int64_t ldx, const int32_t* status) {
  if (*status != GJ_OK) return;
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n;
    const int i = (int)(e - j * n);
    X[i + j * ldx] = Wb[(int64_t)rowat[poscol ? poscol[i] : i] + j * n];
  }
}

// eq. 13: sign and log2|det| from the recorded pivots and interchanges.
__global__ void __launch_bounds__(1024) det_kernel(int n, const double* __restrict__ pivots,
                                                   const int* __restrict__ piv_rows, const int* __restrict__ piv_cols,
                                                   int32_t* status, int8_t* det_sign, double* det_log2,
                                                   int64_t* fail_step) {
  __shared__ double part[32];
  const int tid = threadIdx.x;
  const int ok = (*status == GJ_OK);
  double lg = 0.0;
  int flips = 0;
  if (ok)
    for (int k = tid; k < n; k += blockDim.x) {
      lg += log2(fabs(pivots[k]));
      flips += (pivots[k] < 0.0) + (piv_rows[k] != k) + (piv_cols ? (piv_cols[k] != k) : 0);
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lg += __shfl_xor_sync(0xffffffffu, lg, off);
    flips += __shfl_xor_sync(0xffffffffu, flips, off);
  }
  __shared__ int fl[32];
  if ((tid & 31) == 0) {
    part[tid >> 5] = lg;
    fl[tid >> 5] = flips;
  }
  __syncthreads();
  if (tid < 32) {
    const int nw = blockDim.x >> 5;
    lg = (tid < nw) ? part[tid] : 0.0;
    flips = (tid < nw) ? fl[tid] : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lg += __shfl_xor_sync(0xffffffffu, lg, off);
      flips += __shfl_xor_sync(0xffffffffu, flips, off);
    }
    if (tid == 0) {
      if (det_sign) *det_sign = ok ? ((flips & 1) ? -1 : 1) : 0;
      if (det_log2) *det_log2 = ok ? lg : -INFINITY;
      if (ok && fail_step) *fail_step = -1;
    }
  }
}

// ------------------------------------------------------------------ unblocked path

struct StepState {
  int R, C;
  double inv_q;
};

// Initial candidate scan of A (step 0), one partial result per block.
__global__ void __launch_bounds__(256) scan0_kernel(int n, const double* __restrict__ W, int mode,
                                                    uint64_t* cand_v, int* cand_k) {
  uint64_t bv = 0;
  int bk = kNoKey;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    if (mode == GJ_PIVOT_PARTIAL && j != 0) continue;
    if (mode == GJ_PIVOT_NONE && !(i == 0 && j == 0)) continue;
    const uint64_t a = abs_bits(W[e]);
    const int key = (mode == GJ_PIVOT_FULL) ? j * n + i : i;
    if (key_better(a, key, bv, bk)) {
      bv = a;
      bk = key;
    }
  }
  warp_argmax(bv, bk);
  __shared__ uint64_t sv[8];
  __shared__ int sk[8];
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    sk[threadIdx.x >> 5] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w)
      if (key_better(sv[w], sk[w], bv, bk)) {
        bv = sv[w];
        bk = sk[w];
      }
    cand_v[blockIdx.x] = bv;
    cand_k[blockIdx.x] = bk;
  }
}

__global__ void __launch_bounds__(1024) decide_kernel(int n, int nw, int k, int G, const uint64_t* cand_v,
                                                      const int* cand_k,
                                                      const double* __restrict__ W, int* rowat, int* colat,
                                                      int* posrow, int* poscol, double* prow, double* lcol,
                                                      StepState* ss, double* pivots, int* piv_rows, int* piv_cols,
                                                      int32_t* status, int64_t* fail_step, int mode, double tau) {
  if (*status != GJ_OK) return;
  __shared__ uint64_t sv[32];
  __shared__ int sk[32];
  __shared__ int s_ok, s_R, s_C;
  __shared__ double s_inv;
  uint64_t bv = 0;
  int bk = kNoKey;
  for (int g = threadIdx.x; g < G; g += blockDim.x)
    if (key_better(cand_v[g], cand_k[g], bv, bk)) {
      bv = cand_v[g];
      bk = cand_k[g];
    }
  warp_argmax(bv, bk);
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    sk[threadIdx.x >> 5] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 1; w < nw; ++w)
      if (key_better(sv[w], sk[w], bv, bk)) {
        bv = sv[w];
        bk = sk[w];
      }
    int rp = k, cp = k;
    if (mode == GJ_PIVOT_PARTIAL) rp = bk;
    else if (mode == GJ_PIVOT_FULL) {
      cp = bk / n;
      rp = bk - cp * n;
    }
    int st = GJ_OK;
    if (bk == kNoKey) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
    else if (bv >= kInfBits) st = GJ_NONFINITE;
    else if (__longlong_as_double((long long)bv) <= tau) st = (mode == GJ_PIVOT_NONE) ? GJ_ZERO_PIVOT : GJ_SINGULAR;
    if (st != GJ_OK) {
      *status = st;
      *fail_step = k;
      s_ok = 0;
    } else {
      const int ra = rowat[k], rb = rowat[rp];
      rowat[k] = rb;
      rowat[rp] = ra;
      posrow[rb] = k;
      posrow[ra] = rp;
      const int ca = colat[k], cb = colat[cp];
      colat[k] = cb;
      colat[cp] = ca;
      poscol[cb] = k;
      poscol[ca] = cp;
      const double q = W[(int64_t)rb + (int64_t)cb * n];
      pivots[k] = q;
      piv_rows[k] = rp;
      piv_cols[k] = cp;
      s_ok = 1;
      s_R = rb;
      s_C = cb;
      s_inv = 1.0 / q;
      ss->R = rb;
      ss->C = cb;
      ss->inv_q = s_inv;
    }
  }
  __syncthreads();
  if (!s_ok) return;
  const int R = s_R, C = s_C;
  const double inv_q = s_inv;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) {
    prow[j] = (j == C) ? inv_q : W[(int64_t)R + (int64_t)j * n] * inv_q;
    if (j < n) lcol[j] = (j == R) ? 0.0 : W[(int64_t)j + (int64_t)C * n];
  }
}

__global__ void __launch_bounds__(256) rank1_kernel(int n, int nw, int k, double* __restrict__ W,
                                                    const double* __restrict__ prow, const double* __restrict__ lcol,
                                                    const StepState* ss, const int* __restrict__ posrow,
                                                    const int* __restrict__ poscol, uint64_t* cand_v, int* cand_k,
                                                    const int32_t* status, int mode) {
  if (*status != GJ_OK) return;
  const int R = ss->R, C = ss->C;
  const int kn = k + 1;
  const bool search = kn < n;
  uint64_t bv = 0;
  int bk = kNoKey;
  const int64_t total = (int64_t)n * nw;  // columns of A, then the right-hand sides
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    double nv;
    if (i == R) {
      nv = prow[j];
    } else {
      const double base = (j == C) ? 0.0 : W[e];
      nv = fma(-lcol[i], prow[j], base);
    }
    W[e] = nv;
    if (search && j < n) {
      const int pr = posrow[i];
      if (mode == GJ_PIVOT_PARTIAL) {
        if (j == kn && pr >= kn && key_better(abs_bits(nv), pr, bv, bk)) {
          bv = abs_bits(nv);
          bk = pr;
        }
      } else if (mode == GJ_PIVOT_FULL) {
        const int pc = poscol[j];
        if (pr >= kn && pc >= kn) {
          const int key = pc * n + pr;
          if (key_better(abs_bits(nv), key, bv, bk)) {
            bv = abs_bits(nv);
            bk = key;
          }
        }
      } else if (pr == kn && poscol[j] == kn) {
        bv = abs_bits(nv);
        bk = kn;
      }
    }
  }
  warp_argmax(bv, bk);
  __shared__ uint64_t sv[8];
  __shared__ int sk[8];
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = bv;
    sk[threadIdx.x >> 5] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w)
      if (key_better(sv[w], sk[w], bv, bk)) {
        bv = sv[w];
        bk = sk[w];
      }
    cand_v[blockIdx.x] = bv;
    cand_k[blockIdx.x] = bk;
  }
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <class T>
gj_status ws_alloc(T** p, size_t count, cudaStream_t s, void** list, int& nlist) {
  void* q = nullptr;
  cudaError_t e = lib_malloc_async(&q, sizeof(T) * (count > 0 ? count : 1), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GJ_ERR_NOMEM;
  }
  list[nlist++] = q;
  *p = static_cast<T*>(q);
  return GJ_OK;
}

// Second stream and the two events of the look-ahead schedule; destroyed at scope exit
// (destruction waits for nothing: the runtime releases them once pending work completes).
struct StreamEvents {
  cudaStream_t sb = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  ~StreamEvents() {
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
    if (sb) cudaStreamDestroy(sb);
  }
};

struct WsList {
  void* p[24];
  int n = 0;
  cudaStream_t s;
  explicit WsList(cudaStream_t st) : s(st) {}
  ~WsList() {
    for (int i = 0; i < n; ++i) cudaFreeAsync(p[i], s);
  }
};

#define GJ_WS(ptr, count)                                   \
  do {                                                      \
    gj_status st_ = ws_alloc(&(ptr), (count), s, ws.p, ws.n); \
    if (st_ != GJ_OK) return st_;                           \
  } while (0)

}  // namespace

namespace {
thread_local int t_panel_rows = 256;
}  // namespace

void set_thread_panel_rows(int rows) { t_panel_rows = rows >= 32 ? rows : 256; }

// Choose the cluster size and panel width for order n; returns the shared memory bytes.
static size_t choose_panel(int64_t n, int want_b, int* cs_out, int* b_out, int* rp_out) {
  // rp: rows per CTA, whole 32-row blocks dealt round robin; about t_panel_rows rows per
  // CTA, at most 16 CTAs
  int cs = (int)((n + t_panel_rows - 1) / t_panel_rows);
  if (cs < 1) cs = 1;
  if (cs > 16) cs = 16;
  const size_t limit = 220 * 1024;
  int b = want_b > 0 ? want_b : 32;
  if (b > kPanelMaxB) b = kPanelMaxB;
  for (;;) {
    const int64_t blocks = (n + kRowBlock - 1) / kRowBlock;
    const int rp = (int)((blocks + cs - 1) / cs) * kRowBlock;
    const size_t bytes = PanelSmem::bytes(cs, rp, b);
    if (bytes <= limit || b <= 4) {
      *cs_out = cs;
      *b_out = b;
      *rp_out = rp;
      return bytes;
    }
    b /= 2;
  }
}

gj_status run_blocked(int64_t n64, const double* A, int64_t lda, double* X, int pivot_mode, double tau, int panel,
                      int update, int slices, const CtaOut& out, cudaStream_t s, const Rhs* rhs, int lookahead,
                      int update_sms) {
  if (n64 > 46340) return GJ_ERR_UNSUPPORTED;
  const int n = (int)n64;
  const int64_t m = rhs ? rhs->m : 0;
  if (n + m > 0x3fffffff) return GJ_ERR_UNSUPPORTED;
  const int nw = (int)(n + m);  // columns of the working array: A, then the right-hand sides
  const bool solving = rhs != nullptr;
  int cs = 1, b = 32, rp = n;
  const size_t smem = choose_panel(n, panel, &cs, &b, &rp);
  // Outer panel width: the tensor-core update takes 128-column panels, reduced as
  // 128 / b cluster sub-panels with FP64 updates inside the panel; the FP64 update path
  // uses the cluster panel width directly.
  const bool tc = (update == 2) || (update == 0 && n >= kTensorUpdateMinN);
  const int S = slices > 0 ? slices : 7;  // 7 balanced 8-bit digits: FP64 level
  const int Bw = tc ? 128 : b;
  // look-ahead: the next outer panel is reduced on a second stream while the update of the
  // other columns runs (tensor-core path with at least two outer panels)
  const bool la = tc && n > Bw && (lookahead == 2 || (lookahead == 0 && n >= kLookaheadMinN));

  WsList ws(s);
  double *W, *Lbuf, *U, *pivots = out.pivots;
  int *posrow, *rowat, *prow_ids, *piv_rows = out.piv_rows;
  void* oz_ws = nullptr;
  int32_t* oz_err = nullptr;
  GJ_WS(W, (size_t)n * nw);
  GJ_WS(Lbuf, (size_t)n * b);
  GJ_WS(U, (size_t)nw * b);
  GJ_WS(posrow, (size_t)n);
  GJ_WS(rowat, (size_t)n);
  GJ_WS(prow_ids, (size_t)Bw * 2);  // two buffers: outer panels alternate (look-ahead)
  double* Mbuf;
  GJ_WS(Mbuf, (size_t)kPanelMaxB * kPanelMaxB);
  double* Ufix;  // V of the tensor-core path's product per sub-panel, bb x (outer panel width)
  GJ_WS(Ufix, (size_t)kPanelMaxB * 128);
  GJ_WS(oz_err, 4);
  void* oz_ws_b = nullptr;  // the second stream's updates (columns of one outer panel)
  if (tc) {
    uint8_t* p8;
    GJ_WS(p8, ozaki_workspace_bytes(n, nw, S));
    oz_ws = p8;
    if (la) {
      GJ_WS(p8, ozaki_workspace_bytes(n, Bw, S));
      oz_ws_b = p8;
    }
  }
  if (!pivots) GJ_WS(pivots, (size_t)n);
  if (!piv_rows) GJ_WS(piv_rows, (size_t)n);
  GJ_CUDA(cudaMemsetAsync(oz_err, 0, sizeof(int32_t), s));

  const int sms = num_sms();
  copy_in_kernel<<<sms * 8, 256, 0, s>>>(n, A, lda, W);
  GJ_CUDA(cudaGetLastError());
  if (m > 0) {
    copy_rhs_kernel<<<sms * 8, 256, 0, s>>>(n, m, rhs->B, rhs->ldb, W + (size_t)n * n);
    GJ_CUDA(cudaGetLastError());
  }
  init_positions_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, posrow, nullptr, nullptr, nullptr);
  GJ_CUDA(cudaGetLastError());
  if (out.piv_cols) {  // no column interchanges on this path: position k stays at k
    init_positions_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, out.piv_cols, nullptr, nullptr, nullptr);
    GJ_CUDA(cudaGetLastError());
  }

  GJ_CUDA(allow_max_dynamic_smem((const void*)panel_kernel));
  if (cs > 8) GJ_CUDA(cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  GJ_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, panel_kernel, &cfg));
  if (nclusters < 1) return GJ_ERR_UNSUPPORTED;

  auto fp64_update = [&](int k0, int bb, int c_lo, int c_hi, const int* pids) -> gj_status {
    const int wn = c_hi - c_lo;
    int64_t gblocks = ((int64_t)bb * wn + 255) / 256;
    if (gblocks > sms * 16) gblocks = sms * 16;
    gather_u_kernel<<<(unsigned)gblocks, 256, 0, s>>>(n, k0, bb, c_lo, c_hi, W, pids, U, out.status);
    GJ_CUDA(cudaGetLastError());
    dim3 grid((n + kTM - 1) / kTM, (wn + kTN - 1) / kTN);
    {
      // algorithmic work: n x (wn - bb) columns outside the sub-panel, 2 bb FLOP each;
      // bytes: those columns of W read and written once, L and U read once
      ProfScope ps(s, "update_dfma", 2.0 * n * (double)(wn - bb) * bb, 16.0 * n * (double)wn + 16.0 * n * bb);
      update_dfma_kernel<<<grid, 256, 0, s>>>(n, bb, c_lo, c_hi, Lbuf, U, W, posrow, k0, out.status);
    }
    GJ_CUDA(cudaGetLastError());
    prof_count(2);
    return GJ_OK;
  };

  // One outer panel [K0, K0 + BB): cluster sub-panels of width b, each followed by the
  // fix-up of the rows pivoted earlier and (tensor path) the update of the rest of the outer
  // panel.  pid receives the panel's pivot rows.  `after_first` runs once the first
  // sub-panel is enqueued.
  auto reduce_panel = [&](int K0, int BB, int* pid, cudaStream_t st_, void* ozw,
                          const std::function<gj_status()>& after_first) -> gj_status {
    for (int k0 = K0; k0 < K0 + BB; k0 += b) {
      const int bb = (K0 + BB - k0 < b) ? K0 + BB - k0 : b;
      {
        ProfScope ps(st_, "panel_cluster", 2.0 * n * bb * bb, 16.0 * n * bb);
        cfg.stream = st_;
        GJ_CUDA(cudaLaunchKernelEx(&cfg, panel_kernel, n, k0, bb, rp, K0, BB, W, posrow, Mbuf,
                                   tc ? Ufix : (double*)nullptr, pid + (k0 - K0), pivots, piv_rows, out.status,
                                   out.fail_step, pivot_mode, tau));
      }
      prof_count(1);
      if (k0 == K0 && after_first) {
        gj_status st = after_first();
        if (st != GJ_OK) return st;
      }
      if (tc) {
        // the outer panel [K0, K0 + BB): the product L V (V from the cluster, L the panel's
        // columns as they were at its start, the pivot row of step t replaced by -e_t) is
        // stored on the pivot rows and on the panel's columns and added elsewhere
        OzEpilogue pe;
        pe.row_pos = posrow;
        pe.unit_lo = pe.set_row_lo = k0;
        pe.unit_hi = pe.set_row_hi = k0 + bb;
        pe.set_col_lo = k0 - K0;
        pe.set_col_hi = k0 - K0 + bb;
        gj_status st = ozaki_update(n, BB, bb, W + (size_t)k0 * n, n, nullptr, Ufix, bb, nullptr, 0, 0,
                                    W + (size_t)K0 * n, n, S, ozw, oz_err, out.status, st_, 0, "update_ozaki_panel", pe);
        if (st != GJ_OK) return st;
      } else {
        // the rows that are not pivot rows of this sub-panel: L = -W[i, P] M^-1 (their panel
        // columns at the end of the sub-panel), then into W[i, P]; then the rest of the outer
        // panel by the FP64 update
        ProfScope ps(st_, "fixup_rows", 2.0 * (n - bb) * (double)bb * bb, 16.0 * (n - bb) * (double)bb);
        const unsigned st_blocks = (unsigned)std::min<int64_t>(((int64_t)n * bb + 255) / 256, sms * 8);
        const dim3 fx_grid((n + kFixRows - 1) / kFixRows, (bb + kFixCols - 1) / kFixCols);
        fixup_rows_kernel<<<fx_grid, 256, 0, st_>>>(n, k0, bb, W, posrow, Mbuf, Lbuf, out.status);
        GJ_CUDA(cudaGetLastError());
        fixup_store_kernel<<<st_blocks, 256, 0, st_>>>(n, k0, bb, W, posrow, Lbuf, out.status);
        GJ_CUDA(cudaGetLastError());
        prof_count(2);
        if (BB > bb) {
          gj_status st = fp64_update(k0, bb, K0, K0 + BB, pid + (k0 - K0));
          if (st != GJ_OK) return st;
        }
      }
    }
    return GJ_OK;
  };

  // The rank-BB update of outer panel [K0, K0 + BB) on the columns outside [K0, K0 + skip)
  // (inversion; skip >= BB) or right of K0 + skip (solving).
  auto outer_update = [&](int K0, int BB, int skip, const int* pid, cudaStream_t st_, int max_ctas) -> gj_status {
    // L = the outer panel's columns (final), U = its pivot rows: stored on the pivot rows
    // (M^-1 U: eq. 14 for the panel's rows), added on the others (eq. 15)
    OzEpilogue oe;
    oe.row_pos = posrow;
    oe.set_row_lo = K0;
    oe.set_row_hi = K0 + BB;
    if (!solving) {
      const int zhi = std::min(n, K0 + skip);
      if (K0 == 0 && zhi >= n) return GJ_OK;  // nothing outside
      if (tc)
        return ozaki_update(n, n, BB, W + (size_t)K0 * n, n, nullptr, W, n, pid, K0, zhi, W, n, S, oz_ws, oz_err,
                            out.status, st_, max_ctas, "update_ozaki_wide", oe);
      return fp64_update(K0, BB, 0, n, pid);
    }
    const int c0 = K0 + skip;
    if (c0 >= nw) return GJ_OK;
    if (tc)
      return ozaki_update(n, nw - c0, BB, W + (size_t)K0 * n, n, nullptr, W + (size_t)c0 * n, n, pid, 0, 0,
                          W + (size_t)c0 * n, n, S, oz_ws, oz_err, out.status, st_, max_ctas, "update_ozaki_wide", oe);
    return fp64_update(K0, BB, c0, nw, pid);
  };

  if (!la) {
    for (int K0 = 0; K0 < n; K0 += Bw) {
      const int BB = (n - K0 < Bw) ? n - K0 : Bw;
      gj_status st = reduce_panel(K0, BB, prow_ids, s, oz_ws, nullptr);
      if (st == GJ_OK) st = outer_update(K0, BB, BB, prow_ids, s, 0);
      if (st != GJ_OK) return st;
    }
  } else {
    // Stream sb reduces the panels and updates the next panel's columns (the narrow update);
    // stream s runs the update of all other columns on a capped persistent grid, so that the
    // cluster and sb's other kernels find free SMs.
    // Panel p + 1 is reduced while the wide update of panel p runs.  Events:
    //   ev_b (sb -> s): panel p reduced and panel p + 1's columns updated;
    //   ev_a (s -> sb): wide update of panel p done (panel p + 2's columns current).
    // The wide update is enqueued after the next panel's first cluster, and may not start
    // before the narrow update ends: a 16-CTA cluster needs 16 free SMs of one GPC, which the
    // wide update's persistent CTAs would otherwise scatter over every GPC for the length
    // of the launch.  (Letting the wide update start right after the panel's reduction, beside
    // the narrow update, measured 102.8 ms instead of 66.9: the clusters waited for SMs.)
    StreamEvents se;
    GJ_CUDA(cudaStreamCreateWithFlags(&se.sb, cudaStreamNonBlocking));
    GJ_CUDA(cudaEventCreateWithFlags(&se.ev_a, cudaEventDisableTiming));
    GJ_CUDA(cudaEventCreateWithFlags(&se.ev_b, cudaEventDisableTiming));
    cudaStream_t sb = se.sb;
    GJ_CUDA(cudaEventRecord(se.ev_a, s));  // set-up done
    GJ_CUDA(cudaStreamWaitEvent(sb, se.ev_a, 0));
    // SMs left to sb: the cluster's plus room for its narrow updates, three cluster sizes
    // (the wide update gets 104 of 152: best of 88-120 at n = 8192, 55.4 ms against 57.7 at
    // 96 and 56.2 at 112; the two streams then take about as long)
    const int wide_ctas = update_sms > 0 ? std::min(update_sms, sms) : std::max(1, sms - std::min(3 * cs, sms / 2));
    struct Pending {
      bool valid = false;
      int K0 = 0, BB = 0, skip = 0;
      const int* pid = nullptr;
    } pend;
    auto submit_wide = [&]() -> gj_status {
      if (!pend.valid) return GJ_OK;
      pend.valid = false;
      GJ_CUDA(cudaStreamWaitEvent(s, se.ev_b, 0));
      gj_status st = outer_update(pend.K0, pend.BB, pend.skip, pend.pid, s, wide_ctas);
      if (st != GJ_OK) return st;
      GJ_CUDA(cudaEventRecord(se.ev_a, s));
      return GJ_OK;
    };
    int p = 0;
    for (int K0 = 0; K0 < n; K0 += Bw, ++p) {
      const int BB = (n - K0 < Bw) ? n - K0 : Bw;
      int* pid = prow_ids + (size_t)(p & 1) * Bw;
      // the previous panel's wide update is enqueued once this panel's first cluster is
      gj_status st = reduce_panel(K0, BB, pid, sb, oz_ws_b, submit_wide);
      if (st != GJ_OK) return st;
      const int K1 = K0 + BB;
      const int BBn = (K1 < n) ? std::min(Bw, n - K1) : 0;
      if (BBn > 0) {
        // narrow update: panel p + 1's columns, after the wide update of panel p - 1
        if (p > 0) GJ_CUDA(cudaStreamWaitEvent(sb, se.ev_a, 0));
        OzEpilogue ne;
        ne.row_pos = posrow;
        ne.set_row_lo = K0;
        ne.set_row_hi = K0 + BB;
        st = ozaki_update(n, BBn, BB, W + (size_t)K0 * n, n, nullptr, W + (size_t)K1 * n, n, pid, 0, 0,
                          W + (size_t)K1 * n, n, S, oz_ws_b, oz_err, out.status, sb, 0, "update_ozaki_panel", ne);
        if (st != GJ_OK) return st;
      }
      GJ_CUDA(cudaEventRecord(se.ev_b, sb));
      pend.valid = true;
      pend.K0 = K0;
      pend.BB = BB;
      pend.skip = BB + BBn;
      pend.pid = pid;
    }
    gj_status st = submit_wide();  // the last panel's update; s then follows all of sb's work
    if (st != GJ_OK) return st;
    GJ_CUDA(cudaStreamWaitEvent(s, se.ev_b, 0));
  }
  fold_error_kernel<<<1, 1, 0, s>>>(oz_err, out.status);
  GJ_CUDA(cudaGetLastError());
  rowat_from_posrow_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, posrow, rowat, out.status);
  GJ_CUDA(cudaGetLastError());
  if (!solving)
    unpermute_kernel<<<sms * 8, 256, 0, s>>>(n, W, rowat, posrow, nullptr, nullptr, X, out.status);
  else if (m > 0)
    gather_solution_kernel<<<sms * 8, 256, 0, s>>>(n, m, W + (size_t)n * n, rowat, nullptr, rhs->X, rhs->ldx,
                                                   out.status);
  GJ_CUDA(cudaGetLastError());
  det_kernel<<<1, 1024, 0, s>>>(n, pivots, piv_rows, nullptr, out.status, out.det_sign, out.det_log2, out.fail_step);
  GJ_CUDA(cudaGetLastError());
  prof_count(6);
  return GJ_OK;
}

gj_status run_unblocked(int64_t n64, const double* A, int64_t lda, double* X, int pivot_mode, double tau,
                        const CtaOut& out, cudaStream_t s, const Rhs* rhs) {
  if (n64 > 46340) return GJ_ERR_UNSUPPORTED;
  const int n = (int)n64;
  const int64_t m = rhs ? rhs->m : 0;
  if (n + m > 0x3fffffff) return GJ_ERR_UNSUPPORTED;
  const int nw = (int)(n + m);
  const bool solving = rhs != nullptr;
  WsList ws(s);
  double *W, *prow, *lcol, *pivots = out.pivots;
  int *posrow, *poscol, *rowat, *colat, *piv_rows = out.piv_rows, *piv_cols = out.piv_cols, *cand_k;
  uint64_t* cand_v;
  StepState* ss;
  const int sms = num_sms();
  const int G = sms * 4;
  GJ_WS(W, (size_t)n * nw);
  GJ_WS(prow, (size_t)nw);
  GJ_WS(lcol, (size_t)n);
  GJ_WS(posrow, (size_t)n);
  GJ_WS(poscol, (size_t)n);
  GJ_WS(rowat, (size_t)n);
  GJ_WS(colat, (size_t)n);
  GJ_WS(cand_v, (size_t)G);
  GJ_WS(cand_k, (size_t)G);
  GJ_WS(ss, 1);
  if (!pivots) GJ_WS(pivots, (size_t)n);
  if (!piv_rows) GJ_WS(piv_rows, (size_t)n);
  if (!piv_cols) GJ_WS(piv_cols, (size_t)n);

  copy_in_kernel<<<sms * 8, 256, 0, s>>>(n, A, lda, W);
  GJ_CUDA(cudaGetLastError());
  if (m > 0) {
    copy_rhs_kernel<<<sms * 8, 256, 0, s>>>(n, m, rhs->B, rhs->ldb, W + (size_t)n * n);
    GJ_CUDA(cudaGetLastError());
  }
  init_positions_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, posrow, poscol, rowat, colat);
  GJ_CUDA(cudaGetLastError());
  scan0_kernel<<<G, 256, 0, s>>>(n, W, pivot_mode, cand_v, cand_k);
  GJ_CUDA(cudaGetLastError());
  prof_count(3 + 2 * n + 2);
  for (int k = 0; k < n; ++k) {
    decide_kernel<<<1, 1024, 0, s>>>(n, nw, k, G, cand_v, cand_k, W, rowat, colat, posrow, poscol, prow, lcol, ss,
                                     pivots, piv_rows, piv_cols, out.status, out.fail_step, pivot_mode, tau);
    rank1_kernel<<<G, 256, 0, s>>>(n, nw, k, W, prow, lcol, ss, posrow, poscol, cand_v, cand_k, out.status,
                                   pivot_mode);
  }
  GJ_CUDA(cudaGetLastError());
  if (!solving)
    unpermute_kernel<<<sms * 8, 256, 0, s>>>(n, W, rowat, posrow, colat, poscol, X, out.status);
  else if (m > 0)
    gather_solution_kernel<<<sms * 8, 256, 0, s>>>(n, m, W + (size_t)n * n, rowat, poscol, rhs->X, rhs->ldx,
                                                   out.status);
  GJ_CUDA(cudaGetLastError());
  det_kernel<<<1, 1024, 0, s>>>(n, pivots, piv_rows, piv_cols, out.status, out.det_sign, out.det_log2,
                                out.fail_step);
  GJ_CUDA(cudaGetLastError());
  return GJ_OK;
}

}  // namespace gj
