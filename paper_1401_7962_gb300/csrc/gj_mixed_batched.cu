// gj_mixed_batched.cu -- reduced-precision Gauss-Jordan plus Newton-Schulz refinement over a
// batch of FP32 matrices of different orders (not in the paper; the single-matrix variant of
// eqs. 14-15 is gj_invert_mixed).
//
// One matrix of order 128..1024 fills only part of the GPU: its panel steps are latency-bound
// and its tensor-core updates have few tiles.  The batch therefore runs on a pool of host
// workers, each with its own non-blocking CUDA stream and its own stream-ordered workspace
// (the library's memory pool), which take the matrices largest first from a shared counter.
// The kernels of several matrices then run side by side; the precision ladder of each matrix
// is decided by its worker from that matrix's residuals alone.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "gj_internal.cuh"
#include "gj_ozaki.cuh"
#include "gj_paths.cuh"

extern "C" gj_status gj_invert_mixed_batched(int64_t count, const int32_t* n, const int32_t* lda,
                                             const float* const* A, double* const* X, int x0_slices,
                                             int corr_slices, double tol, int max_iter, int workers,
                                             int32_t* status, double* resid, int32_t* iters, int32_t* rung,
                                             int8_t* det_sign, double* det_log2, void* stream) {
  using namespace gj;
  set_last_error("");
  if (count < 0 || workers < 0 || workers > 64 || x0_slices < 1 || x0_slices > 8 || corr_slices < 1 ||
      corr_slices > 8 || !(tol > 0.0) || max_iter < 0)
    return GJ_ERR_ARG;
  if (count == 0) return GJ_OK;
  if (!n || !lda || !A || !X) return GJ_ERR_ARG;
  for (int64_t m = 0; m < count; ++m) {
    if (n[m] < 0 || lda[m] < std::max(1, n[m]) || (n[m] > 0 && (!A[m] || !X[m]))) {
      set_last_error("gj_invert_mixed_batched: bad order, leading dimension or pointer");
      return GJ_ERR_ARG;
    }
    if (n[m] > 46340) return GJ_ERR_UNSUPPORTED;
  }
  // largest first (ties in matrix order), so the long matrices do not finish last
  std::vector<int64_t> order((size_t)count);
  std::iota(order.begin(), order.end(), (int64_t)0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return n[a] > n[b]; });

  int dev = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  // the batch is ordered after what the caller queued before the call
  GJ_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));

  std::vector<int32_t> st((size_t)count, (int32_t)GJ_ERR_CUDA);  // untouched matrices read as CUDA errors
  std::vector<double> rs((size_t)count, INFINITY), lg((size_t)count, -INFINITY);
  std::vector<int32_t> it((size_t)count, 0), rg((size_t)count, 0);
  std::vector<int8_t> sg((size_t)count, 0);
  std::atomic<int64_t> next{0};
  std::mutex mu;
  std::string first_error;

  const int nw = (int)std::min<int64_t>(count, workers > 0 ? workers : 16);
  int sms = 0;
  GJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // each worker's tensor-core updates take at most twice its share of the SMs, so that a
  // large update of one matrix does not hold the whole GPU while the other workers' panel
  // clusters wait for free SMs
  const int cap = std::max(8, (2 * sms) / nw);
  auto work = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) return;
    set_thread_update_cap(cap);
    set_thread_panel_rows(128);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= count) break;
      const int64_t m = order[(size_t)i];
      double r = INFINITY, l = -INFINITY;
      int k = 0, g = 0, sgn = 0;
      const gj_status sm = gj_invert_mixed(n[m], A[m], lda[m], X[m], x0_slices, corr_slices, tol, max_iter, &r, &k,
                                           &g, &sgn, &l, s);
      st[(size_t)m] = sm;
      rs[(size_t)m] = r;
      it[(size_t)m] = k;
      rg[(size_t)m] = g;
      sg[(size_t)m] = (int8_t)sgn;
      lg[(size_t)m] = l;
      if (sm < 0) {
        std::lock_guard<std::mutex> lk(mu);
        if (first_error.empty()) first_error = gj_last_error();
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    set_thread_update_cap(0);
    set_thread_panel_rows(256);
  };
  std::vector<std::thread> pool;
  pool.reserve((size_t)nw);
  for (int w = 0; w < nw; ++w) {
    try {
      pool.emplace_back(work);
    } catch (...) {  // no more threads: the ones started (or this one) take the rest
      break;
    }
  }
  if (pool.empty()) {
    work();
    cudaSetDevice(dev);
  }
  for (auto& t : pool) t.join();

  // the call's status: the first hard error (negative) in matrix order, else the first
  // positive status (singular, not converged, ...), else GJ_OK
  gj_status result = GJ_OK;
  for (int64_t m = 0; m < count; ++m)
    if (st[(size_t)m] < 0) {
      result = (gj_status)st[(size_t)m];
      break;
    }
  if (result == GJ_OK)
    for (int64_t m = 0; m < count; ++m)
      if (st[(size_t)m] != GJ_OK) {
        result = (gj_status)st[(size_t)m];
        break;
      }
  if (result < 0) set_last_error(first_error.empty() ? "gj_invert_mixed_batched: a worker could not start"
                                                     : first_error.c_str());
  for (int64_t m = 0; m < count; ++m) {
    if (status) status[m] = st[(size_t)m];
    if (resid) resid[m] = rs[(size_t)m];
    if (iters) iters[m] = it[(size_t)m];
    if (rung) rung[m] = rg[(size_t)m];
    if (det_sign) det_sign[m] = sg[(size_t)m];
    if (det_log2) det_log2[m] = lg[(size_t)m];
  }
  return result;
}
