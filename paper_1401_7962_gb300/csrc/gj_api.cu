// gj_api.cu -- the C ABI: argument checks, host/device staging, path selection.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "gj_internal.cuh"
#include "gj_paths.cuh"

namespace gj {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pools[dev], &props);
      if (e != cudaSuccess) {
        g_pools[dev] = nullptr;
        return e;
      }
      uint64_t keep = ~0ull;  // keep freed memory for the next call
      cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

namespace {
std::mutex g_smem_mu;
std::vector<std::pair<const void*, int>> g_smem_done;  // (kernel, device) pairs already raised
}  // namespace

cudaError_t allow_max_dynamic_smem(const void* func) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  for (const auto& d : g_smem_done)
    if (d.first == func && d.second == dev) return cudaSuccess;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) g_smem_done.emplace_back(func, dev);
  return e;
}

gj_status cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return GJ_ERR_CUDA;
}

namespace {

// True when p is memory the device can address directly as global memory.
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stream-ordered scratch allocations released in stream order when the scope ends.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : s_(s) {}
  ~Scratch() {
    for (void* p : ptrs_) cudaFreeAsync(p, s_);
  }
  template <class T>
  gj_status alloc(T** out, size_t count) {
    void* p = nullptr;
    size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = lib_malloc_async(&p, bytes, s_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      snprintf(g_last_error, sizeof(g_last_error), "cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
      return GJ_ERR_NOMEM;
    }
    ptrs_.push_back(p);
    *out = static_cast<T*>(p);
    return GJ_OK;
  }

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
};

#define GJ_TRY(expr)                   \
  do {                                 \
    gj_status st_ = (expr);            \
    if (st_ != GJ_OK) return st_;      \
  } while (0)

struct ResultBlock {
  int32_t status;
  int8_t det_sign;
  int8_t pad[3];
  double det_log2;
  int64_t fail_step;
};

}  // namespace

// Full single-matrix pipeline on device pointers.  Writes status / det / fail step to
// the device result block `res`.
static gj_status run_single_device(const gj_opts& o, int64_t n, const double* dA, int64_t lda, double* dX,
                                   int pivot_mode, int32_t* d_piv_rows, int32_t* d_piv_cols, double* d_pivots,
                                   ResultBlock* res, cudaStream_t s) {
  int path = o.path;
  if (path == 0) {
    if (n <= kCtaMaxN) path = (n >= 64) ? 4 : 1;  // a cluster beats one SM's FP64 units from n = 64
    else if (pivot_mode == GJ_PIVOT_FULL) path = 3;
    else path = 2;
  }
  CtaOut out{};
  out.status = &res->status;
  out.det_sign = &res->det_sign;
  out.det_log2 = &res->det_log2;
  out.fail_step = &res->fail_step;
  out.piv_rows = d_piv_rows;
  out.piv_cols = d_piv_cols;
  out.pivots = d_pivots;
  switch (path) {
    case 1:
      if (n > kCtaMaxN) return GJ_ERR_UNSUPPORTED;
      return launch_cta_single((int)n, dA, lda, dX, pivot_mode, o.tau, out, s);
    case 2:
      if (pivot_mode == GJ_PIVOT_FULL) return GJ_ERR_UNSUPPORTED;
      return run_blocked(n, dA, lda, dX, pivot_mode, o.tau, o.panel, o.update, o.slices, out, s, nullptr,
                         o.lookahead, o.update_sms);
    case 3:
      return run_unblocked(n, dA, lda, dX, pivot_mode, o.tau, out, s);
    case 4:
      if (n > kCtaMaxN) return GJ_ERR_UNSUPPORTED;
      return launch_cluster_single((int)n, dA, lda, dX, pivot_mode, o.tau, out, s);
    default:
      return GJ_ERR_ARG;
  }
}

}  // namespace gj

using namespace gj;

extern "C" {

const char* gj_version(void) { return "gj-gb300 0.1 (sm_103a)"; }

gj_status gj_trim_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < kMaxDevices; ++d)
    if (g_pools[d]) {
      cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolTrimTo");
    }
  return GJ_OK;
}

const char* gj_last_error(void) { return g_last_error; }

const char* gj_status_string(int status) {
  switch (status) {
    case GJ_OK: return "ok";
    case GJ_SINGULAR: return "singular: every pivot candidate of a step was zero (or <= tau)";
    case GJ_ZERO_PIVOT: return "zero pivot without pivoting";
    case GJ_NONFINITE: return "non-finite pivot candidate";
    case GJ_NOT_CONVERGED: return "refinement did not converge";
    case GJ_ERR_ARG: return "invalid argument";
    case GJ_ERR_CUDA: return "CUDA error";
    case GJ_ERR_NOMEM: return "out of device memory";
    case GJ_ERR_TIMEOUT: return "device-side wait timed out";
    case GJ_ERR_UNSUPPORTED: return "unsupported size / option combination";
    default: return "unknown status";
  }
}

gj_status gj_invert_ex(const gj_opts* opts, int64_t n, const double* A, int64_t lda, double* Ainv, int pivot_mode,
                       int* det_sign, double* det_log2) {
  gj_opts o{};
  if (opts) o = *opts;
  g_last_error[0] = '\0';
  if (det_sign) *det_sign = 0;
  if (det_log2) *det_log2 = -INFINITY;
  if (o.fail_step) *o.fail_step = -1;
  if (n < 0 || lda < (n > 0 ? n : 1)) return GJ_ERR_ARG;
  if (pivot_mode < GJ_PIVOT_NONE || pivot_mode > GJ_PIVOT_FULL) return GJ_ERR_ARG;
  if (!(o.tau >= 0.0)) return GJ_ERR_ARG;
  if (o.path < 0 || o.path > 4 || o.update < 0 || o.update > 2 || o.slices < 0 || o.slices > 8) return GJ_ERR_ARG;
  if (o.lookahead < 0 || o.lookahead > 2 || o.update_sms < 0) return GJ_ERR_ARG;
  if (o.panel != 0 && o.panel != 16 && o.panel != 32 && o.panel != 64 && o.panel != 128) return GJ_ERR_ARG;
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    if (det_log2) *det_log2 = 0.0;
    return GJ_OK;
  }
  if (!A || !Ainv) return GJ_ERR_ARG;
  if ((const void*)A == (const void*)Ainv && lda != n) return GJ_ERR_ARG;
  if (n > 2000000000LL / (n > 0 ? n : 1) && n > 46340) return GJ_ERR_UNSUPPORTED;

  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  gj_status result;
  {
    Scratch scr(s);
    const bool a_dev = is_device_ptr(A), x_dev = is_device_ptr(Ainv);
    const double* dA = A;
    double* dX = Ainv;
    int64_t dlda = lda;
    const size_t nn = (size_t)n * (size_t)n;
    if (!x_dev) GJ_TRY(scr.alloc(&dX, nn));
    if (!a_dev) {
      if ((const void*)A == (const void*)Ainv) {
        dA = dX;
      } else {
        double* t;
        GJ_TRY(scr.alloc(&t, (size_t)lda * (size_t)n));
        dA = t;
      }
      GJ_CUDA(cudaMemcpyAsync((void*)dA, A, sizeof(double) * ((size_t)lda * (size_t)(n - 1) + (size_t)n),
                              cudaMemcpyHostToDevice, s));
    }
    int32_t* d_pr = nullptr;
    int32_t* d_pc = nullptr;
    double* d_pv = nullptr;
    const bool pr_dev = is_device_ptr(o.piv_rows), pc_dev = is_device_ptr(o.piv_cols),
               pv_dev = is_device_ptr(o.pivots);
    if (o.piv_rows) {
      if (pr_dev) d_pr = o.piv_rows;
      else GJ_TRY(scr.alloc(&d_pr, (size_t)n));
    }
    if (o.piv_cols) {
      if (pc_dev) d_pc = o.piv_cols;
      else GJ_TRY(scr.alloc(&d_pc, (size_t)n));
    }
    if (o.pivots) {
      if (pv_dev) d_pv = o.pivots;
      else GJ_TRY(scr.alloc(&d_pv, (size_t)n));
    }
    ResultBlock* d_res;
    GJ_TRY(scr.alloc(&d_res, 1));
    GJ_CUDA(cudaMemsetAsync(d_res, 0, sizeof(ResultBlock), s));

    GJ_TRY(run_single_device(o, n, dA, dlda, dX, pivot_mode, d_pr, d_pc, d_pv, d_res, s));

    ResultBlock h{};
    GJ_CUDA(cudaMemcpyAsync(&h, d_res, sizeof(ResultBlock), cudaMemcpyDeviceToHost, s));
    if (!x_dev) GJ_CUDA(cudaMemcpyAsync(Ainv, dX, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
    if (o.piv_rows && !pr_dev) GJ_CUDA(cudaMemcpyAsync(o.piv_rows, d_pr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    if (o.piv_cols && !pc_dev) GJ_CUDA(cudaMemcpyAsync(o.piv_cols, d_pc, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    if (o.pivots && !pv_dev) GJ_CUDA(cudaMemcpyAsync(o.pivots, d_pv, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    GJ_CUDA(cudaStreamSynchronize(s));
    result = (gj_status)h.status;
    if (result == GJ_OK) {
      if (det_sign) *det_sign = h.det_sign;
      if (det_log2) *det_log2 = h.det_log2;
    }
    if (o.fail_step) *o.fail_step = h.fail_step;
  }
  GJ_CUDA(cudaStreamSynchronize(s));  // scratch frees are stream-ordered
  return result;
}

gj_status gj_invert(int64_t n, const double* A, int64_t lda, double* Ainv, int pivot_mode, int* det_sign,
                    double* det_log2) {
  return gj_invert_ex(nullptr, n, A, lda, Ainv, pivot_mode, det_sign, det_log2);
}

gj_status gj_solve_ex(const gj_opts* opts, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B,
                      int64_t ldb, double* X, int64_t ldx, int pivot_mode, int* det_sign, double* det_log2) {
  gj_opts o{};
  if (opts) o = *opts;
  g_last_error[0] = '\0';
  if (det_sign) *det_sign = 0;
  if (det_log2) *det_log2 = -INFINITY;
  if (o.fail_step) *o.fail_step = -1;
  const int64_t ld_min = n > 0 ? n : 1;
  if (n < 0 || nrhs < 0 || lda < ld_min || ldb < ld_min || ldx < ld_min) return GJ_ERR_ARG;
  if (pivot_mode < GJ_PIVOT_NONE || pivot_mode > GJ_PIVOT_FULL) return GJ_ERR_ARG;
  if (!(o.tau >= 0.0)) return GJ_ERR_ARG;
  if (o.path < 0 || o.path > 3 || o.path == 1 || o.update < 0 || o.update > 2 || o.slices < 0 || o.slices > 8 ||
      o.lookahead < 0 || o.lookahead > 2 || o.update_sms < 0)
    return GJ_ERR_ARG;
  if (o.panel != 0 && o.panel != 16 && o.panel != 32 && o.panel != 64 && o.panel != 128) return GJ_ERR_ARG;
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    if (det_log2) *det_log2 = 0.0;
    return GJ_OK;
  }
  if (!A || (nrhs > 0 && (!B || !X))) return GJ_ERR_ARG;
  if (nrhs > 0 && (const void*)X == (const void*)B && ldx != ldb) return GJ_ERR_ARG;
  if (n > 46340 || n + nrhs > 0x3fffffff) return GJ_ERR_UNSUPPORTED;
  int path = o.path;
  if (path == 0) path = (pivot_mode == GJ_PIVOT_FULL) ? 3 : 2;
  if (path == 2 && pivot_mode == GJ_PIVOT_FULL) return GJ_ERR_UNSUPPORTED;

  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  gj_status result;
  {
    Scratch scr(s);
    const double* dA = A;
    const double* dB = B;
    double* dX = X;
    int64_t dlda = lda, dldb = ldb, dldx = ldx;
    const bool x_dev = nrhs == 0 || is_device_ptr(X);
    if (!is_device_ptr(A)) {
      double* t;
      GJ_TRY(scr.alloc(&t, (size_t)n * (size_t)n));
      GJ_CUDA(cudaMemcpy2DAsync(t, sizeof(double) * n, A, sizeof(double) * lda, sizeof(double) * n, n,
                                cudaMemcpyHostToDevice, s));
      dA = t;
      dlda = n;
    }
    if (nrhs > 0 && !is_device_ptr(B)) {
      double* t;
      GJ_TRY(scr.alloc(&t, (size_t)n * (size_t)nrhs));
      GJ_CUDA(cudaMemcpy2DAsync(t, sizeof(double) * n, B, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                                cudaMemcpyHostToDevice, s));
      dB = t;
      dldb = n;
    }
    if (!x_dev) {
      GJ_TRY(scr.alloc(&dX, (size_t)n * (size_t)nrhs));
      dldx = n;
    }
    int32_t* d_pr = nullptr;
    int32_t* d_pc = nullptr;
    double* d_pv = nullptr;
    const bool pr_dev = is_device_ptr(o.piv_rows), pc_dev = is_device_ptr(o.piv_cols),
               pv_dev = is_device_ptr(o.pivots);
    if (o.piv_rows) {
      if (pr_dev) d_pr = o.piv_rows;
      else GJ_TRY(scr.alloc(&d_pr, (size_t)n));
    }
    if (o.piv_cols) {
      if (pc_dev) d_pc = o.piv_cols;
      else GJ_TRY(scr.alloc(&d_pc, (size_t)n));
    }
    if (o.pivots) {
      if (pv_dev) d_pv = o.pivots;
      else GJ_TRY(scr.alloc(&d_pv, (size_t)n));
    }
    ResultBlock* d_res;
    GJ_TRY(scr.alloc(&d_res, 1));
    GJ_CUDA(cudaMemsetAsync(d_res, 0, sizeof(ResultBlock), s));
    CtaOut out{};
    out.status = &d_res->status;
    out.det_sign = &d_res->det_sign;
    out.det_log2 = &d_res->det_log2;
    out.fail_step = &d_res->fail_step;
    out.piv_rows = d_pr;
    out.piv_cols = d_pc;
    out.pivots = d_pv;
    Rhs rhs;
    rhs.m = nrhs;
    rhs.B = dB;
    rhs.ldb = dldb;
    rhs.X = dX;
    rhs.ldx = dldx;
    if (path == 2)
      GJ_TRY(run_blocked(n, dA, dlda, nullptr, pivot_mode, o.tau, o.panel, o.update, o.slices, out, s, &rhs,
                         o.lookahead, o.update_sms));
    else
      GJ_TRY(run_unblocked(n, dA, dlda, nullptr, pivot_mode, o.tau, out, s, &rhs));

    ResultBlock h{};
    GJ_CUDA(cudaMemcpyAsync(&h, d_res, sizeof(ResultBlock), cudaMemcpyDeviceToHost, s));
    if (!x_dev)
      GJ_CUDA(cudaMemcpy2DAsync(X, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n, nrhs,
                                cudaMemcpyDeviceToHost, s));
    if (o.piv_rows && !pr_dev) GJ_CUDA(cudaMemcpyAsync(o.piv_rows, d_pr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    if (o.piv_cols && !pc_dev) GJ_CUDA(cudaMemcpyAsync(o.piv_cols, d_pc, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    if (o.pivots && !pv_dev) GJ_CUDA(cudaMemcpyAsync(o.pivots, d_pv, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    GJ_CUDA(cudaStreamSynchronize(s));
    result = (gj_status)h.status;
    if (result == GJ_OK) {
      if (det_sign) *det_sign = h.det_sign;
      if (det_log2) *det_log2 = h.det_log2;
    }
    if (o.fail_step) *o.fail_step = h.fail_step;
  }
  GJ_CUDA(cudaStreamSynchronize(s));  // scratch frees are stream-ordered
  return result;
}

gj_status gj_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B, int64_t ldb, double* X,
                   int64_t ldx, int pivot_mode, int* det_sign, double* det_log2) {
  return gj_solve_ex(nullptr, n, nrhs, A, lda, B, ldb, X, ldx, pivot_mode, det_sign, det_log2);
}

gj_status gj_invert_batched(int64_t count, int32_t nmax, const int32_t* n, const double* const* A,
                            double* const* Ainv, int pivot_mode, int32_t* status, int8_t* det_sign,
                            double* det_log2, void* stream) {
  g_last_error[0] = '\0';
  if (count < 0 || count > 0x7fffffffLL) return GJ_ERR_ARG;
  if (pivot_mode < GJ_PIVOT_NONE || pivot_mode > GJ_PIVOT_FULL) return GJ_ERR_ARG;
  if (nmax <= 0) nmax = kCtaMaxN;
  if (nmax > kCtaMaxN) return GJ_ERR_UNSUPPORTED;
  if (count == 0) return GJ_OK;
  if (!n || !A || !Ainv || !status) return GJ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch scr(s);
  int32_t* ws;
  GJ_TRY(scr.alloc(&ws, (size_t)count + kCtaMaxN + 3));
  int32_t* order = ws;
  int32_t* hist = ws + count;
  int32_t* counter = hist + kCtaMaxN + 1;
  GJ_TRY(launch_order_by_size(count, n, order, hist, counter, s));
  CtaOut out{};
  out.status = status;
  out.det_sign = det_sign;
  out.det_log2 = det_log2;
  return launch_cta_batched(count, nmax, n, A, Ainv, order, counter, pivot_mode, 0.0, out, s);
}

}  // extern "C"

// ------------------------------------------------------------------ batched plans
//
// A plan fixes the orders of a batch.  It sorts the work largest order first, splits it
// into order bins, and picks for every bin the kernel variant (one warp per matrix, or one
// CTA of 64 / 128 / 256 / 512 threads per matrix) that runs fastest on this GPU: the
// autotuner times each applicable variant on synthetic matrices of the bin's orders and
// keeps the best, remembering the choice per device, pivot mode and bin (in memory, and
// in an optional text cache file).  Executing the plan launches one persistent kernel per
// bin; with use_graph the launches are captured once and replayed as a CUDA graph.

namespace gj {
namespace {

constexpr int kBinEdges[] = {0, 8, 16, 24, 32, 48, 64, 96, 128};  // bin b holds orders (edge[b], edge[b+1]]
constexpr int kNumBins = 8;

struct PlanBin {
  int lo = 0, hi = 0;             // orders lo..hi (inclusive)
  int64_t q_begin = 0, q_end = 0;  // range of the work order
  int nmax = 0;                    // largest order present
  int variant = kVarCta128;
  float tuned_us = -1.0f;          // time of the chosen variant on the tuning sample
};

std::mutex g_tune_mu;
std::map<std::tuple<std::string, int, int, int>, std::pair<int, float>> g_tune_memo;

std::string device_tag() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "_sm" + std::to_string(prop.multiProcessorCount);
}

// Diagonally dominant test matrices for timing (values from a hash of the index).
__global__ void tune_fill_kernel(int64_t count, const int32_t* __restrict__ nv, const int64_t* __restrict__ off,
                                 double* __restrict__ data) {
  for (int64_t m = blockIdx.x; m < count; m += gridDim.x) {
    const int n = nv[m];
    double* A = data + off[m];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int j = e / n, i = e - j * n;
      uint32_t h = (uint32_t)(m * 2654435761u) ^ (uint32_t)(e * 40503u + 12345u);
      h ^= h >> 13;
      h *= 0x5bd1e995u;
      h ^= h >> 15;
      const double v = ((double)(h & 0xffffff) / 16777216.0) * 2.0 - 1.0;
      A[e] = (i == j) ? (double)n + 1.0 + v : v;
    }
  }
}

__global__ void tune_ptrs_kernel(int64_t count, const int64_t* __restrict__ off, double* base_a, double* base_x,
                                 const double** pa, double** px) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < count; m += (int64_t)gridDim.x * blockDim.x) {
    pa[m] = base_a + off[m];
    px[m] = base_x + off[m];
  }
}

bool read_tune_cache(const char* path, const std::string& tag, int mode, int lo, int hi, int* variant) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char t[256];
    int md, l, h, v;
    if (sscanf(line, "gj-tune-v1 %255s %d %d %d %d", t, &md, &l, &h, &v) == 5 && tag == t && md == mode &&
        l == lo && h == hi && v >= 0 && v < kNumVariants) {
      *variant = v;  // the last matching line wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void append_tune_cache(const char* path, const std::string& tag, int mode, int lo, int hi, int variant, float us) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "gj-tune-v1 %s %d %d %d %d %.3f\n", tag.c_str(), mode, lo, hi, variant, us);
  fclose(f);
}

// Time every applicable variant on up to 2048 matrices spread over the bin's orders.
gj_status autotune_bin(const std::vector<int32_t>& sorted_n, PlanBin& b, int mode, int* best, float* best_us) {
  const int64_t cnt = b.q_end - b.q_begin;
  const int64_t sample = std::min<int64_t>(cnt, 2048);
  std::vector<int32_t> ns((size_t)sample);
  std::vector<int64_t> off((size_t)sample);
  int64_t total = 0;
  for (int64_t t = 0; t < sample; ++t) {
    ns[t] = sorted_n[(size_t)(b.q_begin + (t * cnt) / sample)];
    off[t] = total;
    total += (int64_t)ns[t] * ns[t];
  }
  int32_t *d_n = nullptr, *d_status = nullptr, *d_counter = nullptr;
  int64_t* d_off = nullptr;
  double *d_a = nullptr, *d_x = nullptr;
  const double** d_pa = nullptr;
  double** d_px = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gj_status st = GJ_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    st = cuda_fail(e, what);
    return st;
  };
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&d_n, sizeof(int32_t) * sample)) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_status, sizeof(int32_t) * sample)) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_counter, sizeof(int32_t))) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_off, sizeof(int64_t) * sample)) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_a, sizeof(double) * std::max<int64_t>(total, 1))) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_x, sizeof(double) * std::max<int64_t>(total, 1))) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_pa, sizeof(double*) * sample)) != cudaSuccess) { fail(e, "autotune"); break; }
    if ((e = cudaMalloc(&d_px, sizeof(double*) * sample)) != cudaSuccess) { fail(e, "autotune"); break; }
    cudaMemcpy(d_n, ns.data(), sizeof(int32_t) * sample, cudaMemcpyHostToDevice);
    cudaMemcpy(d_off, off.data(), sizeof(int64_t) * sample, cudaMemcpyHostToDevice);
    tune_fill_kernel<<<256, 256>>>(sample, d_n, d_off, d_a);
    tune_ptrs_kernel<<<64, 256>>>(sample, d_off, d_a, d_x, d_pa, d_px);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "autotune"); break; }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    CtaOut out{};
    out.status = d_status;
    *best = -1;
    *best_us = 0.0f;
    for (int v = 0; v < kNumVariants && st == GJ_OK; ++v) {
      if (!batched_variant_applies(v, b.nmax, mode)) continue;
      float t_min = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {  // first run warms up
        cudaMemsetAsync(d_counter, 0, sizeof(int32_t), 0);
        cudaEventRecord(e0, 0);
        gj_status ls = launch_batched_variant(v, 0, sample, b.nmax, d_n, d_pa, d_px, nullptr, d_counter, mode, 0.0,
                                              out, 0);
        cudaEventRecord(e1, 0);
        if (ls != GJ_OK) { st = ls; break; }
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { fail(e, "autotune"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t_min = std::min(t_min, ms * 1000.0f);
      }
      if (st == GJ_OK && (*best < 0 || t_min < *best_us)) {
        *best = v;
        *best_us = t_min;
      }
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  void* ps[] = {d_n, d_status, d_counter, d_off, d_a, d_x, (void*)d_pa, (void*)d_px};
  for (void* q : ps)
    if (q) cudaFree(q);
  return st;
}

}  // namespace
}  // namespace gj

struct gj_plan {
  int64_t count = 0;
  double flops = 0.0;  // sum of 2 n^3 (algorithmic work of one execution)
  double bytes = 0.0;  // 16 sum n^2 (inputs read, inverses written)
  int nmax = 0;
  int pivot_mode = 1;
  int32_t* d_n = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_counter = nullptr;  // one counter per bin
  std::vector<PlanBin> bins;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

static gj_status plan_enqueue(gj_plan* p, const double* const* A, double* const* Ainv, int32_t* status,
                              int8_t* det_sign, double* det_log2, cudaStream_t s) {
  GJ_CUDA(cudaMemsetAsync(p->d_counter, 0, sizeof(int32_t) * kNumBins, s));
  CtaOut out{};
  out.status = status;
  out.det_sign = det_sign;
  out.det_log2 = det_log2;
  for (size_t b = 0; b < p->bins.size(); ++b) {
    const PlanBin& pb = p->bins[b];
    GJ_TRY(launch_batched_variant(pb.variant, pb.q_begin, pb.q_end, pb.nmax, p->d_n, A, Ainv, p->d_order,
                                  p->d_counter + b, p->pivot_mode, 0.0, out, s));
  }
  return GJ_OK;
}

extern "C" {

gj_status gj_batched_plan_create_ex(gj_plan** plan, int64_t count, const int32_t* n_host, int pivot_mode,
                                    const char* tune_cache, int32_t variant) {
  g_last_error[0] = '\0';
  if (!plan) return GJ_ERR_ARG;
  *plan = nullptr;
  if (count < 0 || count > 0x7fffffffLL || (count > 0 && !n_host)) return GJ_ERR_ARG;
  if (pivot_mode < GJ_PIVOT_NONE || pivot_mode > GJ_PIVOT_FULL) return GJ_ERR_ARG;
  if (variant >= kNumVariants) return GJ_ERR_ARG;
  int nmax = 1;
  for (int64_t m = 0; m < count; ++m) {
    if (n_host[m] < 0 || n_host[m] > kCtaMaxN) return GJ_ERR_UNSUPPORTED;
    nmax = std::max(nmax, (int)n_host[m]);
  }
  gj_plan* p = new gj_plan();
  p->count = count;
  p->nmax = nmax;
  p->pivot_mode = pivot_mode;
  // largest order first (longest-processing-time order for the persistent queues)
  std::vector<int32_t> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return n_host[a] > n_host[b]; });
  std::vector<int32_t> sorted_n((size_t)count);
  for (int64_t q = 0; q < count; ++q) sorted_n[q] = n_host[order[q]];
  for (int64_t m = 0; m < count; ++m) {
    const double nm = (double)n_host[m];
    p->flops += 2.0 * nm * nm * nm;
    p->bytes += 16.0 * nm * nm;
  }
  // order bins: contiguous ranges of the descending work order
  for (int b = kNumBins - 1; b >= 0; --b) {
    PlanBin pb;
    pb.lo = (b == 0) ? 0 : kBinEdges[b] + 1;
    pb.hi = kBinEdges[b + 1];
    const auto first = std::lower_bound(sorted_n.begin(), sorted_n.end(), pb.hi, std::greater<int32_t>());
    const auto last = std::upper_bound(sorted_n.begin(), sorted_n.end(), pb.lo, std::greater<int32_t>());
    pb.q_begin = first - sorted_n.begin();
    pb.q_end = last - sorted_n.begin();
    if (pb.q_end <= pb.q_begin) continue;
    pb.nmax = std::max(1, (int)sorted_n[pb.q_begin]);
    p->bins.push_back(pb);
  }
  cudaError_t e = cudaMalloc(&p->d_n, sizeof(int32_t) * (count > 0 ? count : 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_order, sizeof(int32_t) * (count > 0 ? count : 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, sizeof(int32_t) * kNumBins);
  if (e == cudaSuccess && count > 0) e = cudaMemcpy(p->d_n, n_host, sizeof(int32_t) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && count > 0)
    e = cudaMemcpy(p->d_order, order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    gj_batched_plan_destroy(p);
    return cuda_fail(e, "gj_batched_plan_create");
  }
  // kernel variant per bin: forced, cached, or measured
  const std::string tag = device_tag();
  for (PlanBin& pb : p->bins) {
    const int fallback = (pb.nmax > 64) ? kVarCta256 : kVarCta128;
    if (variant >= 0) {
      pb.variant = batched_variant_applies(variant, pb.nmax, pivot_mode) ? variant : fallback;
      continue;
    }
    const auto key = std::make_tuple(tag, pivot_mode, pb.lo, pb.hi);
    int v = -1;
    // the caller's cache file first, then this process's earlier measurements
    if (read_tune_cache(tune_cache, tag, pivot_mode, pb.lo, pb.hi, &v) &&
        batched_variant_applies(v, pb.nmax, pivot_mode)) {
      pb.variant = v;
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_memo.find(key);
      if (it != g_tune_memo.end() && batched_variant_applies(it->second.first, pb.nmax, pivot_mode)) {
        pb.variant = it->second.first;
        continue;
      }
    }
    float us = 0.0f;
    gj_status st = autotune_bin(sorted_n, pb, pivot_mode, &v, &us);
    if (st != GJ_OK || v < 0) {
      gj_batched_plan_destroy(p);
      return st != GJ_OK ? st : GJ_ERR_UNSUPPORTED;
    }
    pb.variant = v;
    pb.tuned_us = us;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_memo[key] = {v, us};
    }
    append_tune_cache(tune_cache, tag, pivot_mode, pb.lo, pb.hi, v, us);
  }
  *plan = p;
  return GJ_OK;
}

gj_status gj_batched_plan_create(gj_plan** plan, int64_t count, const int32_t* n_host, int pivot_mode) {
  return gj_batched_plan_create_ex(plan, count, n_host, pivot_mode, nullptr, -1);
}

int32_t gj_batched_plan_bins(const gj_plan* p, int32_t* lo, int32_t* hi, int64_t* count, int32_t* variant,
                             float* tuned_us, int32_t max_bins) {
  if (!p) return 0;
  const int32_t nb = (int32_t)p->bins.size();
  for (int32_t b = 0; b < nb && b < max_bins; ++b) {
    const PlanBin& pb = p->bins[b];
    if (lo) lo[b] = pb.lo;
    if (hi) hi[b] = pb.hi;
    if (count) count[b] = pb.q_end - pb.q_begin;
    if (variant) variant[b] = pb.variant;
    if (tuned_us) tuned_us[b] = pb.tuned_us;
  }
  return nb;
}

gj_status gj_batched_plan_execute(gj_plan* p, const double* const* A, double* const* Ainv, int32_t* status,
                                  int8_t* det_sign, double* det_log2, void* stream, int use_graph) {
  g_last_error[0] = '\0';
  if (!p) return GJ_ERR_ARG;
  if (p->count == 0) return GJ_OK;
  if (!A || !Ainv || !status) return GJ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!use_graph) return plan_enqueue(p, A, Ainv, status, det_sign, det_log2, s);
  const void* key[6] = {A, Ainv, status, det_sign, det_log2, stream};
  bool same = p->exec != nullptr;
  for (int i = 0; i < 6 && same; ++i) same = (key[i] == p->key[i]);
  if (!same) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    if (p->graph) {
      cudaGraphDestroy(p->graph);
      p->graph = nullptr;
    }
    cudaStream_t cap;
    GJ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    gj_status st = plan_enqueue(p, A, Ainv, status, det_sign, det_log2, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != GJ_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    p->graph = g;
    GJ_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
    for (int i = 0; i < 6; ++i) p->key[i] = key[i];
  }
  {
    ProfScope ps(s, "batched_plan", p->flops, p->bytes);
    GJ_CUDA(cudaGraphLaunch(p->exec, s));
  }
  prof_count(1);
  return GJ_OK;
}

void gj_batched_plan_destroy(gj_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_n) cudaFree(p->d_n);
  if (p->d_order) cudaFree(p->d_order);
  if (p->d_counter) cudaFree(p->d_counter);
  delete p;
}

}  // extern "C"
