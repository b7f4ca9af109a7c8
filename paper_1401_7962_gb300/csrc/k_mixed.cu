// k_mixed.cu -- reduced-precision Gauss-Jordan followed by Newton-Schulz refinement.
//
// X0 comes from the blocked Gauss-Jordan of eqs. 14-15 whose rank-128 updates run on the
// BF16 tensor cores with only S digit slices (8 bits each: S = 1 about BF16's 8-bit
// significand, S = 2 a split-BF16 pair of 16 bits, S = 3 24 bits, FP32's significand, of
// each row / column scale) while pivot search, division and the determinant stay in FP64.
// Accuracy is then recovered by Newton-Schulz refinement
//     R_k = I - A X_k,   X_{k+1} = X_k + X_k R_k,   so   I - A X_{k+1} = R_k^2,
// with R_k formed to FP64 level: the K = n product A X_k is summed in exact 128-wide
// chunks of the tensor-core update (7 slices), and the correction X_k R_k -- which only
// has to be accurate relative to the small R_k -- uses fewer slices.  The iteration stops
// when ||A X - I||_F / (||A||_F ||X||_F) <= tol.  If the residual does not contract (the
// first X0 was too inaccurate for this condition number) the next rung of precision is
// taken: 5 slices for X0, and finally the FP64-level update (7 slices); the 5-slice rung is
// skipped when the failed rung's first residual norm shows that 5 slices cannot contract
// either (each extra slice lowers the truncation by 2^-8).
#include <math.h>

#include <algorithm>

#include "gj_ozaki.cuh"
#include "gj_paths.cuh"

namespace gj {
namespace {

constexpr int kFp64Slices = 7;  // digit slices of the FP64-level update

__global__ void f32_to_f64_kernel(int64_t n, const float* __restrict__ A, int64_t lda, double* __restrict__ D,
                                  double* __restrict__ negD) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const double v = (double)A[i + j * lda];
    D[e] = v;
    negD[e] = -v;
  }
}

__global__ void identity_kernel(int64_t n, double* __restrict__ R) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    R[e] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void copy_kernel(int64_t total, const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// Partial sums of squares, one per block (fixed block order: deterministic).
__global__ void __launch_bounds__(256) sumsq_partial_kernel(int64_t total, const double* __restrict__ x,
                                                            double* __restrict__ part) {
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[e], x[e], s);
  __shared__ double red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    *out = t;
  }
}

}  // namespace

// sum of squares of x (device) -> host, synchronous on s
static gj_status sumsq(int64_t total, const double* x, double* part, double* dres, int nparts, cudaStream_t s,
                       double* host) {
  sumsq_partial_kernel<<<nparts, 256, 0, s>>>(total, x, part);
  GJ_CUDA(cudaGetLastError());
  sum_kernel<<<1, 32, 0, s>>>(nparts, part, dres);
  GJ_CUDA(cudaGetLastError());
  prof_count(2);
  GJ_CUDA(cudaMemcpyAsync(host, dres, sizeof(double), cudaMemcpyDeviceToHost, s));
  GJ_CUDA(cudaStreamSynchronize(s));
  return GJ_OK;
}

// C += L U with K = n, summed in exact chunks of 128 (each chunk an emulated update).
static gj_status product_chunks(int64_t n, const double* L, const double* U, double* C, int S, void* ws,
                                int32_t* err, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < n; k0 += 128) {
    const int kk = (int)std::min<int64_t>(128, n - k0);
    gj_status st = ozaki_update(n, n, kk, L + k0 * n, n, nullptr, U + k0, n, nullptr, 0, 0, C, n, S, ws, err, nullptr,
                                s);
    if (st != GJ_OK) return st;
  }
  return GJ_OK;
}

}  // namespace gj

using namespace gj;

extern "C" gj_status gj_invert_mixed(int64_t n, const float* A, int64_t lda, double* X, int x0_slices,
                                     int corr_slices, double tol, int max_iter, double* resid_out, int* iters_out,
                                     int* rung_out, int* det_sign, double* det_log2, void* stream) {
  set_last_error("");
  if (det_sign) *det_sign = 0;
  if (det_log2) *det_log2 = -INFINITY;
  if (resid_out) *resid_out = INFINITY;
  if (iters_out) *iters_out = 0;
  if (rung_out) *rung_out = 0;
  if (n < 0 || lda < (n > 0 ? n : 1) || x0_slices < 1 || x0_slices > 8 || corr_slices < 1 || corr_slices > 8 ||
      !(tol > 0.0) || max_iter < 0)
    return GJ_ERR_ARG;
  if (n == 0) {
    if (det_sign) *det_sign = 1;
    if (det_log2) *det_log2 = 0.0;
    if (resid_out) *resid_out = 0.0;
    return GJ_OK;
  }
  if (!A || !X) return GJ_ERR_ARG;
  if (n > 46340) return GJ_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)n * (size_t)n;
  const int nparts = 1024;
  double *Ad = nullptr, *negA = nullptr, *R = nullptr, *Xn = nullptr, *part = nullptr, *dres = nullptr;
  void* ws = nullptr;
  int32_t* err = nullptr;
  struct ResultBlock {
    int32_t status;
    int8_t det_sign;
    int8_t pad[3];
    double det_log2;
    int64_t fail_step;
  }* res = nullptr;
  auto cleanup = [&]() {
    void* ps[] = {Ad, negA, R, Xn, part, dres, ws, err, res};
    for (void* p : ps)
      if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  };
  auto alloc = [&](void** p, size_t bytes) {
    if (lib_malloc_async(p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!alloc((void**)&Ad, nn * 8) || !alloc((void**)&negA, nn * 8) || !alloc((void**)&R, nn * 8) ||
      !alloc((void**)&Xn, nn * 8) || !alloc((void**)&part, nparts * 8) || !alloc((void**)&dres, 8) ||
      !alloc(&ws, ozaki_workspace_bytes(n, n, 8)) || !alloc((void**)&err, 16) ||
      !alloc((void**)&res, sizeof(ResultBlock))) {
    cleanup();
    return GJ_ERR_NOMEM;
  }
  gj_status result = GJ_OK;
  do {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    f32_to_f64_kernel<<<sms * 8, 256, 0, s>>>(n, A, lda, Ad, negA);
    if (cudaGetLastError() != cudaSuccess) { result = GJ_ERR_CUDA; break; }
    prof_count(1);
    double hA2 = 0.0;
    if ((result = sumsq((int64_t)nn, Ad, part, dres, nparts, s, &hA2)) != GJ_OK) break;
    const double normA = sqrt(hA2);

    // precision ladder for X0: requested slices, then 5, then the FP64-level 7.  The update
    // error is below (S + 2) 128 2^-8S of the scales per panel; Newton-Schulz needs roughly
    // that times kappa below 1: 5 slices (~1e-9) serve kappa up to ~1e8.
    int rungs[3] = {std::min(x0_slices, kFp64Slices), std::min(std::max(x0_slices, 5), kFp64Slices), kFp64Slices};
    double r = INFINITY;
    int iters = 0, rung_used = 0;
    bool converged = false;
    for (int rg = 0; rg < 3 && !converged; ++rg) {
      if (rg > 0 && rungs[rg] == rungs[rg - 1]) continue;
      rung_used = rg;
      cudaMemsetAsync(res, 0, sizeof(ResultBlock), s);
      cudaMemsetAsync(err, 0, 16, s);
      CtaOut out{};
      out.status = &res->status;
      out.det_sign = &res->det_sign;
      out.det_log2 = &res->det_log2;
      out.fail_step = &res->fail_step;
      gj_status st = run_blocked(n, Ad, n, X, GJ_PIVOT_PARTIAL, 0.0, 0, 2, rungs[rg], out, s);
      if (st != GJ_OK) { result = st; break; }
      ResultBlock h{};
      if (cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        result = GJ_ERR_CUDA;
        break;
      }
      if (h.status != GJ_OK) { result = (gj_status)h.status; break; }
      if (det_sign) *det_sign = h.det_sign;
      if (det_log2) *det_log2 = h.det_log2;
      double prev = INFINITY, R0 = INFINITY;
      iters = 0;
      for (;;) {
        // R = I - A X (FP64-level: 7 slices, exact 128-wide chunks)
        identity_kernel<<<sms * 8, 256, 0, s>>>(n, R);
        prof_count(1);
        if ((st = product_chunks(n, negA, X, R, kFp64Slices, ws, err, s)) != GJ_OK) { result = st; break; }
        double hR2 = 0.0, hX2 = 0.0;
        if ((st = sumsq((int64_t)nn, R, part, dres, nparts, s, &hR2)) != GJ_OK) { result = st; break; }
        if ((st = sumsq((int64_t)nn, X, part, dres, nparts, s, &hX2)) != GJ_OK) { result = st; break; }
        r = sqrt(hR2) / (normA * sqrt(hX2));
        if (!(r == r)) r = INFINITY;
        if (iters == 0 && hR2 == hR2) R0 = sqrt(hR2);
        if (r <= tol) {
          converged = true;
          break;
        }
        // stop this rung when the residual no longer contracts (or the budget is spent)
        if (iters >= max_iter || !(r < 0.5 * prev) || sqrt(hR2) >= 1.0 * sqrt((double)n)) break;
        prev = r;
        // X <- X + X R
        copy_kernel<<<sms * 8, 256, 0, s>>>((int64_t)nn, X, Xn);
        prof_count(1);
        if ((st = product_chunks(n, X, R, Xn, corr_slices, ws, err, s)) != GJ_OK) { result = st; break; }
        copy_kernel<<<sms * 8, 256, 0, s>>>((int64_t)nn, Xn, X);
        prof_count(1);
        ++iters;
      }
      if (result != GJ_OK) break;
      // next rung: the lowest one whose X0 (error 2^-8 smaller per extra slice) would bring
      // this rung's first ||I - A X0||_F below 1/4, else the FP64-level rung; so a matrix
      // whose 3-slice X0 is far off goes to 7 slices without a 5-slice X0 between
      if (!converged && rg < 2) {
        int nxt = 2;
        for (int q = rg + 1; q < 2; ++q)
          if (R0 * ldexp(1.0, -8 * (rungs[q] - rungs[rg])) <= 0.25) {
            nxt = q;
            break;
          }
        rg = nxt - 1;  // the loop's increment lands on nxt
      }
    }
    int32_t herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (result == GJ_OK && herr != 0) result = GJ_ERR_TIMEOUT;
    if (resid_out) *resid_out = r;
    if (iters_out) *iters_out = iters;
    if (rung_out) *rung_out = rung_used;
    if (result == GJ_OK && !converged) result = GJ_NOT_CONVERGED;
  } while (false);
  cleanup();
  return result;
}

extern "C" gj_status gj_invert_mixed_prec(int64_t n, const float* A, int64_t lda, double* X, int prec, double tol,
                                          int max_iter, double* resid_out, int* iters_out, int* rung_out,
                                          int* det_sign, double* det_log2, void* stream) {
  // digit slices of the first inverse's update for each named arithmetic
  int x0;
  switch (prec) {
    case GJ_PREC_FP64: x0 = kFp64Slices; break;
    case GJ_PREC_BF16: x0 = 1; break;
    case GJ_PREC_FP16: x0 = 2; break;
    case GJ_PREC_SPLIT_BF16_3: x0 = 2; break;
    case GJ_PREC_TF32x3: x0 = 3; break;
    default:
      set_last_error("gj_invert_mixed_prec: unknown gj_prec value");
      return GJ_ERR_ARG;
  }
  return gj_invert_mixed(n, A, lda, X, x0, 4, tol, max_iter, resid_out, iters_out, rung_out, det_sign, det_log2,
                         stream);
}
