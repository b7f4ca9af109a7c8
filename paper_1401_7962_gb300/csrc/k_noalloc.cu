// k_noalloc.cu -- batched inversion that allocates no device memory.
//
// gj_invert_batched takes its scratch (the largest-first work order, the order-size
// histogram and the queue counter) from the stream-ordered allocator.  Some callers
// cannot allocate at the point where they invert: real-time loops that must not take the
// allocator's locks or risk its latency or failure, programs that handed all device
// memory to their own pool, code that allocates only during initialisation.  This
// variant keeps that scratch in a file-scope device array instead: it is loaded with the
// library and every GPU that loads the library holds it (about 4 MiB) until the process
// exits.
//
// The array's name is a host-side stand-in in host code, not a device address, so the
// host asks the runtime for the address (cudaGetSymbolAddress) once per device, with
// that device current, and passes the result to the kernels.  The first call on a
// device does this set-up; make that first call before any stream capture.  The address
// is kept together with the identifier of the context it was looked up in, and looked up
// again when the device's current context is another one (a cudaDeviceReset destroys the
// context the address belonged to).
//
// All calls share the one array, and it keeps the last call's contents: the histogram
// and the queue counter are cleared by every call before use.  Calls whose execution
// overlaps on the GPU (different streams, or concurrent host threads) race on the
// array and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "gj_internal.cuh"

namespace gj {
namespace {

constexpr int64_t kNoAllocMaxCount = GJ_NOALLOC_MAX_COUNT;
constexpr int64_t kNoAllocWords = kNoAllocMaxCount + kCtaMaxN + 3;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identifier of the calling thread's current context, 0 when none is current or the driver
// does not offer context identifiers (the address is then looked up on every call).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up once per device and
// context.
gj_status scratch_address(int32_t** out) {
  int dev = 0;
  GJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GJ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_addr[dev] = static_cast<int32_t*>(p);
    g_ctx[dev] = current_context_id();  // the lookup makes the device's primary context current
  }
  *out = g_addr[dev];
  return GJ_OK;
}

}  // namespace
}  // namespace gj

using namespace gj;

extern "C" gj_status gj_invert_batched_noalloc(int64_t count, int32_t nmax, const int32_t* n, const double* const* A,
                                               double* const* Ainv, int pivot_mode, int32_t* status,
                                               int8_t* det_sign, double* det_log2, void* stream) {
  set_last_error("");
  if (count < 0) return GJ_ERR_ARG;
  if (count > kNoAllocMaxCount) {
    set_last_error("gj_invert_batched_noalloc: count exceeds GJ_NOALLOC_MAX_COUNT (1048576); split the batch");
    return GJ_ERR_UNSUPPORTED;
  }
  if (pivot_mode < GJ_PIVOT_NONE || pivot_mode > GJ_PIVOT_FULL) return GJ_ERR_ARG;
  if (nmax <= 0) nmax = kCtaMaxN;
  if (nmax > kCtaMaxN) return GJ_ERR_UNSUPPORTED;
  if (count == 0) return GJ_OK;
  if (!n || !A || !Ainv || !status) return GJ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* ws = nullptr;
  gj_status st = scratch_address(&ws);
  if (st != GJ_OK) return st;
  int32_t* order = ws;
  int32_t* hist = ws + count;
  int32_t* counter = hist + kCtaMaxN + 1;
  st = launch_order_by_size(count, n, order, hist, counter, s);  // clears hist and counter first
  if (st != GJ_OK) return st;
  CtaOut out{};
  out.status = status;
  out.det_sign = det_sign;
  out.det_log2 = det_log2;
  return launch_cta_batched(count, nmax, n, A, Ainv, order, counter, pivot_mode, 0.0, out, s);
}
