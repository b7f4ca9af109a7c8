// gj_profile.cu -- optional kernel timing: CUDA events around selected launches.
//
// When enabled (gj_profile_begin), launch sites wrapped in a ProfScope record an event
// pair on the launching stream; gj_profile_end waits for the events and reports, per
// kernel name, the number of launches, the summed device time and the algorithmic
// FLOP and byte counts the launch site declared.  Every library launch site also bumps
// a launch counter while profiling is on.
#include <mutex>
#include <string>
#include <vector>

#include "gj_internal.cuh"

namespace gj {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
int64_t g_launches = 0;

}  // namespace

bool prof_enabled() { return g_on; }

void prof_count(int launches) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_launches += launches;
}

ProfScope::ProfScope(cudaStream_t s, const char* name, double flops, double bytes) : s_(s), rec_(-1) {
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // no event records inside a graph capture
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, nullptr, nullptr, flops, bytes};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  rec_ = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (rec_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (rec_ < (int)g_recs.size()) cudaEventRecord(g_recs[rec_].b, s_);
}

}  // namespace gj

using namespace gj;

extern "C" {

gj_status gj_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  g_launches = 0;
  g_on = true;
  return GJ_OK;
}

int gj_profile_end(gj_profile_entry* out, int max_entries, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  std::vector<gj_profile_entry> agg;
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess) cudaEventElapsedTime(&ms, r.a, r.b);
    cudaGetLastError();
    gj_profile_entry* e = nullptr;
    for (auto& x : agg)
      if (std::string(x.kernel) == r.name) e = &x;
    if (!e) {
      agg.push_back(gj_profile_entry{r.name, 0, 0.0, 0.0, 0.0});
      e = &agg.back();
    }
    e->launches += 1;
    e->total_ms += ms;
    e->flops += r.flops;
    e->bytes += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  if (launches) *launches = g_launches;
  const int cnt = (int)agg.size();
  for (int i = 0; i < cnt && i < max_entries && out; ++i) out[i] = agg[i];
  return cnt;
}

}  // extern "C"
