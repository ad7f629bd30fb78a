// Host-side launch accounting: a counter of kernel launches issued by the
// library, and (while enabled) a CUDA event pair recorded on the launching
// stream around every launch, grouped by kernel class.  Used by the
// benchmark to time the dominant kernel inside the timed region.
#include "internal.cuh"
#include "profile.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace sorsvd {
namespace {

std::atomic<uint64_t> g_launches{0};
std::mutex g_mu;
bool g_on = false;
unsigned g_mask = 0;
struct Rec { int cls; cudaEvent_t a, b; };
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int prof_start(int cls, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || !((g_mask >> cls) & 1u)) return -1;
  Rec r{cls, take_event(), take_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_stop(int slot, cudaStream_t st) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].b, st);
}

}  // namespace sorsvd

using namespace sorsvd;

extern "C" {

uint64_t sorsvd_launch_count(void) { return g_launches.load(); }

int sorsvd_profile_begin(unsigned class_mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_mask = class_mask;
  for (auto& r : g_recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  g_recs.clear();
  g_on = true;
  return SORSVD_OK;
}

int sorsvd_profile_end(double* ms, int* launches, int nclass) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  for (int c = 0; c < nclass; ++c) { if (ms) ms[c] = 0.0; if (launches) launches[c] = 0; }
  int rc = SORSVD_OK;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) { rc = SORSVD_ERR_CUDA; continue; }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { rc = SORSVD_ERR_CUDA; continue; }
    if (r.cls >= 0 && r.cls < nclass) {
      if (ms) ms[r.cls] += t;
      if (launches) launches[r.cls] += 1;
    }
  }
  for (auto& r : g_recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  g_recs.clear();
  return rc;
}

}  // extern "C"
