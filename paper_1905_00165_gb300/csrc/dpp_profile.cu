// Optional per-kernel timing: while enabled, every launch of a tracked kernel
// is bracketed by CUDA events recorded on its own stream; the totals are read
// back (after an event synchronise) by dpp_profile_stop. A process-wide launch
// counter counts every kernel the library enqueues.
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "dpp.h"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

struct Rec {
  int cat;
  cudaEvent_t a, b;
  double flops, bytes;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<unsigned long long> g_launches{0};

const char* kNames[kProfCategories] = {"panel_decide_solve", "update_fp64", "update_f32_simt",
                                       "update_tc", "convert", "recompute", "other",
                                       "batched", "adjoint_batched", "lensemble_batched",
                                       "panel_rows_below", "elementary"};

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(int cat, cudaStream_t s, double flops, double bytes) : idx_(-1), s_(s) {
  count_launch(1);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  Rec r;
  r.cat = cat;
  r.a = get_event();
  r.b = get_event();
  r.flops = flops;
  r.bytes = bytes;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  idx_ = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, s_);
}

}  // namespace dpp

using namespace dpp;

extern "C" {

void dpp_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = true;
}

int32_t dpp_profile_stop(dpp_kernel_stat* out, int32_t max_entries) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  dpp_kernel_stat acc[kProfCategories];
  memset(acc, 0, sizeof(acc));
  for (int c = 0; c < kProfCategories; ++c) {
    strncpy(acc[c].name, kNames[c], sizeof(acc[c].name) - 1);
  }
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      acc[r.cat].launches += 1;
      acc[r.cat].total_ms += ms;
      acc[r.cat].flops += r.flops;
      acc[r.cat].bytes += r.bytes;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  int n = 0;
  for (int c = 0; c < kProfCategories && n < max_entries; ++c) {
    if (acc[c].launches == 0) continue;
    if (out) out[n] = acc[c];
    ++n;
  }
  return n;
}

uint64_t dpp_launch_count(void) { return g_launches.load(); }

}  // extern "C"
