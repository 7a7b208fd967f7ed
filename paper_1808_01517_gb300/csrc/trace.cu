// Optional per-launch timing (tracing): when enabled, each traced launch group is
// bracketed by CUDA events recorded on its launch stream; the summary reports,
// per name, the number of launches and their total device time.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/delimit.h"
#include "kernels.h"

namespace delimit {

namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void recycle_all() {
  for (auto& r : g_recs) {
    if (r.a) g_pool.push_back(r.a);
    if (r.b) g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t st) : idx_(-1), st_(st) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, take_event(), take_event()};
  if (!r.a || !r.b || cudaEventRecord(r.a, st) != cudaSuccess) {
    if (r.a) g_pool.push_back(r.a);
    if (r.b) g_pool.push_back(r.b);
    return;
  }
  g_recs.push_back(r);
  idx_ = int(g_recs.size()) - 1;
}

TraceScope::~TraceScope() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx_ < int(g_recs.size())) cudaEventRecord(g_recs[idx_].b, st_);
}

}  // namespace delimit

using namespace delimit;

extern "C" {

delimit_status delimit_trace_enable(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  recycle_all();
  g_on.store(enable != 0);
  return DELIMIT_OK;
}

int64_t delimit_trace_summary(char* buf, size_t cap) {
  std::map<std::string, std::pair<long, double>> agg;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
      auto& v = agg[r.name];
      v.first += 1;
      v.second += ms;
    }
  }
  std::string out = "{";
  char item[256];
  bool first = true;
  for (auto& kv : agg) {
    std::snprintf(item, sizeof item, "%s\"%s\": {\"n\": %ld, \"ms\": %.6f}", first ? "" : ", ", kv.first.c_str(),
                  kv.second.first, kv.second.second);
    out += item;
    first = false;
  }
  out += "}";
  if (buf && cap > 0) {
    const size_t n = out.size() < cap - 1 ? out.size() : cap - 1;
    out.copy(buf, n);
    buf[n] = '\0';
  }
  return int64_t(out.size());
}

}  // extern "C"
