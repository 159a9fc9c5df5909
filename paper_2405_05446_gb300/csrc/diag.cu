// Diagnostics: a process-wide count of kernels this library enqueued, and an
// opt-in per-kernel timer built from CUDA events recorded on the launching
// stream around each launch (aggregated by kernel name when read back).
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "gdgs_internal.cuh"

namespace gdgs {

namespace {

struct Rec {
  const char *name;
  cudaEvent_t a, b;
};

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_profiling{0};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local long t_open = -1;
thread_local bool t_capturing = false;

cudaEvent_t take_event() {
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

bool pdl_enabled() {
  static const bool on = [] {
    const char *v = getenv("GDGS_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

bool diag_profiling() { return g_profiling.load(std::memory_order_acquire) != 0; }

void diag_set_capturing(bool on) { t_capturing = on; }

void diag_before(const char *name, cudaStream_t st) {
  t_open = -1;
  if (t_capturing) return;  // counted when the graph runs
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return;  // recorded into a caller's graph: runs (and is counted by it) at replay
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_profiling.load(std::memory_order_acquire)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, take_event(), take_event()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  t_open = (long)g_recs.size() - 1;
}

void diag_after(cudaStream_t st) {
  if (t_open < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_open < (long)g_recs.size()) cudaEventRecord(g_recs[t_open].b, st);
  t_open = -1;
}

}  // namespace gdgs

using namespace gdgs;

extern "C" {

uint64_t gdgs_kernel_launch_count(void) { return g_launches.load() + graph_kernel_count(); }

int gdgs_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_profiling.store(1, std::memory_order_release);
  return GDGS_OK;
}

int gdgs_profile_end(gdgs_kernel_time *out, int32_t max_entries, int32_t *n_entries) {
  g_profiling.store(0, std::memory_order_release);
  std::lock_guard<std::mutex> lk(g_mu);
  int n = 0;
  int status = GDGS_OK;
  for (auto &r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      status = GDGS_ERR_CUDA;
      continue;
    }
    int k = 0;
    while (k < n && strncmp(out[k].name, r.name, sizeof(out[k].name)) != 0) ++k;
    if (k == n) {
      if (!out || n >= max_entries) continue;
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, r.name, sizeof(out[k].name) - 1);
      ++n;
    }
    out[k].launches += 1;
    out[k].total_ms += ms;
  }
  for (auto &r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  if (n_entries) *n_entries = n;
  return status;
}

}  // extern "C"
