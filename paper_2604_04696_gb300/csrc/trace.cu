// Per-kernel tracing: when enabled, every kernel launch of the library is
// bracketed by CUDA events recorded on its launch stream, so callers can read
// device durations per kernel (the paper profiles per kernel with Nsight
// Compute, Sec. 4.2 / Sec. 5.1.2; these are the same durations, live).
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.h"

namespace gpir {
namespace {

struct Rec {
  char name[32];
  cudaEvent_t e0, e1;
};

std::mutex g_mu;
bool g_on = false;
bool g_count_roles = false;   // tracing level 2
std::vector<Rec> g_recs;
std::vector<unsigned long long> g_counters;   // last kernel's wait-cycle counters

}  // namespace

bool trace_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

bool trace_counters_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on && g_count_roles;
}

// Copy a kernel's device counters to the host (synchronizes `s`).
void trace_counters(const unsigned long long *dev, int n, cudaStream_t s) {
  try {   // tracing only: an allocation failure drops the counters
    std::vector<unsigned long long> h(n, 0);
    if (cudaMemcpyAsync(h.data(), dev, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_mu);
      g_counters = h;
    }
  } catch (...) {
  }
}

int trace_begin(const char *name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Rec r;
  strncpy(r.name, name, sizeof(r.name) - 1);
  r.name[sizeof(r.name) - 1] = 0;
  if (cudaEventCreate(&r.e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&r.e1) != cudaSuccess) {
    cudaEventDestroy(r.e0);
    return -1;
  }
  try {   // tracing only: an allocation failure drops the record
    g_recs.push_back(r);
  } catch (...) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
    return -1;
  }
  cudaEventRecord(r.e0, s);
  return (int)g_recs.size() - 1;
}

void trace_end(int id, cudaStream_t s) {
  if (id < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (id < (int)g_recs.size()) cudaEventRecord(g_recs[id].e1, s);
}

}  // namespace gpir

extern "C" {

int gpir_trace_enable(int on) {
  if (on < 0 || on > 2) return GPIR_EINVAL;
  std::lock_guard<std::mutex> lk(gpir::g_mu);
  gpir::g_on = on != 0;
  gpir::g_count_roles = on == 2;
  return GPIR_OK;
}

int gpir_trace_read(gpir_trace_record_t *out, uint32_t max_records, uint32_t *count) {
  if (!count) return GPIR_EINVAL;
  std::lock_guard<std::mutex> lk(gpir::g_mu);
  uint32_t n = 0;
  int rc = GPIR_OK;
  for (auto &r : gpir::g_recs) {
    if (out && n < max_records) {
      float ms = -1.f;
      if (cudaEventSynchronize(r.e1) == cudaSuccess) cudaEventElapsedTime(&ms, r.e0, r.e1);
      memcpy(out[n].name, r.name, sizeof(out[n].name));
      out[n].ms = ms;
      ++n;
    }
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  gpir::g_recs.clear();
  *count = n;
  return rc;
}

int gpir_trace_counters(unsigned long long *out, uint32_t max_counters, uint32_t *count) {
  if (!count) return GPIR_EINVAL;
  std::lock_guard<std::mutex> lk(gpir::g_mu);
  uint32_t n = 0;
  for (auto v : gpir::g_counters) {
    if (out && n < max_counters) out[n] = v;
    ++n;
  }
  *count = n < max_counters ? n : max_counters;
  return GPIR_OK;
}

}  // extern "C"
