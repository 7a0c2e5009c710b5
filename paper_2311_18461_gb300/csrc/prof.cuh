// Per-kernel launch timing with CUDA events (the library's tracing hook). When a handle has
// profiling enabled, each API call installs the handle's profiler as the current one; every launch
// site brackets its kernel (or a short run of kernels, counted as such) with prof_begin / prof_end,
// which record events on the launch stream. Durations and kernel launch counts are collected by
// stst_profile_read. Graph-captured launches are never profiled. Scopes do not nest.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>

struct ProfRecord {
  std::string name;
  cudaEvent_t a, b;
  int kernels;  // kernel launches inside the bracket
};

struct Profiler {
  std::vector<ProfRecord> pending;
  std::vector<std::string> names;   // aggregated
  std::vector<double> total_ms;
  std::vector<long long> count;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

extern thread_local Profiler *g_prof;
extern thread_local cudaStream_t g_prof_stream;

void prof_begin(const char *name, cudaStream_t s, int kernels);
void prof_end(cudaStream_t s);
void prof_flush(Profiler *p);

struct ProfScope {
  bool on;
  ProfScope(const char *name, cudaStream_t s, int kernels = 1) : on(g_prof != nullptr) {
    if (on) prof_begin(name, s, kernels);
  }
  ~ProfScope() {
    if (on) prof_end(g_prof_stream);
  }
};
#define STST_PROF(name, stream) ProfScope prof_scope_##__LINE__(name, stream)
#define STST_PROF_N(name, stream, kernels) ProfScope prof_scope_##__LINE__(name, stream, kernels)
