// Event-based per-kernel timing (see prof.cuh).
#include "prof.cuh"

thread_local Profiler *g_prof = nullptr;
thread_local cudaStream_t g_prof_stream = nullptr;

static cudaEvent_t take_event(Profiler *p) {
  if (p->pool_used == p->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p->pool.push_back(e);
  }
  return p->pool[p->pool_used++];
}

void prof_begin(const char *name, cudaStream_t s, int kernels) {
  Profiler *p = g_prof;
  ProfRecord r;
  r.name = name;
  r.kernels = kernels;
  r.a = take_event(p);
  r.b = take_event(p);
  cudaEventRecord(r.a, s);
  p->pending.push_back(r);
  g_prof_stream = s;
}

void prof_end(cudaStream_t s) {
  Profiler *p = g_prof;
  if (p->pending.empty()) return;
  cudaEventRecord(p->pending.back().b, s);
}

void prof_flush(Profiler *p) {
  if (!p || p->pending.empty()) return;
  cudaEventSynchronize(p->pending.back().b);
  for (const ProfRecord &r : p->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    size_t k = 0;
    for (; k < p->names.size(); ++k)
      if (p->names[k] == r.name) break;
    if (k == p->names.size()) {
      p->names.push_back(r.name);
      p->total_ms.push_back(0.0);
      p->count.push_back(0);
    }
    p->total_ms[k] += ms;
    p->count[k] += r.kernels;
  }
  p->pending.clear();
  p->pool_used = 0;
}
