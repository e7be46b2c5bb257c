// Kernel timing hooks of a plan (see profile.hpp) and their C entry points.
#include <cstring>

#include "plan.hpp"
#include "profile.hpp"

namespace dda {

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void Profiler::begin(int id, cudaStream_t s, double nbytes) {
  if (!on) return;
  Rec r{id, nbytes, get(), get()};
  cudaEventRecord(r.a, s);
  recs.push_back(r);
}

void Profiler::end(cudaStream_t s) {
  if (!on || recs.empty()) return;
  cudaEventRecord(recs.back().b, s);
  if (recs.size() >= 4096) collect();
}

void Profiler::collect() {
  for (Rec& r : recs) {
    cudaEventSynchronize(r.b);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.id] += t;
      count[r.id] += 1;
      bytes[r.id] += r.bytes;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

Profiler::~Profiler() {
  for (Rec& r : recs) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_profile_enable(dda_plan_t p, int32_t on) {
  if (!p) return fail(DDA_ERR_INVALID_ARG, "dda_profile_enable: NULL plan");
  p->prof.collect();
  p->prof.on = on != 0;
  return DDA_OK;
}

extern "C" dda_status_t dda_profile_read(dda_plan_t p, double* h_ms, int64_t* h_count,
                                         double* h_bytes, int32_t n, int32_t reset) {
  if (!p || !h_ms || !h_count) return fail(DDA_ERR_INVALID_ARG, "dda_profile_read: NULL argument");
  p->prof.collect();
  for (int i = 0; i < n && i < PROF_COUNT; ++i) {
    h_ms[i] = p->prof.ms[i];
    h_count[i] = p->prof.count[i];
    if (h_bytes) h_bytes[i] = p->prof.bytes[i];
  }
  if (reset) {
    std::memset(p->prof.ms, 0, sizeof(p->prof.ms));
    std::memset(p->prof.count, 0, sizeof(p->prof.count));
    std::memset(p->prof.bytes, 0, sizeof(p->prof.bytes));
  }
  return check_cuda("dda_profile_read");
}
