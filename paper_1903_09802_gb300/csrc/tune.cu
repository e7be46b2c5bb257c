// Launch schedules and the autotuner (dda_schedule_set / _get, dda_autotune).
//
// A schedule only selects among launch forms that compute the same thing
// (launch.cuh: the register-resident or the all-shared-memory z pass, launches
// with or without programmatic dependent launch).  The autotuner times the
// plan's matvec under each schedule with CUDA events on the caller's stream
// and keeps the fastest; the choice is remembered per (device, box, precision,
// right-hand sides) for the rest of the process, so plans of the same shape
// (an uneven batch of prisms repeats a few box sizes) pay for the timing once.
#include <map>
#include <mutex>
#include <tuple>

#include "plan.hpp"

using namespace dda;

namespace {

using TuneKey = std::tuple<int, int, int, int, int, int>;  // device, l, m, n, prec, nrhs

std::mutex g_tune_mu;
std::map<TuneKey, Schedule> g_tune_table;

dda_schedule_t to_c(const Schedule& s) {
  return dda_schedule_t{s.rr_z ? 1 : 0, s.pdl ? 1 : 0, s.graph ? 1 : 0, s.z_occ ? 1 : 0};
}

// Mean milliseconds per matvec under the plan's current schedule.
dda_status_t time_matvec(dda_plan_t p, int32_t prec, int32_t nrhs, const void* x, void* y,
                         int32_t reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                         float* ms) {
  for (int i = 0; i < 2; ++i) {
    const dda_status_t st = dda_matvec(p, prec, nrhs, x, y, s);
    if (st != DDA_OK) return st;
  }
  if (cudaEventRecord(e0, s) != cudaSuccess) return check_cuda("dda_autotune: event");
  for (int i = 0; i < reps; ++i) {
    const dda_status_t st = dda_matvec(p, prec, nrhs, x, y, s);
    if (st != DDA_OK) return st;
  }
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
    return check_cuda("dda_autotune: event");
  float t = 0.f;
  if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return check_cuda("dda_autotune: event");
  *ms = t / reps;
  return DDA_OK;
}

}  // namespace

extern "C" dda_status_t dda_schedule_set(dda_plan_t p, const dda_schedule_t* sched) {
  if (!p || !sched) return fail(DDA_ERR_INVALID_ARG, "dda_schedule_set: NULL argument");
  if ((sched->rr_z != 0 && sched->rr_z != 1) || (sched->pdl != 0 && sched->pdl != 1) ||
      (sched->graph != 0 && sched->graph != 1) || (sched->z_occ != 0 && sched->z_occ != 1))
    return fail(DDA_ERR_INVALID_ARG, "dda_schedule_set: fields must be 0 or 1");
  p->sched.rr_z = sched->rr_z == 1;
  p->sched.pdl = sched->pdl == 1;
  p->sched.graph = sched->graph == 1;
  p->sched.z_occ = sched->z_occ == 1;
  return DDA_OK;
}

extern "C" dda_status_t dda_schedule_get(dda_plan_t p, dda_schedule_t* out) {
  if (!p || !out) return fail(DDA_ERR_INVALID_ARG, "dda_schedule_get: NULL argument");
  *out = to_c(p->sched);
  return DDA_OK;
}

extern "C" dda_status_t dda_autotune(dda_plan_t p, int32_t prec, int32_t nrhs, const void* d_x,
                                     void* d_y, int32_t reps, int32_t flags,
                                     dda_tune_report_t* h_report, void* stream) {
  if (!p || !d_x || !d_y) return fail(DDA_ERR_INVALID_ARG, "dda_autotune: NULL argument");
  if (reps < 1 || reps > 1000) return fail(DDA_ERR_INVALID_ARG, "dda_autotune: reps must be 1..1000");
  if (prec != DDA_C128 && prec != DDA_C64)
    return fail(DDA_ERR_INVALID_ARG, "dda_autotune: prec must be DDA_C128 or DDA_C64");
  if ((prec == DDA_C128 && !p->has128) || (prec == DDA_C64 && !p->has64))
    return fail(DDA_ERR_INVALID_ARG, "dda_autotune: plan lacks that precision");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_autotune: nrhs must be 1..(incidences set)");
  if (d_x == d_y) return fail(DDA_ERR_INVALID_ARG, "dda_autotune: x and y must not overlap");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("dda_autotune");
  const TuneKey key{dev, p->l, p->m, p->n, prec, nrhs};
  dda_tune_report_t rep{};
  if (!(flags & 1)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_table.find(key);
    if (it != g_tune_table.end()) {
      p->sched.rr_z = it->second.rr_z;
      p->sched.pdl = it->second.pdl;
      p->sched.z_occ = it->second.z_occ;
      rep.chosen = to_c(p->sched);
      rep.cached = 1;
      if (h_report) *h_report = rep;
      return DDA_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return check_cuda("dda_autotune: event");
  }
  const Schedule saved = p->sched;
  dda_status_t st = DDA_OK;
  int best = -1;
  for (int c = 0; c < 8 && st == DDA_OK; ++c) {
    Schedule cand = saved;  // the solve-loop choice (graph) is not tuned here
    cand.rr_z = (c & 1) == 0;
    cand.pdl = (c & 2) != 0;
    cand.z_occ = (c & 4) == 0;
    p->sched = cand;
    float ms = 0.f;
    st = time_matvec(p, prec, nrhs, d_x, d_y, reps, s, e0, e1, &ms);
    if (st != DDA_OK) break;
    rep.cand[c] = to_c(cand);
    rep.ms_per_matvec[c] = ms;
    rep.ncand = c + 1;
    if (best < 0 || ms < rep.ms_per_matvec[best]) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DDA_OK) {
    p->sched = saved;
    return st;
  }
  p->sched.rr_z = rep.cand[best].rr_z == 1;
  p->sched.pdl = rep.cand[best].pdl == 1;
  p->sched.z_occ = rep.cand[best].z_occ == 1;
  rep.chosen = rep.cand[best];
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_table[key] = p->sched;
  }
  if (h_report) *h_report = rep;
  return DDA_OK;
}
