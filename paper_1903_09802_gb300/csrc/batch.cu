// Several independent systems solved concurrently (dda_solve_many): the
// solves of all plans captured into one CUDA graph, one independent chain
// per plan with device-side loop control, and launched once; where that is
// not possible (kernel timing on, a plan's schedule without graphs) one host
// thread per plan drives that plan's solve loop on its own stream.  A small
// prism's solve is a chain of short kernels that leaves most of the GPU idle;
// with several chains in flight on different streams their kernels share the
// SMs.  The plans do not interact: every plan owns its workspace, pinned
// polling words and kernel timing, so each result equals the one the same
// solve gives alone.
#include <string>
#include <thread>
#include <vector>

#include "plan.hpp"

using namespace dda;

extern "C" dda_status_t dda_solve_many(int32_t nplans, const dda_plan_t* plans,
                                       const int32_t* nrhs, const void* const* d_b,
                                       void* const* d_x, const dda_solve_opts_t* opts,
                                       dda_rhs_stats_t* const* h_stats, void* const* streams) {
  if (nplans < 1 || !plans || !nrhs || !d_x || !opts)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve_many: NULL argument or nplans < 1");
  if (opts->h_history != nullptr)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve_many: h_history must be NULL (one row set per plan)");
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || !d_x[i]) return fail(DDA_ERR_INVALID_ARG, "dda_solve_many: NULL plan or x");
    for (int k = 0; k < i; ++k) {
      if (plans[k] == plans[i])
        return fail(DDA_ERR_INVALID_ARG, "dda_solve_many: a plan appears twice");
      if (streams && streams[k] && streams[k] == streams[i])
        return fail(DDA_ERR_INVALID_ARG, "dda_solve_many: two plans share a stream");
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("dda_solve_many");
  std::vector<dda_status_t> st(nplans, DDA_OK);
  std::vector<std::string> why(nplans);
  if (solve_many_as_graph(nplans, plans, nrhs, d_b, d_x, opts, h_stats, streams, st.data(),
                          why.data())) {
    for (int i = 0; i < nplans; ++i)
      if (st[i] != DDA_OK)
        return fail(st[i], "dda_solve_many: plan " + std::to_string(i) + ": " + why[i]);
    return DDA_OK;
  }
  std::vector<std::thread> workers;
  workers.reserve(nplans);
  for (int i = 0; i < nplans; ++i) {
    workers.emplace_back([&, i] {
      cudaSetDevice(dev);
      st[i] = dda_solve(plans[i], nrhs[i], d_b ? d_b[i] : nullptr, d_x[i], opts,
                        h_stats ? h_stats[i] : nullptr, streams ? streams[i] : nullptr);
      if (st[i] != DDA_OK) why[i] = dda_last_error();
    });
  }
  for (std::thread& t : workers) t.join();
  for (int i = 0; i < nplans; ++i)
    if (st[i] != DDA_OK)
      return fail(st[i], "dda_solve_many: plan " + std::to_string(i) + ": " + why[i]);
  return DDA_OK;
}
