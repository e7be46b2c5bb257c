// Kernel launch with programmatic dependent launch (PDL).
//
// Kernels of the solver loop follow one another on one stream, most of them
// short (tens of microseconds at 64^3).  A launch made with the
// programmatic-stream-serialization attribute may be scheduled while the
// previous kernel of the stream is still finishing; it must then wait, with
// griddepcontrol.wait, before touching anything that kernel writes.  Every
// kernel of the library starts with pdl_entry(): the wait (a no-op when the
// kernel was launched the ordinary way), then launch_dependents, which lets
// the next kernel's CTAs become resident as soon as all of this grid's CTAs
// are running.  Because every CTA waits before its first memory access, a
// kernel completes only after its predecessor has, so ordering stays
// transitive along the stream.  DDA_PDL=0 in the environment turns the
// attribute off (ordinary launches).
//
// Schedule: the launch choices a plan may tune (dda_autotune).  The entry
// points of the library install their plan's schedule for the calling thread
// (ScheduleScope) before launching; the defaults are the choices measured
// fastest on the 64^3 workloads.  The environment switches above override a
// schedule towards the plain forms.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <utility>

namespace dda {

__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

struct Schedule {
  bool rr_z = true;  // register-resident z pass of the complex64 matvec (lengths 64, 128)
  // programmatic dependent launch: off by default (with the register-bounded
  // z pass and the graph-driven loop it measured 8-15% slower on the 64^3
  // solves: the next kernel's early-resident blocks take SM room from the
  // draining one)
  bool pdl = false;
  bool graph = true; // dda_solve as one CUDA graph launch (device-side loop control)
  bool z_occ = true; // register-resident z pass with 256-thread tiles bounded to three blocks per SM
};

inline thread_local Schedule tl_schedule;

struct ScheduleScope {
  Schedule saved;
  explicit ScheduleScope(const Schedule& s) : saved(tl_schedule) { tl_schedule = s; }
  ~ScheduleScope() { tl_schedule = saved; }
  ScheduleScope(const ScheduleScope&) = delete;
  ScheduleScope& operator=(const ScheduleScope&) = delete;
};

inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("DDA_PDL");
    return !(e && e[0] == '0');
  }();
  return on && tl_schedule.pdl;
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace dda
