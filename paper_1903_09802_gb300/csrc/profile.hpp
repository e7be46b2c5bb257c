// Per-plan kernel timing: when enabled, CUDA events bracket selected
// launches and their elapsed times are summed per kernel class at read-out.
#pragma once

#include <cuda_runtime.h>

#include <vector>

struct dda_plan_s;

namespace dda {

enum ProfId {
  PROF_MV_XF = 0,  // matvec pass 1: x forward
  PROF_MV_YF,      // matvec pass 2: y forward
  PROF_MV_Z,       // matvec pass 3: z forward, spectrum multiply, z inverse
  PROF_MV_YI,      // matvec pass 4: y inverse
  PROF_MV_XI,      // matvec pass 5: x inverse and diagonal
  PROF_PC_XF,      // preconditioner passes
  PROF_PC_YF,
  PROF_PC_Z,
  PROF_PC_YI,
  PROF_PC_XI,
  PROF_AR_DOT,     // Gram-Schmidt dot products
  PROF_AR_UPD,     // Gram-Schmidt update and norm
  PROF_P2_BLOCK,   // 2-level preconditioner: dense block per frequency pair
  PROF_MV128_XF,   // the matvec's passes in complex128 (FP64 residuals), same order
  PROF_MV128_YF,
  PROF_MV128_Z,
  PROF_MV128_YI,
  PROF_MV128_XI,
  PROF_PC128_XF,   // the preconditioner's passes in complex128, same order
  PROF_PC128_YF,
  PROF_PC128_Z,
  PROF_PC128_YI,
  PROF_PC128_XI,
  PROF_COUNT
};

struct Profiler {
  bool on = false;
  struct Rec {
    int id;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;   // events recorded since the last read
  std::vector<cudaEvent_t> pool;
  double ms[PROF_COUNT] = {};
  long count[PROF_COUNT] = {};
  double bytes[PROF_COUNT] = {};
  cudaEvent_t get();
  // bytes: algorithmic bytes the bracketed launch moves (0 if not stated)
  void begin(int id, cudaStream_t s, double nbytes = 0.0);
  void end(cudaStream_t s);
  void collect();           // synchronises the recorded events and accumulates
  ~Profiler();
};

}  // namespace dda
