// Host-side plan object, workspace layout and shared launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dda.h"
#include "cx.cuh"
#include "dfloat.cuh"
#include "fft_core.cuh"
#include "profile.hpp"

namespace dda {

// Thread-local error text, set by fail().
void set_error(const std::string& msg);
dda_status_t fail(dda_status_t st, const std::string& msg);
dda_status_t check_cuda(const char* where);

inline bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

// Length of the plan's twiddle table exp(-2 pi i t / Lmax): a multiple of
// every transform length of the box (2l, 2m, 2n and l, m, n), i.e. their
// least common multiple; the largest edge's 2e for power-of-two boxes.
inline long twiddle_length(long l, long m, long n) {
  auto gcd = [](long a, long b) {
    while (b) {
      const long t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  long v = 2 * l;
  for (long e : {2 * m, 2 * n}) v = v / gcd(v, e) * e;
  return v;
}
constexpr long kMaxTwiddleLength = 1L << 20;

// Weight of the Toeplitz entry at offset p (side 0) or p - L (side 1) in
// entry p of a level's circulant: T. Chan's eq. 13 ((L - p)/L and p/L) or
// Strang's (the nearer of the two offsets; both halves at p = L/2).
__host__ __device__ inline double circ_weight(long p, long L, int side, int strang) {
  if (side == 1 && p == 0) return 0.0;
  if (!strang) return side ? (double)p / L : (double)(L - p) / L;
  if (2 * p == L) return 0.5;
  return (2 * p < L) == (side == 0) ? 1.0 : 0.0;
}

// Process-wide count of kernel launches made by the library (dda_launch_count).
void note_launch();

// Bump allocator over the caller's workspace; with base == 0 it only measures.
struct Carver {
  uintptr_t base;
  size_t off = 0;
  explicit Carver(void* b) : base(reinterpret_cast<uintptr_t>(b)) {}
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = reinterpret_cast<void*>(base + off);
    off += bytes;
    return p;
  }
};

// Device-side GMRES state per right-hand side (FP64).
struct SolverState {
  double2* H;        // [rhs][(m+1) * m], column-major: H[j*(m+1) + i]
  double* cs;        // [rhs][m]
  double2* sn;       // [rhs][m]
  double2* g;        // [rhs][m+1]
  double2* y;        // [rhs][m]
  double2* hcol;     // [rhs][m+1]   current column (dots of this step)
  double2* partial;  // [rhs][nblk][m+2] block partial sums
  double* scal;      // [rhs][16]: 0 beta, 2 bnorm, 3 target, 4 resid estimate,
                     //   5 1/h(j+1,j), 6 r-norm (FP64), 7 ||w||^2 before Gram-Schmidt,
                     //   8 ||w||^2 after it
  int* active;       // [rhs] 1 while the current cycle of this RHS is running
  int* jlen;         // [rhs] Arnoldi steps taken in the current cycle
  int* flags;        // [rhs] error bits (1 nan, 2 breakdown)
  int* iters;        // [rhs] inner iterations so far
  int* run;          // [rhs] 1 when the right-hand side takes part in this cycle
  int* reorth;       // [rhs] 1 when this step needs a second Gram-Schmidt pass
  int* reorth_count; // [rhs] steps that took a second pass
  int* tickets;      // [2][rhs] last-block counters of the Gram-Schmidt kernels
  double* bscal;     // [rhs][16] BiCG-Stab scalars
  int* counters;     // [16] 0: RHS still iterating in the current cycle
  int* ctl;          // [4] step index of the cycle, steps allowed, RHS running
  void* out;         // [rhs] outcome per right-hand side (krylov.cu's RhsOut)
  double* hist;      // [rhs][kHistCap] relative residual after each inner iteration
  unsigned long long* t0;  // solve start, device global timer (ns)
  long long* nlaunch;      // kernels run by a graph-driven solve
  // s-step GMRES (desc.sstep > 0)
  double2* Hraw;     // [rhs][(m+1) * m] the unrotated Hessenberg matrix
  double2* theta;    // [rhs][8] Newton shifts
  double2* cb;       // [rhs][2][(m+1+s) s] block coefficients: pass 1 C, pass 2 C and Gram
  double2* rinv;     // [rhs][64] inverse of the block's Cholesky factor
  double2* bpart;    // [blocks][(m+1+s) s] block partial sums (k_sdots)
};

// Residual-history entries kept per right-hand side on the device.
constexpr int kHistCap = 4096;
// Bytes of one right-hand side's outcome record (krylov.cu's RhsOut).
constexpr int kRhsOutBytes = 32;

// A plan's solve captured as one CUDA graph (krylov.cu), reused while the
// solve's arguments stay the same.
struct SolveGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;     // capture stream
  std::vector<char> key;         // arguments the graph was captured for
  bool failed = false;           // capture did not work: host-driven loop only
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    key.clear();
  }
  ~SolveGraph() {
    reset();
    if (cs) cudaStreamDestroy(cs);
  }
};

// Library launch counter (dda_launch_count): current value, and a signed
// adjustment (kernels a graph ran on the device; launches only captured).
long long launch_counter();
void add_launches(long long n);

// Whether dda_solve may run as one graph launch (DDA_SOLVE_GRAPH=0 in the
// environment forces the host-driven loop).
bool solve_graph_enabled();

// dda_solve_many's batch as one graph launch (krylov.cu); false when the
// plans cannot take part (then nothing was launched).
bool solve_many_as_graph(int32_t nplans, const dda_plan_t* plans, const int32_t* nrhs,
                         const void* const* d_b, void* const* d_x, const dda_solve_opts_t* opts,
                         dda_rhs_stats_t* const* h_stats, void* const* streams,
                         dda_status_t* st_out, std::string* why);

struct Layout {
  // spectra, octant-compressed: [(hz)(hy)(hx)][6]
  void* G128 = nullptr;
  void* G64 = nullptr;
  void* C128 = nullptr;
  void* C64 = nullptr;
  void* P2 = nullptr;   // 2-level preconditioner: l m (3n)^2 complex64 inverse blocks
  void* C2 = nullptr;   // its build scratch: 6 (2n-1) l m complex128
  void* mat2 = nullptr; // material mask in the relabelled frame (Toeplitz level x or y)
  // twiddles for the largest transform length
  void* tw128 = nullptr;
  void* tw64 = nullptr;
  // double-float copies of the twiddles, the kernel spectrum and alpha^{-1},
  // for the complex128 matvec that runs in double-float arithmetic
  void* twdf = nullptr;
  void* Gdf = nullptr;
  void* ainvdf = nullptr;
  // alpha^{-1} per (rhs, material 0..K); entry 0 is alpha_tilde^{-1}
  void* ainv128 = nullptr;
  void* ainv64 = nullptr;
  double* incd = nullptr;  // [rhs][6]: direction, polarisation
  // per-voxel permittivity (desc.voxel_eps): eps [nvox] complex128 and
  // alpha^{-1} per (rhs, voxel) in complex128, complex64 and double-float
  void* eps_vox = nullptr;
  void* pv128 = nullptr;
  void* pv64 = nullptr;
  void* pvdf = nullptr;
  void* dainv128 = nullptr;  // d(alpha^{-1})/d(eps) per (rhs, material), entry 0 unused
  int nblk = 1;            // reduction blocks per right-hand side
  // FFT scratch
  void* buf1 = nullptr;
  void* buf2 = nullptr;
  // solver vectors
  void* V = nullptr;       // [(m+1)][rhs][nu] inner precision
  void* Wv = nullptr;      // [rhs][nu] inner precision (A P^-1 v)
  void* Zv = nullptr;      // [rhs][nu] inner precision (P^-1 v)
  void* Wb = nullptr;      // [s][rhs][nu] inner precision: s-step Newton vectors
  void* R128 = nullptr;    // [rhs][nu] complex128 residual
  void* B128 = nullptr;    // [rhs][nu] complex128 right-hand side
  SolverState st{};
  void* err_flag = nullptr;  // int, device status bits of kernels
  size_t total = 0;
};

}  // namespace dda

struct dda_plan_s {
  dda_plan_desc_t d;
  int l, m, n;        // box
  int Lx, Ly, Lz;     // padded transform lengths (2l, 2m, 2n)
  int Lmax;           // largest transform length (twiddle table size)
  long nvox;          // l*m*n
  long P;             // Lx*Ly*Lz
  int hx, hy, hz;     // compressed kernel spectrum extents (L/2 + 1)
  int cx_, cy_, cz_;  // compressed circulant spectrum extents (l/2 + 1, ...)
  int K;              // materials
  int rhs_chunk;      // right-hand sides per pass through the FFT scratch
  const uint8_t* mat;
  std::vector<double> eps;  // 2K
  std::vector<long> mat_count;  // voxels per material 0..K
  dda::Layout w;
  bool has128, has64;
  bool precond_built = false;
  bool precond2_built = false;
  int nrhs_inc = 0;                      // RHS count of the last dda_set_incidence
  bool voxel_eps_on = false;             // dda_set_voxel_eps holds a table
  std::vector<dda_incidence_t> inc;      // incidence per RHS
  std::vector<double> ainv_host;         // [rhs][K+1][2]
  std::vector<float> ainv_host32;
  std::vector<double> dainv_host;        // [rhs][K+1][2]
  int* pinned = nullptr;                 // host-pinned words polled by the solver
  dda::Profiler prof;                    // optional kernel timing
  dda::Schedule sched;                   // launch choices (dda_schedule_set, dda_autotune)
  dda::SolveGraph graph;                 // the last captured solve
  dda::SolveGraph batch;                 // the last batch (dda_solve_many) led by this plan
  long long id = 0;                      // creation number (graph cache keys)
};

namespace dda {

// Loads the no-allocation apply's static scratch into the current context
// (noalloc.cu); dda_plan_create calls it.
dda_status_t noalloc_prepare();

// Layout of a plan's workspace; with ws == nullptr only the size is computed.
bool make_layout(const dda_plan_desc_t& d, void* ws, Layout& L, std::string& why);

// FFT launch helpers (fft_launch.cu), in place when in == out.
template <typename T, bool INV>
void launch_contig(const cx<T>* in, cx<T>* out, const uint8_t* mask, const uint8_t* omask,
                   long mask_lines, long nlines,
                   int L, int Lin, long in_ld, int Lout, long out_ld, T scale, const cx<T>* tw,
                   int Lmax, cudaStream_t s);
template <typename T, bool INV>
void launch_strided(const cx<T>* in, cx<T>* out, long ncols, long nslabs, int L, int Lin,
                    long in_js, long in_ss, int Lout, long out_js, long out_ss, T scale,
                    const cx<T>* tw, int Lmax, cudaStream_t s);
// Full in-place 3-D transform of nbatch arrays [batch][Lz][Ly][Lx].
template <typename T, bool INV>
void fft3d_inplace(cx<T>* data, long nbatch, int Lx, int Ly, int Lz, T scale, const cx<T>* tw,
                   int Lmax, cudaStream_t s);

// Operator pieces (matvec.cu, precond.cu), nrhs fields of the box.
template <typename T>
void matvec_impl(dda_plan_s* p, int nrhs, const cx<T>* x, cx<T>* y, cudaStream_t s);
template <>
void matvec_impl<float>(dda_plan_s* p, int nrhs, const cx<float>* x, cx<float>* y, cudaStream_t s);
template <>
void matvec_impl<double>(dda_plan_s* p, int nrhs, const cx<double>* x, cx<double>* y,
                         cudaStream_t s);
template <typename T>
void precond_apply_impl(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s);
template <typename T>
void precond2_apply(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s);
template <typename T>
void precond_apply_into(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cx<T>* t,
                        cudaStream_t s);

// Templated accessors of the plan's precision-specific buffers.
template <typename T> inline const cx<T>* tw_of(const dda_plan_s* p);
template <> inline const cx<double>* tw_of<double>(const dda_plan_s* p) {
  return static_cast<const cx<double>*>(p->w.tw128);
}
template <> inline const cx<float>* tw_of<float>(const dda_plan_s* p) {
  return static_cast<const cx<float>*>(p->w.tw64);
}
template <> inline const cx<df>* tw_of<df>(const dda_plan_s* p) {
  return static_cast<const cx<df>*>(p->w.twdf);
}
template <typename T> inline const cx<T>* G_of(const dda_plan_s* p);
template <> inline const cx<df>* G_of<df>(const dda_plan_s* p) {
  return static_cast<const cx<df>*>(p->w.Gdf);
}
template <> inline const cx<double>* G_of<double>(const dda_plan_s* p) {
  return static_cast<const cx<double>*>(p->w.G128);
}
template <> inline const cx<float>* G_of<float>(const dda_plan_s* p) {
  return static_cast<const cx<float>*>(p->w.G64);
}
template <typename T> inline const cx<T>* C_of(const dda_plan_s* p);
template <> inline const cx<double>* C_of<double>(const dda_plan_s* p) {
  return static_cast<const cx<double>*>(p->w.C128);
}
template <> inline const cx<float>* C_of<float>(const dda_plan_s* p) {
  return static_cast<const cx<float>*>(p->w.C64);
}
// Per-voxel alpha^{-1} [rhs][nvox] of the plan's precision, or nullptr when
// the plan has no per-voxel permittivity.
template <typename T> inline const cx<T>* pv_of(const dda_plan_s* p);
template <> inline const cx<double>* pv_of<double>(const dda_plan_s* p) {
  return p->voxel_eps_on ? static_cast<const cx<double>*>(p->w.pv128) : nullptr;
}
template <> inline const cx<float>* pv_of<float>(const dda_plan_s* p) {
  return p->voxel_eps_on ? static_cast<const cx<float>*>(p->w.pv64) : nullptr;
}
template <> inline const cx<df>* pv_of<df>(const dda_plan_s* p) {
  return p->voxel_eps_on ? static_cast<const cx<df>*>(p->w.pvdf) : nullptr;
}

template <typename T> inline const cx<T>* ainv_of(const dda_plan_s* p);
template <> inline const cx<double>* ainv_of<double>(const dda_plan_s* p) {
  return static_cast<const cx<double>*>(p->w.ainv128);
}
template <> inline const cx<float>* ainv_of<float>(const dda_plan_s* p) {
  return static_cast<const cx<float>*>(p->w.ainv64);
}
template <> inline const cx<df>* ainv_of<df>(const dda_plan_s* p) {
  return static_cast<const cx<df>*>(p->w.ainvdf);
}

}  // namespace dda
