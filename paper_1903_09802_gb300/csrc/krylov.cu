// Restarted, right-preconditioned GMRES for the DDA system, batched over
// right-hand sides that advance in lock step.
//
// The paper solves with full GMRES and a relative-residual stopping test
// (Section 4) and points to restarted GMRES as the memory-bounded variant
// (Sections 4 and 5).  Here every restart cycle
//   1. recomputes the residual r = b - A x in complex128 (FP64 iterative
//      refinement when the cycle itself runs in complex64; the complex128
//      matvec computes in double-float arithmetic, about 48 bits),
//   2. runs Arnoldi on A P^{-1} from v0 = r/||r||: w = A P^{-1} v_j,
//      classical Gram-Schmidt (h = V^H w, w -= V h) with a second pass when
//      the first left less than eta of ||w|| (selective reorthogonalisation,
//      eta = 1/sqrt(2) by default), FP64
//      Hessenberg column, complex Givens rotations and the residual estimate
//      |g_{j+1}| on the device,
//   3. ends when the estimate reaches max(tol ||b||, inner_tol ||r||), after
//      `restart` steps or on breakdown, then solves the triangular system,
//      forms u = V y and adds P^{-1} u to x in complex128.
// With method = 1 each cycle runs right-preconditioned BiCG-Stab instead
// (restart = iterations per cycle), on the same refinement loop.
// Dots and norms of complex64 vectors multiply in FP32 and sum per thread
// with compensated (Neumaier) FP32 addition, then across threads and blocks
// in FP64 in a fixed order, so results are reproducible run to run; the
// last block of each Gram-Schmidt kernel (ticket counter) does the
// cross-block sum, so no separate reduction launches are needed.
// The host keeps at most two Arnoldi steps queued ahead of the GPU and polls
// a pinned word to stop launching once every right-hand side has finished
// its cycle.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "plan.hpp"

namespace dda {

namespace {

constexpr int kNT = 256;  // threads of the vector kernels
constexpr int kUpdDepth = 5;  // basis vectors in flight per thread in the complex64 update

// Device time in nanoseconds (the global timer of the GPU).
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Control of the solve loop from the device.  When the loop runs as one
// CUDA graph (conditional WHILE and IF nodes), the kernels that decide
// whether another restart cycle or Arnoldi step follows set the graph's
// condition values themselves; graph == 0 is the host-driven loop, whose
// kernels get the step index as an argument and whose host reads the
// decisions back.  The same kernels serve both.
struct LoopCtl {
  int graph;                          // 1: graph-driven (handles valid)
  cudaGraphConditionalHandle h_cycle; // WHILE over restart cycles
  cudaGraphConditionalHandle h_run;   // IF: this cycle has right-hand sides to run
  cudaGraphConditionalHandle h_step;  // WHILE over the steps of a cycle
  int* jstep;                         // step index within the cycle
  int* steps;                         // steps allowed in this cycle
  int* nrun;                          // right-hand sides running this cycle
  long long* nlaunch;                 // kernels run by the graph (counted on the device)
  int k_head, k_run, k_step;          // kernels per cycle head, cycle start + end, step
  const unsigned long long* t0;       // solve start (global timer)
  long long timeout_ns;               // 0: no limit
  double* hist;                       // [rhs][hcap] relative residual per inner iteration
  int hcap;
  int max_iters;
  // s-step GMRES: WHILE over the blocks of a cycle, kernels per block, and
  // the count of cycles started (the first is Arnoldi, later ones blocks)
  cudaGraphConditionalHandle h_blk;
  int k_blk;
  int* scount;                        // nullptr: not s-step
};

// Outcome of one right-hand side, written by k_cycle_decide.
struct RhsOut {
  int conv, nan, cycles, timeout;
  double rel;
  int last_it;  // inner iterations when the last cycle that ran started
  int stalled;  // a cycle ran without a single iteration (BiCG-Stab breakdown)
};
static_assert(sizeof(RhsOut) == kRhsOutBytes, "RhsOut layout");

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warp sum of compensated FP32 pairs (value s, correction c) without FP64
// arithmetic (FP64 runs at 1/58 of the FP32 rate on this GPU); lane 0
// returns s + c in double.
__device__ __forceinline__ double warp_sum_comp(float s, float c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float so = __shfl_down_sync(0xffffffffu, s, o);
    const float co = __shfl_down_sync(0xffffffffu, c, o);
    float e;
    two_sum(s, so, s, e);
    c = c + co + e;
  }
  return (double)s + (double)c;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Per-thread accumulator: plain FP64, or FP32 with Neumaier compensation.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double warp_total() const {
    return warp_sum(make_double2(s, 0.0)).x;
  }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
  __device__ __forceinline__ double warp_total() const { return warp_sum_comp(s, c); }
};

// Sum over the block in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : make_double2(0.0, 0.0);
    v = warp_sum(v);
  }
  return v;
}

// Chunk of a block: an even number of elements, so pairs of complex values
// stay 16-byte aligned when the vector length is even.
__device__ __forceinline__ void chunk_of(long nu, int nblk, long& k0, long& k1) {
  long chunk = (nu + nblk - 1) / nblk;
  chunk += chunk & 1;
  k0 = min(nu, blockIdx.x * chunk);
  k1 = min(nu, k0 + chunk);
}

// Two neighbouring complex values (k, k+1): one 16-byte load in complex64,
// two in complex128.
template <typename T>
struct Pair {
  cx<T> a, b;
};
template <typename T>
__device__ __forceinline__ Pair<T> ld2(const cx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return Pair<T>{mk<T>(v.x, v.y), mk<T>(v.z, v.w)};
  } else {
    return Pair<T>{p[0], p[1]};
  }
}
// The same load without allocating in L1 (normal L2 policy): basis vectors
// stream through once per pass, so they should not evict the w chunk that
// the warps of a block share from L1.
template <typename T>
__device__ __forceinline__ Pair<T> ld2_na(const cx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return Pair<T>{mk<T>(v.x, v.y), mk<T>(v.z, v.w)};
  } else {
    double2 a, b;
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];\n"
                 : "=d"(a.x), "=d"(a.y)
                 : "l"(p));
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];\n"
                 : "=d"(b.x), "=d"(b.y)
                 : "l"(p + 1));
    return Pair<T>{mk<T>(a.x, a.y), mk<T>(b.x, b.y)};
  }
}

template <typename T>
__device__ __forceinline__ void st2(cx<T>* p, const Pair<T>& v) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
  } else {
    p[0] = v.a;
    p[1] = v.b;
  }
}

// partial[(r * nblk + blk) * pst + i] = sum_k conj(V_i[k]) w[k], i < jc (the
// dot products of Gram-Schmidt), eight per sweep over the block's chunk;
// with want_norm also ||w||^2 into slot pst - 2.  Elements are read in
// 16-byte pairs, two pairs per thread and trip, so every thread keeps 18
// wide loads in flight (VEC; the scalar path serves odd vector lengths).
// Each warp reduces its eight sums with shuffles into shared memory, then
// eight threads add the warps' shares in a fixed order.  `mask` selects
// the right-hand sides that take part (active, or needing a second pass).
template <typename T, bool VEC>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? 3 : 1)
    k_multidot(const cx<T>* __restrict__ V, const cx<T>* __restrict__ W, long nu, long vstride,
               int jc, double2* __restrict__ partial, int pst, const int* __restrict__ mask,
               const int* __restrict__ mask2, int want_norm, int* __restrict__ tickets,
               double2* __restrict__ hcol, double2* __restrict__ H, int m, int j, int pass,
               double* __restrict__ scal, const int* __restrict__ jdev) {
  pdl_entry();
  if (jdev != nullptr) {  // graph-driven loop: the step index lives on the device
    j = *jdev;
    jc = j + 1;
  }
  constexpr int ND = 8;
  constexpr int NW = kNT / 32;
  __shared__ double2 sh[ND][NW];
  __shared__ int s_last;
  const int r = blockIdx.y;
  if (!mask[r] || (mask2 != nullptr && !mask2[r])) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  const cx<T>* w = W + r * nu;
  const cx<T>* vb = V + r * nu;
  double2* out = partial + ((long)r * gridDim.x + blockIdx.x) * pst;
  const int ntot = jc + (want_norm ? 1 : 0);  // index jc stands for ||w||^2
  for (int i0 = 0; i0 < ntot; i0 += ND) {
    Acc<T> ar[ND], ai[ND];
    auto acc = [&](int d, const cx<T>& vk, const cx<T>& wk) {
      ar[d].add(vk.x * wk.x + vk.y * wk.y);
      ai[d].add(vk.x * wk.y - vk.y * wk.x);
    };
    if (VEC) {
      for (long k = k0 + 2 * threadIdx.x; k < k1; k += 2 * kNT) {
        const Pair<T> w0 = ld2(w + k);
        Pair<T> v0[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          const int i = i0 + d;
          v0[d] = i < jc ? ld2(vb + (long)i * vstride + k) : w0;  // i == jc: ||w||^2
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          if (i0 + d < ntot) {
            acc(d, v0[d].a, w0.a);
            acc(d, v0[d].b, w0.b);
          }
        }
      }
    } else {
      for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
        const cx<T> wk = w[k];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          const int i = i0 + d;
          if (i < jc) acc(d, vb[(long)i * vstride + k], wk);
          else if (i == jc && want_norm) acc(d, wk, wk);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const double tr = ar[d].warp_total();
      const double ti = ai[d].warp_total();
      if (lane == 0) sh[d][wid] = make_double2(tr, ti);
    }
    __syncthreads();
    if (threadIdx.x < ND && i0 + (int)threadIdx.x < ntot) {
      double2 a = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        a.x += sh[threadIdx.x][q].x;
        a.y += sh[threadIdx.x][q].y;
      }
      const int i = i0 + threadIdx.x;
      out[i < jc ? i : pst - 2] = a;
    }
    __syncthreads();
  }
  // The last block of this right-hand side to finish adds the blocks'
  // partial sums (warp i handles slots i, i + 8, ...; lanes stride over the
  // blocks in a fixed order) and writes the Hessenberg column.  Every
  // writer fences its partials before the barrier that precedes the ticket.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tickets[r], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nblk = gridDim.x;
  for (int i = wid; i < ntot; i += NW) {
    const int slot = i < jc ? i : pst - 2;
    double2 a = make_double2(0.0, 0.0);
    for (int b = lane; b < nblk; b += 32) {
      const double2 v = __ldcg(&partial[((long)r * nblk + b) * pst + slot]);
      a.x += v.x;
      a.y += v.y;
    }
    a = warp_sum(a);
    if (lane == 0) {
      if (i < jc) {
        hcol[(long)r * (m + 2) + i] = a;
        double2* h = H + (long)r * (m + 1) * m + (long)j * (m + 1) + i;
        if (pass == 0) {
          *h = a;
        } else {
          h->x += a.x;
          h->y += a.y;
        }
      } else {
        scal[(long)r * 16 + 7] = a.x;  // ||w||^2 before Gram-Schmidt
      }
    }
  }
  if (threadIdx.x == 0) tickets[r] = 0;
}

// The same dot products with one warp per basis vector: warp q of a block
// sums conj(V_i[k]) w[k] over the block's chunk for i = q, q + NW, ...
// (index jc stands for ||w||^2), one compensated accumulator pair per lane
// and one shuffle reduction per vector, no block barrier between vectors.
// w is re-read by every warp of the block from L1.  Needs an even vector
// length (16-byte pairs).  The last block of each right-hand side sums the
// blocks' partials (four slots per warp at a time) into the Hessenberg
// column as k_multidot does.
constexpr int kDotNT = 128;
template <typename T>
__global__ void __launch_bounds__(kDotNT)
    k_dots_w(const cx<T>* __restrict__ V, const cx<T>* __restrict__ W, long nu, long vstride,
             int jc, double2* __restrict__ partial, int pst, const int* __restrict__ mask,
             const int* __restrict__ mask2, int want_norm, int* __restrict__ tickets,
             double2* __restrict__ hcol, double2* __restrict__ H, int m, int j, int pass,
             double* __restrict__ scal, const int* __restrict__ jdev) {
  pdl_entry();
  if (jdev != nullptr) {
    j = *jdev;
    jc = j + 1;
  }
  constexpr int NW = kDotNT / 32;
  __shared__ int s_last;
  const int r = blockIdx.y;
  if (!mask[r] || (mask2 != nullptr && !mask2[r])) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  const cx<T>* w = W + r * nu;
  const cx<T>* vb = V + r * nu;
  double2* out = partial + ((long)r * gridDim.x + blockIdx.x) * pst;
  const int ntot = jc + (want_norm ? 1 : 0);
  for (int i = wid; i < ntot; i += NW) {
    Acc<T> ar, ai;
    // Trips go in batches of U whose loads are all issued before the first
    // use (a tail trip past k1 is masked, not run on its own), so a lane
    // keeps U loads in flight down to the end of its chunk.
    constexpr int U = sizeof(T) == 4 ? 4 : 2;
    if (i < jc) {
      const cx<T>* v = vb + (long)i * vstride;
      for (long kb = k0 + 2 * lane; kb < k1; kb += 64 * U) {
        Pair<T> a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long k = kb + 64 * u;
          if (k < k1) {
            a[u] = ld2_na(v + k);
            b[u] = ld2(w + k);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (kb + 64 * u < k1) {
            ar.add(a[u].a.x * b[u].a.x + a[u].a.y * b[u].a.y);
            ai.add(a[u].a.x * b[u].a.y - a[u].a.y * b[u].a.x);
            ar.add(a[u].b.x * b[u].b.x + a[u].b.y * b[u].b.y);
            ai.add(a[u].b.x * b[u].b.y - a[u].b.y * b[u].b.x);
          }
        }
      }
    } else {
      for (long kb = k0 + 2 * lane; kb < k1; kb += 64 * U) {
        Pair<T> b[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (kb + 64 * u < k1) b[u] = ld2(w + kb + 64 * u);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (kb + 64 * u < k1) {
            ar.add(norm2(b[u].a));
            ar.add(norm2(b[u].b));
          }
        }
      }
    }
    const double tr = ar.warp_total();
    const double ti = ai.warp_total();
    if (lane == 0) out[i < jc ? i : pst - 2] = make_double2(tr, ti);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tickets[r], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nblk = gridDim.x;
  constexpr int SB = 4;  // slots per warp at a time: more loads in flight
  for (int i0 = wid * SB; i0 < ntot; i0 += NW * SB) {
    double2 a[SB];
#pragma unroll
    for (int u = 0; u < SB; ++u) a[u] = make_double2(0.0, 0.0);
    for (int b = lane; b < nblk; b += 32) {
      const double2* pb = partial + ((long)r * nblk + b) * pst;
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int i = i0 + u;
        if (i < ntot) {
          const double2 v = __ldcg(pb + (i < jc ? i : pst - 2));
          a[u].x += v.x;
          a[u].y += v.y;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < SB; ++u) {
      const int i = i0 + u;
      const double2 t = warp_sum(a[u]);
      if (lane == 0 && i < ntot) {
        if (i < jc) {
          hcol[(long)r * (m + 2) + i] = t;
          double2* h = H + (long)r * (m + 1) * m + (long)j * (m + 1) + i;
          if (pass == 0) {
            *h = t;
          } else {
            h->x += t.x;
            h->y += t.y;
          }
        } else {
          scal[(long)r * 16 + 7] = t.x;  // ||w||^2 before Gram-Schmidt
        }
      }
    }
  }
  if (threadIdx.x == 0) tickets[r] = 0;
}

// w -= sum_{i < jc} h_i V_i, and the block's share of ||w||^2 into
// partial[...][pst - 1].  16-byte pairs, two per thread and trip (VEC).
template <typename T, bool VEC>
__global__ void __launch_bounds__(kNT)
    k_update(const cx<T>* __restrict__ V, cx<T>* __restrict__ W, long nu, long vstride, int jc,
             const double2* __restrict__ hcol, int m, double2* __restrict__ partial, int pst,
             const int* __restrict__ mask, const int* __restrict__ mask2, int* __restrict__ tickets,
             double* __restrict__ scal, int pass, int* __restrict__ reorth,
             int* __restrict__ reorth_count, double eta2, const int* __restrict__ jdev) {
  pdl_entry();
  if (jdev != nullptr) jc = *jdev + 1;
  __shared__ cx<T> hs[520];
  __shared__ double2 sh[32];
  __shared__ int s_last;
  // Blocks run roughly in launch order; the dots pass just walked the basis
  // from the first right-hand side's first chunk to the last one's last
  // chunk, so this pass walks it backwards and starts on what is still in L2.
  const int r = gridDim.y - 1 - blockIdx.y;
  if (!mask[r] || (mask2 != nullptr && !mask2[r])) return;
  for (int i = threadIdx.x; i < jc; i += kNT) {
    const double2 h = hcol[(long)r * (m + 2) + i];
    hs[i] = mk<T>((T)h.x, (T)h.y);
  }
  __syncthreads();
  long k0, k1;
  {
    long chunk = (nu + gridDim.x - 1) / gridDim.x;
    chunk += chunk & 1;
    k0 = min(nu, (long)(gridDim.x - 1 - blockIdx.x) * chunk);
    k1 = min(nu, k0 + chunk);
  }
  cx<T>* w = W + r * nu;
  const cx<T>* vb = V + r * nu;
  Acc<T> nn;
  if constexpr (VEC && sizeof(T) == 4) {
    // complex64: the basis pairs a thread needs are copied asynchronously
    // into its own slots of a shared ring, kUpdDepth basis vectors ahead,
    // so many loads stay in flight without holding registers (the update is
    // bound by memory latency otherwise).  Each thread reads only what it
    // copied itself: no block barrier; the arithmetic and its order are
    // those of the plain loop.
    constexpr int D = kUpdDepth;
    __shared__ float4 ring[D][2][kNT];
    const int tid = threadIdx.x;
    auto copy = [&](int slot, int i, long k, bool two) {
      const cx<T>* src = vb + (long)i * vstride + k;
      const unsigned d0 = (unsigned)__cvta_generic_to_shared(&ring[slot][0][tid]);
      const unsigned d1 = (unsigned)__cvta_generic_to_shared(&ring[slot][1][tid]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d0), "l"(src) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d1),
                   "l"(two ? src + 2 * kNT : src), "r"(two ? 16 : 0)
                   : "memory");
    };
    for (long k = k0 + 2 * tid; k < k1; k += 4 * kNT) {
      const bool two = k + 2 * kNT < k1;
      Pair<T> a0 = ld2(w + k);
      Pair<T> a1 = two ? ld2(w + k + 2 * kNT) : Pair<T>{zero<T>(), zero<T>()};
#pragma unroll
      for (int q = 0; q < D; ++q) {
        if (q < jc) copy(q, q, k, two);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
      int slot = 0;
      for (int i = 0; i < jc; ++i) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 1) : "memory");
        const float4 p0 = ring[slot][0][tid], p1 = ring[slot][1][tid];
        const cx<T> h = hs[i];
        a0.a = a0.a - h * mk<T>(p0.x, p0.y);
        a0.b = a0.b - h * mk<T>(p0.z, p0.w);
        a1.a = a1.a - h * mk<T>(p1.x, p1.y);
        a1.b = a1.b - h * mk<T>(p1.z, p1.w);
        // refill the slot just consumed (its values are in registers and used)
        if (i + D < jc) copy(slot, i + D, k, two);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        slot = slot + 1 == D ? 0 : slot + 1;
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      st2(w + k, a0);
      nn.add(norm2(a0.a));
      nn.add(norm2(a0.b));
      if (two) {
        st2(w + k + 2 * kNT, a1);
        nn.add(norm2(a1.a));
        nn.add(norm2(a1.b));
      }
    }
  } else if (VEC) {
    for (long k = k0 + 2 * threadIdx.x; k < k1; k += 4 * kNT) {
      const bool two = k + 2 * kNT < k1;
      Pair<T> a0 = ld2(w + k);
      Pair<T> a1 = two ? ld2(w + k + 2 * kNT) : Pair<T>{zero<T>(), zero<T>()};
#pragma unroll 8
      for (int i = 0; i < jc; ++i) {
        const cx<T> h = hs[i];
        const Pair<T> v0 = ld2(vb + (long)i * vstride + k);
        const Pair<T> v1 = two ? ld2(vb + (long)i * vstride + k + 2 * kNT) : Pair<T>{zero<T>(), zero<T>()};
        a0.a = a0.a - h * v0.a;
        a0.b = a0.b - h * v0.b;
        a1.a = a1.a - h * v1.a;
        a1.b = a1.b - h * v1.b;
      }
      st2(w + k, a0);
      nn.add(norm2(a0.a));
      nn.add(norm2(a0.b));
      if (two) {
        st2(w + k + 2 * kNT, a1);
        nn.add(norm2(a1.a));
        nn.add(norm2(a1.b));
      }
    }
  } else {
    for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
      cx<T> acc = w[k];
      for (int i = 0; i < jc; ++i) acc = acc - hs[i] * vb[(long)i * vstride + k];
      w[k] = acc;
      nn.add(norm2(acc));
    }
  }
  const double2 t = block_sum(make_double2(nn.get(), 0.0), sh);
  if (threadIdx.x == 0) partial[((long)r * gridDim.x + blockIdx.x) * pst + pst - 1] = t;
  // Last block: ||w||^2 after this pass, and after the first pass the
  // selective-reorthogonalisation test (Daniel, Gragg, Kaufman & Stewart):
  // a second pass runs when ||w_after||^2 < eta^2 ||w_before||^2.
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(&tickets[r], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  double n2 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
    n2 += __ldcg(&partial[((long)r * gridDim.x + b) * pst + pst - 1]).x;
  n2 = warp_sum(make_double2(n2, 0.0)).x;
  if (threadIdx.x == 0) {
    scal[(long)r * 16 + 8] = n2;
    if (pass == 0) {
      const int need = !(n2 >= eta2 * scal[(long)r * 16 + 7]);
      reorth[r] = need;
      reorth_count[r] += need;
    }
    tickets[r] = 0;
  }
}

// Complex Givens rotation [c s; -conj(s) c] with real c taking (a, b) to (rho, 0).
__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& rho) {
  const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
  if (nb == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
    rho = a;
    return;
  }
  if (na == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    rho = b;
    return;
  }
  const double nr = hypot(na, nb);
  c = na / nr;
  const double2 ph = make_double2(a.x / na, a.y / na);  // a/|a|
  // s = (a/|a|) conj(b) / nr
  s = make_double2((ph.x * b.x + ph.y * b.y) / nr, (ph.y * b.x - ph.x * b.y) / nr);
  rho = make_double2(ph.x * nr, ph.y * nr);
}

// One warp per right-hand side: the warp stages column j of H and the
// earlier rotations in shared memory with parallel loads, lane 0 applies the
// rotations (a dependent chain: from shared memory it takes cycles, not
// memory latencies), computes the new rotation, updates g and the residual
// estimate and decides whether the cycle of this right-hand side goes on; the
// warp writes the column back.  With count_out, the last block (ticket) also
// counts the right-hand sides still iterating.
__global__ void __launch_bounds__(32)
    k_givens(double2* __restrict__ H, double* __restrict__ cs, double2* __restrict__ sn,
             double2* __restrict__ g, double* __restrict__ scal, int* __restrict__ active,
             int* __restrict__ jlen, int* __restrict__ flags, int* __restrict__ iters, int nrhs,
             int m, int j, double brk, int* __restrict__ count_out, int* __restrict__ ticket,
             LoopCtl ctl, double2* __restrict__ Hraw) {
  pdl_entry();
  if (ctl.graph) j = *ctl.jstep;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* hs = reinterpret_cast<double2*>(smem_raw);  // [j + 2]
  double2* ss = hs + (j + 2);                           // [j]
  double* cc = reinterpret_cast<double*>(ss + j);       // [j]
  const int r = blockIdx.x, lane = threadIdx.x;
  if (active[r]) {
    double2* h = H + (long)r * (m + 1) * m + (long)j * (m + 1);
    double* c = cs + (long)r * m;
    double2* sv = sn + (long)r * m;
    for (int i = lane; i <= j; i += 32) hs[i] = h[i];
    for (int i = lane; i < j; i += 32) {
      ss[i] = sv[i];
      cc[i] = c[i];
    }
    __syncwarp();
    if (Hraw != nullptr) {  // the unrotated column (s-step shifts come from it)
      double2* hr = Hraw + (long)r * (m + 1) * m + (long)j * (m + 1);
      for (int i = lane; i <= j; i += 32) hr[i] = hs[i];
      if (lane == 0) hr[j + 1] = make_double2(sqrt(scal[(long)r * 16 + 8]), 0.0);
    }
    if (lane == 0) {
      const double n2 = scal[(long)r * 16 + 8];  // ||w||^2 after Gram-Schmidt
      const double hn = sqrt(n2);
      double colnorm2 = n2;
      for (int i = 0; i <= j; ++i) colnorm2 += hs[i].x * hs[i].x + hs[i].y * hs[i].y;
      for (int i = 0; i < j; ++i) {
        const double2 a = hs[i], b = hs[i + 1], si = ss[i];
        const double ci = cc[i];
        hs[i] = make_double2(ci * a.x + (si.x * b.x - si.y * b.y),
                             ci * a.y + (si.x * b.y + si.y * b.x));
        // -conj(s) a + c b
        hs[i + 1] = make_double2(-(si.x * a.x + si.y * a.y) + ci * b.x,
                                 -(si.x * a.y - si.y * a.x) + ci * b.y);
      }
      double cj;
      double2 sj, rho;
      givens(hs[j], make_double2(hn, 0.0), cj, sj, rho);
      c[j] = cj;
      sv[j] = sj;
      hs[j] = rho;
      hs[j + 1] = make_double2(0.0, 0.0);
      double2* gg = g + (long)r * (m + 1);
      const double2 gj = gg[j];
      gg[j + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));
      gg[j] = make_double2(cj * gj.x, cj * gj.y);
      const double res = hypot(gg[j + 1].x, gg[j + 1].y);
      double* sc = scal + (long)r * 16;
      sc[4] = res;
      sc[5] = hn > 0.0 ? 1.0 / hn : 0.0;
      jlen[r] = j + 1;
      const int it = iters[r] + 1;
      iters[r] = it;
      if (ctl.hist != nullptr && it < ctl.hcap) {
        const double bn = sc[2];
        ctl.hist[(long)r * ctl.hcap + it] = bn > 0.0 ? res / bn : res;
      }
      if (ctl.timeout_ns > 0 && (long long)(now_ns() - *ctl.t0) > ctl.timeout_ns) {
        flags[r] |= 4;  // time limit of the solve reached
        active[r] = 0;
      } else if (!isfinite(res) || !isfinite(hn)) {
        flags[r] |= 1;
        active[r] = 0;
      } else if (res <= sc[3]) {
        active[r] = 0;
      } else if (hn <= brk * sqrt(colnorm2)) {
        flags[r] |= 2;  // breakdown: the Krylov space is invariant, the cycle's solution is exact
        active[r] = 0;
      } else if (it >= ctl.max_iters) {
        active[r] = 0;  // this right-hand side's iteration cap
      }
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += 32) h[i] = hs[i];
  }
  if (count_out != nullptr) {
    __shared__ int s_last;
    __threadfence();
    if (lane == 0) s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncwarp();
    if (s_last) {
      __threadfence();
      int cnt = 0;
      for (int q = lane; q < nrhs; q += 32) cnt += __ldcg(&active[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      if (lane == 0) {
        *count_out = cnt;
        *ticket = 0;
        if (ctl.graph) {  // the next step runs while some RHS iterate and the cycle has room
          const int jn = j + 1;
          *ctl.jstep = jn;
          cudaGraphSetConditional(ctl.h_step, (cnt > 0 && jn < *ctl.steps) ? 1u : 0u);
          *ctl.nlaunch += ctl.k_step;
        }
      }
    }
  }
}

// v_{j+1} = w / h_{j+1,j} into the basis (slot Vn, or with jdev the slot of
// the device's step index, which the Givens kernel has just advanced), and
// the same vector into Zc when given: the graph-driven loop feeds the next
// step's preconditioner and matvec from that fixed buffer.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_scale(const cx<T>* __restrict__ W, cx<T>* __restrict__ Vn, long nu,
            const double* __restrict__ scal, const int* __restrict__ active,
            cx<T>* __restrict__ V, long vstride, const int* __restrict__ jdev,
            cx<T>* __restrict__ Zc) {
  pdl_entry();
  const int r = blockIdx.y;
  if (!active[r]) return;
  if (jdev != nullptr) Vn = V + (long)(*jdev) * vstride;
  const T inv = (T)scal[(long)r * 16 + 5];
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const cx<T> v = inv * W[r * nu + k];
    Vn[r * nu + k] = v;
    if (Zc != nullptr) Zc[r * nu + k] = v;
  }
}

// Number of right-hand sides still iterating (one warp).  Also the
// BiCG-Stab loop's step control: the time limit, the residual history
// (sqrt of bs[10], the last ||r||^2, relative to ||b||) and, graph-driven,
// the next step's condition.
__global__ void k_count_active(int* __restrict__ active, int nrhs, int* __restrict__ out,
                               int* __restrict__ flags, const int* __restrict__ iters,
                               const double* __restrict__ bs, const double* __restrict__ scal,
                               LoopCtl ctl) {
  pdl_entry();
  const bool late = ctl.timeout_ns > 0 && (long long)(now_ns() - *ctl.t0) > ctl.timeout_ns;
  int c = 0;
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    if (late && active[r]) {
      flags[r] |= 4;
      active[r] = 0;
    }
    c += active[r];
    const int it = iters[r];
    if (ctl.hist != nullptr && it < ctl.hcap && bs != nullptr) {
      const double bn = scal[(long)r * 16 + 2], rn = sqrt(bs[(long)r * 16 + 10]);
      ctl.hist[(long)r * ctl.hcap + it] = bn > 0.0 ? rn / bn : rn;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if (threadIdx.x == 0) {
    *out = c;
    if (ctl.graph) {
      const int jn = *ctl.jstep + 1;
      *ctl.jstep = jn;
      cudaGraphSetConditional(ctl.h_step, (c > 0 && jn < *ctl.steps) ? 1u : 0u);
      *ctl.nlaunch += ctl.k_step;
    }
  }
}

// Start of a restart cycle, after the FP64 residual: per right-hand side
// converged (||r|| <= tol ||b||), non-finite, out of time or out of
// iterations, or running another cycle; the cycle's step count (restart
// length, at most the iterations the running RHS have left); the true
// relative residual into the history at the current iteration count.
// Graph-driven, it sets the conditions of the cycle loop, of this cycle's
// body and of its step loop.  One block.
__global__ void __launch_bounds__(256)
    k_cycle_decide(const double* __restrict__ scal, const int* __restrict__ iters,
                   int* __restrict__ flags, int* __restrict__ run, RhsOut* __restrict__ out,
                   int nrhs, double tol, int m, LoopCtl ctl) {
  pdl_entry();
  __shared__ int s_n[8], s_l[8];
  const bool late = ctl.timeout_ns > 0 && (long long)(now_ns() - *ctl.t0) > ctl.timeout_ns;
  int nrun = 0, left = 0;
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    const double bn = scal[(long)r * 16 + 2], rn = scal[(long)r * 16 + 6];
    const double rel = bn > 0.0 ? rn / bn : rn;
    const int nan = !isfinite(rn) || (flags[r] & 1);
    const int conv = isfinite(rn) && (rn <= tol * bn || bn == 0.0);
    if (late && !conv && !nan) flags[r] |= 4;
    const int to = (flags[r] & 4) != 0;
    const int it = iters[r];
    RhsOut o = out[r];
    // a cycle that ended without one iteration (a breakdown at its first
    // step) would repeat forever: such a right-hand side stops here, and so
    // does any that has run more cycles than it has iterations to spend
    const int stalled = o.stalled || (o.cycles > 0 && it == o.last_it) ||
                        o.cycles > ctl.max_iters;
    const int rr = !conv && !nan && !to && !stalled && it < ctl.max_iters;
    run[r] = rr;
    o.conv = conv;
    o.nan = nan;
    o.timeout = to && !conv;
    o.rel = rel;
    o.stalled = stalled && !conv;
    o.cycles += rr;
    if (rr) o.last_it = it;
    out[r] = o;
    if (ctl.hist != nullptr && it < ctl.hcap) ctl.hist[(long)r * ctl.hcap + it] = rel;
    nrun += rr;
    if (rr) left = max(left, ctl.max_iters - it);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrun += __shfl_down_sync(0xffffffffu, nrun, o);
    left = max(left, __shfl_down_sync(0xffffffffu, left, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_n[wid] = nrun;
    s_l[wid] = left;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0, l = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      n += s_n[w];
      l = max(l, s_l[w]);
    }
    const int steps = min(m, l);
    *ctl.steps = steps;
    *ctl.jstep = 0;
    *ctl.nrun = n;
    // s-step: the first cycle that runs is Arnoldi, the later ones blocks
    const int started = ctl.scount != nullptr ? *ctl.scount : 0;
    const bool blk = ctl.scount != nullptr && started >= 1;
    if (ctl.scount != nullptr && n > 0) *ctl.scount = started + 1;
    if (ctl.graph) {
      cudaGraphSetConditional(ctl.h_cycle, n > 0 ? 1u : 0u);
      cudaGraphSetConditional(ctl.h_run, n > 0 ? 1u : 0u);
      cudaGraphSetConditional(ctl.h_step, (n > 0 && steps > 0 && !blk) ? 1u : 0u);
      if (ctl.scount != nullptr)
        cudaGraphSetConditional(ctl.h_blk, (n > 0 && steps > 0 && blk) ? 1u : 0u);
      *ctl.nlaunch += ctl.k_head + (n > 0 ? ctl.k_run : 0);
    }
  }
}

// Start of the solve: the global timer's reading for the time limit.
__global__ void k_solve_begin(unsigned long long* __restrict__ t0) {
  pdl_entry();
  *t0 = now_ns();
}

// Back substitution R y = g with the rotated (upper triangular) H.
__global__ void k_trisolve(const double2* __restrict__ H, const double2* __restrict__ g,
                           const int* __restrict__ jlen, double2* __restrict__ y, int nrhs, int m) {
  pdl_entry();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int jl = jlen[r];
  const double2* h = H + (long)r * (m + 1) * m;
  const double2* gg = g + (long)r * (m + 1);
  double2* yy = y + (long)r * m;
  for (int i = jl - 1; i >= 0; --i) {
    double2 acc = gg[i];
    for (int k = i + 1; k < jl; ++k) {
      const double2 a = h[(long)k * (m + 1) + i], b = yy[k];
      acc.x -= a.x * b.x - a.y * b.y;
      acc.y -= a.x * b.y + a.y * b.x;
    }
    const double2 d = h[(long)i * (m + 1) + i];
    const double dn = d.x * d.x + d.y * d.y;
    yy[i] = dn > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn)
                     : make_double2(0.0, 0.0);
  }
}

// u = sum_{i < jlen} y_i V_i.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_combine(const cx<T>* __restrict__ V, const double2* __restrict__ y,
              const int* __restrict__ jlen, cx<T>* __restrict__ U, long nu, long vstride, int m) {
  pdl_entry();
  __shared__ cx<T> ys[520];
  const int r = blockIdx.y;
  const int jl = jlen[r];
  for (int i = threadIdx.x; i < jl; i += kNT) {
    const double2 v = y[(long)r * m + i];
    ys[i] = mk<T>((T)v.x, (T)v.y);
  }
  __syncthreads();
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  const cx<T>* vb = V + r * nu;
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    cx<T> acc = zero<T>();
    for (int i = 0; i < jl; ++i) acc = acc + ys[i] * vb[(long)i * vstride + k];
    U[r * nu + k] = acc;
  }
}

// x += z (complex128 += inner precision) for right-hand sides that iterated.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_add_x(double2* __restrict__ x, const cx<T>* __restrict__ z, const int* __restrict__ jlen,
            long nu) {
  pdl_entry();
  const int r = blockIdx.y;
  if (jlen[r] == 0) return;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const cx<T> v = z[r * nu + k];
    double2 a = x[r * nu + k];
    a.x += (double)v.x;
    a.y += (double)v.y;
    x[r * nu + k] = a;
  }
}

// r = b - (A x) in place on ax; block shares of ||r||^2 and ||b||^2.
__global__ void __launch_bounds__(kNT)
    k_residual(const double2* __restrict__ b, double2* __restrict__ ax, long nu,
               double2* __restrict__ part) {
  pdl_entry();
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  double rr = 0.0, bb = 0.0;
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const double2 bv = b[r * nu + k];
    const double2 av = ax[r * nu + k];
    const double2 d = make_double2(bv.x - av.x, bv.y - av.y);
    ax[r * nu + k] = d;
    rr += d.x * d.x + d.y * d.y;
    bb += bv.x * bv.x + bv.y * bv.y;
  }
  const double2 t = block_sum(make_double2(rr, bb), sh);
  if (threadIdx.x == 0) part[(long)r * gridDim.x + blockIdx.x] = t;
}

__global__ void k_finish_norms(const double2* __restrict__ part, int nblk, int nrhs,
                               double* __restrict__ scal) {
  pdl_entry();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double rr = 0.0, bb = 0.0;
  for (int b = 0; b < nblk; ++b) {
    rr += part[(long)r * nblk + b].x;
    bb += part[(long)r * nblk + b].y;
  }
  scal[(long)r * 16 + 6] = sqrt(rr);
  scal[(long)r * 16 + 2] = sqrt(bb);
}

// Start a cycle: v0 = r/||r||, g = (||r||, 0, ...), target estimate, flags.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_start_cycle(const double2* __restrict__ R, cx<T>* __restrict__ V0, long nu,
                  double* __restrict__ scal, double2* __restrict__ g, int m,
                  const int* __restrict__ run, int* __restrict__ active, int* __restrict__ jlen,
                  double tol, double inner_tol, cx<T>* __restrict__ Zc) {
  pdl_entry();
  const int r = blockIdx.y;
  const double beta = scal[(long)r * 16 + 6];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    active[r] = run[r];
    jlen[r] = 0;
    g[(long)r * (m + 1)] = make_double2(beta, 0.0);
    scal[(long)r * 16 + 0] = beta;
    scal[(long)r * 16 + 3] = fmax(tol * scal[(long)r * 16 + 2], inner_tol * beta);
  }
  if (!run[r] || !(beta > 0.0)) return;
  const double inv = 1.0 / beta;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const double2 v = R[r * nu + k];
    const cx<T> w = mk<T>((T)(v.x * inv), (T)(v.y * inv));
    V0[r * nu + k] = w;
    if (Zc != nullptr) Zc[r * nu + k] = w;
  }
}

// ---------------------------------------------------------------------------
// BiCG-Stab (van der Vorst), right-preconditioned, the paper's second solver
// (Section 4).  Per right-hand side the device holds rho, alpha, omega and two
// dot products in bs[r * 16 + ...]: 0-1 rho, 2-3 alpha, 4-5 omega, 6-7 dot A,
// 8-9 dot B, 10 ||s||^2 or ||r||^2, 11 target^2, 12 state (1: converged at the
// half step).

// bs[slot..slot+1] = conj(a) . b per right-hand side, and optionally
// bs[slot+2..slot+3] = conj(a2) . b2; last block reduces in a fixed order.
template <typename T, int ND>
__global__ void __launch_bounds__(kNT)
    k_bdots(const cx<T>* __restrict__ a, const cx<T>* __restrict__ b,
            const cx<T>* __restrict__ a2, const cx<T>* __restrict__ b2, long nu,
            const int* __restrict__ mask, double2* __restrict__ partial,
            int* __restrict__ tickets, double* __restrict__ bs, int slot) {
  pdl_entry();
  __shared__ double2 sh[ND][kNT / 32];
  __shared__ int s_last;
  const int r = blockIdx.y;
  if (!mask[r]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  Acc<T> ar[ND], ai[ND];
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const cx<T> x = a[r * nu + k], y = b[r * nu + k];
    ar[0].add(x.x * y.x + x.y * y.y);
    ai[0].add(x.x * y.y - x.y * y.x);
    if (ND > 1) {
      const cx<T> x2 = a2[r * nu + k], y2 = b2[r * nu + k];
      ar[ND - 1].add(x2.x * y2.x + x2.y * y2.y);
      ai[ND - 1].add(x2.x * y2.y - x2.y * y2.x);
    }
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const double tr = ar[d].warp_total(), ti = ai[d].warp_total();
    if (lane == 0) sh[d][wid] = make_double2(tr, ti);
  }
  __syncthreads();
  if (threadIdx.x < ND) {
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < kNT / 32; ++q) {
      acc.x += sh[threadIdx.x][q].x;
      acc.y += sh[threadIdx.x][q].y;
    }
    partial[((long)r * gridDim.x + blockIdx.x) * ND + threadIdx.x] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&tickets[r], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  for (int d = 0; d < ND; ++d) {
    double2 acc = make_double2(0.0, 0.0);
    for (int bb = threadIdx.x; bb < (int)gridDim.x; bb += 32) {
      const double2 v = __ldcg(&partial[((long)r * gridDim.x + bb) * ND + d]);
      acc.x += v.x;
      acc.y += v.y;
    }
    acc = warp_sum(acc);
    if (threadIdx.x == 0) {
      bs[(long)r * 16 + slot + 2 * d] = acc.x;
      bs[(long)r * 16 + slot + 2 * d + 1] = acc.y;
    }
  }
  if (threadIdx.x == 0) tickets[r] = 0;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double dn = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / dn, (a.y * b.x - a.x * b.y) / dn);
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// op 0: beta = (rho_new/rho)(alpha/omega) -> slots 8-9, rho = rho_new (dot A);
// op 1: alpha = rho / (rhat . v) (dot A); op 2: omega = (t . s)/(t . t) (dots A, B);
// op 3: mark the half-step correction of d as applied.
// A zero denominator is a breakdown: the cycle of that right-hand side ends.
__global__ void k_bscalar(int op, double* __restrict__ bs, int* __restrict__ active,
                          int* __restrict__ flags, int nrhs) {
  pdl_entry();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double* q = bs + (long)r * 16;
  if (op == 3) {  // the half-step update of d has been applied
    if (q[12] == 1.0) q[12] = 2.0;
    return;
  }
  if (!active[r]) return;
  const double2 rho = make_double2(q[0], q[1]), alpha = make_double2(q[2], q[3]);
  const double2 omega = make_double2(q[4], q[5]), da = make_double2(q[6], q[7]);
  const double2 db = make_double2(q[8], q[9]);
  double2 out;
  if (op == 0) {
    if (!(rho.x * rho.x + rho.y * rho.y > 0.0) || !(omega.x * omega.x + omega.y * omega.y > 0.0)) {
      flags[r] |= 2;
      active[r] = 0;
      return;
    }
    out = cmul2(cdiv(da, rho), cdiv(alpha, omega));
    q[0] = da.x;
    q[1] = da.y;
    q[8] = out.x;
    q[9] = out.y;
  } else if (op == 1) {
    if (!(da.x * da.x + da.y * da.y > 0.0)) {
      flags[r] |= 2;
      active[r] = 0;
      return;
    }
    out = cdiv(rho, da);
    q[2] = out.x;
    q[3] = out.y;
  } else {
    if (!(db.x * db.x + db.y * db.y > 0.0)) {
      flags[r] |= 2;
      active[r] = 0;
      return;
    }
    out = cdiv(da, db);
    q[4] = out.x;
    q[5] = out.y;
  }
  if (!isfinite(out.x) || !isfinite(out.y)) {
    flags[r] |= 1;
    active[r] = 0;
  }
}

// mode 0: p = r + beta (p - omega v)
// mode 1: s = r - alpha v, and ||s||^2 (last block: converged at the half step?)
// mode 2: d += alpha ph (right-hand sides converged at the half step only)
// mode 3: d += alpha ph + omega sh, r = s - omega t, and ||r||^2 (last block:
//         converged?)
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_baxpy(int mode, cx<T>* __restrict__ X, cx<T>* __restrict__ Y, const cx<T>* __restrict__ A1,
            const cx<T>* __restrict__ A2, const cx<T>* __restrict__ A3,
            cx<T>* __restrict__ D, long nu, const double* __restrict__ bs_in,
            double* __restrict__ bs, int* __restrict__ active, int* __restrict__ iters,
            double2* __restrict__ partial, int* __restrict__ tickets) {
  pdl_entry();
  __shared__ double2 sh[32];
  __shared__ int s_last;
  const int r = blockIdx.y;
  const double* q = bs_in + (long)r * 16;
  if (mode == 2) {
    if (q[12] != 1.0) return;
  } else if (!active[r]) {
    return;
  }
  const cx<T> beta = mk<T>((T)q[8], (T)q[9]), alpha = mk<T>((T)q[2], (T)q[3]);
  const cx<T> omega = mk<T>((T)q[4], (T)q[5]);
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  const long o = r * nu;
  Acc<T> nn;
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    if (mode == 0) {  // X = p, A1 = r, A2 = v
      X[o + k] = A1[o + k] + beta * (X[o + k] - omega * A2[o + k]);
    } else if (mode == 1) {  // Y = s, A1 = r, A2 = v
      const cx<T> v = A1[o + k] - alpha * A2[o + k];
      Y[o + k] = v;
      nn.add(norm2(v));
    } else if (mode == 2) {  // D += alpha ph (A1 = ph)
      D[o + k] = D[o + k] + alpha * A1[o + k];
    } else {  // D += alpha ph + omega sh; X = r = s - omega t (A1 ph, A2 sh, A3 t, Y s)
      D[o + k] = D[o + k] + alpha * A1[o + k] + omega * A2[o + k];
      const cx<T> v = Y[o + k] - omega * A3[o + k];
      X[o + k] = v;
      nn.add(norm2(v));
    }
  }
  if (mode == 0 || mode == 2) return;
  const double2 t = block_sum(make_double2(nn.get(), 0.0), sh);
  if (threadIdx.x == 0) partial[(long)r * gridDim.x + blockIdx.x] = t;
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(&tickets[r], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  double n2 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
    n2 += __ldcg(&partial[(long)r * gridDim.x + b]).x;
  n2 = warp_sum(make_double2(n2, 0.0)).x;
  if (threadIdx.x == 0) {
    double* w = bs + (long)r * 16;
    w[10] = n2;
    const bool conv = !(n2 > w[11]);
    if (mode == 1) {
      w[12] = conv ? 1.0 : 0.0;
      if (conv) {
        active[r] = 0;
        iters[r] += 1;
      }
    } else {
      iters[r] += 1;
      if (conv || !isfinite(n2)) active[r] = 0;
    }
    tickets[r] = 0;
  }
}

// Start a BiCG-Stab cycle on the residual R (complex128): r = rhat = R in the
// inner precision, p = v = d = 0, rho = alpha = omega = 1, target^2.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_bstart(const double2* __restrict__ R, cx<T>* __restrict__ r0, cx<T>* __restrict__ rhat,
             cx<T>* __restrict__ p, cx<T>* __restrict__ v, cx<T>* __restrict__ D, long nu,
             const double* __restrict__ scal, double* __restrict__ bs, const int* __restrict__ run,
             int* __restrict__ active, double tol, double inner_tol) {
  pdl_entry();
  const int r = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    active[r] = run[r];
    double* q = bs + (long)r * 16;
    q[0] = 1.0; q[1] = 0.0; q[2] = 1.0; q[3] = 0.0; q[4] = 1.0; q[5] = 0.0;
    q[12] = 0.0;
    const double beta = scal[(long)r * 16 + 6];
    const double tgt = fmax(tol * scal[(long)r * 16 + 2], inner_tol * beta);
    q[11] = tgt * tgt;
  }
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const double2 a = R[r * nu + k];
    const cx<T> x = mk<T>((T)a.x, (T)a.y);
    r0[r * nu + k] = x;
    rhat[r * nu + k] = x;
    p[r * nu + k] = zero<T>();
    v[r * nu + k] = zero<T>();
    D[r * nu + k] = zero<T>();
  }
}

// x += d for right-hand sides that ran this cycle.
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_badd_x(double2* __restrict__ x, const cx<T>* __restrict__ d, const int* __restrict__ run,
             long nu) {
  pdl_entry();
  const int r = blockIdx.y;
  if (!run[r]) return;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) {
    const cx<T> v = d[r * nu + k];
    double2 a = x[r * nu + k];
    a.x += (double)v.x;
    a.y += (double)v.y;
    x[r * nu + k] = a;
  }
}

// ---------------------------------------------------------------------------
// Host side.  One restart cycle is: the FP64 residual and the decision
// (cycle_head), the cycle's start, its Arnoldi (or BiCG-Stab) steps, and its
// end (x update).  The same launch sequences serve the host-driven loop
// (step index as an argument, the host polls the device's decisions) and
// the graph-driven one, where the whole solve is captured once into a CUDA
// graph: WHILE(cycle) { head; IF(run) { start; WHILE(step) { step }; end } },
// with the conditions set by the device (k_cycle_decide, k_givens,
// k_count_active), so one graph launch runs the solve to the end.

#include "sstep.cuh"

template <typename T>
struct Ctx {
  dda_plan_s* p;
  int nrhs;
  const double2* b;
  double2* x;
  dda_solve_opts_t o;
  long nu;
  int m;
  int nblk, pst;
  SolverState* st;
  cx<T>* V;
  cx<T>* W;
  cx<T>* Z;
  double2* R;
  long vstride;
  dim3 vgrid, dgrid;
  bool prec, vec;
  double brk, eta2;
  // s-step GMRES (method 2): block size, Newton vectors, block dot grid
  int S = 0, bnb = 1;
  cx<T>* Wb = nullptr;
  dim3 bgrid;

  Ctx(dda_plan_s* p_, int nrhs_, const double2* b_, double2* x_, const dda_solve_opts_t& o_)
      : p(p_), nrhs(nrhs_), b(b_), x(x_), o(o_) {
    nu = 3 * p->nvox;
    m = o.restart;
    // one wave of 3 blocks per SM over the whole batch
    nblk = std::max(1, std::min(p->w.nblk, (456 + nrhs - 1) / nrhs));
    pst = m + 2;
    st = &p->w.st;
    V = static_cast<cx<T>*>(p->w.V);
    W = static_cast<cx<T>*>(p->w.Wv);
    Z = static_cast<cx<T>*>(p->w.Zv);
    R = static_cast<double2*>(p->w.R128);
    vstride = (long)nrhs * nu;
    vgrid = dim3(nblk, nrhs);
    dgrid = dim3(p->w.nblk, nrhs);  // warp-per-vector dots: the plan's full block count
    prec = o.precond != 0;
    vec = (nu % 2) == 0;  // 16-byte pairs stay aligned
    brk = sizeof(T) == 8 ? 1e-13 : 1e-6;
    eta2 = o.reorth_eta * o.reorth_eta;
    if (o.method == 2) {
      S = p->d.sstep;
      Wb = static_cast<cx<T>*>(p->w.Wb);
      // at least two blocks of 8 warps per SM over the batch, and chunks of
      // at most 8192 / S values, so that a block's chunk of the S Newton
      // vectors (64 KB in complex64), which every warp reads, stays in L1
      bnb = (int)std::max<long>((304 + nrhs - 1) / nrhs, (nu * S + 8191) / 8192);
      // whole waves: a batch of at least one wave of resident blocks (152
      // SMs x 3 in complex64) is rounded to the nearest multiple of it, so
      // that no short last wave doubles the pass (480 blocks were 1.05
      // waves); that adds at most half a wave, within the partial-sum store
      {
        const long resident = 152L * (sizeof(T) == 4 ? 3 : 1);
        const long total = (long)bnb * nrhs;
        if (total >= resident) {
          const long waves = (total + resident / 2) / resident;
          bnb = (int)std::max<long>(1, waves * resident / nrhs);
        }
      }
      bgrid = dim3(bnb, nrhs);
    }
  }

  void apply_prec(const cx<T>* in, cx<T>* out, cudaStream_t s) const {
    if (o.precond == 2)
      precond2_apply<T>(p, nrhs, in, out, s);
    else
      precond_apply_impl<T>(p, nrhs, in, out, s);
  }

  LoopCtl ctl_base() const {
    LoopCtl c{};
    c.jstep = st->ctl;
    c.steps = st->ctl + 1;
    c.nrun = st->ctl + 2;
    c.nlaunch = st->nlaunch;
    c.t0 = st->t0;
    c.timeout_ns = o.timeout_ns;
    c.hist = st->hist;
    c.hcap = kHistCap;
    c.max_iters = o.max_iters;
    c.scount = o.method == 2 ? st->ctl + 3 : nullptr;
    return c;
  }

  // The FP64 residual r = b - A x and the cycle decision.
  void cycle_head(const LoopCtl& c, cudaStream_t s) const {
    matvec_impl<double>(p, nrhs, reinterpret_cast<const cx<double>*>(x),
                        reinterpret_cast<cx<double>*>(R), s);
    note_launch();
    k_residual<<<vgrid, kNT, 0, s>>>(b, R, nu, st->partial);
    note_launch();
    k_finish_norms<<<(nrhs + 127) / 128, 128, 0, s>>>(st->partial, nblk, nrhs, st->scal);
    note_launch();
    k_cycle_decide<<<1, 256, 0, s>>>(st->scal, st->iters, st->flags, st->run,
                                     reinterpret_cast<RhsOut*>(st->out), nrhs, o.tol, m, c);
  }

  // GMRES -------------------------------------------------------------------
  void gmres_start(cx<T>* Zc, cudaStream_t s) const {
    cudaMemsetAsync(st->counters + 8, 0, sizeof(int), s);  // Givens kernel's ticket
    note_launch();
    k_start_cycle<T><<<vgrid, kNT, 0, s>>>(R, V, nu, st->scal, st->g, m, st->run, st->active,
                                           st->jlen, o.tol, o.inner_tol, Zc);
  }

  // Arnoldi step j (host-driven) or the device's step (graph: jdev != null,
  // the step's vector in Z, the preconditioner applied in place).
  void gmres_step(int j, bool scale_next, const LoopCtl& c, cudaStream_t s) const {
    const bool dev = c.graph != 0;
    const int* jdev = dev ? c.jstep : nullptr;
    const cx<T>* src = dev ? Z : V + (long)j * vstride;
    if (prec) {
      apply_prec(src, Z, s);
      src = Z;
    }
    matvec_impl<T>(p, nrhs, src, W, s);
    for (int pass = 0; pass < 2; ++pass) {
      const int* mask2 = pass == 0 ? nullptr : st->reorth;
      // kernel timing brackets the first pass (the second runs only for
      // some right-hand sides, so its work is not known on the host)
      const double vb = (double)nrhs * nu * sizeof(cx<T>);
      if (pass == 0) p->prof.begin(PROF_AR_DOT, s, (j + 2) * vb);
      note_launch();
      if (vec)
        launch_k(k_dots_w<T>, dgrid, kDotNT, 0, s, V, W, nu, vstride, j + 1, st->partial, pst,
                 st->active, mask2, pass == 0, st->tickets, st->hcol, st->H, m, j, pass, st->scal,
                 jdev);
      else
        launch_k(k_multidot<T, false>, vgrid, kNT, 0, s, V, W, nu, vstride, j + 1, st->partial,
                 pst, st->active, mask2, pass == 0, st->tickets, st->hcol, st->H, m, j, pass,
                 st->scal, jdev);
      if (pass == 0) p->prof.end(s);
      if (pass == 0) p->prof.begin(PROF_AR_UPD, s, (j + 3) * vb);
      note_launch();
      if (vec)
        launch_k(k_update<T, true>, vgrid, kNT, 0, s, V, W, nu, vstride, j + 1, st->hcol, m,
                 st->partial, pst, st->active, mask2, st->tickets + nrhs, st->scal, pass,
                 st->reorth, st->reorth_count, eta2, jdev);
      else
        launch_k(k_update<T, false>, vgrid, kNT, 0, s, V, W, nu, vstride, j + 1, st->hcol, m,
                 st->partial, pst, st->active, mask2, st->tickets + nrhs, st->scal, pass,
                 st->reorth, st->reorth_count, eta2, jdev);
      if (pass == 0) p->prof.end(s);
    }
    note_launch();
    // the Givens kernel also counts the right-hand sides still iterating
    const int jsm = dev ? m : j;
    launch_k(k_givens, nrhs, 32, (size_t)(jsm + 2) * 16 + (size_t)jsm * 24, s, st->H, st->cs,
             st->sn, st->g, st->scal, st->active, st->jlen, st->flags, st->iters, nrhs, m, j, brk,
             st->counters + (j & 1), st->counters + 8, c, o.method == 2 ? st->Hraw : nullptr);
    if (dev || scale_next) {
      note_launch();
      launch_k(k_scale<T>, vgrid, kNT, 0, s, W, V + (long)(j + 1) * vstride, nu, st->scal,
               st->active, V, vstride, jdev, dev ? Z : nullptr);
    }
  }

  // x += P^{-1} V y
  void gmres_end(cudaStream_t s) const {
    note_launch();
    k_trisolve<<<(nrhs + 63) / 64, 64, 0, s>>>(st->H, st->g, st->jlen, st->y, nrhs, m);
    note_launch();
    k_combine<T><<<vgrid, kNT, 0, s>>>(V, st->y, st->jlen, W, nu, vstride, m);
    const cx<T>* upd = W;
    if (prec) {
      apply_prec(W, Z, s);
      upd = Z;
    }
    note_launch();
    k_add_x<T><<<vgrid, kNT, 0, s>>>(x, upd, st->jlen, nu);
  }

  // BiCG-Stab ---------------------------------------------------------------
  cx<T>* bv(int i) const { return V + (long)i * vstride; }
  cx<T>* b_ph() const { return prec ? bv(6) : bv(2); }
  cx<T>* b_sh() const { return prec ? bv(7) : bv(4); }

  void bicg_start(cudaStream_t s) const {
    note_launch();
    k_bstart<T><<<vgrid, kNT, 0, s>>>(R, bv(0), bv(1), bv(2), bv(3), Z, nu, st->scal, st->bscal,
                                      st->run, st->active, o.tol, o.inner_tol);
  }

  void bicg_step(int it, const LoopCtl& c, cudaStream_t s) const {
    cx<T>* Vr = bv(0);
    cx<T>* Vrh = bv(1);
    cx<T>* Vp = bv(2);
    cx<T>* Vv = bv(3);
    cx<T>* Vs = bv(4);
    cx<T>* Vt = bv(5);
    cx<T>* Vph = b_ph();
    cx<T>* Vsh = b_sh();
    cx<T>* D = Z;
    double* bs = st->bscal;
    int* tk2 = st->tickets + nrhs;
    const unsigned sg = (nrhs + 63) / 64;
    note_launch();
    launch_k(k_bdots<T, 1>, vgrid, kNT, 0, s, Vrh, Vr, nullptr, nullptr, nu, st->active,
             st->partial, st->tickets, bs, 6);
    note_launch();
    launch_k(k_bscalar, sg, 64, 0, s, 0, bs, st->active, st->flags, nrhs);
    note_launch();
    launch_k(k_baxpy<T>, vgrid, kNT, 0, s, 0, Vp, nullptr, Vr, Vv, nullptr, nullptr, nu, bs, bs,
             st->active, st->iters, st->partial, tk2);
    if (prec) apply_prec(Vp, Vph, s);
    matvec_impl<T>(p, nrhs, Vph, Vv, s);
    note_launch();
    launch_k(k_bdots<T, 1>, vgrid, kNT, 0, s, Vrh, Vv, nullptr, nullptr, nu, st->active,
             st->partial, st->tickets, bs, 6);
    note_launch();
    launch_k(k_bscalar, sg, 64, 0, s, 1, bs, st->active, st->flags, nrhs);
    note_launch();
    launch_k(k_baxpy<T>, vgrid, kNT, 0, s, 1, nullptr, Vs, Vr, Vv, nullptr, nullptr, nu, bs, bs,
             st->active, st->iters, st->partial, tk2);
    note_launch();
    launch_k(k_baxpy<T>, vgrid, kNT, 0, s, 2, nullptr, nullptr, Vph, nullptr, nullptr, D, nu, bs,
             bs, st->active, st->iters, st->partial, tk2);
    note_launch();
    launch_k(k_bscalar, sg, 64, 0, s, 3, bs, st->active, st->flags, nrhs);
    if (prec) apply_prec(Vs, Vsh, s);
    matvec_impl<T>(p, nrhs, Vsh, Vt, s);
    note_launch();
    launch_k(k_bdots<T, 2>, vgrid, kNT, 0, s, Vt, Vs, Vt, Vt, nu, st->active, st->partial,
             st->tickets, bs, 6);
    note_launch();
    launch_k(k_bscalar, sg, 64, 0, s, 2, bs, st->active, st->flags, nrhs);
    note_launch();
    launch_k(k_baxpy<T>, vgrid, kNT, 0, s, 3, Vr, Vs, Vph, Vsh, Vt, D, nu, bs, bs, st->active,
             st->iters, st->partial, tk2);
    note_launch();
    launch_k(k_count_active, 1, 32, 0, s, st->active, nrhs, st->counters + (it & 1), st->flags,
             st->iters, st->bscal, st->scal, c);
  }

  void bicg_end(cudaStream_t s) const {
    note_launch();
    k_badd_x<T><<<vgrid, kNT, 0, s>>>(x, Z, st->run, nu);
  }

  // s-step GMRES --------------------------------------------------------------
  // One block of S columns from column j (host-driven) or the device's step
  // index (graph); q_j is in Z.
  template <int SB>
  void sstep_block_t(int j, const LoopCtl& c, cudaStream_t s) const {
    const bool dev = c.graph != 0;
    const int* jdev = dev ? c.jstep : nullptr;
    for (int t = 0; t < SB; ++t) {
      const cx<T>* in = t == 0 ? Z : Wb + (long)(t - 1) * vstride;
      cx<T>* out = Wb + (long)t * vstride;
      const cx<T>* src = in;
      if (prec) {
        apply_prec(in, W, s);
        src = W;
      }
      matvec_impl<T>(p, nrhs, src, out, s);
      note_launch();
      launch_k(k_shift<T>, vgrid, kNT, 0, s, out, in, nu, st->theta, t, st->active);
    }
    const int slots = (m + 1 + SB) * SB;
    const dim3 rgrid((slots + 7) / 8, nrhs);
    const double vb = (double)nrhs * nu * sizeof(cx<T>);
    for (int pass = 0; pass < 2; ++pass) {
      p->prof.begin(PROF_AR_DOT, s, (j + 1 + SB) * vb);
      note_launch();
      launch_k(k_sdots<T, SB>, bgrid, kBNT, 0, s, V, Wb, nu, vstride, j, jdev, pass,
               st->active, st->bpart, slots);
      note_launch();
      launch_k(k_sdots_reduce, rgrid, 256, 0, s, st->bpart, bnb, slots, SB, j, jdev, pass,
               st->active, st->cb, slots, pass);
      p->prof.end(s);
      if (pass == 0) {
        p->prof.begin(PROF_AR_UPD, s, (j + 1 + 2 * SB) * vb);
        note_launch();
        launch_k(k_supd<T, SB>, vgrid, kNT, 0, s, V, Wb, nu, vstride, j, jdev, 0, st->cb, slots,
                 0, nullptr, st->active, nullptr);
        p->prof.end(s);
      }
    }
    const int jsm = dev ? m - SB : j;
    const int nrow = jsm + SB + 1;
    const size_t smem = (size_t)16 * ((size_t)nrow * SB + (size_t)(jsm + 1) * SB + 3 * SB * SB +
                                      nrow + (jsm + SB)) +
                        (size_t)8 * (jsm + SB);
    note_launch();
    launch_k(k_ssmall, nrhs, 32, smem, s, SB, st->Hraw, st->H, st->cs, st->sn, st->g, st->scal,
             st->active, st->reorth, st->jlen, st->flags, st->iters, st->cb, slots, st->rinv,
             st->theta, nrhs, m, j, brk, st->counters + ((j / SB) & 1), st->counters + 8, c);
    p->prof.begin(PROF_AR_UPD, s, (j + 1 + 2 * SB) * vb);
    note_launch();
    launch_k(k_supd<T, SB>, vgrid, kNT, 0, s, V, Wb, nu, vstride, j, jdev, SB, st->cb, slots, 1,
             st->rinv, st->reorth, Z);
    p->prof.end(s);
  }

  void sstep_block(int j, const LoopCtl& c, cudaStream_t s) const {
    switch (S) {
      case 2: sstep_block_t<2>(j, c, s); break;
      case 3: sstep_block_t<3>(j, c, s); break;
      case 4: sstep_block_t<4>(j, c, s); break;
      case 5: sstep_block_t<5>(j, c, s); break;
      case 6: sstep_block_t<6>(j, c, s); break;
      case 7: sstep_block_t<7>(j, c, s); break;
      default: sstep_block_t<8>(j, c, s); break;
    }
  }

  void start(cudaStream_t s, bool graph) const {
    if (o.method == 1)
      bicg_start(s);
    else
      gmres_start(graph || o.method == 2 ? Z : nullptr, s);
  }
  void end(cudaStream_t s) const {
    if (o.method == 1) {
      bicg_end(s);
    } else {
      gmres_end(s);
      if (o.method == 2) {  // the shifts, after the first cycle
        note_launch();
        launch_k(k_ritz, nrhs, 32, 0, s, st->Hraw, st->jlen, st->theta, S, m, st->ctl + 3);
      }
    }
  }
};

// State reset at the start of every solve (both drivers).
template <typename T>
void solve_prologue(const Ctx<T>& c, cudaStream_t s) {
  SolverState& st = *c.st;
  const int nrhs = c.nrhs;
  cudaMemsetAsync(st.iters, 0, sizeof(int) * nrhs, s);
  cudaMemsetAsync(st.reorth_count, 0, sizeof(int) * nrhs, s);
  cudaMemsetAsync(st.tickets, 0, sizeof(int) * 2 * nrhs, s);
  cudaMemsetAsync(st.flags, 0, sizeof(int) * nrhs, s);
  cudaMemsetAsync(st.out, 0, sizeof(RhsOut) * nrhs, s);
  cudaMemsetAsync(st.nlaunch, 0, sizeof(long long), s);
  cudaMemsetAsync(st.ctl + 3, 0, sizeof(int), s);  // cycles started (s-step)
  cudaMemsetAsync(c.p->w.err_flag, 0, 4, s);
  note_launch();
  k_solve_begin<<<1, 1, 0, s>>>(st.t0);
}

// Host-driven loop: the host reads each cycle's decision and polls the
// step count (at most two Arnoldi steps queued ahead of the GPU).  Used
// when kernel timing is on (events bracket launches) and as the fallback.
template <typename T>
dda_status_t drive_host(const Ctx<T>& c, cudaStream_t s) {
  dda_plan_s* p = c.p;
  SolverState& st = *c.st;
  LoopCtl ctl = c.ctl_base();
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  dda_status_t status = DDA_OK;
  int cycles = 0;
  for (;;) {
    c.cycle_head(ctl, s);
    cudaMemcpyAsync(p->pinned + 2, st.ctl + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      status = check_cuda("dda_solve");
      break;
    }
    const int steps = p->pinned[2], nrun = p->pinned[3];
    if (nrun == 0) break;
    c.start(s, false);
    // s-step: Arnoldi in the first cycle, blocks of S columns afterwards
    const bool blocks = c.o.method == 2 && cycles > 0;
    const int stride = blocks ? c.S : 1;
    for (int j = 0, q = 0; j < steps; j += stride, ++q) {
      if (blocks)
        c.sstep_block(j, ctl, s);
      else if (c.o.method == 1)
        c.bicg_step(j, ctl, s);
      else
        c.gmres_step(j, j + 1 < steps, ctl, s);
      cudaMemcpyAsync(p->pinned + (q & 1), st.counters + (q & 1), sizeof(int),
                      cudaMemcpyDeviceToHost, s);
      cudaEventRecord(ev[q & 1], s);
      if (q >= 1) {
        cudaEventSynchronize(ev[(q - 1) & 1]);
        if (p->pinned[(q - 1) & 1] == 0) break;
      }
    }
    c.end(s);
    ++cycles;
    if ((status = check_cuda("dda_solve")) != DDA_OK) break;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return status;
}

// What a captured solve graph depends on: a new graph is captured when any
// of it changes (pointers and scalars are baked into the kernel nodes).
struct GraphKey {
  const void* plan;
  long long plan_id;
  int nrhs, tsize, method, precond, restart, max_iters, rr_z, pdl;
  const void* b;
  void* x;
  double tol, inner_tol, eta;
  long long timeout_ns;
};

template <typename T>
GraphKey graph_key(const Ctx<T>& c) {
  GraphKey key{};
  key.plan = c.p;
  key.plan_id = c.p->id;
  key.nrhs = c.nrhs;
  key.tsize = sizeof(T);
  key.method = c.o.method;
  key.precond = c.o.precond;
  key.restart = c.o.restart;
  key.max_iters = c.o.max_iters;
  key.rr_z = tl_schedule.rr_z;
  key.pdl = pdl_enabled();
  key.b = c.b;
  key.x = c.x;
  key.tol = c.o.tol;
  key.inner_tol = c.o.inner_tol;
  key.eta = c.o.reorth_eta;
  key.timeout_ns = c.o.timeout_ns;
  return key;
}

// A conditional node on the capturing stream, after everything captured so
// far; returns its body graph, to be captured separately.
cudaGraph_t add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, bool& ok) {
  if (!ok) return nullptr;
  cudaStreamCaptureStatus stt;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, &deps, &edata, &nd) != cudaSuccess ||
      stt != cudaStreamCaptureStatusActive) {
    ok = false;
    return nullptr;
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np) != cudaSuccess ||
      cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies) != cudaSuccess) {
    ok = false;
    return nullptr;
  }
  return np.conditional.phGraph_out[0];
}

// Run fn() captured on cs into graph g (appended after g's roots: a new
// independent chain); ok turns false on any capture error.
template <typename F>
void capture(cudaStream_t cs, cudaGraph_t g, bool& ok, F&& fn) {
  if (!ok || g == nullptr) {
    ok = false;
    return;
  }
  if (cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
      cudaSuccess) {
    ok = false;
    return;
  }
  fn();
  cudaGraph_t out = nullptr;
  if (cudaStreamEndCapture(cs, &out) != cudaSuccess) ok = false;
}

// Capture one plan's whole solve into `top` as an independent chain:
// prologue (state reset, start time), then
// WHILE(cycle) { head; IF(run) { start; WHILE(step) { step }; end } }.
// The kernel counts per part go into the kernel arguments (the device
// counts what the graph runs), so a throwaway capture counts them first.
// Launches made while capturing are not counted as launches.
template <typename T>
bool capture_into(const Ctx<T>& c, cudaGraph_t top, cudaStream_t cs) {
  ScheduleScope scope(c.p->sched);
  const long long before = launch_counter();
  bool ok = true;
  const bool ss = c.o.method == 2;
  cudaGraphConditionalHandle hc = 0, hr = 0, hs = 0, hb = 0;
  ok = cudaGraphConditionalHandleCreate(&hc, top, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
       cudaGraphConditionalHandleCreate(&hr, top, 0, 0) == cudaSuccess &&
       cudaGraphConditionalHandleCreate(&hs, top, 0, 0) == cudaSuccess &&
       (!ss || cudaGraphConditionalHandleCreate(&hb, top, 0, 0) == cudaSuccess);
  LoopCtl ctl = c.ctl_base();
  ctl.graph = 1;
  ctl.h_cycle = hc;
  ctl.h_run = hr;
  ctl.h_step = hs;
  ctl.h_blk = hb;
  {
    cudaGraph_t dry = nullptr;
    ok = ok && cudaGraphCreate(&dry, 0) == cudaSuccess;
    long long t = launch_counter();
    capture(cs, dry, ok, [&] { c.cycle_head(ctl, cs); });
    ctl.k_head = (int)(launch_counter() - t);
    t = launch_counter();
    capture(cs, dry, ok, [&] {
      c.start(cs, true);
      c.end(cs);
    });
    ctl.k_run = (int)(launch_counter() - t);
    t = launch_counter();
    capture(cs, dry, ok, [&] {
      if (c.o.method == 1)
        c.bicg_step(0, ctl, cs);
      else
        c.gmres_step(0, true, ctl, cs);
    });
    ctl.k_step = (int)(launch_counter() - t);
    if (ss) {
      t = launch_counter();
      capture(cs, dry, ok, [&] { c.sstep_block(0, ctl, cs); });
      ctl.k_blk = (int)(launch_counter() - t);
    }
    if (dry) cudaGraphDestroy(dry);
  }
  cudaGraph_t body_cycle = nullptr, body_run = nullptr, body_step = nullptr, body_blk = nullptr;
  capture(cs, top, ok, [&] {
    solve_prologue(c, cs);
    body_cycle = add_conditional(cs, hc, cudaGraphCondTypeWhile, ok);
  });
  capture(cs, body_cycle, ok, [&] {
    c.cycle_head(ctl, cs);
    body_run = add_conditional(cs, hr, cudaGraphCondTypeIf, ok);
  });
  capture(cs, body_run, ok, [&] {
    c.start(cs, true);
    body_step = add_conditional(cs, hs, cudaGraphCondTypeWhile, ok);
    if (ss) body_blk = add_conditional(cs, hb, cudaGraphCondTypeWhile, ok);
    c.end(cs);
  });
  if (ss) capture(cs, body_blk, ok, [&] { c.sstep_block(0, ctl, cs); });
  capture(cs, body_step, ok, [&] {
    if (c.o.method == 1)
      c.bicg_step(0, ctl, cs);
    else
      c.gmres_step(0, true, ctl, cs);
  });
  add_launches(before - launch_counter());  // captured, not run
  if (!ok) cudaGetLastError();
  return ok;
}

// Make (or reuse) the graph of `keys` in G: one chain per context.
template <typename T>
bool ensure_graph(SolveGraph& G, const std::vector<const Ctx<T>*>& ctxs) {
  std::vector<GraphKey> keys;
  for (const Ctx<T>* c : ctxs) {
    ScheduleScope scope(c->p->sched);
    keys.push_back(graph_key(*c));
  }
  const size_t nb = keys.size() * sizeof(GraphKey);
  if (G.exec && G.key.size() == nb && std::memcmp(G.key.data(), keys.data(), nb) == 0) return true;
  G.reset();
  if (!G.cs && cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    G.cs = nullptr;
    return false;
  }
  bool ok = cudaGraphCreate(&G.graph, 0) == cudaSuccess;
  for (const Ctx<T>* c : ctxs) {
    if (!ok) break;
    ok = capture_into(*c, G.graph, G.cs);
  }
  ok = ok && cudaGraphInstantiate(&G.exec, G.graph, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    G.reset();
    return false;
  }
  G.key.assign(reinterpret_cast<const char*>(keys.data()),
               reinterpret_cast<const char*>(keys.data()) + nb);
  return true;
}

// Copy a finished solve's outcome to the host (queued on s; the caller
// synchronises) and turn it into stats and a status.
struct Collected {
  std::vector<RhsOut> out;
  std::vector<int> hits, hreo;
  int perr = 0;
  long long nl = 0;
};

template <typename T>
void collect_async(const Ctx<T>& c, Collected& r, cudaStream_t s) {
  const SolverState& st = *c.st;
  const int nrhs = c.nrhs;
  r.out.resize(nrhs);
  r.hits.resize(nrhs);
  r.hreo.resize(nrhs);
  cudaMemcpyAsync(r.out.data(), st.out, sizeof(RhsOut) * nrhs, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(r.hits.data(), st.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(r.hreo.data(), st.reorth_count, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&r.perr, c.p->w.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&r.nl, st.nlaunch, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (c.o.h_history != nullptr && c.o.history_cap > 0) {
    const int w = std::min(c.o.history_cap, kHistCap);
    cudaMemcpy2DAsync(c.o.h_history, sizeof(double) * c.o.history_cap, st.hist,
                      sizeof(double) * kHistCap, sizeof(double) * w, nrhs, cudaMemcpyDeviceToHost,
                      s);
  }
}

template <typename T>
dda_status_t finish_stats(const Ctx<T>& c, const Collected& r, bool graph, float ms,
                          dda_rhs_stats_t* stats) {
  const dda_solve_opts_t& o = c.o;
  bool any_nan = false, any_nc = false, any_to = false, any_brk = false;
  for (int i = 0; i < c.nrhs; ++i) {
    const RhsOut& q = r.out[i];
    any_nan |= q.nan != 0;
    any_to |= !q.conv && !q.nan && q.timeout;
    any_brk |= !q.conv && !q.nan && !q.timeout && q.stalled;
    any_nc |= !q.conv;
    if (stats) {
      stats[i].iters = r.hits[i];
      stats[i].cycles = q.cycles;
      stats[i].reorth = r.hreo[i];
      stats[i].converged = q.conv;
      stats[i].rel_resid = q.rel;
      stats[i].status = q.nan ? DDA_ERR_NAN
                        : q.conv ? DDA_OK
                        : q.timeout ? DDA_ERR_TIMEOUT
                        : q.stalled ? DDA_ERR_BREAKDOWN
                                    : DDA_ERR_NOT_CONVERGED;
      stats[i].history_len =
          (o.h_history != nullptr && o.history_cap > 0)
              ? std::min(r.hits[i] + 1, std::min(o.history_cap, kHistCap))
              : 0;
      stats[i].graph = graph ? 1 : 0;
      stats[i].ms = ms;
    }
  }
  if (r.perr) return fail(DDA_ERR_SINGULAR_PRECOND, "dda_solve: preconditioner symbol is singular");
  if (any_nan) return fail(DDA_ERR_NAN, "dda_solve: non-finite residual");
  if (any_to) return fail(DDA_ERR_TIMEOUT, "dda_solve: time limit reached");
  if (any_brk)
    return fail(DDA_ERR_BREAKDOWN, "dda_solve: a restart cycle made no progress (BiCG-Stab "
                                   "breakdown at its first step)");
  if (any_nc) return fail(DDA_ERR_NOT_CONVERGED, "dda_solve: tolerance not reached within max_iters");
  return DDA_OK;
}

bool ensure_pinned(dda_plan_s* p) {
  if (p->pinned) return true;
  if (cudaHostAlloc(&p->pinned, 64, cudaHostAllocDefault) != cudaSuccess) {
    p->pinned = nullptr;
    return false;
  }
  return true;
}

template <typename T>
dda_status_t solve_impl(dda_plan_s* p, int nrhs, const double2* b, double2* x,
                        const dda_solve_opts_t& o, dda_rhs_stats_t* stats, cudaStream_t s) {
  const auto t_begin = std::chrono::steady_clock::now();
  Ctx<T> c(p, nrhs, b, x, o);
  if (!ensure_pinned(p)) return check_cuda("dda_solve: pinned host word");
  dda_status_t status = DDA_OK;
  bool graph = tl_schedule.graph && !p->prof.on && solve_graph_enabled() && !p->graph.failed;
  if (graph && !ensure_graph<T>(p->graph, {&c})) {
    p->graph.failed = true;  // this plan keeps to the host-driven loop
    graph = false;
  }
  if (graph) {
    if (cudaGraphLaunch(p->graph.exec, s) != cudaSuccess) status = check_cuda("dda_solve: graph");
  } else {
    solve_prologue(c, s);
    status = drive_host(c, s);
  }
  if (status != DDA_OK) return status;
  Collected r;
  collect_async(c, r, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_cuda("dda_solve");
  if (graph) add_launches(r.nl + 1);  // the graph's kernels and its prologue kernel
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() -
                                                            t_begin).count();
  return finish_stats(c, r, graph, ms, stats);
}

// dda_solve_many as one graph launch: every plan's solve an independent
// chain of one graph, so the uneven batch runs concurrently on the GPU with
// no host thread per plan.  Returns false (nothing launched) when a plan
// cannot take part; the caller then falls back to one thread per plan.
template <typename T>
bool solve_many_graph(int nplans, const dda_plan_t* plans, const int32_t* nrhs,
                      const void* const* d_b, void* const* d_x, const dda_solve_opts_t& o,
                      dda_rhs_stats_t* const* h_stats, void* const* streams,
                      dda_status_t* st_out, std::string* why) {
  const auto t_begin = std::chrono::steady_clock::now();
  std::vector<std::unique_ptr<Ctx<T>>> ctxs;
  std::vector<const Ctx<T>*> cptr;
  for (int i = 0; i < nplans; ++i) {
    dda_plan_s* p = plans[i];
    if (!p->sched.graph || p->prof.on || !ensure_pinned(p)) return false;
    const double2* b = d_b && d_b[i] ? static_cast<const double2*>(d_b[i])
                                     : static_cast<const double2*>(p->w.B128);
    ctxs.emplace_back(new Ctx<T>(p, nrhs[i], b, static_cast<double2*>(d_x[i]), o));
    cptr.push_back(ctxs.back().get());
  }
  // the batch graph lives with the first plan
  SolveGraph& G = plans[0]->batch;
  if (!ensure_graph<T>(G, cptr)) return false;
  cudaStream_t s0 = streams ? static_cast<cudaStream_t>(streams[0]) : nullptr;
  // the launch stream waits for every plan's stream (their b and x), and
  // every plan's stream waits for the launch
  std::vector<cudaEvent_t> evs;
  for (int i = 1; i < nplans && streams; ++i) {
    if (!streams[i]) continue;
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventRecord(e, static_cast<cudaStream_t>(streams[i]));
    cudaStreamWaitEvent(s0, e, 0);
    evs.push_back(e);
  }
  dda_status_t status = DDA_OK;
  if (cudaGraphLaunch(G.exec, s0) != cudaSuccess) status = check_cuda("dda_solve_many: graph");
  std::vector<Collected> r(nplans);
  for (int i = 0; i < nplans && status == DDA_OK; ++i) collect_async(*cptr[i], r[i], s0);
  if (status == DDA_OK && cudaStreamSynchronize(s0) != cudaSuccess)
    status = check_cuda("dda_solve_many");
  cudaEvent_t done;
  cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  cudaEventRecord(done, s0);
  for (int i = 1; i < nplans && streams; ++i)
    if (streams[i]) cudaStreamWaitEvent(static_cast<cudaStream_t>(streams[i]), done, 0);
  cudaEventDestroy(done);
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() -
                                                            t_begin).count();
  for (int i = 0; i < nplans; ++i) {
    if (status != DDA_OK) {
      st_out[i] = status;
      continue;
    }
    add_launches(r[i].nl + 1);
    st_out[i] = finish_stats(*cptr[i], r[i], true, ms, h_stats ? h_stats[i] : nullptr);
    if (st_out[i] != DDA_OK) why[i] = dda_last_error();
  }
  return true;
}

// Options and plan checks shared by dda_solve and dda_solve_many.
dda_status_t check_solve(dda_plan_t p, int32_t nrhs, const dda_solve_opts_t& o) {
  if (p->d.krylov_m < 1) return fail(DDA_ERR_INVALID_ARG, "dda_solve: plan has krylov_m = 0");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: nrhs must be 1..(incidences set)");
  if (!(o.tol > 0) || o.max_iters < 1 || o.restart < 1 ||
      (o.method == 0 && o.restart > p->d.krylov_m) ||
      !(o.inner_tol >= 0) || !(o.reorth_eta >= 0) ||
      (o.precond != 0 && o.precond != 2 && o.precond != 3))
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: invalid options");
  if (o.precond == 3 && !p->precond_built)
    return fail(DDA_ERR_NO_PRECOND, "dda_solve: call dda_precond_build first");
  if (o.precond == 2 && !p->precond2_built)
    return fail(DDA_ERR_NO_PRECOND, "dda_solve: call dda_precond2_build first");
  if (!p->has128) return fail(DDA_ERR_INVALID_ARG, "dda_solve: the residual needs complex128 data");
  if (o.method == 0 && o.restart + 2 > 518)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: restart above 512");
  if (o.method != 0 && o.method != 1 && o.method != 2)
    return fail(DDA_ERR_INVALID_ARG,
                "dda_solve: method must be 0 (GMRES), 1 (BiCG-Stab) or 2 (s-step GMRES)");
  if (o.method == 2) {
    const int sb = p->d.sstep;
    if (sb < 2)
      return fail(DDA_ERR_INVALID_ARG, "dda_solve: method 2 needs a plan with sstep >= 2");
    if (o.restart % sb != 0 || o.restart > p->d.krylov_m || o.restart > kSRestart)
      return fail(DDA_ERR_INVALID_ARG,
                  "dda_solve: method 2 needs restart a multiple of sstep, <= krylov_m and <= 64");
    if ((3 * p->nvox) % 2 != 0)
      return fail(DDA_ERR_INVALID_ARG, "dda_solve: method 2 needs an even number of unknowns");
  }
  if (o.method == 1 && p->d.krylov_m < 7)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: BiCG-Stab needs a plan with krylov_m >= 7");
  if (o.history_cap < 0 || o.timeout_ns < 0 || (o.h_history != nullptr && o.history_cap < 1))
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: history_cap and timeout_ns must be >= 0");
  if (o.inner_prec != DDA_C128 && o.inner_prec != DDA_C64)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: inner_prec must be DDA_C128 or DDA_C64");
  if (o.inner_prec == DDA_C64 && !p->has64)
    return fail(DDA_ERR_INVALID_ARG, "dda_solve: plan holds no complex64 data");
  if (o.inner_prec == DDA_C128 && p->d.krylov_c64)
    return fail(DDA_ERR_INVALID_ARG,
                "dda_solve: the plan's Krylov basis is complex64 (krylov_c64): inner_prec must be "
                "DDA_C64");
  return DDA_OK;
}

}  // namespace

// One graph launch for a batch of plans (dda_solve_many); false: use threads.
bool solve_many_as_graph(int32_t nplans, const dda_plan_t* plans, const int32_t* nrhs,
                         const void* const* d_b, void* const* d_x, const dda_solve_opts_t* opts,
                         dda_rhs_stats_t* const* h_stats, void* const* streams,
                         dda_status_t* st_out, std::string* why) {
  if (!solve_graph_enabled()) return false;
  for (int i = 0; i < nplans; ++i) {
    if (check_solve(plans[i], nrhs[i], *opts) != DDA_OK) return false;  // dda_solve reports it
    if (!(d_b && d_b[i])) {
      cudaStream_t si = streams ? static_cast<cudaStream_t>(streams[i]) : nullptr;
      if (dda_incident_field(plans[i], nrhs[i], plans[i]->w.B128, si) != DDA_OK) return false;
    }
  }
  if (opts->inner_prec == DDA_C128)
    return solve_many_graph<double>(nplans, plans, nrhs, d_b, d_x, *opts, h_stats, streams, st_out,
                                    why);
  return solve_many_graph<float>(nplans, plans, nrhs, d_b, d_x, *opts, h_stats, streams, st_out,
                                 why);
}

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_ritz_shifts(const void* d_hraw, int32_t m, const int32_t* d_jlen,
                                        int32_t nrhs, int32_t s, void* d_theta, void* stream) {
  if (!d_hraw || !d_jlen || !d_theta)
    return fail(DDA_ERR_INVALID_ARG, "dda_ritz_shifts: NULL argument");
  if (m < 1 || nrhs < 1 || s < 1 || s > kSMax)
    return fail(DDA_ERR_INVALID_ARG, "dda_ritz_shifts: need m >= 1, nrhs >= 1, 1 <= s <= 8");
  note_launch();
  k_ritz<<<nrhs, 32, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const double2*>(d_hraw), d_jlen, static_cast<double2*>(d_theta), s, m, nullptr);
  return check_cuda("dda_ritz_shifts");
}

extern "C" dda_status_t dda_solve(dda_plan_t p, int32_t nrhs, const void* d_b, void* d_x,
                                  const dda_solve_opts_t* opts, dda_rhs_stats_t* h_stats,
                                  void* stream) {
  if (!p || !d_x || !opts) return fail(DDA_ERR_INVALID_ARG, "dda_solve: NULL argument");
  const dda_solve_opts_t& o = *opts;
  const dda_status_t chk = check_solve(p, nrhs, o);
  if (chk != DDA_OK) return chk;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScheduleScope scope(p->sched);
  const double2* b = static_cast<const double2*>(d_b);
  if (!b) {
    dda_status_t st = dda_incident_field(p, nrhs, p->w.B128, stream);
    if (st != DDA_OK) return st;
    b = static_cast<const double2*>(p->w.B128);
  }
  if (o.inner_prec == DDA_C128)
    return solve_impl<double>(p, nrhs, b, static_cast<double2*>(d_x), o, h_stats, s);
  return solve_impl<float>(p, nrhs, b, static_cast<double2*>(d_x), o, h_stats, s);
}
