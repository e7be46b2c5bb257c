// Shared-memory Stockham FFT used by every transform of the DDA operator and
// preconditioner.
//
// A CTA transforms NB independent lines of power-of-two length L held in
// shared memory, element (line b, position j) at s[j * ld + b].  Threads are
// mapped with the line index fastest, so a warp touches consecutive words.
// Each stage of radix R (2, 4, 8 or 16) is the self-sorting Stockham step:
//   butterfly jb (0 <= jb < L/R) of a line reads x[jb + q L/R], q < R,
//   multiplies by w_L^{q k L/(Ns R)} with k = jb mod Ns (Ns = product of the
//   radices already applied), takes an R-point DFT in registers and writes
//   y[(jb - k) R + k + q Ns].
// After the last stage the line holds its DFT in natural order.  Every
// thread owns E = 16 complex values per stage (16/R butterflies), so a CTA
// has NB * L / 16 threads.  Reads of a stage complete (barrier) before its
// writes, so one buffer suffices.
#pragma once

#include "cx.cuh"

namespace dda {

void note_launch();

constexpr int kElemsPerThread = 16;

// cos(2 pi j / 32), j = 0..8 (plain trigonometry: cos(pi j / 16)).
constexpr double kCos32[9] = {1.0,
                              0.98078528040323044913,
                              0.92387953251128675613,
                              0.83146961230254523708,
                              0.70710678118654752440,
                              0.55557023301960222474,
                              0.38268343236508977173,
                              0.19509032201612826785,
                              0.0};

// cos(2 pi j / 32) for any j, by the quarter-wave symmetries.
__host__ __device__ constexpr double cos32(int j) {
  return ((j & 31) <= 8)    ? kCos32[j & 31]
         : ((j & 31) <= 16) ? -kCos32[16 - (j & 31)]
         : ((j & 31) <= 24) ? -kCos32[(j & 31) - 16]
                            : kCos32[32 - (j & 31)];
}
// sin(x) = cos(x - pi/2)
__host__ __device__ constexpr double sin32(int j) { return cos32(j - 8); }

// a * exp(-+ 2 pi i Q / R) (minus sign forward, plus sign inverse), R | 32.
template <int R, int Q, bool INV, typename T>
__device__ __forceinline__ cx<T> twc(cx<T> a) {
  static_assert(32 % R == 0, "radix up to 32");
  constexpr int j = (Q * (32 / R)) & 31;
  if constexpr (j == 0) {
    return a;
  } else if constexpr (j == 8) {
    return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
  } else if constexpr (j == 16) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (j == 24) {
    return INV ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
  } else {
    constexpr T c = (T)cos32(j);
    constexpr T s = INV ? (T)sin32(j) : -(T)sin32(j);
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

template <int R, int Q, bool INV, typename T>
__device__ __forceinline__ void dft_combine(cx<T>* v, const cx<T>* e, const cx<T>* o) {
  if constexpr (Q < R / 2) {
    const cx<T> t = twc<R, Q, INV>(o[Q]);
    v[Q] = e[Q] + t;
    v[Q + R / 2] = e[Q] - t;
    dft_combine<R, Q + 1, INV>(v, e, o);
  }
}

// In-register R-point DFT, natural order in and out (radix-2 decimation in
// time: X[q] = E[q] + w^q O[q], X[q + R/2] = E[q] - w^q O[q]).
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R > 1) {
    cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<R / 2, INV>(e);
    dft<R / 2, INV>(o);
    dft_combine<R, 0, INV>(v, e, o);
  }
}

template <int R, int Q, bool INV, typename T>
__device__ __forceinline__ void twiddle_into(cx<T>* o, const cx<T>* v) {
  if constexpr (Q < R / 2) {
    o[Q] = twc<R, Q, INV>(v[Q]);
    twiddle_into<R, Q + 1, INV>(o, v);
  }
}

// R-point DFT of an input whose upper half v[R/2..R) is zero (first stage
// of a zero-padded transform): X[2k] = DFT_{R/2}(v)[k],
// X[2k+1] = DFT_{R/2}(v w_R^q)[k].
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_half_in(cx<T>* v) {
  if constexpr (R == 2) {
    v[1] = v[0];
  } else if constexpr (R > 2) {
    cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int q = 0; q < R / 2; ++q) e[q] = v[q];
    twiddle_into<R, 0, INV>(o, v);
    dft<R / 2, INV>(e);
    dft<R / 2, INV>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      v[2 * k] = e[k];
      v[2 * k + 1] = o[k];
    }
  }
}

template <int R, int Q, bool INV, typename T>
__device__ __forceinline__ void dft_combine_lo(cx<T>* v, const cx<T>* e, const cx<T>* o) {
  if constexpr (Q < R / 2) {
    v[Q] = e[Q] + twc<R, Q, INV>(o[Q]);
    dft_combine_lo<R, Q + 1, INV>(v, e, o);
  }
}

// R-point DFT of which only the outputs X[0..R/2) are needed (last stage of
// a transform whose upper half is discarded).
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_half_out(cx<T>* v) {
  if constexpr (R > 1) {
    cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<R / 2, INV>(e);
    dft<R / 2, INV>(o);
    dft_combine_lo<R, 0, INV>(v, e, o);
  }
}

// Radix sequence of a transform: at most 4 stages (L <= 65536); lg = log2 L.
struct RadixPlan {
  int nst;
  int lg;
  int r[4];
};

inline int ilog2i(long v) {
  int b = 0;
  while ((1L << b) < v) ++b;
  return b;
}

inline RadixPlan make_radix_plan(int L) {
  RadixPlan p{0, 0, {1, 1, 1, 1}};
  int bits = 0;
  while ((1 << bits) < L) ++bits;
  p.lg = bits;
  if (bits == 0) return p;
  const int nst = (bits + 3) / 4;
  int left = bits;
  for (int s = 0; s < nst; ++s) {
    const int b = (left + (nst - s) - 1) / (nst - s);  // ceil: larger radices first
    p.r[s] = 1 << b;
    left -= b;
  }
  p.nst = nst;
  return p;
}

// Line count of a tile: (1 << sh) or 3 * (1 << sh) lines (MUL3), so that
// the line / butterfly split of an index needs no run-time division.
template <bool MUL3>
__device__ __forceinline__ void split_line(int u, int sh, int& b, int& jb) {
  const int hi = u >> sh;
  jb = MUL3 ? hi / 3 : hi;
  b = u - ((jb * (MUL3 ? 3 : 1)) << sh);
}

// MODE 0: full stage; 1: first stage of a transform whose input's upper
// half is zero (those values are neither read nor used); 2: last stage of a
// transform whose output's upper half is discarded (not computed, not written).
template <int R, bool INV, bool MUL3, int MODE, typename T>
__device__ __forceinline__ void smem_stage(cx<T>* s, const cx<T>* tw, int L, int sh, int ld,
                                           int Ns, int tid, int nth) {
  constexpr int G = kElemsPerThread / R;
  constexpr int QIN = MODE == 1 ? R / 2 : R;
  constexpr int QOUT = MODE == 2 ? R / 2 : R;
  cx<T> v[kElemsPerThread];
  const int LR = L / R;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * nth;
    int b, jb;
    split_line<MUL3>(u, sh, b, jb);
#pragma unroll
    for (int q = 0; q < QIN; ++q) v[g * R + q] = s[(jb + q * LR) * ld + b];
  }
  __syncthreads();
  const int tstep = L / (Ns * R);  // powers of two: compiles to a shift
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * nth;
    int b, jb;
    split_line<MUL3>(u, sh, b, jb);
    const int k = jb & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) v[g * R + q] = mulc<INV>(v[g * R + q], tw[q * k * tstep]);
    }
    if constexpr (MODE == 1)
      dft_half_in<R, INV>(&v[g * R]);
    else if constexpr (MODE == 2)
      dft_half_out<R, INV>(&v[g * R]);
    else
      dft<R, INV>(&v[g * R]);
    const int base = (jb - k) * R + k;
#pragma unroll
    for (int q = 0; q < QOUT; ++q) s[(base + q * Ns) * ld + b] = v[g * R + q];
  }
  __syncthreads();
}

template <int R, bool INV, bool MUL3, typename T>
__device__ __forceinline__ void smem_stage_any(int mode, cx<T>* s, const cx<T>* tw, int L, int sh,
                                               int ld, int Ns, int tid, int nth) {
  if (mode == 1)
    smem_stage<R, INV, MUL3, 1>(s, tw, L, sh, ld, Ns, tid, nth);
  else if (mode == 2)
    smem_stage<R, INV, MUL3, 2>(s, tw, L, sh, ld, Ns, tid, nth);
  else
    smem_stage<R, INV, MUL3, 0>(s, tw, L, sh, ld, Ns, tid, nth);
}

// Full transform of NB = (MUL3 ? 3 : 1) << sh lines in shared memory.
// tw[t] = exp(-2 pi i t / L), t < L, also in shared memory.  Caller
// synchronises before the call.
// half_in: the input's upper half (positions >= L/2) is zero and need not
// be present in shared memory; half_out: only positions < L/2 of the result
// are wanted (the rest of shared memory is left stale).
template <bool INV, bool MUL3 = false, typename T>
__device__ __forceinline__ void smem_fft(cx<T>* s, const cx<T>* tw, int L, int sh, int ld,
                                         const RadixPlan& rp, bool half_in = false,
                                         bool half_out = false) {
  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  int Ns = 1;
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    if (st >= rp.nst) break;
    const int R = rp.r[st];
    const int mode = (st == 0 && half_in) ? 1 : ((st == rp.nst - 1 && half_out) ? 2 : 0);
    switch (R) {
      case 16: smem_stage_any<16, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      case 8: smem_stage_any<8, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      case 4: smem_stage_any<4, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      default: smem_stage_any<2, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
    }
    Ns *= R;
  }
}

// Asynchronous global -> shared copy of one complex value (cp.async); with
// valid == false nothing is read and the shared word is zero filled.  The
// source pointer must be a valid address either way.
template <typename T>
__device__ __forceinline__ void cp_async_cx(cx<T>* sdst, const cx<T>* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  const int nbytes = valid ? (int)sizeof(cx<T>) : 0;
  if constexpr (sizeof(cx<T>) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gsrc),
                 "r"(nbytes)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(gsrc),
                 "r"(nbytes)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Copy the L-point twiddles out of the plan's Lmax-point table.
template <typename T>
__device__ __forceinline__ void load_twiddles(cx<T>* stw, const cx<T>* __restrict__ tw, int L,
                                              int twshift) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) stw[t] = tw[(size_t)t * twshift];
}

}  // namespace dda
