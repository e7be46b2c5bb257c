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
// Mixed-radix kernels hold 8 values per thread: the odd radices' butterflies
// then fit in registers in every precision (no local stack frame).
constexpr int kElemsMR = 8;
template <bool MR>
__host__ __device__ constexpr int elems_per_thread() {
  return MR ? kElemsMR : kElemsPerThread;
}

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

// Radix sequence of a transform of length L.  Powers of two: at most 4
// stages of radix 2..16 (L <= 65536), lg = log2 L.  Other 7-smooth lengths
// (mixed radix): stages of radix 2, 4, 3, 5, 7, an even one first and, when
// the power of two allows, last (at most 8 stages for L <= 1024); lg is
// then unused.  hin / hout: the first / last radix is even,
// so a zero upper input half can be skipped in the first stage and the upper
// output half left uncomputed in the last.
struct RadixPlan {
  int nst;
  int lg;
  int L;
  int pow2;
  int hin, hout;
  int r[8];
};

inline int ilog2i(long v) {
  int b = 0;
  while ((1L << b) < v) ++b;
  return b;
}

inline bool is_7smooth(long v) {
  if (v < 1) return false;
  for (int f : {2, 3, 5, 7})
    while (v % f == 0) v /= f;
  return v == 1;
}

inline RadixPlan make_radix_plan(int L) {
  RadixPlan p{0, 0, L, 1, 0, 0, {1, 1, 1, 1, 1, 1, 1, 1}};
  if ((L & (L - 1)) == 0) {
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
    p.hin = p.hout = 1;
    return p;
  }
  p.pow2 = 0;
  int rest = L, a = 0;
  while (rest % 2 == 0) rest /= 2, ++a;
  // power-of-two part as radix-4 stages (one radix 2 when a is odd), one of
  // them first and one last, the odd primes and the other radix-4 stages
  // between them (only radices 2, 3, 4, 5, 7: the mixed-radix stages stay
  // small, and so does their compile time in every precision)
  int p2[8], n2 = 0;
  if (a % 2) p2[n2++] = 2;
  for (int i = 0; i < a / 2 && n2 < 8; ++i) p2[n2++] = 4;
  int k = 0;
  if (n2 > 0) p.r[p.nst++] = p2[k++];
  for (int f : {7, 5, 3})
    while (rest % f == 0 && p.nst < 8) rest /= f, p.r[p.nst++] = f;
  while (k < n2 - 1 && p.nst < 8) p.r[p.nst++] = p2[k++];
  if (k < n2 && p.nst < 8) p.r[p.nst++] = p2[k++];
  p.hin = n2 > 0;
  p.hout = n2 > 1;
  if (rest != 1 || k != n2) p.nst = -1;  // not 7-smooth, or over 8 stages: rejected
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

// cos and sin of 2 pi t / R for the odd radices (plain trigonometric values).
__host__ __device__ constexpr double odd_cos(int R, int t) {
  t %= R;
  if (2 * t > R) t = R - t;
  return t == 0 ? 1.0
         : R == 3 ? -0.5
         : R == 5 ? (t == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
                  : (t == 1 ? 0.623489801858733530525
                            : t == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double odd_sin(int R, int t) {
  t %= R;
  const double sg = 2 * t > R ? -1.0 : 1.0;
  if (2 * t > R) t = R - t;
  return t == 0 ? 0.0
         : sg * (R == 3 ? 0.8660254037844386467637
                 : R == 5 ? (t == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
                          : (t == 1 ? 0.7818314824680298087084
                                    : t == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758));
}

// In-register R-point DFT for odd R (3, 5, 7), natural order in and out:
// with s_j = v_j + v_{R-j} and d_j = v_j - v_{R-j} (0 < j <= (R-1)/2),
//   X_0 = v_0 + sum_j s_j,
//   X_k, X_{R-k} = v_0 + sum_j cos(2 pi jk/R) s_j  -/+ i sum_j sin(2 pi jk/R) d_j
// (forward; the inverse swaps the two signs).
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_odd(cx<T>* v) {
  constexpr int H = (R - 1) / 2;
  cx<T> sp[H], sm[H];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    sp[j - 1] = v[j] + v[R - j];
    sm[j - 1] = v[j] - v[R - j];
  }
  const cx<T> x0 = v[0];
  cx<T> out[R];
  out[0] = x0;
#pragma unroll
  for (int j = 0; j < H; ++j) out[0] = out[0] + sp[j];
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cx<T> a = x0, b = zero<T>();
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      const T c = (T)odd_cos(R, j * k), sn = (T)odd_sin(R, j * k);
      a = mk<T>(a.x + c * sp[j - 1].x, a.y + c * sp[j - 1].y);
      b = mk<T>(b.x + sn * sm[j - 1].x, b.y + sn * sm[j - 1].y);
    }
    // -i b = (b.y, -b.x), +i b = (-b.y, b.x)
    const cx<T> lo = mk<T>(a.x + b.y, a.y - b.x), hi = mk<T>(a.x - b.y, a.y + b.x);
    out[k] = INV ? hi : lo;
    out[R - k] = INV ? lo : hi;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

// One Stockham stage of radix R on lines of any length L (mixed radix): the
// same indexing as smem_stage with k = jb mod Ns by division.  A thread holds
// up to ceil(8 / R) butterflies (NB L / R of them in the tile, 8 values per
// thread).
template <int R, bool INV, bool MUL3, int MODE, typename T>
__device__ __forceinline__ void smem_stage_mr(cx<T>* s, const cx<T>* tw, int L, int sh, int ld,
                                              int Ns, int tid, int nth) {
  constexpr int G = (kElemsMR + R - 1) / R;
  constexpr int QIN = MODE == 1 ? R / 2 : R;
  constexpr int QOUT = MODE == 2 ? R / 2 : R;
  const int nbf = nth * kElemsMR / R;
  const int LR = L / R;
  cx<T> v[G][R];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * nth;
    if (u < nbf) {
      int b, jb;
      split_line<MUL3>(u, sh, b, jb);
#pragma unroll
      for (int q = 0; q < QIN; ++q) v[g][q] = s[(jb + q * LR) * ld + b];
    }
  }
  __syncthreads();
  const int tstep = L / (Ns * R);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * nth;
    if (u < nbf) {
      int b, jb;
      split_line<MUL3>(u, sh, b, jb);
      const int k = jb % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int q = 1; q < R; ++q) v[g][q] = mulc<INV>(v[g][q], tw[q * k * tstep]);
      }
      if constexpr (R % 2 == 1)
        dft_odd<R, INV>(v[g]);
      else if constexpr (MODE == 1)
        dft_half_in<R, INV>(v[g]);
      else if constexpr (MODE == 2)
        dft_half_out<R, INV>(v[g]);
      else
        dft<R, INV>(v[g]);
      const int base = (jb - k) * R + k;
#pragma unroll
      for (int q = 0; q < QOUT; ++q) s[(base + q * Ns) * ld + b] = v[g][q];
    }
  }
  __syncthreads();
}

template <int R, bool INV, bool MUL3, typename T>
__device__ __forceinline__ void smem_stage_mr_any(int mode, cx<T>* s, const cx<T>* tw, int L,
                                                  int sh, int ld, int Ns, int tid, int nth) {
  if constexpr (R % 2 == 0) {
    if (mode == 1) {
      smem_stage_mr<R, INV, MUL3, 1>(s, tw, L, sh, ld, Ns, tid, nth);
      return;
    }
    if (mode == 2) {
      smem_stage_mr<R, INV, MUL3, 2>(s, tw, L, sh, ld, Ns, tid, nth);
      return;
    }
  }
  smem_stage_mr<R, INV, MUL3, 0>(s, tw, L, sh, ld, Ns, tid, nth);
}

// Mixed-radix transform of the tile's lines (any 7-smooth L of the plan);
// same contract as smem_fft, with 8 values per thread (kElemsMR).  half_in /
// half_out must only be asked for when the plan's first / last radix is even
// (rp.hin / rp.hout).  Used by the mixed-radix kernels only (kernel template
// flag MR), so that power-of-two kernels carry none of it.
template <bool INV, bool MUL3, typename T>
__device__ __forceinline__ void smem_fft_mr(cx<T>* s, const cx<T>* tw, int L, int sh, int ld,
                                            const RadixPlan& rp, bool half_in, bool half_out) {
  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  int Ns = 1;
  for (int st = 0; st < rp.nst; ++st) {
    const int R = rp.r[st];
    const int mode = (st == 0 && half_in) ? 1 : ((st == rp.nst - 1 && half_out) ? 2 : 0);
    switch (R) {
      case 7: smem_stage_mr_any<7, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      case 5: smem_stage_mr_any<5, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      case 4: smem_stage_mr_any<4, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      case 3: smem_stage_mr_any<3, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
      default: smem_stage_mr_any<2, INV, MUL3>(mode, s, tw, L, sh, ld, Ns, tid, nth); break;
    }
    Ns *= R;
  }
}

// Either form: MR (a kernel template flag) selects the mixed-radix one.
template <bool INV, bool MUL3, bool MR, typename T>
__device__ __forceinline__ void smem_fft_plan(cx<T>* s, const cx<T>* tw, int sh, int ld,
                                              const RadixPlan& rp, bool half_in, bool half_out) {
  if constexpr (MR)
    smem_fft_mr<INV, MUL3, T>(s, tw, rp.L, sh, ld, rp, half_in, half_out);
  else
    smem_fft<INV, MUL3>(s, tw, rp.L, sh, ld, rp, half_in, half_out);
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
// 16 bytes (two complex64 values), both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gsrc) : "memory");
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
