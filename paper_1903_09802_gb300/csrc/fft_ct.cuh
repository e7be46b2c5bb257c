// Compile-time specialised shared-memory FFT.
//
// Same Stockham algorithm as fft_core.cuh, but the transform length L, the
// shared-memory row pitch LD, the number of lines NB and therefore the
// radix sequence, the stride Ns of every stage and the thread count are
// template constants.  Every butterfly then addresses shared memory as
// (per-butterfly base register) + (compile-time immediate), the line /
// butterfly split of a thread index is a shift (or a multiply by the
// reciprocal of 3 for three-component tiles), and twiddle indices advance by
// additions; this removes most of the integer work of the run-time version,
// which dominated its instruction count.
#pragma once

#include "fft_kernels.cuh"

namespace dda {

__host__ __device__ constexpr int ct_log2(int v) { return v <= 1 ? 0 : 1 + ct_log2(v / 2); }

// Same stage split as make_radix_plan: ceil(bits/4) stages, larger radices first.
__host__ __device__ constexpr int ct_nst(int L) { return (ct_log2(L) + 3) / 4; }
__host__ __device__ constexpr int ct_bits(int L, int st) {
  int left = ct_log2(L), n = ct_nst(L), b = 0;
  for (int s = 0; s <= st; ++s) {
    b = (left + (n - s) - 1) / (n - s);
    left -= b;
  }
  return b;
}
__host__ __device__ constexpr int ct_radix(int L, int st) { return 1 << ct_bits(L, st); }

// DDA_RR_FFT3C=0 in the environment, or a schedule with rr_z off, selects the
// all-shared-memory z pass.
inline bool rr_fft3c_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("DDA_RR_FFT3C");
    return !(e && e[0] == '0');
  }();
  return on && tl_schedule.rr_z;
}

// One stage: radix R, NS = product of the radices already applied.  The tile
// holds NB lines (NB = NBP or 3 * NBP) of length L; element (b, j) at
// s[j * LD + b]; the block has NB * L / 16 threads.
template <int R, int NS, int MODE, int L, int LD, int NB, bool INV, typename T>
__device__ __forceinline__ void ct_stage(cx<T>* s, const cx<T>* tw, int tid) {
  constexpr int NTH = NB * L / kElemsPerThread;
  constexpr int G = kElemsPerThread / R;
  constexpr int LR = L / R;
  constexpr int QIN = MODE == 1 ? R / 2 : R;
  constexpr int QOUT = MODE == 2 ? R / 2 : R;
  constexpr int TSTEP = L / (NS * R);
  cx<T> v[kElemsPerThread];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * NTH;
    const int jb = u / NB;
    const int b = u - jb * NB;
    const cx<T>* src = s + jb * LD + b;
#pragma unroll
    for (int q = 0; q < QIN; ++q) v[g * R + q] = src[q * LR * LD];
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int u = tid + g * NTH;
    const int jb = u / NB;
    const int b = u - jb * NB;
    if constexpr (NS > 1) {
      const int k = jb & (NS - 1);
      const int kt = k * TSTEP;
      int idx = kt;
#pragma unroll
      for (int q = 1; q < R; ++q, idx += kt) v[g * R + q] = mulc<INV>(v[g * R + q], tw[idx]);
    }
    if constexpr (MODE == 1)
      dft_half_in<R, INV>(&v[g * R]);
    else if constexpr (MODE == 2)
      dft_half_out<R, INV>(&v[g * R]);
    else
      dft<R, INV>(&v[g * R]);
    const int k = jb & (NS - 1);
    cx<T>* dst = s + ((jb - k) * R + k) * LD + b;
#pragma unroll
    for (int q = 0; q < QOUT; ++q) dst[q * NS * LD] = v[g * R + q];
  }
  __syncthreads();
}

template <int ST, int NS, int L, int LD, int NB, bool INV, bool HALF_IN, bool HALF_OUT, typename T>
__device__ __forceinline__ void ct_stages(cx<T>* s, const cx<T>* tw, int tid) {
  if constexpr (ST < ct_nst(L)) {
    constexpr int R = ct_radix(L, ST);
    constexpr int MODE = (ST == 0 && HALF_IN) ? 1 : ((ST == ct_nst(L) - 1 && HALF_OUT) ? 2 : 0);
    ct_stage<R, NS, MODE, L, LD, NB, INV>(s, tw, tid);
    ct_stages<ST + 1, NS * R, L, LD, NB, INV, HALF_IN, HALF_OUT>(s, tw, tid);
  }
}

// Full transform of the NB lines of a tile (caller synchronises before).
template <int L, int LD, int NB, bool INV, bool HALF_IN, bool HALF_OUT, typename T>
__device__ __forceinline__ void ct_fft(cx<T>* s, const cx<T>* tw) {
  ct_stages<0, 1, L, LD, NB, INV, HALF_IN, HALF_OUT>(s, tw, threadIdx.x);
}

// ---------------------------------------------------------------------------
// Kernels.  Tile shapes: strided NB columns, contiguous NB lines, three-
// component tiles 3 * NBC columns.

// Lines along a strided axis (see k_fft_strided); HALF_IN / HALF_OUT when
// the input has Lin = L/2 rows / only Lout = L/2 output rows are kept.
template <typename T, bool INV, int L, int NB, bool HALF_IN, bool HALF_OUT>
__global__ void __launch_bounds__(NB * L / kElemsPerThread, 1024 / (NB * L / kElemsPerThread))
    k_ct_strided(const cx<T>* in, cx<T>* out, long ncols, int Lin, long in_js, long in_ss,
                 int Lout, long out_js, long out_ss, T scale, const cx<T>* __restrict__ tw,
                 int twshift) {
  pdl_entry();
  constexpr int NTH = NB * L / kElemsPerThread;
  constexpr int JSTEP = NTH / NB;  // = L / 16
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + L * NB;
  const int tid = threadIdx.x;
  const long tiles = ncols / NB;
  const long slab = blockIdx.x / tiles;
  const long col0 = (blockIdx.x - slab * tiles) * NB;
  const int b = tid & (NB - 1);
  const int j0 = tid / NB;
  {
    const cx<T>* g = in + slab * in_ss + col0 + (long)j0 * in_js + b;
    const long gstep = (long)JSTEP * in_js;
    constexpr int NLOAD = HALF_IN ? kElemsPerThread / 2 : kElemsPerThread;
#pragma unroll
    for (int i = 0; i < NLOAD; ++i, g += gstep) {
      const int j = j0 + i * JSTEP;
      const bool ok = j < Lin;
      cp_async_cx(s + tid + i * NTH, ok ? g : in, ok);
    }
  }
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  ct_fft<L, NB, NB, INV, HALF_IN, HALF_OUT>(s, stw);
  cx<T>* g = out + slab * out_ss + col0 + (long)j0 * out_js + b;
  const long gstep = (long)JSTEP * out_js;
  constexpr int NSTORE = HALF_OUT ? kElemsPerThread / 2 : kElemsPerThread;
#pragma unroll
  for (int i = 0; i < NSTORE; ++i, g += gstep) {
    const int j = j0 + i * JSTEP;
    if (j < Lout) *g = scale * s[tid + i * NTH];
  }
}

// Lines along the contiguous axis (see k_fft_contig), NB lines per CTA,
// pitch NB + 1; NB >= 16 so that each thread keeps one position j.
template <typename T, bool INV, int L, int NB, bool HALF_IN, bool HALF_OUT>
__global__ void __launch_bounds__(NB * L / kElemsPerThread, 1024 / (NB * L / kElemsPerThread))
    k_ct_contig(const cx<T>* in, cx<T>* out, const uint8_t* __restrict__ mask,
                const uint8_t* __restrict__ omask, long mask_lines, long nlines, int Lin,
                long in_ld, int Lout, long out_ld, T scale, const cx<T>* __restrict__ tw,
                int twshift) {
  pdl_entry();
  static_assert(NB >= 16, "one position per thread");
  constexpr int NTH = NB * L / kElemsPerThread;
  constexpr int LD = NB + 1;
  constexpr int BSTEP = NTH / L;  // = NB / 16
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + L * LD;
  const int tid = threadIdx.x;
  const long line0 = (long)blockIdx.x * NB;
  const int j = tid & (L - 1);
  const int b0 = tid / L;
  if (!(HALF_IN && 2 * j >= L)) {
    // the mask bytes of all 16 elements first (independent loads in
    // flight together), then the 16 copies
    unsigned ok = 0;
    {
      long line = line0 + b0;
      long mrow = line % mask_lines;
#pragma unroll
      for (int i = 0; i < kElemsPerThread; ++i, line += BSTEP) {
        bool v = line < nlines && j < Lin;
        if (v && mask != nullptr) v = __ldg(mask + mrow * Lin + j) != 0;
        ok |= (unsigned)v << i;
        mrow += BSTEP;
        if (mrow >= mask_lines) mrow = mrow >= 2 * mask_lines ? mrow % mask_lines : mrow - mask_lines;
      }
    }
    const cx<T>* g = in + (line0 + b0) * in_ld + j;
    cx<T>* q = s + j * LD + b0;
#pragma unroll
    for (int i = 0; i < kElemsPerThread; ++i, g += BSTEP * in_ld, q += BSTEP) {
      const bool v = (ok >> i) & 1u;
      cp_async_cx(q, v ? g : in, v);
    }
  }
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  ct_fft<L, LD, NB, INV, HALF_IN, HALF_OUT>(s, stw);
  if (j < Lout) {
    long line = line0 + b0;
    long mrow = line % mask_lines;
    cx<T>* g = out + line * out_ld + j;
    const cx<T>* q = s + j * LD + b0;
#pragma unroll 4
    for (int i = 0; i < kElemsPerThread && line < nlines;
         ++i, line += BSTEP, g += BSTEP * out_ld, q += BSTEP) {
      cx<T> w = scale * *q;
      if (omask != nullptr && omask[mrow * Lout + j] == 0) w = zero<T>();
      *g = w;
      mrow += BSTEP;
      if (mrow >= mask_lines) mrow = mrow >= 2 * mask_lines ? mrow % mask_lines : mrow - mask_lines;
    }
  }
}

// Three components of NBC neighbouring columns (see k_fft3c).
template <typename T, class Op, int L, int NBC, bool HALF_IN, bool HALF_OUT>
__global__ void __launch_bounds__(3 * NBC * L / kElemsPerThread,
                                  (768 / (3 * NBC * L / kElemsPerThread)) > 0
                                      ? 768 / (3 * NBC * L / kElemsPerThread)
                                      : 1)
    k_ct_fft3c(cx<T>* data, long ncols, int Lin, long js, long cs, long ss, int Lout, Op op,
               const cx<T>* __restrict__ tw, int twshift, int row_len, int nrows) {
  pdl_entry();
  constexpr int LD = 3 * NBC;
  constexpr int NTH = LD * L / kElemsPerThread;
  constexpr int JSTEP = L / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + L * LD;
  const int tid = threadIdx.x;
  const long tiles = ncols / NBC;
  const long slab = blockIdx.x / tiles;
  const int tt = (int)(blockIdx.x - slab * tiles);
  long col0;
  if (row_len >= NBC && nrows > 0 && row_len % NBC == 0) {
    const int row_tiles = row_len / NBC;
    const int r = tt / row_tiles;
    const int ti = tt - r * row_tiles;
    col0 = (long)mirror_perm(r, nrows) * row_len + (long)mirror_perm(ti, row_tiles) * NBC;
  } else {
    col0 = (long)tt * NBC;
  }
  cx<T>* base = data + slab * ss + col0;
  const int b0 = tid & (NBC - 1);
  const int t0 = tid / NBC;  // 3 j0 + c0
  const int j0 = t0 / 3, c0 = t0 - 3 * j0;
  {
    const cx<T>* g = base + c0 * cs + (long)j0 * js + b0;
    const long gstep = (long)JSTEP * js;
    constexpr int NLOAD = HALF_IN ? kElemsPerThread / 2 : kElemsPerThread;
#pragma unroll
    for (int i = 0; i < NLOAD; ++i, g += gstep) {
      const bool ok = j0 + i * JSTEP < Lin;
      cp_async_cx(s + tid + i * NTH, ok ? g : data, ok);
    }
  }
  op.prefetch(col0, NBC, L);
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  ct_fft<L, LD, LD, false, HALF_IN, false>(s, stw);
  {
    // every thread keeps one column (NTH is a multiple of NBC)
    const auto ctx = op.column(slab, col0 + b0);
    constexpr int PSTEP = NTH / NBC;
#pragma unroll 2
    for (int j = tid / NBC; j < L; j += PSTEP) {
      cx<T>* q = s + j * LD + b0;
      cx<T> x0 = q[0], x1 = q[NBC], x2 = q[2 * NBC];
      op.point(ctx, j, x0, x1, x2);
      q[0] = x0;
      q[NBC] = x1;
      q[2 * NBC] = x2;
    }
  }
  __syncthreads();
  ct_fft<L, LD, LD, true, false, HALF_OUT>(s, stw);
  {
    cx<T>* g = base + c0 * cs + (long)j0 * js + b0;
    const long gstep = (long)JSTEP * js;
    constexpr int NSTORE = HALF_OUT ? kElemsPerThread / 2 : kElemsPerThread;
#pragma unroll
    for (int i = 0; i < NSTORE; ++i, g += gstep)
      if (j0 + i * JSTEP < Lout) *g = s[tid + i * NTH];
  }
}

// Three-component pass of the matvec (zero-padded input, half output kept)
// with the middle of the transform held in registers.  The forward transform
// runs radix R1 then R2, the inverse R2 then R1 (Stockham, natural order at
// both ends), so the butterfly a thread computes last in the forward
// transform covers exactly the frequencies jb + R1 q (q < R2) that its first
// inverse butterfly needs:
//   A  cp.async: rows j < L/2 of the 3 x NBC lines into shared memory;
//   B  forward radix R1 (NS = 1, upper input half zero), shared -> shared;
//   C  forward radix R2 (NS = R1) for all three components of column b,
//      shared -> registers;
//   D  3x3 point operation on the R2 frequencies in registers;
//   E  inverse radix R2 (NS = 1), registers -> shared;
//   F  inverse radix R1 (NS = R2), only outputs j < L/2, shared -> global.
// Every element crosses shared memory about 5.5 times instead of 12.  Tile:
// NBC columns (16: 128-byte rows) x 3 components; in C-E thread tid owns
// column b = tid % NBC, butterfly jb = tid / NBC.
template <class Op, int L, int R1, int R2, int NBC, bool HALF>
__device__ __forceinline__ void rr_fft3c_body(cx<float>* data, long ncols, long js, long cs,
                                              long ss, const Op& op,
                                              const cx<float>* __restrict__ tw, int twshift,
                                              int row_len, int nrows) {
  static_assert(R1 * R2 == L, "two stages");
  using T = float;
  constexpr int NL = 3 * NBC;  // lines (component, column) of the tile
  constexpr int LD = NL;       // shared row pitch
  // With 24 lines (8-column tiles) every group of 8 rows is followed by 8
  // unused values: the stores of stage E (rows jb R2 + q, four jb per warp)
  // and B then fall on distinct banks (2 wavefronts per access instead of 4).
  constexpr int PADR = NL == 24 ? 8 : 0;
  constexpr int NTH = R1 * NBC;
  constexpr int NBF = NL * R2;                // butterflies of stage B (and F)
  constexpr int GB = (NBF + NTH - 1) / NTH;   // per thread
  constexpr int H = L / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + L * LD + (L / 8) * PADR;
  // row(a + b) = row(a) + row(b) when a or b is a multiple of 8: the
  // compile-time part of each index below is kept apart
  auto row = [](int j) { return j * LD + (j >> 3) * PADR; };
  const int tid = threadIdx.x;
  const long tiles = ncols / NBC;
  const long slab = blockIdx.x / tiles;
  const int tt = (int)(blockIdx.x - slab * tiles);
  long col0;
  if (row_len >= NBC && nrows > 0 && row_len % NBC == 0) {
    const int row_tiles = row_len / NBC;
    const int r = tt / row_tiles;
    const int ti = tt - r * row_tiles;
    col0 = (long)mirror_perm(r, nrows) * row_len + (long)mirror_perm(ti, row_tiles) * NBC;
  } else {
    col0 = (long)tt * NBC;
  }
  cx<T>* base = data + slab * ss + col0;
  constexpr int ROWS_IN = HALF ? H : L;  // rows loaded (the rest are zero padding)
  // A: 16-byte copies of two neighbouring columns (tiles start on even
  // columns, rows and component planes are even strides, shared rows even)
  constexpr int NLH = NL / 2;
#pragma unroll 3
  for (int e = tid; e < ROWS_IN * NLH; e += NTH) {
    const int j = e / NLH, line = 2 * (e - j * NLH);
    const int c = line / NBC, b = line - c * NBC;
    cp_async_16(s + row(j) + line, base + c * cs + (long)j * js + b);
  }
  op.prefetch(col0, NBC, L);
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  // B: inputs rows jb + q R2 (with HALF only q < R1/2 non-zero), outputs rows jb R1 + q
  {
    cx<T> v[GB][R1];
#pragma unroll
    for (int g = 0; g < GB; ++g) {
      const int u = tid + g * NTH;
      if (u < NBF) {
        const int jb = u / NL, line = u - jb * NL;
#pragma unroll
        for (int q = 0; q < (HALF ? R1 / 2 : R1); ++q) v[g][q] = s[row(jb) + row(q * R2) + line];
      }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < GB; ++g) {
      const int u = tid + g * NTH;
      if (u < NBF) {
        const int jb = u / NL, line = u - jb * NL;
        if constexpr (HALF)
          dft_half_in<R1, false>(v[g]);
        else
          dft<R1, false>(v[g]);
#pragma unroll
        for (int q = 0; q < R1; ++q) s[row(jb * R1) + row(q) + line] = v[g][q];
      }
    }
    __syncthreads();
  }
  const int b = tid % NBC, jb = tid / NBC;  // jb < R1
  cx<T> x[3][R2];
  // the spectrum of the first frequency is requested before stage C, that of
  // each next one before the current one is multiplied (D)
  const auto ctx = op.column(slab, col0 + b);
  typename Op::G6r gn;
  op.load_raw(ctx, jb, gn);
  // C: inputs rows jb + q R1, twiddle w^(q jb), outputs frequencies jb + q R1
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int q = 0; q < R2; ++q) x[c][q] = s[row(jb) + row(q * R1) + c * NBC + b];
#pragma unroll
    for (int q = 1; q < R2; ++q) x[c][q] = mulc<false>(x[c][q], stw[q * jb]);
    dft<R2, false>(x[c]);
  }
  // D
#pragma unroll
  for (int q = 0; q < R2; ++q) {
    const typename Op::G6r g = gn;
    if (q + 1 < R2) op.load_raw(ctx, jb + (q + 1) * R1, gn);
    op.mul_raw(g, x[0][q], x[1][q], x[2][q]);
  }
  // E: inverse radix R2 on the same frequencies, outputs rows jb R2 + q
#pragma unroll
  for (int c = 0; c < 3; ++c) dft<R2, true>(x[c]);
  __syncthreads();  // every thread has read its stage-C inputs
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < R2; ++q) s[row(jb * R2) + row(q) + c * NBC + b] = x[c][q];
  __syncthreads();
  // F: inputs rows j2 + q R2, twiddle conj(w)^(q j2), outputs rows j2 + q R2 < L/2
#pragma unroll
  for (int g = 0; g < GB; ++g) {
    const int u = tid + g * NTH;
    if (u < NBF) {
      const int j2 = u / NL, line = u - j2 * NL;
      const int c = line / NBC, bb = line - c * NBC;
      cx<T> v[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) v[q] = s[row(j2) + row(q * R2) + line];
#pragma unroll
      for (int q = 1; q < R1; ++q) v[q] = mulc<true>(v[q], stw[q * j2]);
      if constexpr (HALF)
        dft_half_out<R1, true>(v);
      else
        dft<R1, true>(v);
      cx<T>* g = base + c * cs + bb;
#pragma unroll
      for (int q = 0; q < (HALF ? R1 / 2 : R1); ++q) g[(long)(j2 + q * R2) * js] = v[q];
    }
  }
}

// The pass as a kernel: registers left to the compiler (k_rr_fft3c), or
// bounded so that MINB blocks fit on an SM (k_rr_fft3c_mb: more warps in
// flight, fewer registers per thread).
template <class Op, int L, int R1, int R2, int NBC, bool HALF>
__global__ void __launch_bounds__(R1 * NBC)
    k_rr_fft3c(cx<float>* data, long ncols, long js, long cs, long ss, Op op,
               const cx<float>* __restrict__ tw, int twshift, int row_len, int nrows) {
  pdl_entry();
  rr_fft3c_body<Op, L, R1, R2, NBC, HALF>(data, ncols, js, cs, ss, op, tw, twshift, row_len,
                                           nrows);
}
template <class Op, int L, int R1, int R2, int NBC, bool HALF, int MINB>
__global__ void __launch_bounds__(R1 * NBC, MINB)
    k_rr_fft3c_mb(cx<float>* data, long ncols, long js, long cs, long ss, Op op,
                  const cx<float>* __restrict__ tw, int twshift, int row_len, int nrows) {
  pdl_entry();
  rr_fft3c_body<Op, L, R1, R2, NBC, HALF>(data, ncols, js, cs, ss, op, tw, twshift, row_len,
                                           nrows);
}

// The same pass with three stages each way, for lengths where two stages
// would need too many registers (L = 512 = 8 x 8 x 8): forward radix R1a
// (first input half zero) and R1b in shared memory, R2 from shared memory
// into registers, the 3x3 point operation on the R2 frequencies a thread
// holds (jb + q L/R2), inverse R2 from registers to shared memory, then
// inverse R1b and R1a (only outputs j < L/2) back to global memory.  Stockham
// indexing per stage (NS = product of the radices already applied):
// butterfly jb reads x[jb + q L/R], twiddle w^{q (jb mod NS) L/(NS R)},
// writes y[(jb - jb mod NS) R + jb mod NS + q NS].
template <class Op, int L, int R1A, int R1B, int R2, int NBC, bool HALF>
__global__ void __launch_bounds__(NBC * (L / R2))
    k_rr3_fft3c(cx<float>* data, long ncols, long js, long cs, long ss, Op op,
                const cx<float>* __restrict__ tw, int twshift, int row_len, int nrows) {
  pdl_entry();
  static_assert(R1A * R1B * R2 == L, "three stages");
  using T = float;
  constexpr int NL = 3 * NBC;
  constexpr int LD = NL;
  constexpr int NTH = NBC * (L / R2);
  constexpr int H = L / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + L * LD;
  const int tid = threadIdx.x;
  const long tiles = ncols / NBC;
  const long slab = blockIdx.x / tiles;
  const int tt = (int)(blockIdx.x - slab * tiles);
  long col0;
  if (row_len >= NBC && nrows > 0 && row_len % NBC == 0) {
    const int row_tiles = row_len / NBC;
    const int r = tt / row_tiles;
    const int ti = tt - r * row_tiles;
    col0 = (long)mirror_perm(r, nrows) * row_len + (long)mirror_perm(ti, row_tiles) * NBC;
  } else {
    col0 = (long)tt * NBC;
  }
  cx<T>* base = data + slab * ss + col0;
  constexpr int ROWS_IN = HALF ? H : L;
  // A: rows j < L/2 (HALF) or all rows of the 3 x NBC lines
#pragma unroll 4
  for (int e = tid; e < ROWS_IN * NL; e += NTH) {
    const int j = e / NL, line = e - j * NL;
    const int c = line / NBC, b = line - c * NBC;
    cp_async_cx(s + j * LD + line, base + c * cs + (long)j * js + b, true);
  }
  op.prefetch(col0, NBC, L);
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  // B1: radix R1A, NS = 1, input rows jb + q L/R1A (q < R1A/2 non-zero)
  {
    constexpr int NB1 = NL * (L / R1A);
    constexpr int G = (NB1 + NTH - 1) / NTH;
    cx<T> v[G][R1A];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB1) {
        const int jb = u / NL, line = u - jb * NL;
#pragma unroll
        for (int q = 0; q < (HALF ? R1A / 2 : R1A); ++q)
          v[g][q] = s[(jb + q * (L / R1A)) * LD + line];
      }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB1) {
        const int jb = u / NL, line = u - jb * NL;
        if constexpr (HALF)
          dft_half_in<R1A, false>(v[g]);
        else
          dft<R1A, false>(v[g]);
#pragma unroll
        for (int q = 0; q < R1A; ++q) s[(jb * R1A + q) * LD + line] = v[g][q];
      }
    }
    __syncthreads();
  }
  // B2: radix R1B, NS = R1A
  {
    constexpr int NB2 = NL * (L / R1B);
    constexpr int G = (NB2 + NTH - 1) / NTH;
    cx<T> v[G][R1B];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB2) {
        const int jb = u / NL, line = u - jb * NL;
#pragma unroll
        for (int q = 0; q < R1B; ++q) v[g][q] = s[(jb + q * (L / R1B)) * LD + line];
      }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB2) {
        const int jb = u / NL, line = u - jb * NL;
        const int k = jb % R1A;
#pragma unroll
        for (int q = 1; q < R1B; ++q) v[g][q] = mulc<false>(v[g][q], stw[q * k * R2]);
        dft<R1B, false>(v[g]);
#pragma unroll
        for (int q = 0; q < R1B; ++q) s[((jb - k) * R1B + k + q * R1A) * LD + line] = v[g][q];
      }
    }
    __syncthreads();
  }
  // C: radix R2, NS = L/R2, rows jb + q L/R2 of all three components of column b
  const int b = tid % NBC, jb = tid / NBC;  // jb < L/R2
  cx<T> x[3][R2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int q = 0; q < R2; ++q) x[c][q] = s[(jb + q * (L / R2)) * LD + c * NBC + b];
#pragma unroll
    for (int q = 1; q < R2; ++q) x[c][q] = mulc<false>(x[c][q], stw[q * jb]);
    dft<R2, false>(x[c]);
  }
  // D
  {
    const auto ctx = op.column(slab, col0 + b);
#pragma unroll
    for (int q = 0; q < R2; ++q) op.point(ctx, jb + q * (L / R2), x[0][q], x[1][q], x[2][q]);
  }
  // E: inverse radix R2, NS = 1, outputs rows jb R2 + q
#pragma unroll
  for (int c = 0; c < 3; ++c) dft<R2, true>(x[c]);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < R2; ++q) s[(jb * R2 + q) * LD + c * NBC + b] = x[c][q];
  __syncthreads();
  // F1: inverse radix R1B, NS = R2
  {
    constexpr int NB2 = NL * (L / R1B);
    constexpr int G = (NB2 + NTH - 1) / NTH;
    cx<T> v[G][R1B];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB2) {
        const int j2 = u / NL, line = u - j2 * NL;
#pragma unroll
        for (int q = 0; q < R1B; ++q) v[g][q] = s[(j2 + q * (L / R1B)) * LD + line];
      }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = tid + g * NTH;
      if (u < NB2) {
        const int j2 = u / NL, line = u - j2 * NL;
        const int k = j2 % R2;
#pragma unroll
        for (int q = 1; q < R1B; ++q) v[g][q] = mulc<true>(v[g][q], stw[q * k * R1A]);
        dft<R1B, true>(v[g]);
#pragma unroll
        for (int q = 0; q < R1B; ++q) s[((j2 - k) * R1B + k + q * R2) * LD + line] = v[g][q];
      }
    }
    __syncthreads();
  }
  // F2: inverse radix R1A, NS = L/R1A, only outputs j < L/2, to global memory
  {
    constexpr int NB1 = NL * (L / R1A);
#pragma unroll 2
    for (int u = tid; u < NB1; u += NTH) {
      const int j2 = u / NL, line = u - j2 * NL;
      const int c = line / NBC, bb = line - c * NBC;
      cx<T> v[R1A];
#pragma unroll
      for (int q = 0; q < R1A; ++q) v[q] = s[(j2 + q * (L / R1A)) * LD + line];
#pragma unroll
      for (int q = 1; q < R1A; ++q) v[q] = mulc<true>(v[q], stw[q * j2]);
      if constexpr (HALF)
        dft_half_out<R1A, true>(v);
      else
        dft<R1A, true>(v);
      cx<T>* g = base + c * cs + bb;
#pragma unroll
      for (int q = 0; q < (HALF ? R1A / 2 : R1A); ++q) g[(long)(j2 + q * (L / R1A)) * js] = v[q];
    }
  }
}

template <int L, int R1A, int R1B, int R2, int NBC, bool HALF, class Op>
void rr3_fft3c_launch(cx<float>* data, long ncols, long nslabs, long js, long cs, long ss,
                      const Op& op, const cx<float>* tw, int Lmax, int row_len, int nrows,
                      cudaStream_t s) {
  const size_t smem = ((size_t)3 * NBC * L + L) * sizeof(cx<float>);
  auto kern = k_rr3_fft3c<Op, L, R1A, R1B, R2, NBC, HALF>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long grid = nslabs * (ncols / NBC);
  note_launch();
  launch_k(kern, (unsigned)grid, NBC * (L / R2), smem, s, data, ncols, js, cs, ss, op, tw,
           Lmax / L, row_len, nrows);
}

template <int L, int R1, int R2, int NBC, bool HALF, class Op>
void rr_fft3c_launch(cx<float>* data, long ncols, long nslabs, long js, long cs, long ss,
                     const Op& op, const cx<float>* tw, int Lmax, int row_len, int nrows,
                     cudaStream_t s) {
  // tile, its row padding (8 values per 8 rows with 8-column tiles) and the twiddles
  const size_t smem =
      ((size_t)3 * NBC * L + (3 * NBC == 24 ? L : 0) + L) * sizeof(cx<float>);
  // 256-thread tiles (lengths 128 and 256) with registers bounded so that
  // three blocks share an SM (schedule z_occ, the default): measured 11%
  // faster at length 256 and 4% at 128 than the compiler's own count (two
  // blocks); four blocks spill.
  auto kern = (R1 * NBC == 256 && tl_schedule.z_occ) ? k_rr_fft3c_mb<Op, L, R1, R2, NBC, HALF, 3>
                                                     : k_rr_fft3c<Op, L, R1, R2, NBC, HALF>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long grid = nslabs * (ncols / NBC);
  note_launch();
  launch_k(kern, (unsigned)grid, R1 * NBC, smem, s, data, ncols, js, cs, ss, op, tw, Lmax / L,
           row_len, nrows);
}

// Three-component pass: compile-time kernel for complex64 when the tile
// shape allows (L in 32..512, 8-column tiles), the run-time kernel otherwise.
template <int L, class Op, bool HI, bool HO>
void ct_fft3c_launch(cx<float>* data, long ncols, long nslabs, int Lin, long js, long cs, long ss,
                     int Lout, const Op& op, const cx<float>* tw, int Lmax, int row_len, int nrows,
                     cudaStream_t s) {
  constexpr int NBC = 8;
  constexpr int NTH = 3 * NBC * L / kElemsPerThread;
  const size_t smem = ((size_t)3 * NBC * L + L) * sizeof(cx<float>);
  auto kern = k_ct_fft3c<float, Op, L, NBC, HI, HO>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long grid = nslabs * (ncols / NBC);
  note_launch();
  launch_k(kern, (unsigned)grid, NTH, smem, s, data, ncols, Lin, js, cs, ss, Lout, op, tw, Lmax / L,
                                         row_len, nrows);
}

template <class Op, bool HI, bool HO>
bool ct_fft3c_dispatch(cx<float>* data, long ncols, long nslabs, int L, int Lin, long js, long cs,
                       long ss, int Lout, const Op& op, const cx<float>* tw, int Lmax, int row_len,
                       int nrows, cudaStream_t s) {
  // Register-resident forms: the last forward and the first inverse stage
  // in registers, the point operation between them; the matvec's pass (HI
  // and HO: zero-padded input, half of the output kept) at lengths 64 to
  // 512.  (Length 256 as 16 x 16 needs 48 register values per thread and
  // 180 registers: measured slower than the all-shared-memory kernel; as
  // 32 x 8 the register stage holds 3 x 8 values.  The preconditioner's pass
  // (full input and output) measured 10-15% slower in these forms than in
  // the all-shared-memory kernel, so it keeps that one.)
  if constexpr (HI && HO) {
    if (rr_fft3c_enabled()) {
      if (ncols % 16 == 0 && L == 64) {
        rr_fft3c_launch<64, 8, 8, 16, HI>(data, ncols, nslabs, js, cs, ss, op, tw, Lmax, row_len,
                                          nrows, s);
        return true;
      }
      if (ncols % 16 == 0 && L == 128) {
        rr_fft3c_launch<128, 16, 8, 16, HI>(data, ncols, nslabs, js, cs, ss, op, tw, Lmax,
                                            row_len, nrows, s);
        return true;
      }
      if (ncols % 8 == 0 && L == 256) {
        rr_fft3c_launch<256, 32, 8, 8, HI>(data, ncols, nslabs, js, cs, ss, op, tw, Lmax, row_len,
                                           nrows, s);
        return true;
      }
      if (ncols % 8 == 0 && L == 512) {
        rr3_fft3c_launch<512, 8, 8, 8, 8, HI>(data, ncols, nslabs, js, cs, ss, op, tw, Lmax,
                                              row_len, nrows, s);
        return true;
      }
    }
  }
  switch (L) {
    case 32: ct_fft3c_launch<32, Op, HI, HO>(data, ncols, nslabs, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s); return true;
    case 64: ct_fft3c_launch<64, Op, HI, HO>(data, ncols, nslabs, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s); return true;
    case 128: ct_fft3c_launch<128, Op, HI, HO>(data, ncols, nslabs, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s); return true;
    case 256: ct_fft3c_launch<256, Op, HI, HO>(data, ncols, nslabs, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s); return true;
    case 512: ct_fft3c_launch<512, Op, HI, HO>(data, ncols, nslabs, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s); return true;
    default: return false;
  }
}

// Dispatcher used by the operator: HI / HO are fixed per call site (the
// matvec's z pass has both, the preconditioner's neither).
template <bool HI, bool HO, typename T, class Op>
void launch_fft3c_any(cx<T>* data, long ncols, long nslabs, int L, int Lin, long js, long cs,
                      long ss, int Lout, const Op& op, const cx<T>* tw, int Lmax, int row_len,
                      int nrows, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const bool hi = 2 * Lin <= L, ho = 2 * Lout <= L;
    if (hi == HI && ho == HO && ncols % 8 == 0 && ncols >= 8 &&
        ct_fft3c_dispatch<Op, HI, HO>(data, ncols, nslabs, L, Lin, js, cs, ss, Lout, op, tw, Lmax,
                                      row_len, nrows, s))
      return;
  }
  launch_fft3c<T>(data, ncols, nslabs, L, Lin, js, cs, ss, Lout, op, tw, Lmax, row_len, nrows, s);
}

}  // namespace dda
