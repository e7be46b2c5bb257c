// Batched line-FFT kernels over HBM arrays, built on the shared-memory
// Stockham core.  Three shapes cover every transform of the library:
//   k_fft_contig  lines along the contiguous axis (x)
//   k_fft_strided lines along a strided axis (y or z), tiles of NB
//                 neighbouring columns so each row of a tile is one
//                 coalesced segment
//   k_fft3c       the three field components of a strided tile together,
//                 forward transform, a per-frequency 3x3 operation, inverse
//                 transform, in one pass over HBM
// Tiles are loaded with asynchronous global -> shared copies (cp.async,
// zero filled where the input is padding or masked), 16 per thread issued
// back to back, so each SM keeps many loads in flight without staging them
// in registers.  An optional uint8 mask (one row of Lin / Lout flags per
// line, repeating every mask_lines lines) zeroes inputs or outputs of
// contiguous lines.  Inputs shorter than the transform are zero padded
// (Lin < L); outputs can be truncated (Lout < L), which is how the circulant
// embedding of the BTTB matvec is pruned.  A CTA reads all of its lines
// before it writes any, so every kernel may run in place (in == out).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "dfloat.cuh"
#include "fft_core.cuh"

namespace dda {

// Threads per CTA of the three-component pass: double-float values need
// twice the registers of their arithmetic, so that kernel keeps 256 threads
// (255 registers each) instead of 512.
template <typename T>
__host__ __device__ constexpr int fft3c_max_threads() {
  return sizeof(T) == 4 ? 768 : (std::is_same<T, df>::value ? 256 : 512);
}

template <typename T, bool INV, bool MR>
__global__ void __launch_bounds__(256)
    k_fft_contig(const cx<T>* in, cx<T>* out, const uint8_t* __restrict__ mask,
                 const uint8_t* __restrict__ omask, long mask_lines, long nlines, int Lin,
                 long in_ld, int Lout, long out_ld, T scale, const cx<T>* __restrict__ tw,
                 int twshift, RadixPlan rp, int nb_sh) {
  pdl_entry();
  constexpr int EPT = elems_per_thread<MR>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int L = rp.L;
  const int NB = 1 << nb_sh;
  const int ld = NB + 1;
  cx<T>* stw = s + (size_t)L * ld;
  const int nth = blockDim.x, tid = threadIdx.x;
  const long line0 = (long)blockIdx.x << nb_sh;
  const bool half_in = 2 * Lin <= L && L > 1 && rp.hin;
  const bool half_out = 2 * Lout <= L && L > 1 && rp.hout;
  // Thread tid keeps position j = tid mod L of lines b0 + i * (nth / L)
  // (nth / L >= 1 since nth = NB L / 16 and NB >= 16 whenever L < nth); a
  // mixed-radix length takes the per-element loops below.
  const int j = MR ? 0 : tid & (L - 1);
  const int b0 = MR ? 0 : tid >> rp.lg;
  const int bstep = MR ? 0 : nth >> rp.lg;
  if (bstep > 0) {
    if (!(half_in && 2 * j >= L)) {  // the pruned first stage never reads j >= L/2
      long line = line0 + b0;
      long mrow = line % mask_lines;  // mask row, advanced incrementally
      const cx<T>* g = in + line * in_ld + j;
      const long gstep = (long)bstep * in_ld;
      cx<T>* q = s + j * ld + b0;
#pragma unroll 4
      for (int i = 0; i < EPT; ++i, line += bstep, g += gstep, q += bstep) {
        bool ok = line < nlines && j < Lin;
        if (ok && mask != nullptr) ok = mask[mrow * Lin + j] != 0;
        cp_async_cx(q, ok ? g : in, ok);
        mrow += bstep;
        if (mrow >= mask_lines) mrow = mrow >= 2 * mask_lines ? mrow % mask_lines : mrow - mask_lines;
      }
    }
  } else {
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nth;
      const int jj = MR ? e % L : e & (L - 1);
      const int b = MR ? e / L : e >> rp.lg;
      const long line = line0 + b;
      if (half_in && 2 * jj >= L) continue;
      bool ok = line < nlines && jj < Lin;
      if (ok && mask != nullptr) ok = mask[(line % mask_lines) * Lin + jj] != 0;
      cp_async_cx(s + jj * ld + b, ok ? in + line * in_ld + jj : in, ok);
    }
  }
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  smem_fft_plan<INV, false, MR>(s, stw, nb_sh, ld, rp, half_in, half_out);
  if (bstep > 0) {
    if (j < Lout) {
      long line = line0 + b0;
      long mrow = line % mask_lines;
      cx<T>* g = out + line * out_ld + j;
      const long gstep = (long)bstep * out_ld;
      const cx<T>* q = s + j * ld + b0;
#pragma unroll 4
      for (int i = 0; i < EPT && line < nlines;
           ++i, line += bstep, g += gstep, q += bstep) {
        cx<T> w = scale * *q;
        if (omask != nullptr && omask[mrow * Lout + j] == 0) w = zero<T>();
        *g = w;
        mrow += bstep;
        if (mrow >= mask_lines) mrow = mrow >= 2 * mask_lines ? mrow % mask_lines : mrow - mask_lines;
      }
    }
  } else {
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nth;
      const int jj = MR ? e % L : e & (L - 1);
      const int b = MR ? e / L : e >> rp.lg;
      const long line = line0 + b;
      if (line < nlines && jj < Lout) {
        cx<T> w = scale * s[jj * ld + b];
        if (omask != nullptr && omask[(line % mask_lines) * Lout + jj] == 0) w = zero<T>();
        out[line * out_ld + jj] = w;
      }
    }
  }
}

template <typename T, bool INV, bool FIX, bool MR>
__global__ void __launch_bounds__(MR ? 256 : 512)
    k_fft_strided(const cx<T>* in, cx<T>* out, long ncols, int Lin, long in_js, long in_ss,
                  int Lout, long out_js, long out_ss, T scale, const cx<T>* __restrict__ tw,
                  int twshift, RadixPlan rp, int nb_sh) {
  pdl_entry();
  constexpr int EPT = elems_per_thread<MR>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int L = rp.L;
  const int NB = 1 << nb_sh;
  cx<T>* stw = s + ((size_t)L << nb_sh);
  const int nth = blockDim.x, tid = threadIdx.x;
  const long tiles = (ncols + NB - 1) >> nb_sh;
  const long slab = blockIdx.x / tiles;
  const long col0 = (blockIdx.x - slab * tiles) << nb_sh;
  const cx<T>* src = in + slab * in_ss + col0;
  const bool half_in = 2 * Lin <= L && L > 1 && rp.hin;
  const bool half_out = 2 * Lout <= L && L > 1 && rp.hout;
  const int nload = half_in ? EPT / 2 : EPT;  // rows < L/2 only
  // Thread tid keeps column b = tid mod NB and rows j0 + i * (nth / NB):
  // addresses advance by constant strides.
  // (FIX: L a multiple of 16, so nth / NB = L / 16 >= 1; other lengths take
  // the generic loop).
  const int b = tid & (NB - 1);
  const int j0 = tid >> nb_sh;
  const int jstep = nth >> nb_sh;
  const bool colok = col0 + b < ncols;
  if constexpr (FIX) {
    const cx<T>* g = src + (long)j0 * in_js + b;
    const long gstep = (long)jstep * in_js;
    cx<T>* q = s + tid;
#pragma unroll 4
    for (int i = 0, j = j0; i < nload; ++i, j += jstep, g += gstep, q += nth) {
      const bool ok = colok && j < Lin;
      cp_async_cx(q, ok ? g : in, ok);
    }
  } else {
    for (int i = 0; i < nload; ++i) {
      const int e = tid + i * nth;
      const int bb = e & (NB - 1);
      const int j = e >> nb_sh;
      const bool ok = col0 + bb < ncols && j < Lin;
      cp_async_cx(s + e, ok ? src + j * in_js + bb : in, ok);
    }
  }
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  smem_fft_plan<INV, false, MR>(s, stw, nb_sh, NB, rp, half_in, half_out);
  if constexpr (FIX) {
    if (colok) {
      cx<T>* g = out + slab * out_ss + col0 + (long)j0 * out_js + b;
      const long gstep = (long)jstep * out_js;
      const cx<T>* q = s + tid;
#pragma unroll 4
      for (int j = j0; j < Lout; j += jstep, g += gstep, q += nth) *g = scale * *q;
    }
  } else {
    cx<T>* dst = out + slab * out_ss + col0;
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nth;
      const int bb = e & (NB - 1);
      const int j = e >> nb_sh;
      if (col0 + bb < ncols && j < Lout) dst[j * out_js + bb] = scale * s[e];
    }
  }
}

// Launch order of the tiles of one slab.  Columns form nrows rows of
// row_len; frequency r and its mirror (-r) use the same stored spectrum
// entry (parity folding), so rows are visited 0, 1, -1, 2, -2, ... and the
// tiles of a row likewise, which keeps both users of a spectrum line in
// flight at the same time and the line in L2.
__device__ __forceinline__ int mirror_perm(int r, int n) {
  return r == 0 ? 0 : ((r & 1) ? (r + 1) >> 1 : n - (r >> 1));
}

// Three components of a strided tile: forward FFT, op.point(op.column(slab,
// col), j, x0, x1, x2) at every frequency j of every column, inverse FFT; in place on
// `data` (first Lout of L outputs kept).  Lines of the tile are ordered
// (component, column) with the column fastest, so shared-memory index and
// tile index coincide.
template <typename T, class Op, bool FIX, bool MR>
__global__ void __launch_bounds__(MR ? 256 : fft3c_max_threads<T>())
    k_fft3c(cx<T>* data, long ncols, int Lin, long js, long cs, long ss, int Lout, Op op,
            const cx<T>* __restrict__ tw, int twshift, RadixPlan rp, int nbc_sh, int row_len,
            int nrows) {
  pdl_entry();
  constexpr int EPT = elems_per_thread<MR>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int L = rp.L;
  const int NBc = 1 << nbc_sh;
  const int ld = 3 * NBc;
  cx<T>* stw = s + (size_t)L * ld;
  const int nth = blockDim.x, tid = threadIdx.x;
  const long tiles = (ncols + NBc - 1) >> nbc_sh;
  const long slab = blockIdx.x / tiles;
  const int tt = (int)(blockIdx.x - slab * tiles);
  long col0;
  if (row_len >= NBc && nrows > 0 && (row_len & (NBc - 1)) == 0) {
    const int row_tiles = row_len >> nbc_sh;
    const int r = tt / row_tiles;
    const int ti = tt - r * row_tiles;
    col0 = (long)mirror_perm(r, nrows) * row_len + ((long)mirror_perm(ti, row_tiles) << nbc_sh);
  } else {
    col0 = (long)tt << nbc_sh;
  }
  cx<T>* base = data + slab * ss + col0;
  const bool half_in = 2 * Lin <= L && L > 1 && rp.hin;
  const bool half_out = 2 * Lout <= L && L > 1 && rp.hout;
  const int nload = half_in ? EPT / 2 : EPT;  // rows < L/2 only
  // With L a multiple of 16 every thread keeps one (component, column) pair
  // and rows j0 + i * L/16, so addresses advance by constant strides.
  constexpr bool fixed = FIX;
  {
    const int e0 = tid;
    const int b0 = e0 & (NBc - 1);
    const int t0 = e0 >> nbc_sh;
    const int j0 = t0 / 3, c0 = t0 - 3 * (t0 / 3);
    if constexpr (fixed) {
      const int jstep = L / EPT;  // nth / (3 NBc)
      const bool colok = col0 + b0 < ncols;
      const cx<T>* g = base + c0 * cs + (long)j0 * js + b0;
      const long gstep = (long)jstep * js;
      cx<T>* q = s + e0;
#pragma unroll 4
      for (int i = 0, j = j0; i < nload; ++i, j += jstep, g += gstep, q += nth) {
        const bool ok = colok && j < Lin;
        cp_async_cx(q, ok ? g : data, ok);
      }
    } else {
      for (int i = 0; i < nload; ++i) {
        const int e = tid + i * nth;
        const int b = e & (NBc - 1);
        const int t = e >> nbc_sh;  // 3 j + c
        const int j = t / 3;
        const int c = t - 3 * j;
        const bool ok = col0 + b < ncols && j < Lin;
        cp_async_cx(s + e, ok ? base + c * cs + j * js + b : data, ok);
      }
    }
  }
  op.prefetch(col0, NBc, L);
  load_twiddles(stw, tw, L, twshift);
  cp_async_wait_all();
  __syncthreads();
  smem_fft_plan<false, true, MR>(s, stw, nbc_sh, ld, rp, half_in, false);
  if ((nth & (NBc - 1)) == 0) {
    // every thread keeps one column: its per-column state is set up once
    const int b = tid & (NBc - 1);
    if (col0 + b < ncols) {
      const auto ctx = op.column(slab, col0 + b);
      const int jstep = nth >> nbc_sh;
      for (int j = tid >> nbc_sh; j < L; j += jstep) {
        cx<T>* q = s + j * ld + b;
        cx<T> x0 = q[0], x1 = q[NBc], x2 = q[2 * NBc];
        op.point(ctx, j, x0, x1, x2);
        q[0] = x0;
        q[NBc] = x1;
        q[2 * NBc] = x2;
      }
    }
  } else {
    for (int p = tid; p < (L << nbc_sh); p += nth) {
      const int b = p & (NBc - 1);
      const int j = p >> nbc_sh;
      if (col0 + b < ncols) {
        cx<T>* q = s + j * ld + b;
        cx<T> x0 = q[0], x1 = q[NBc], x2 = q[2 * NBc];
        op.point(op.column(slab, col0 + b), j, x0, x1, x2);
        q[0] = x0;
        q[NBc] = x1;
        q[2 * NBc] = x2;
      }
    }
  }
  __syncthreads();
  smem_fft_plan<true, true, MR>(s, stw, nbc_sh, ld, rp, false, half_out);
  if constexpr (fixed) {
    const int b0 = tid & (NBc - 1);
    const int t0 = tid >> nbc_sh;
    const int j0 = t0 / 3, c0 = t0 - 3 * (t0 / 3);
    if (col0 + b0 < ncols) {
      const int jstep = L / EPT;
      cx<T>* g = base + c0 * cs + (long)j0 * js + b0;
      const long gstep = (long)jstep * js;
      const cx<T>* q = s + tid;
#pragma unroll 4
      for (int j = j0; j < Lout; j += jstep, g += gstep, q += nth) *g = *q;
    }
  } else {
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nth;
      const int b = e & (NBc - 1);
      const int t = e >> nbc_sh;
      const int j = t / 3;
      const int c = t - 3 * j;
      if (col0 + b < ncols && j < Lout) base[c * cs + j * js + b] = s[e];
    }
  }
}

// Parity of the six unique Green-function blocks (order xx, xy, xz, yy, yz,
// zz): a block is odd along an axis when that axis appears once in its
// index pair, because g_ab is proportional to r_a r_b plus a multiple of
// delta_ab.  Mirroring a frequency along an odd axis flips the sign of the
// block's spectrum.
__device__ __forceinline__ int fold_axis(int k, int L, bool& flip) {
  flip = 2 * k > L;
  return flip ? L - k : k;
}
// Six spectrum entries of one frequency (48 bytes in complex64: three
// 16-byte loads) with the parity signs of the fold: flip_xy = flip_x != flip_y etc.
template <typename T>
__device__ __forceinline__ void load_sym6(const cx<T>* __restrict__ g6, bool fxy, bool fxz,
                                          bool fyz, cx<T>& xx, cx<T>& xy, cx<T>& xz, cx<T>& yy,
                                          cx<T>& yz, cx<T>& zz) {
  if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(g6);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    xx = mk<T>(a.x, a.y);
    xy = mk<T>(a.z, a.w);
    xz = mk<T>(b.x, b.y);
    yy = mk<T>(b.z, b.w);
    yz = mk<T>(c.x, c.y);
    zz = mk<T>(c.z, c.w);
  } else {
    xx = g6[0];
    xy = g6[1];
    xz = g6[2];
    yy = g6[3];
    yz = g6[4];
    zz = g6[5];
  }
  if (fxy) xy = mk<T>(-xy.x, -xy.y);
  if (fxz) xz = mk<T>(-xz.x, -xz.y);
  if (fyz) yz = mk<T>(-yz.x, -yz.y);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

inline int floor_pow2_l(long v) {
  int p = 1;
  while ((long)p * 2 <= v) p *= 2;
  return p;
}

// Launch k_fft3c with tiles of NBc columns: NBc * 3 * L complex values per
// CTA (16 per thread), NBc shrunk for small grids so that at least two CTAs
// per SM exist.  Columns are rows of row_len (see mirror_perm).
template <typename T, class Op>
void launch_fft3c(cx<T>* data, long ncols, long nslabs, int L, int Lin, long js, long cs, long ss,
                  int Lout, const Op& op, const cx<T>* tw, int Lmax, int row_len, int nrows,
                  cudaStream_t s) {
  if (ncols <= 0 || nslabs <= 0) return;
  const RadixPlan rp = make_radix_plan(L);
  const int ept = rp.pow2 ? kElemsPerThread : kElemsMR;  // values per thread
  // mixed-radix kernels: 256 threads (their stages need the registers)
  const int cap = (rp.pow2 ? fft3c_max_threads<T>() : 256) * ept;
  static const int nbc_env = [] {
    const char* v = getenv("DDA_FFT3C_COLS");
    return v ? atoi(v) : 0;
  }();
  int NBc = nbc_env > 0 ? nbc_env : 8;  // 8 columns: two or more CTAs per SM
  NBc = (int)std::min<long>(NBc, floor_pow2_l(ncols));
  while (3 * NBc * L > cap && NBc > 1) NBc /= 2;
  while (NBc > 1 && 3 * NBc * L > 1536 && nslabs * ((ncols + NBc - 1) / NBc) < 2 * 152) NBc /= 2;
  while (3 * NBc * L < ept * 32) NBc *= 2;
  while ((3 * NBc * L) % ept != 0) NBc *= 2;  // mixed-radix lengths
  const int nth = 3 * NBc * L / ept;
  const size_t smem = ((size_t)3 * NBc * L + L) * sizeof(cx<T>);
  const long grid = nslabs * ((ncols + NBc - 1) / NBc);
  const bool fix = L >= ept && L % ept == 0;
  auto kern = rp.pow2 ? (fix ? k_fft3c<T, Op, true, false> : k_fft3c<T, Op, false, false>)
                      : (fix ? k_fft3c<T, Op, true, true> : k_fft3c<T, Op, false, true>);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  launch_k(kern, (unsigned)grid, nth, smem, s, data, ncols, Lin, js, cs, ss, Lout, op, tw, Lmax / L,
                                         rp, ilog2i(NBc), row_len, nrows);
}

}  // namespace dda
