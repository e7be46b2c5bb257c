// Batched line-FFT kernels over HBM arrays, built on the shared-memory
// Stockham core.  Three shapes cover every transform of the library:
//   k_fft_contig  lines along the contiguous axis (x)
//   k_fft_strided lines along a strided axis (y or z), tiles of NB
//                 neighbouring columns so each row of a tile is one
//                 coalesced segment
//   k_fft3c       the three field components of a strided tile together,
//                 forward transform, a per-frequency 3x3 operation, inverse
//                 transform, in one pass over HBM
// Inputs shorter than the transform are zero padded (Lin < L); outputs can
// be truncated (Lout < L), which is how the circulant embedding of the BTTB
// matvec is pruned.  A CTA reads all of its lines before it writes any, so
// every kernel may run in place (in == out).
#pragma once

#include <algorithm>
#include <cstdint>

#include "fft_core.cuh"

namespace dda {

template <typename T, bool INV>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
    k_fft_contig(const cx<T>* in, cx<T>* out,
                 const uint8_t* __restrict__ mask, long mask_lines, long nlines, int L, int Lin,
                 long in_ld, int Lout, long out_ld, T scale, const cx<T>* __restrict__ tw,
                 int twshift, RadixPlan rp, int NB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int ld = NB + 1;
  cx<T>* stw = s + (size_t)L * ld;
  const long line0 = (long)blockIdx.x * NB;
  load_twiddles(stw, tw, L, twshift);
  for (int e = threadIdx.x; e < NB * L; e += blockDim.x) {
    const int j = e & (L - 1);
    const int b = e / L;
    const long line = line0 + b;
    cx<T> v = zero<T>();
    if (line < nlines && j < Lin) {
      v = in[line * in_ld + j];
      if (mask != nullptr && mask[(line % mask_lines) * Lin + j] == 0) v = zero<T>();
    }
    s[j * ld + b] = v;
  }
  __syncthreads();
  smem_fft<INV>(s, stw, L, NB, ld, rp);
  for (int e = threadIdx.x; e < NB * L; e += blockDim.x) {
    const int j = e & (L - 1);
    const int b = e / L;
    const long line = line0 + b;
    if (line < nlines && j < Lout) out[line * out_ld + j] = scale * s[j * ld + b];
  }
}

template <typename T, bool INV>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
    k_fft_strided(const cx<T>* in, cx<T>* out, long ncols, int L,
                  int Lin, long in_js, long in_ss, int Lout, long out_js, long out_ss, T scale,
                  const cx<T>* __restrict__ tw, int twshift, RadixPlan rp, int NB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + (size_t)L * NB;
  const long tiles = (ncols + NB - 1) / NB;
  const long slab = blockIdx.x / tiles;
  const long col0 = (blockIdx.x % tiles) * NB;
  load_twiddles(stw, tw, L, twshift);
  const cx<T>* src = in + slab * in_ss + col0;
  for (int e = threadIdx.x; e < NB * L; e += blockDim.x) {
    const int b = e & (NB - 1);
    const int j = e / NB;
    cx<T> v = zero<T>();
    if (col0 + b < ncols && j < Lin) v = src[j * in_js + b];
    s[j * NB + b] = v;
  }
  __syncthreads();
  smem_fft<INV>(s, stw, L, NB, NB, rp);
  cx<T>* dst = out + slab * out_ss + col0;
  for (int e = threadIdx.x; e < NB * L; e += blockDim.x) {
    const int b = e & (NB - 1);
    const int j = e / NB;
    if (col0 + b < ncols && j < Lout) dst[j * out_js + b] = scale * s[j * NB + b];
  }
}

// Three components of a strided tile: forward FFT, op(slab, col, j, x0, x1,
// x2) at every frequency j of every column, inverse FFT; in place on
// `data` (first Lout of L outputs kept).  Lines of the tile are ordered
// (component, column) with the column fastest.
template <typename T, class Op>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 768)
    k_fft3c(cx<T>* data, long ncols, int L, int Lin, long js, long cs, long ss,
            int Lout, Op op, const cx<T>* __restrict__ tw, int twshift, RadixPlan rp, int NBc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int ld = 3 * NBc;
  cx<T>* stw = s + (size_t)L * ld;
  const long tiles = (ncols + NBc - 1) / NBc;
  const long slab = blockIdx.x / tiles;
  const long col0 = (blockIdx.x % tiles) * NBc;
  load_twiddles(stw, tw, L, twshift);
  cx<T>* base = data + slab * ss + col0;
  for (int e = threadIdx.x; e < ld * L; e += blockDim.x) {
    const int b = e & (NBc - 1);
    const int c = (e / NBc) % 3;
    const int j = e / ld;
    cx<T> v = zero<T>();
    if (col0 + b < ncols && j < Lin) v = base[c * cs + j * js + b];
    s[j * ld + c * NBc + b] = v;
  }
  __syncthreads();
  smem_fft<false>(s, stw, L, ld, ld, rp);
  for (int p = threadIdx.x; p < L * NBc; p += blockDim.x) {
    const int b = p & (NBc - 1);
    const int j = p / NBc;
    if (col0 + b < ncols) {
      cx<T>* q = s + j * ld + b;
      cx<T> x0 = q[0], x1 = q[NBc], x2 = q[2 * NBc];
      op(slab, col0 + b, j, x0, x1, x2);
      q[0] = x0;
      q[NBc] = x1;
      q[2 * NBc] = x2;
    }
  }
  __syncthreads();
  smem_fft<true>(s, stw, L, ld, ld, rp);
  for (int e = threadIdx.x; e < ld * L; e += blockDim.x) {
    const int b = e & (NBc - 1);
    const int c = (e / NBc) % 3;
    const int j = e / ld;
    if (col0 + b < ncols && j < Lout) base[c * cs + j * js + b] = s[j * ld + c * NBc + b];
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
template <typename T>
__device__ __forceinline__ void load_sym6(const cx<T>* __restrict__ g6, const bool* flip,
                                          cx<T>& xx, cx<T>& xy, cx<T>& xz, cx<T>& yy,
                                          cx<T>& yz, cx<T>& zz) {
  xx = g6[0];
  xy = g6[1];
  xz = g6[2];
  yy = g6[3];
  yz = g6[4];
  zz = g6[5];
  if (flip[0] != flip[1]) xy = mk<T>(-xy.x, -xy.y);
  if (flip[0] != flip[2]) xz = mk<T>(-xz.x, -xz.y);
  if (flip[1] != flip[2]) yz = mk<T>(-yz.x, -yz.y);
}

inline int floor_pow2_l(long v) {
  int p = 1;
  while ((long)p * 2 <= v) p *= 2;
  return p;
}

// Launch k_fft3c with tiles of NBc columns: NBc * 3 * L complex values per
// CTA (16 per thread), NBc shrunk for small grids so that at least two CTAs
// per SM exist.
template <typename T, class Op>
void launch_fft3c(cx<T>* data, long ncols, long nslabs, int L, int Lin, long js, long cs, long ss,
                  int Lout, const Op& op, const cx<T>* tw, int Lmax, cudaStream_t s) {
  if (ncols <= 0 || nslabs <= 0) return;
  const int cap = (sizeof(T) == 8 ? 512 : 768) * kElemsPerThread;
  int NBc = sizeof(T) == 8 ? 8 : 16;
  NBc = (int)std::min<long>(NBc, floor_pow2_l(ncols));
  while (3 * NBc * L > cap && NBc > 1) NBc /= 2;
  while (NBc > 1 && 3 * NBc * L > 1536 && nslabs * ((ncols + NBc - 1) / NBc) < 2 * 152) NBc /= 2;
  while (3 * NBc * L < kElemsPerThread * 32) NBc *= 2;
  const int nth = 3 * NBc * L / kElemsPerThread;
  const size_t smem = ((size_t)3 * NBc * L + L) * sizeof(cx<T>);
  const long grid = nslabs * ((ncols + NBc - 1) / NBc);
  auto kern = k_fft3c<T, Op>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<(unsigned)grid, nth, smem, s>>>(data, ncols, L, Lin, js, cs, ss, Lout, op, tw, Lmax / L,
                                         make_radix_plan(L), NBc);
}

}  // namespace dda
