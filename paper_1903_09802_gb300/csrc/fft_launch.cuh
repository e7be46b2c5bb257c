// Launch geometry of the batched FFT kernels and the full 3-D transform
// (instantiated per precision by fft_launch.cu, fft_launch_f64.cu and
// fft_launch_df.cu).
//
// Tiles are sized so that a CTA holds 2-16K complex values in shared memory
// (16 per thread), strided tiles span at least 8 (complex128) or 16
// (complex64) neighbouring columns so that every row is one 128-byte
// segment, and small problems shrink tiles until the grid covers the 152
// SMs at least twice.
#pragma once

#include <algorithm>

#include "fft_ct.cuh"
#include "plan.hpp"

namespace dda {

namespace {

constexpr int kSMs = 152;

template <typename T>
constexpr int max_threads() {
  return sizeof(T) == 8 ? 512 : 1024;
}

inline int floor_pow2(long v) {
  int p = 1;
  while ((long)p * 2 <= v) p *= 2;
  return p;
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Compile-time kernels (complex64): lengths 32..512.
template <bool INV, int L, bool HI, bool HO>
void ct_strided_launch(const cx<float>* in, cx<float>* out, long ncols, long nslabs, int Lin,
                       long in_js, long in_ss, int Lout, long out_js, long out_ss, float scale,
                       const cx<float>* tw, int Lmax, cudaStream_t s) {
  constexpr int NB = 16;
  const size_t smem = ((size_t)L * NB + L) * sizeof(cx<float>);
  auto kern = k_ct_strided<float, INV, L, NB, HI, HO>;
  allow_smem(kern, smem);
  note_launch();
  launch_k(kern, (unsigned)(nslabs * (ncols / NB)), NB * L / kElemsPerThread, smem, s,
      in, out, ncols, Lin, in_js, in_ss, Lout, out_js, out_ss, scale, tw, Lmax / L);
}

template <bool INV, bool HI, bool HO>
bool ct_strided(const cx<float>* in, cx<float>* out, long ncols, long nslabs, int L, int Lin,
                long in_js, long in_ss, int Lout, long out_js, long out_ss, float scale,
                const cx<float>* tw, int Lmax, cudaStream_t s) {
#define DDA_CT_S(LL)                                                                          \
  case LL:                                                                                   \
    ct_strided_launch<INV, LL, HI, HO>(in, out, ncols, nslabs, Lin, in_js, in_ss, Lout, out_js, \
                                       out_ss, scale, tw, Lmax, s);                          \
    return true;
  switch (L) {
    DDA_CT_S(32)
    DDA_CT_S(64)
    DDA_CT_S(128)
    DDA_CT_S(256)
    DDA_CT_S(512)
    default: return false;
  }
#undef DDA_CT_S
}

template <bool INV, int L, bool HI, bool HO>
void ct_contig_launch(const cx<float>* in, cx<float>* out, const uint8_t* mask,
                      const uint8_t* omask, long mask_lines, long nlines, int Lin, long in_ld,
                      int Lout, long out_ld, float scale, const cx<float>* tw, int Lmax,
                      cudaStream_t s) {
  constexpr int NB = (2048 / L) > 16 ? 2048 / L : 16;
  const size_t smem = ((size_t)L * (NB + 1) + L) * sizeof(cx<float>);
  auto kern = k_ct_contig<float, INV, L, NB, HI, HO>;
  allow_smem(kern, smem);
  note_launch();
  launch_k(kern, (unsigned)((nlines + NB - 1) / NB), NB * L / kElemsPerThread, smem, s,
      in, out, mask, omask, mask_lines, nlines, Lin, in_ld, Lout, out_ld, scale, tw, Lmax / L);
}

template <bool INV, bool HI, bool HO>
bool ct_contig(const cx<float>* in, cx<float>* out, const uint8_t* mask, const uint8_t* omask,
               long mask_lines, long nlines, int L, int Lin, long in_ld, int Lout, long out_ld,
               float scale, const cx<float>* tw, int Lmax, cudaStream_t s) {
#define DDA_CT_C(LL)                                                                          \
  case LL:                                                                                   \
    ct_contig_launch<INV, LL, HI, HO>(in, out, mask, omask, mask_lines, nlines, Lin, in_ld, Lout, \
                                      out_ld, scale, tw, Lmax, s);                           \
    return true;
  switch (L) {
    DDA_CT_C(32)
    DDA_CT_C(64)
    DDA_CT_C(128)
    DDA_CT_C(256)
    DDA_CT_C(512)
    default: return false;
  }
#undef DDA_CT_C
}

}  // namespace

template <typename T, bool INV>
void launch_contig(const cx<T>* in, cx<T>* out, const uint8_t* mask, const uint8_t* omask,
                   long mask_lines, long nlines,
                   int L, int Lin, long in_ld, int Lout, long out_ld, T scale, const cx<T>* tw,
                   int Lmax, cudaStream_t s) {
  if (nlines <= 0) return;
  if constexpr (sizeof(T) == 4) {
    // forward passes with a zero-padded input, inverse passes with a halved
    // output, or neither: the combinations the operator uses
    const bool hi = 2 * Lin <= L, ho = 2 * Lout <= L;
    bool done = false;
    if (!INV && hi)
      done = ct_contig<INV, true, false>(in, out, mask, omask, mask_lines, nlines, L, Lin, in_ld,
                                         Lout, out_ld, scale, tw, Lmax, s);
    else if (!hi && !ho)
      done = ct_contig<INV, false, false>(in, out, mask, omask, mask_lines, nlines, L, Lin, in_ld,
                                          Lout, out_ld, scale, tw, Lmax, s);
    if (done) return;
  }
  int per_cta = 4096;  // complex values per CTA: at most 256 threads
  while (per_cta > 512 && per_cta > L && (nlines * L + per_cta - 1) / per_cta < 2 * kSMs)
    per_cta /= 2;
  const RadixPlan rp = make_radix_plan(L);
  const int ept = rp.pow2 ? kElemsPerThread : kElemsMR;  // values per thread
  if (!rp.pow2) per_cta /= 2;                               // 256 threads at most
  int NB = floor_pow2(std::max(1, per_cta / L));
  while (NB * L < ept * 32) NB *= 2;  // at least one warp
  while ((NB * L) % ept != 0) NB *= 2;  // mixed-radix lengths
  const int nth = NB * L / ept;
  const size_t smem = ((size_t)L * (NB + 1) + L) * sizeof(cx<T>);
  const long grid = (nlines + NB - 1) / NB;
  auto kern = rp.pow2 ? k_fft_contig<T, INV, false> : k_fft_contig<T, INV, true>;
  allow_smem(kern, smem);
  note_launch();
  launch_k(kern, (unsigned)grid, nth, smem, s, in, out, mask, omask, mask_lines, nlines, Lin, in_ld, Lout,
                                         out_ld, scale, tw, Lmax / L, rp,
                                         ilog2i(NB));
}

template <typename T, bool INV>
void launch_strided(const cx<T>* in, cx<T>* out, long ncols, long nslabs, int L, int Lin,
                    long in_js, long in_ss, int Lout, long out_js, long out_ss, T scale,
                    const cx<T>* tw, int Lmax, cudaStream_t s) {
  if (ncols <= 0 || nslabs <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (ncols % 16 == 0 && ncols >= 16) {
      const bool hi = 2 * Lin <= L, ho = 2 * Lout <= L;
      bool done = false;
      if (!INV && hi)
        done = ct_strided<INV, true, false>(in, out, ncols, nslabs, L, Lin, in_js, in_ss, Lout,
                                            out_js, out_ss, scale, tw, Lmax, s);
      else if (INV && ho)
        done = ct_strided<INV, false, true>(in, out, ncols, nslabs, L, Lin, in_js, in_ss, Lout,
                                            out_js, out_ss, scale, tw, Lmax, s);
      else if (!hi && !ho)
        done = ct_strided<INV, false, false>(in, out, ncols, nslabs, L, Lin, in_js, in_ss, Lout,
                                             out_js, out_ss, scale, tw, Lmax, s);
      if (done) return;
    }
  }
  const RadixPlan rp = make_radix_plan(L);
  const int ept = rp.pow2 ? kElemsPerThread : kElemsMR;  // values per thread
  const int cap = (rp.pow2 ? 512 : 256) * ept;  // threads: 512, mixed radix 256
  int NB = sizeof(T) == 8 ? 8 : 16;
  NB = std::min<long>(NB, floor_pow2(ncols));
  while (NB * L > cap && NB > 1) NB /= 2;
  while (NB > 1 && NB * L > 1024 && nslabs * ((ncols + NB - 1) / NB) < 2 * kSMs) NB /= 2;
  while (NB * L < ept * 32) NB *= 2;
  while ((NB * L) % ept != 0) NB *= 2;  // mixed-radix lengths
  const int nth = NB * L / ept;
  const size_t smem = ((size_t)L * NB + L) * sizeof(cx<T>);
  const long grid = nslabs * ((ncols + NB - 1) / NB);
  const bool fix = L >= ept && L % ept == 0;
  auto kern = rp.pow2 ? (fix ? k_fft_strided<T, INV, true, false> : k_fft_strided<T, INV, false, false>)
                      : (fix ? k_fft_strided<T, INV, true, true> : k_fft_strided<T, INV, false, true>);
  allow_smem(kern, smem);
  note_launch();
  launch_k(kern, (unsigned)grid, nth, smem, s, in, out, ncols, Lin, in_js, in_ss, Lout, out_js, out_ss,
                                         scale, tw, Lmax / L, rp, ilog2i(NB));
}

template <typename T, bool INV>
void fft3d_inplace(cx<T>* data, long nbatch, int Lx, int Ly, int Lz, T scale, const cx<T>* tw,
                   int Lmax, cudaStream_t s) {
  const long plane = (long)Lx * Ly;
  const long vol = plane * Lz;
  if (Lx > 1)
    launch_contig<T, INV>(data, data, nullptr, nullptr, 1, nbatch * Ly * Lz, Lx, Lx, Lx, Lx, Lx, T(1), tw,
                          Lmax, s);
  if (Ly > 1)
    launch_strided<T, INV>(data, data, Lx, nbatch * Lz, Ly, Ly, Lx, plane, Ly, Lx, plane, T(1), tw,
                           Lmax, s);
  if (Lz > 1 || scale != T(1))
    launch_strided<T, INV>(data, data, plane, nbatch, Lz, Lz, plane, vol, Lz, plane, vol, scale,
                           tw, Lmax, s);
}

}  // namespace dda
