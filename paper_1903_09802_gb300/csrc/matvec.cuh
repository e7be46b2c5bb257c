// Pieces of the BTTB matvec shared by its complex64 (matvec.cu) and
// double-float (matvec_df.cu) translation units: the spectrum multiply of the
// z pass, the x-inverse epilogue kernels and the five-pass driver.  Kept in
// an unnamed namespace: each translation unit instantiates its own precision.
#pragma once

#include "fft_ct.cuh"
#include "plan.hpp"

namespace dda {

namespace {

// sum_b Ghat_ab(k) x_b at frequency (kx, ky, kz) of the padded grid; the
// spectrum is stored for 0 <= k <= L/2 on every axis and mirrored with the
// block's parity.
template <typename T>
struct KernelMul {
  // complex64: three planes of component pairs per (z, y) row (see
  // k_compress); other precisions: the six components of a frequency together
  static constexpr bool kPlanar = std::is_same<T, float>::value;
  const cx<T>* G;
  int Lx, Ly, Lz, hx, hy, lxs;
  // Pull the spectrum entries of this tile (all kz) towards L2 before the
  // field tile is loaded and transformed.
  // x and y frequency of a column (lxs = log2 Lx, or -1 for a mixed-radix Lx)
  __device__ __forceinline__ int xof(long col) const {
    return lxs >= 0 ? (int)(col & (Lx - 1)) : (int)(col % Lx);
  }
  __device__ __forceinline__ int yof(long col) const {
    return lxs >= 0 ? (int)(col >> lxs) : (int)(col / Lx);
  }
  __device__ __forceinline__ void prefetch(long col0, int ncol, int L) const {
    const int ky = yof(col0);
    bool fl;
    const int fy = fold_axis(ky, Ly, fl);
    const int nz = Lz / 2 + 1;
    if constexpr (kPlanar) {
      // the tile's x frequencies are one contiguous run of each pair plane:
      // its two ends cover it
      const int fa = fold_axis(xof(col0), Lx, fl);
      const int fb = fold_axis(xof(col0 + ncol - 1), Lx, fl);
      for (int i = threadIdx.x; i < nz * 6; i += blockDim.x) {
        const int fz = i / 6, pr = (i >> 1) % 3;
        const int fx = (i & 1) ? fb : fa;
        prefetch_l2(G + ((((size_t)fz * hy + fy) * 3 + pr) * hx + fx) * 2);
      }
    } else {
      for (int i = threadIdx.x; i < ncol * nz; i += blockDim.x) {
        const int b = i % ncol, fz = i / ncol;
        const int fx = fold_axis(xof(col0 + b), Lx, fl);
        prefetch_l2(G + ((size_t)(fz * hy + fy) * hx + fx) * 6);
      }
    }
  }
  struct Col {
    const cx<T>* g;  // spectrum at (fx, fy, fz = 0)
    bool flx, fly;
  };
  __device__ __forceinline__ Col column(long, long col) const {
    Col c;
    const int fx = fold_axis(xof(col), Lx, c.flx);
    const int fy = fold_axis(yof(col), Ly, c.fly);
    c.g = kPlanar ? G + ((size_t)fy * 3 * hx + fx) * 2 : G + ((size_t)fy * hx + fx) * 6;
    return c;
  }
  // The spectrum entries of frequency j as loaded (complex64), their signs
  // applied only in mul_raw: the register-resident z pass issues the loads of
  // the next frequency before it multiplies the current one.
  struct G6r {
    float4 a, b, c;
    bool fxy, fxz, fyz;
  };
  __device__ __forceinline__ void load_raw(const Col& c, int j, G6r& g) const {
    static_assert(kPlanar, "pair planes: the complex64 store");
    bool flz;
    const int fz = fold_axis(j, Lz, flz);
    const float4* p = reinterpret_cast<const float4*>(c.g + (size_t)fz * hy * hx * 6);
    g.a = __ldg(p);
    g.b = __ldg(p + hx);
    g.c = __ldg(p + 2 * hx);
    g.fxy = c.flx != c.fly;
    g.fxz = c.flx != flz;
    g.fyz = c.fly != flz;
  }
  __device__ __forceinline__ void mul_raw(const G6r& g, cx<T>& x0, cx<T>& x1, cx<T>& x2) const {
    const cx<T> gxx = mk<T>(g.a.x, g.a.y), gyy = mk<T>(g.b.z, g.b.w), gzz = mk<T>(g.c.z, g.c.w);
    const cx<T> gxy = g.fxy ? mk<T>(-g.a.z, -g.a.w) : mk<T>(g.a.z, g.a.w);
    const cx<T> gxz = g.fxz ? mk<T>(-g.b.x, -g.b.y) : mk<T>(g.b.x, g.b.y);
    const cx<T> gyz = g.fyz ? mk<T>(-g.c.x, -g.c.y) : mk<T>(g.c.x, g.c.y);
    const cx<T> y0 = gxx * x0 + gxy * x1 + gxz * x2;
    const cx<T> y1 = gxy * x0 + gyy * x1 + gyz * x2;
    const cx<T> y2 = gxz * x0 + gyz * x1 + gzz * x2;
    x0 = y0;
    x1 = y1;
    x2 = y2;
  }
  __device__ __forceinline__ void point(const Col& c, int j, cx<T>& x0, cx<T>& x1,
                                        cx<T>& x2) const {
    if constexpr (kPlanar) {
      G6r g;
      load_raw(c, j, g);
      mul_raw(g, x0, x1, x2);
    } else {
      bool flz;
      const int fz = fold_axis(j, Lz, flz);
      cx<T> gxx, gxy, gxz, gyy, gyz, gzz;
      load_sym6(c.g + (size_t)fz * hy * hx * 6, c.flx != c.fly, c.flx != flz, c.fly != flz, gxx,
                gxy, gxz, gyy, gyz, gzz);
      const cx<T> y0 = gxx * x0 + gxy * x1 + gxz * x2;
      const cx<T> y1 = gxy * x0 + gyy * x1 + gyz * x2;
      const cx<T> y2 = gxz * x0 + gyz * x1 + gzz * x2;
      x0 = y0;
      x1 = y1;
      x2 = y2;
    }
  }
};

// Pass 5: inverse FFT along x of each padded line, then
//   y = a x - coef * conv   (scatterer voxel, a = alpha^{-1} of its material)
//   y = a x                 (air voxel, a = alpha_tilde^{-1})
// with coef = dx^3 / (2l 2m 2n) (the inverse transforms are unnormalised).
template <typename T, bool MR>
__global__ void __launch_bounds__((MR || std::is_same<T, df>::value) ? 256 : 512)
    k_mv_epilogue(const cx<T>* __restrict__ buf1, const cx<T>* __restrict__ x,
                  cx<T>* __restrict__ y, const uint8_t* __restrict__ mat,
                  const cx<T>* __restrict__ ainv, int K1, long nlines, long nm, int l, int Lx,
                  T coef, const cx<T>* __restrict__ tw, int twshift, RadixPlan rp, int nb_sh,
                  const cx<T>* __restrict__ pv) {
  pdl_entry();
  constexpr int EPT = elems_per_thread<MR>();
  const int NB = 1 << nb_sh;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  const int ld = NB + 1;
  cx<T>* stw = s + (size_t)Lx * ld;
  const long line0 = (long)blockIdx.x * NB;
  const int nth = blockDim.x, tid = threadIdx.x;
#pragma unroll 4
  for (int i = 0; i < EPT; ++i) {
    const int e = tid + i * nth;
    const int j = MR ? e % Lx : e & (Lx - 1);
    const int b = MR ? e / Lx : e >> rp.lg;
    const long line = line0 + b;
    const bool ok = line < nlines;
    cp_async_cx(s + j * ld + b, ok ? buf1 + line * Lx + j : buf1, ok);
  }
  load_twiddles(stw, tw, Lx, twshift);
  cp_async_wait_all();
  __syncthreads();
  smem_fft_plan<true, false, MR>(s, stw, nb_sh, ld, rp, false, 2 * l <= Lx && Lx > 1 && rp.hout);
  // Stores: element e = tid + i * nth of the NB x l outputs; when l divides
  // nth every thread keeps one column j and steps over lines by nth / l, so
  // the voxel row and right-hand side advance incrementally.
  const int lsh = rp.lg - 1;  // l = Lx / 2
  if (!MR && 2 * l == Lx && (nth & (l - 1)) == 0) {
    const int j = tid & (l - 1);
    const int b0 = tid >> lsh;
    const int bstep = nth >> lsh;
    long line = line0 + b0;
    long vrow = line % nm;  // (z, y) row of the voxel
    long rhs = line / (3 * nm);
    long rem = line - rhs * 3 * nm;
    for (int b = b0; b < NB && line < nlines; b += bstep, line += bstep) {
      const int mt = mat[vrow * l + j];
      const cx<T> a = (pv != nullptr && mt != 0) ? pv[(rhs * nm + vrow) * l + j]
                                                 : ainv[rhs * K1 + mt];
      const cx<T> xv = x[line * l + j];
      cx<T> out = a * xv;
      if (mt != 0) out = out - coef * s[j * ld + b];
      y[line * l + j] = out;
      vrow += bstep;
      rem += bstep;
      if (vrow >= nm) vrow = vrow >= 2 * nm ? vrow % nm : vrow - nm;
      if (rem >= 3 * nm) {
        rhs += rem / (3 * nm);
        rem %= 3 * nm;
      }
    }
  } else {
    for (int e = tid; e < NB * l; e += nth) {
      const int j = e % l;
      const int b = e / l;
      const long line = line0 + b;
      if (line < nlines) {
        const long vox = (line % nm) * l + j;
        const long rhs = line / (3 * nm);
        const int mt = mat[vox];
        const cx<T> a = (pv != nullptr && mt != 0) ? pv[rhs * nm * l + vox] : ainv[rhs * K1 + mt];
        const cx<T> xv = x[line * l + j];
        cx<T> out = a * xv;
        if (mt != 0) out = out - coef * s[j * ld + b];
        y[line * l + j] = out;
      }
    }
  }
}

// Compile-time variant of pass 5 (complex64, Lx in 32..512): NB lines of
// pitch NB + 1, every thread keeps one position j (NB >= 16).
template <typename T, int LX, int NB>
__global__ void __launch_bounds__(NB * LX / kElemsPerThread, 1024 / (NB * LX / kElemsPerThread))
    k_ct_mv_epilogue(const cx<T>* __restrict__ buf1, const cx<T>* __restrict__ x,
                     cx<T>* __restrict__ y, const uint8_t* __restrict__ mat,
                     const cx<T>* __restrict__ ainv, int K1, long nlines, long nm, T coef,
                     const cx<T>* __restrict__ tw, int twshift, const cx<T>* __restrict__ pv) {
  pdl_entry();
  static_assert(NB >= 16, "one position per thread");
  constexpr int NTH = NB * LX / kElemsPerThread;
  constexpr int LD = NB + 1;
  constexpr int BSTEP = NTH / LX;
  constexpr int l = LX / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stw = s + LX * LD;
  cx<T>* sx = stw + LX;  // the NB x l input values of the diagonal term
  const int tid = threadIdx.x;
  const long line0 = (long)blockIdx.x * NB;
  {
    const int j = tid & (LX - 1);
    const int b0 = tid / LX;
    long line = line0 + b0;
    const cx<T>* g = buf1 + line * LX + j;
    cx<T>* q = s + j * LD + b0;
#pragma unroll 4
    for (int i = 0; i < kElemsPerThread; ++i, line += BSTEP, g += BSTEP * LX, q += BSTEP) {
      const bool ok = line < nlines;
      cp_async_cx(q, ok ? g : buf1, ok);
    }
  }
  // outputs: NB lines x l positions; thread keeps j = tid mod l.  Its x
  // values are copied and its material bytes loaded now, so that their
  // latency passes under the transform.
  const int j = tid & (l - 1);
  const int b0 = tid / l;
  constexpr int OSTEP = NTH / l;
  constexpr int NOUT = NB / OSTEP;  // outputs per thread
  int mts[NOUT];
  {
    long line = line0 + b0;
    long vrow = line % nm;
#pragma unroll
    for (int i = 0; i < NOUT; ++i, line += OSTEP) {
      const bool ok = line < nlines;
      cp_async_cx(sx + (b0 + i * OSTEP) * l + j, ok ? x + line * l + j : x, ok);
      mts[i] = ok ? (int)__ldg(mat + vrow * l + j) : 0;
      vrow += OSTEP;
      if (vrow >= nm) vrow = vrow >= 2 * nm ? vrow % nm : vrow - nm;
    }
  }
  load_twiddles(stw, tw, LX, twshift);
  cp_async_wait_all();
  __syncthreads();
  ct_fft<LX, LD, NB, true, false, true>(s, stw);
  long line = line0 + b0;
  long vrow = line % nm;
  long rhs = line / (3 * nm);
  long rem = line - rhs * 3 * nm;
#pragma unroll
  for (int i = 0; i < NOUT; ++i, line += OSTEP) {
    if (line >= nlines) break;
    const int b = b0 + i * OSTEP;
    const int mt = mts[i];
    const cx<T> a = (pv != nullptr && mt != 0) ? pv[(rhs * nm + vrow) * l + j]
                                               : ainv[rhs * K1 + mt];
    const cx<T> xv = sx[b * l + j];
    cx<T> out = a * xv;
    if (mt != 0) out = out - coef * s[j * LD + b];
    y[line * l + j] = out;
    vrow += OSTEP;
    rem += OSTEP;
    if (vrow >= nm) vrow = vrow >= 2 * nm ? vrow % nm : vrow - nm;
    if (rem >= 3 * nm) {
      rhs += rem / (3 * nm);
      rem %= 3 * nm;
    }
  }
}

template <int LX>
void ct_epilogue_launch(dda_plan_s* p, const cx<float>* b1, const cx<float>* x, cx<float>* y,
                        long lines, long nm, float coef, cudaStream_t s, int rhs0) {
  constexpr int NB = (2048 / LX) > 16 ? 2048 / LX : 16;
  const size_t smem = ((size_t)LX * (NB + 1) + LX + (size_t)NB * (LX / 2)) * sizeof(cx<float>);
  auto kern = k_ct_mv_epilogue<float, LX, NB>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  launch_k(kern, (unsigned)((lines + NB - 1) / NB), NB * LX / kElemsPerThread, smem, s,
      b1, x, y, p->mat, ainv_of<float>(p) + (long)rhs0 * (p->K + 1), p->K + 1, lines, nm, coef,
      tw_of<float>(p), p->Lmax / LX,
      pv_of<float>(p) ? pv_of<float>(p) + (long)rhs0 * p->nvox : nullptr);
}

bool ct_epilogue(dda_plan_s* p, const cx<float>* b1, const cx<float>* x, cx<float>* y, long lines,
                 long nm, float coef, cudaStream_t s, int rhs0) {
  switch (p->Lx) {
    case 32: ct_epilogue_launch<32>(p, b1, x, y, lines, nm, coef, s, rhs0); return true;
    case 64: ct_epilogue_launch<64>(p, b1, x, y, lines, nm, coef, s, rhs0); return true;
    case 128: ct_epilogue_launch<128>(p, b1, x, y, lines, nm, coef, s, rhs0); return true;
    case 256: ct_epilogue_launch<256>(p, b1, x, y, lines, nm, coef, s, rhs0); return true;
    case 512: ct_epilogue_launch<512>(p, b1, x, y, lines, nm, coef, s, rhs0); return true;
    default: return false;
  }
}

inline int ilog2(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

template <typename T>
void matvec_core(dda_plan_s* p, int nrhs, const cx<T>* x, cx<T>* y, cudaStream_t s, int rhs0) {
  const cx<T>* tw = tw_of<T>(p);
  cx<T>* b1 = static_cast<cx<T>*>(p->w.buf1);
  cx<T>* b2 = static_cast<cx<T>*>(p->w.buf2);
  const long l = p->l, m = p->m, n = p->n, Lx = p->Lx, Ly = p->Ly, Lz = p->Lz;
  const long nm = n * m;
  const long lines = (long)nrhs * 3 * nm;
  const long plane = Ly * Lx;
  const double u = (double)nrhs * 3 * p->nvox * sizeof(cx<T>);  // box fields of the batch
  const double spec = 6.0 * p->hx * p->hy * p->hz * sizeof(cx<T>);
  // complex128 launches are timed apart from the complex64 ones
  constexpr int pc = std::is_same<T, float>::value ? 0 : PROF_MV128_XF - PROF_MV_XF;
  // 1: x forward of the masked field, l -> 2l
  p->prof.begin(PROF_MV_XF + pc, s, 3 * u + p->nvox);
  launch_contig<T, false>(x, b1, p->mat, nullptr, nm, lines, (int)Lx, (int)l, l, (int)Lx, Lx, T(1), tw,
                          p->Lmax, s);
  p->prof.end(s);
  // 2: y forward, m -> 2m
  p->prof.begin(PROF_MV_YF + pc, s, 6 * u);
  launch_strided<T, false>(b1, b2, Lx, (long)nrhs * 3 * n, (int)Ly, (int)m, Lx, m * Lx, (int)Ly,
                           Lx, plane, T(1), tw, p->Lmax, s);
  p->prof.end(s);
  // 3: z forward, spectrum multiply, z inverse (n live planes in and out)
  KernelMul<T> op{G_of<T>(p), (int)Lx, (int)Ly, (int)Lz, p->hx, p->hy,
                  is_pow2(Lx) ? ilog2((int)Lx) : -1};
  p->prof.begin(PROF_MV_Z + pc, s, 8 * u + spec);
  launch_fft3c_any<true, true>(b2, plane, nrhs, (int)Lz, (int)n, plane, n * plane, 3 * n * plane,
                               (int)n, op, tw, p->Lmax, (int)Lx, (int)Ly, s);
  p->prof.end(s);
  // 4: y inverse, 2m -> m
  p->prof.begin(PROF_MV_YI + pc, s, 6 * u);
  launch_strided<T, true>(b2, b1, Lx, (long)nrhs * 3 * n, (int)Ly, (int)Ly, Lx, plane, (int)m, Lx,
                          m * Lx, T(1), tw, p->Lmax, s);
  p->prof.end(s);
  // 5: x inverse and the diagonal
  if constexpr (sizeof(T) == 4) {
    if (is_pow2(Lx) && Lx >= 32 && Lx <= 512) {
      const float coef = (float)(p->d.dx * p->d.dx * p->d.dx / (double)p->P);
      p->prof.begin(PROF_MV_XI + pc, s, 4 * u + p->nvox);
      ct_epilogue(p, b1, x, y, lines, nm, coef, s, rhs0);
      p->prof.end(s);
      return;
    }
  }
  {
    const RadixPlan rp = make_radix_plan((int)Lx);
    const int ept = rp.pow2 ? kElemsPerThread : kElemsMR;  // values per thread
    const int cap = ((!rp.pow2 || std::is_same<T, df>::value) ? 256 : 512) * ept;
    int per_cta = std::min(4096, cap);
    while (per_cta > 512 && per_cta > Lx && (lines * Lx + per_cta - 1) / per_cta < 2 * 152)
      per_cta /= 2;
    int NB = 1;
    while (2 * NB * Lx <= per_cta) NB *= 2;
    while (NB * Lx < ept * 32) NB *= 2;
    while ((NB * Lx) % ept != 0) NB *= 2;  // mixed-radix lengths
    const int nth = NB * (int)Lx / ept;
    const size_t smem = ((size_t)Lx * (NB + 1) + Lx) * sizeof(cx<T>);
    auto kern = rp.pow2 ? k_mv_epilogue<T, false> : k_mv_epilogue<T, true>;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const T coef = (T)(p->d.dx * p->d.dx * p->d.dx / (double)p->P);
    p->prof.begin(PROF_MV_XI + pc, s, 4 * u + p->nvox);
    note_launch();
    launch_k(kern, (unsigned)((lines + NB - 1) / NB), nth, smem, s,
        b1, x, y, p->mat, ainv_of<T>(p) + (long)rhs0 * (p->K + 1), p->K + 1, lines, nm, (int)l,
        (int)Lx, coef, tw, p->Lmax / (int)Lx, rp, ilog2i(NB),
        pv_of<T>(p) ? pv_of<T>(p) + (long)rhs0 * p->nvox : nullptr);
    p->prof.end(s);
  }
}

}  // namespace

}  // namespace dda
