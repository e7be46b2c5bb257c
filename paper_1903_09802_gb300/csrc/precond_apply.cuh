// The 3-level preconditioner's apply, shared by its complex64 (precond.cu)
// and complex128 (precond_f64.cu) translation units: the per-frequency 3x3
// solve of the z pass and the five-pass driver (see precond.cu).
#pragma once

#include <algorithm>

#include "fft_ct.cuh"
#include "plan.hpp"

namespace dda {

namespace {

// z(w) = Lambda(w)^{-1} x(w) / (l m n) (the inverse transforms are unnormalised).
template <typename T>
struct CircSolve {
  const cx<T>* C;
  const cx<T>* ainv;
  int* err;
  int K1, l, m, n, hx, hy, lxs;
  T dx3, inv_n;
  __device__ __forceinline__ void prefetch(long, int, int) const {}
  struct Col {
    const cx<T>* c;  // spectrum at (fx, fy, fz = 0)
    cx<T> at;        // alpha_tilde^{-1} of this right-hand side
    bool flx, fly;
  };
  __device__ __forceinline__ Col column(long rhs, long col) const {
    Col q;
    // lxs = log2 l, or -1 for a mixed-radix l
    const int fx = fold_axis(lxs >= 0 ? (int)(col & (l - 1)) : (int)(col % l), l, q.flx);
    const int fy = fold_axis(lxs >= 0 ? (int)(col >> lxs) : (int)(col / l), m, q.fly);
    q.c = C + ((size_t)fy * hx + fx) * 6;
    q.at = ainv[rhs * K1];
    return q;
  }
  __device__ __forceinline__ void point(const Col& q, int j, cx<T>& x0, cx<T>& x1,
                                        cx<T>& x2) const {
    bool flz;
    const int fz = fold_axis(j, n, flz);
    cx<T> cxx, cxy, cxz, cyy, cyz, czz;
    load_sym6(q.c + (size_t)fz * hy * hx * 6, q.flx != q.fly, q.flx != flz, q.fly != flz, cxx, cxy,
              cxz, cyy, cyz, czz);
    const cx<T> at = q.at;
    // Lambda = [[a b c] [b d e] [c e f]]
    const cx<T> a = at - dx3 * cxx, d = at - dx3 * cyy, ff = at - dx3 * czz;
    const cx<T> b = -dx3 * cxy, c = -dx3 * cxz, e = -dx3 * cyz;
    // adjugate of a symmetric matrix
    const cx<T> A00 = d * ff - e * e, A01 = c * e - b * ff, A02 = b * e - c * d;
    const cx<T> A11 = a * ff - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
    const cx<T> det = a * A00 + b * A01 + c * A02;
    const T dn = norm2(det);
    if (!(dn > T(0)) || !isfinite(dn)) {
      atomicOr(err, 1);
      return;
    }
    // inv_n / det
    const cx<T> sdet = mk<T>(inv_n * det.x / dn, -inv_n * det.y / dn);
    const cx<T> y0 = A00 * x0 + A01 * x1 + A02 * x2;
    const cx<T> y1 = A01 * x0 + A11 * x1 + A12 * x2;
    const cx<T> y2 = A02 * x0 + A12 * x1 + A22 * x2;
    x0 = sdet * y0;
    x1 = sdet * y1;
    x2 = sdet * y2;
  }
};

inline int ilog2(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

}  // namespace

template <typename T>
void precond_apply_chunk(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s,
                         int rhs0) {
  const cx<T>* tw = tw_of<T>(p);
  cx<T>* t = static_cast<cx<T>*>(p->w.buf2);
  const long l = p->l, m = p->m, n = p->n;
  const long lines = (long)nrhs * 3 * n * m;
  const long plane = l * m;
  const double u = (double)nrhs * 3 * p->nvox * sizeof(cx<T>);
  const double circ = 6.0 * p->cx_ * p->cy_ * p->cz_ * sizeof(cx<T>);
  // complex128 launches are timed apart from the complex64 ones
  constexpr int pc = std::is_same<T, float>::value ? 0 : PROF_PC128_XF - PROF_PC_XF;
  p->prof.begin(PROF_PC_XF + pc, s, 2 * u + p->nvox);
  launch_contig<T, false>(v, t, p->mat, nullptr, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                          p->Lmax, s);
  p->prof.end(s);
  p->prof.begin(PROF_PC_YF + pc, s, 2 * u);
  if (m > 1)
    launch_strided<T, false>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                             T(1), tw, p->Lmax, s);
  CircSolve<T> op{C_of<T>(p), ainv_of<T>(p) + (long)rhs0 * (p->K + 1),
                  static_cast<int*>(p->w.err_flag), p->K + 1,
                  (int)l, (int)m, (int)n, p->cx_, p->cy_, is_pow2(l) ? ilog2((int)l) : -1,
                  (T)(p->d.dx * p->d.dx * p->d.dx), (T)(1.0 / (double)p->nvox)};
  p->prof.end(s);
  p->prof.begin(PROF_PC_Z + pc, s, 2 * u + circ);
  launch_fft3c_any<false, false>(t, plane, nrhs, (int)n, (int)n, plane, n * plane, 3 * n * plane,
                                 (int)n, op, tw, p->Lmax, (int)l, (int)m, s);
  p->prof.end(s);
  p->prof.begin(PROF_PC_YI + pc, s, 2 * u);
  if (m > 1)
    launch_strided<T, true>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                            T(1), tw, p->Lmax, s);
  p->prof.end(s);
  p->prof.begin(PROF_PC_XI + pc, s, 2 * u + p->nvox);
  launch_contig<T, true>(t, z, nullptr, p->mat, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                         p->Lmax, s);
  p->prof.end(s);
}

// Right-hand sides in chunks of the plan's rhs_chunk (the transform scratch
// holds that many).
template <typename T>
void precond_apply_impl(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s) {
  const long nu = 3 * p->nvox;
  for (int r0 = 0; r0 < nrhs; r0 += p->rhs_chunk) {
    const int nr = std::min(p->rhs_chunk, nrhs - r0);
    precond_apply_chunk<T>(p, nr, v + r0 * nu, z + r0 * nu, s, r0);
  }
}

// The same five passes with the transform held in caller-chosen scratch
// `t` (nrhs * 3 * l m n values) instead of the plan's workspace, and no
// kernel timing.
template <typename T>
void precond_apply_into(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cx<T>* t,
                        cudaStream_t s) {
  const cx<T>* tw = tw_of<T>(p);
  const long l = p->l, m = p->m, n = p->n;
  const long lines = (long)nrhs * 3 * n * m;
  const long plane = l * m;
  launch_contig<T, false>(v, t, p->mat, nullptr, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                          p->Lmax, s);
  if (m > 1)
    launch_strided<T, false>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                             T(1), tw, p->Lmax, s);
  CircSolve<T> op{C_of<T>(p), ainv_of<T>(p), static_cast<int*>(p->w.err_flag), p->K + 1,
                  (int)l, (int)m, (int)n, p->cx_, p->cy_, is_pow2(l) ? ilog2((int)l) : -1,
                  (T)(p->d.dx * p->d.dx * p->d.dx), (T)(1.0 / (double)p->nvox)};
  launch_fft3c_any<false, false>(t, plane, nrhs, (int)n, (int)n, plane, n * plane, 3 * n * plane,
                                 (int)n, op, tw, p->Lmax, (int)l, (int)m, s);
  if (m > 1)
    launch_strided<T, true>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                            T(1), tw, p->Lmax, s);
  launch_contig<T, true>(t, z, nullptr, p->mat, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                         p->Lmax, s);
}

}  // namespace dda
