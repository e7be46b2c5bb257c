// The BTTB matvec of the DDA system (Section 2.2): y = alpha^{-1} x - dx^3 G x
// on the scatterer, y = alpha_tilde^{-1} x on air, with G x evaluated as a
// circulant convolution on the (2l, 2m, 2n) padded grid (the FFT acceleration
// the paper relies on, Sections 1 and 2.2).
//
// Five passes over HBM per right-hand side (u = l m n complex values):
//   1 x forward   masked x (3u)        -> buf1 (3 n m 2l = 6u), zero-pad pruned
//   2 y forward   buf1                 -> buf2 (3 n 2m 2l = 12u), zero-pad pruned
//   3 z           buf2, kernel spectrum -> buf2: forward FFT along z of the n
//                 live planes, 3x3 symmetric multiply by the spectrum, inverse
//                 FFT, only the n box planes written back
//   4 y inverse   buf2 -> buf1 (rows m..2m-1 dropped)
//   5 x inverse   buf1 -> y: columns l..2l-1 dropped, diagonal term added
#include "matvec.cuh"

namespace dda {

// Right-hand sides go through the five passes in chunks of the plan's
// rhs_chunk (the FFT scratch holds that many).
template <>
void matvec_impl<float>(dda_plan_s* p, int nrhs, const cx<float>* x, cx<float>* y,
                        cudaStream_t s) {
  const long nu = 3 * p->nvox;
  for (int r0 = 0; r0 < nrhs; r0 += p->rhs_chunk) {
    const int nr = std::min(p->rhs_chunk, nrhs - r0);
    matvec_core<float>(p, nr, x + r0 * nu, y + r0 * nu, s, r0);
  }
}

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_matvec(dda_plan_t p, int32_t prec, int32_t nrhs, const void* d_x,
                                   void* d_y, void* stream) {
  if (!p || !d_x || !d_y) return fail(DDA_ERR_INVALID_ARG, "dda_matvec: NULL argument");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_matvec: nrhs must be 1..(incidences set)");
  if (d_x == d_y) return fail(DDA_ERR_INVALID_ARG, "dda_matvec: x and y must not overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScheduleScope scope(p->sched);
  if (prec == DDA_C128) {
    if (!p->has128) return fail(DDA_ERR_INVALID_ARG, "dda_matvec: plan holds no complex128 data");
    matvec_impl<double>(p, nrhs, static_cast<const cx<double>*>(d_x), static_cast<cx<double>*>(d_y), s);
  } else if (prec == DDA_C64) {
    if (!p->has64) return fail(DDA_ERR_INVALID_ARG, "dda_matvec: plan holds no complex64 data");
    matvec_impl<float>(p, nrhs, static_cast<const cx<float>*>(d_x), static_cast<cx<float>*>(d_y), s);
  } else {
    return fail(DDA_ERR_INVALID_ARG, "dda_matvec: prec must be DDA_C128 or DDA_C64");
  }
  return check_cuda("dda_matvec");
}
