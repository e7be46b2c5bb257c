// The BTTB matvec in complex128 (double-float arithmetic): the same five
// passes as the complex64 operator (matvec.cu), compiled in a translation
// unit of its own.
#include "matvec.cuh"

namespace dda {

// complex128 fields, double-float arithmetic (about 48 bits, at FP32 rates):
// y <- x converted, the five passes in place on y (the epilogue reads each
// input value before writing the output value of the same thread), y
// converted back.  x and y must not overlap unless they are the same buffer.
template <>
void matvec_impl<double>(dda_plan_s* p, int nrhs, const cx<double>* x, cx<double>* y,
                         cudaStream_t s) {
  const long n = (long)nrhs * 3 * p->nvox;
  const unsigned g = (unsigned)std::min<long>((n + 255) / 256, 152L * 32);
  cx<df>* ydf = reinterpret_cast<cx<df>*>(y);
  note_launch();
  launch_k(k_to_df, g, 256, 0, s, reinterpret_cast<const double2*>(x), ydf, n);
  const long nu = 3 * p->nvox;
  for (int r0 = 0; r0 < nrhs; r0 += p->rhs_chunk) {
    const int nr = std::min(p->rhs_chunk, nrhs - r0);
    matvec_core<df>(p, nr, ydf + r0 * nu, ydf + r0 * nu, s, r0);
  }
  note_launch();
  launch_k(k_from_df, g, 256, 0, s, static_cast<const cx<df>*>(ydf),
           reinterpret_cast<double2*>(y), n);
}

}  // namespace dda
