// Batched FFT launchers, double-float complex instantiations (forward; the
// inverse ones are in fft_launch_dfi.cu, to halve the compile time).
#include "fft_launch.cuh"

namespace dda {

#define DDA_INST_FFT(T, INV)                                                                      \
  template void launch_contig<T, INV>(const cx<T>*, cx<T>*, const uint8_t*, const uint8_t*, long,  \
                                      long, int, int,                                             \
                                      long, int, long, T, const cx<T>*, int, cudaStream_t);        \
  template void launch_strided<T, INV>(const cx<T>*, cx<T>*, long, long, int, int, long, long,     \
                                       int, long, long, T, const cx<T>*, int, cudaStream_t);       \
  template void fft3d_inplace<T, INV>(cx<T>*, long, int, int, int, T, const cx<T>*, int,           \
                                      cudaStream_t);
DDA_INST_FFT(df, false)

}  // namespace dda
