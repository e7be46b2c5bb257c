// The 3-level preconditioner's apply in complex128 (the complex64 one and the
// build are in precond.cu).
#include "precond_apply.cuh"

namespace dda {

template void precond_apply_into<double>(dda_plan_s*, int, const cx<double>*, cx<double>*,
                                         cx<double>*, cudaStream_t);
template void precond_apply_impl<double>(dda_plan_s*, int, const cx<double>*, cx<double>*,
                                         cudaStream_t);

}  // namespace dda
