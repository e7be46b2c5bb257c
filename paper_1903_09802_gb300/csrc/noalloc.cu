// dda_precond_apply_noalloc: the preconditioner apply for callers that must
// not allocate device memory while they run.  Examples are real-time or
// embedded hosts whose device memory is fixed at start-up, and frameworks
// that own every byte of the device through their own pool and forbid
// allocations from outside it.  The ordinary entry
// point keeps its transform in the plan's workspace; this one keeps it in a
// fixed array compiled into the library, so the call itself reserves
// nothing.
#include <cstring>

#include "plan.hpp"

namespace dda {
namespace {

// 32 MiB, reserved on every device that loads the library until the
// process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array in the current context.  The host-side
// symbol is not a device address.  Once the library's device code is loaded
// in the context (noalloc_prepare, called by dda_plan_create), the lookup is
// a host-side table read that allocates nothing; it is repeated on every call
// so that a context torn down and made again (cudaDeviceReset) never leaves
// a stale address behind.
dda_status_t scratch_address(void** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr)
    return fail(DDA_ERR_CUDA, std::string("dda_precond_apply_noalloc: cudaGetSymbolAddress: ") +
                                  cudaGetErrorString(e));
  *out = ptr;
  return DDA_OK;
}

}  // namespace

// Loads this file's device code (and with it the 32 MiB array) into the
// current context.  With lazy module loading the first symbol lookup is what
// loads it, and loading reserves the array's memory; plan creation, which
// the caller makes while it may still allocate, does that lookup so that the
// apply itself never reserves anything.
dda_status_t noalloc_prepare() {
  void* ptr = nullptr;
  return scratch_address(&ptr);
}

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_precond_apply_noalloc(dda_plan_t p, int32_t prec, int32_t nrhs,
                                                  const void* d_v, void* d_z, void* stream) {
  if (!p || !d_v || !d_z)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply_noalloc: NULL argument");
  if (!p->precond_built)
    return fail(DDA_ERR_NO_PRECOND, "dda_precond_apply_noalloc: call dda_precond_build first");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply_noalloc: nrhs must be 1..(incidences set)");
  if (prec != DDA_C128 && prec != DDA_C64)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply_noalloc: prec must be DDA_C128 or DDA_C64");
  if ((prec == DDA_C128 && !p->has128) || (prec == DDA_C64 && !p->has64))
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply_noalloc: plan lacks that precision");
  // Mixed-radix transforms in FP64 run kernels with a local stack frame,
  // whose first launch may make the driver enlarge the context's
  // local-memory reservation, an allocation: power-of-two boxes only.
  if (!is_pow2(p->l) || !is_pow2(p->m) || !is_pow2(p->n))
    return fail(DDA_ERR_UNSUPPORTED_SIZE,
                "dda_precond_apply_noalloc: box edges must be powers of two (mixed-radix "
                "transforms may enlarge the local-memory reservation)");
  const size_t esz = prec == DDA_C128 ? 16 : 8;
  const size_t need = (size_t)nrhs * 3 * (size_t)p->nvox * esz;
  if (need > kNoAllocScratchBytes)
    return fail(DDA_ERR_WORKSPACE,
                "dda_precond_apply_noalloc: nrhs * 3 * l*m*n complex values need " +
                    std::to_string(need) + " bytes, above the 33554432-byte static scratch");
  void* scratch = nullptr;
  const dda_status_t st = scratch_address(&scratch);
  if (st != DDA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScheduleScope scope(p->sched);
  if (prec == DDA_C128)
    precond_apply_into<double>(p, nrhs, static_cast<const cx<double>*>(d_v),
                               static_cast<cx<double>*>(d_z), static_cast<cx<double>*>(scratch), s);
  else
    precond_apply_into<float>(p, nrhs, static_cast<const cx<float>*>(d_v),
                              static_cast<cx<float>*>(d_z), static_cast<cx<float>*>(scratch), s);
  return check_cuda("dda_precond_apply_noalloc");
}
