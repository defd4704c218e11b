// dm_solve_band_noalloc: the batched banded solve of dm_solve_band with all
// of its device scratch in a fixed array of this file, for callers that may
// not allocate device memory.  The kernels are the same as dm_solve_band's.
#include <string>

#include "dm_internal.h"

namespace dm {
size_t band_scratch_bytes(int32_t nsys, int64_t ntot);
bool check_band_batch(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                      const double *band, const double *rhs, const double *x);
dm_status run_band_solve(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                         const double *band, const double *rhs, double *x, char *scr,
                         cudaStream_t st);
}  // namespace dm

namespace {

// Scratch for DM_NOALLOC_MAX_SYSTEMS systems and DM_NOALLOC_MAX_DOFS DOFs:
// band copy, right-hand side and substitution vectors (13 doubles per DOF),
// six ints and one residual word per system, four counters.  About 3.3 MiB.
// The driver allocates it on a device when it loads this file's module
// there: at the first call of this entry point on that device under CUDA's
// default lazy module loading, at context creation under eager loading.
// It is then held until the process exits.
constexpr size_t kScratchBytes =
    13 * (size_t)DM_NOALLOC_MAX_DOFS * sizeof(double) +
    ((6 * (size_t)DM_NOALLOC_MAX_SYSTEMS * sizeof(int32_t) + 255) & ~(size_t)255) +
    ((DM_NOALLOC_MAX_SYSTEMS * sizeof(unsigned long long) + 255) & ~(size_t)255) + 256;

static __device__ __align__(256) char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch in the current context.  In host code
// the symbol name only stands for the array; the kernels must be given this
// address.  It is looked up on every call (cudaGetSymbolAddress allocates
// nothing once the module is loaded), so it is never stale after a device
// reset or under another context of the same device.
dm_status scratch_for_current_context(char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    dm::set_error(std::string("dm_solve_band_noalloc: cudaGetSymbolAddress: ") +
                  cudaGetErrorString(e));
    return DM_ERR_CUDA;
  }
  *out = (char *)p;
  return DM_OK;
}

}  // namespace

extern "C" dm_status dm_solve_band_noalloc(int32_t nsys, const int32_t *sys_dof0,
                                           const int32_t *sys_ndof, int64_t ntot,
                                           const double *band, const double *rhs, double *x,
                                           void *stream) {
  using namespace dm;
  if (!check_band_batch(nsys, sys_dof0, sys_ndof, ntot, band, rhs, x)) return DM_ERR_INVALID_ARG;
  if (nsys > DM_NOALLOC_MAX_SYSTEMS || ntot > DM_NOALLOC_MAX_DOFS) {
    set_error("dm_solve_band_noalloc: batch of " + std::to_string(nsys) + " systems / " +
              std::to_string(ntot) + " DOFs exceeds the fixed scratch limit of " +
              std::to_string(DM_NOALLOC_MAX_SYSTEMS) + " systems / " +
              std::to_string(DM_NOALLOC_MAX_DOFS) + " DOFs");
    return DM_ERR_INVALID_ARG;
  }
  if (band_scratch_bytes(nsys, ntot) > kScratchBytes) {
    set_error("dm_solve_band_noalloc: internal scratch layout exceeds the fixed array");
    return DM_ERR_INVALID_ARG;
  }
  if (nsys == 0 || ntot == 0) return DM_OK;
  char *scr = nullptr;
  dm_status st = scratch_for_current_context(&scr);
  if (st != DM_OK) return st;
  // run_band_solve clears every part of the scratch the kernel reads
  // before it reads it (band copy, right-hand side, counters, flags).
  return run_band_solve(nsys, sys_dof0, sys_ndof, ntot, band, rhs, x, scr, (cudaStream_t)stream);
}
