// Public batched banded solve (dm_solve_band): the twisted LDL^T kernel of
// the Newton step (k_solve_rod) applied to caller-provided systems.
#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

namespace {

__global__ void k_band_prepare(int nsys, int64_t ntot, const double *rhs, double *f,
                               int32_t *order, int32_t *active, int32_t *iters,
                               int32_t *status, unsigned long long *res, int32_t *ctrl) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ntot) f[i] = -rhs[i];  // the kernel solves J dq = -f
  if (i < nsys) {
    order[i] = (int32_t)i;
    active[i] = 1;
    iters[i] = 0;
    status[i] = 0;
    res[i] = 0x7ff0000000000000ull;  // +inf: never counted as converged
  }
  if (i == 0) {
    ctrl[0] = 0;
    ctrl[1] = 0;
    ctrl[2] = INT_MAX;
    ctrl[3] = 0;
  }
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// Bytes of scratch the banded solve needs for a batch.
size_t band_scratch_bytes(int32_t nsys, int64_t ntot) {
  size_t b = align256(13 * (size_t)ntot * sizeof(double));  // band copy, f, dq
  b += align256(6 * (size_t)nsys * sizeof(int32_t));        // per-system ints
  b += align256((size_t)nsys * sizeof(unsigned long long)); // residual slots
  b += align256(4 * sizeof(int32_t));                       // queue / counters
  return b;
}

bool check_band_batch(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                      const double *band, const double *rhs, const double *x) {
  if (nsys < 0 || ntot < 0 || (nsys > 0 && (!dof0 || !ndof || !band || !rhs || !x))) {
    set_error("dm_solve_band: bad arguments");
    return false;
  }
  if (ntot > INT_MAX / 16) {
    set_error("dm_solve_band: ntot too large");
    return false;
  }
  for (int k = 0; k < nsys; ++k)
    if (ndof[k] < 1 || dof0[k] < 0 || (int64_t)dof0[k] + ndof[k] > ntot) {
      set_error("dm_solve_band: system " + std::to_string(k) + " outside [0, ntot)");
      return false;
    }
  // the kernel updates each system's rows in place and accumulates into x:
  // systems may not share rows
  std::vector<int32_t> by_start(nsys);
  for (int k = 0; k < nsys; ++k) by_start[k] = k;
  std::sort(by_start.begin(), by_start.end(),
            [&](int32_t u, int32_t v) { return dof0[u] < dof0[v]; });
  for (int k = 1; k < nsys; ++k) {
    const int32_t u = by_start[k - 1], v = by_start[k];
    if ((int64_t)dof0[u] + ndof[u] > dof0[v]) {
      set_error("dm_solve_band: systems " + std::to_string(u) + " and " + std::to_string(v) +
                " overlap");
      return false;
    }
  }
  // x is written while band and rhs are still read
  auto overlaps = [](const void *p, size_t pn, const void *q, size_t qn) {
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + qn && b < a + pn;
  };
  const size_t vb = (size_t)ntot * sizeof(double);
  if (nsys > 0 && ntot > 0 && (overlaps(x, vb, rhs, vb) || overlaps(x, vb, band, 11 * vb))) {
    set_error("dm_solve_band: x overlaps band or rhs");
    return false;
  }
  return true;
}

// Runs the banded solve with all scratch inside `scr` (band_scratch_bytes
// bytes, 256-byte aligned) and waits for it.  h_ctrl: 4 host ints.
dm_status run_band_solve(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                         const double *band, const double *rhs, double *x, char *scr,
                         cudaStream_t st) {
  if (nsys == 0 || ntot == 0) return DM_OK;
  double *bcopy = (double *)scr;  // [11][ntot] band copy (becomes L)
  double *f = bcopy + 11 * ntot;  // [ntot] -rhs
  double *dq = f + ntot;          // [ntot] y / D
  char *q = scr + align256(13 * (size_t)ntot * sizeof(double));
  int32_t *ib = (int32_t *)q;
  int32_t *d_dof0 = ib, *d_ndof = ib + nsys, *order = ib + 2 * nsys;
  int32_t *active = ib + 3 * nsys, *iters = ib + 4 * nsys, *status = ib + 5 * nsys;
  q += align256(6 * (size_t)nsys * sizeof(int32_t));
  unsigned long long *res = (unsigned long long *)q;
  q += align256((size_t)nsys * sizeof(unsigned long long));
  int32_t *ctrl = (int32_t *)q;
#define BS_CK(call)                                                           \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      set_error(std::string("dm_solve_band: ") + cudaGetErrorString(e_));     \
      return DM_ERR_CUDA;                                                     \
    }                                                                         \
  } while (0)
  BS_CK(cudaMemcpyAsync(bcopy, band, 11 * ntot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  BS_CK(cudaMemcpyAsync(d_dof0, dof0, nsys * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  BS_CK(cudaMemcpyAsync(d_ndof, ndof, nsys * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  BS_CK(cudaMemsetAsync(x, 0, ntot * sizeof(double), st));
  const int64_t nthr = ntot > nsys ? ntot : nsys;
  k_band_prepare<<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(nsys, ntot, rhs, f, order,
                                                                  active, iters, status, res, ctrl);
  BS_CK(cudaGetLastError());
  SolveArgs va{};
  va.nsys = nsys;
  va.nd = (int)ntot;
  va.tol = 0.0;
  va.max_iter = 1;
  va.order = order;
  va.sys_dof0 = d_dof0;
  va.sys_ndof = d_ndof;
  va.fixed = nullptr;
  va.f = f;
  va.band = bcopy;
  va.q = x;
  va.dq = dq;
  va.sys_active = active;
  va.sys_iters = iters;
  va.sys_status = status;
  va.sys_res = res;
  va.ctrl = ctrl;
  va.units = nullptr;
  const int rods_per_block = 4 * kSolveRodsPerWarp;  // four warps
  const size_t smem = rods_per_block * kSolveRodDoubles * sizeof(double);
  int dev = 0, sms = 1, per_sm = 1;
  BS_CK(cudaGetDevice(&dev));
  BS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BS_CK(cudaFuncSetAttribute(k_solve_rod, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_rod, 128, smem));
  int nblk = (nsys + rods_per_block - 1) / rods_per_block;
  if (nblk > per_sm * sms) nblk = per_sm * sms;
  if (nblk > sms) nblk = sms;  // one block of four warps per SM, as in dm_step
  if (nblk < 1) nblk = 1;
  k_solve_rod<<<nblk, 128, smem, st>>>(va);
  BS_CK(cudaGetLastError());
  int32_t h[4] = {0, 0, 0, 0};
  BS_CK(cudaMemcpyAsync(h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st));
  BS_CK(cudaStreamSynchronize(st));
#undef BS_CK
  if (h[1] > 0) {
    set_error("dm_solve_band: zero or non-finite pivot in system " + std::to_string(h[2]));
    return DM_ERR_DEGENERATE;
  }
  return DM_OK;
}

}  // namespace dm

extern "C" dm_status dm_solve_band(int32_t nsys, const int32_t *sys_dof0,
                                   const int32_t *sys_ndof, int64_t ntot, const double *band,
                                   const double *rhs, double *x, void *stream) {
  using namespace dm;
  if (!check_band_batch(nsys, sys_dof0, sys_ndof, ntot, band, rhs, x)) return DM_ERR_INVALID_ARG;
  if (nsys == 0 || ntot == 0) return DM_OK;
  char *scr = nullptr;
  const size_t bytes = band_scratch_bytes(nsys, ntot);
  cudaError_t e = cudaMalloc(&scr, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("dm_solve_band: cudaMalloc: ") + cudaGetErrorString(e));
    return DM_ERR_OOM;
  }
  dm_status st = run_band_solve(nsys, sys_dof0, sys_ndof, ntot, band, rhs, x, scr,
                                (cudaStream_t)stream);
  cudaFree(scr);
  return st;
}
