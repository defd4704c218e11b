// Step bookkeeping kernels: predictor, commit and rollback (DisMech,
// arXiv 2311.18126, Sec. III-C: q_dot_{n+1} = (q_{n+1} - q_n)/dt; Sec. III:
// reference frames carried between steps by time-parallel transport).
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

// Start of a step: every system active, Newton guess q = q_n + dt qdot_n
// (reading C23), fixed DOFs keep q_n.
__global__ void k_begin_step(StepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nsys) {
    a.sys_active[i] = 1;
    a.sys_iters[i] = 0;
    a.sys_status[i] = 0;
    a.sys_res[i] = 0ull;
  }
  if (i < a.nd) a.q[i] = a.fixed[i] ? a.qn[i] : fma(a.dt, a.vn[i], a.qn[i]);
}

// Commit the converged step: velocities, then q_n, the transported reference
// directors and tangents of every edge, and the reference twist of every
// stencil (all computed at the converged iterate).
__global__ void k_commit(StepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double idt = 1.0 / a.dt;
  if (i < a.nd) {
    const double q = a.q[i];
    a.vn[i] = a.vnew ? a.vnew[i] : (q - a.qn[i]) * idt;
    a.qn[i] = q;
  }
  if (i < a.ne) {
    const int NE = a.ne;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.tn[c * NE + i] = a.ef[c * NE + i];
      a.d1n[c * NE + i] = a.ef[(4 + c) * NE + i];
    }
  }
  if (i < a.ns) a.beta_n[i] = a.beta_it[i];
}

// Implicit midpoint, solved as backward Euler over dt/2 (a.dt) for the
// midpoint configuration y (held in q): with y = (q_n + q_{n+1})/2 the
// midpoint residual 2M/dt^2 (q_{n+1} - q_n - dt qdot_n) - F(y) is the
// backward-Euler residual 4M/dt^2 (y - q_n - (dt/2) qdot_n) - F(y), and the
// velocity of velocity-dependent forces (x_{n+1} - x_n)/dt = (y - x_n)/(dt/2).
// Here: q <- q_{n+1} = 2y - q_n and the staged velocity qdot_{n+1} =
// 2 (q_{n+1} - q_n)/dt - qdot_n = 2 (y - q_n)/(dt/2) - qdot_n (zero on fixed
// DOFs); every system is marked active so that the frames and the reference
// twist can be evaluated at q_{n+1} before the commit.
__global__ void k_midpoint_finish(StepArgs a, double *vnew) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nd) {
    const double y = a.q[i], qn = a.qn[i];
    vnew[i] = a.fixed[i] ? 0.0 : 2.0 * (y - qn) / a.dt - a.vn[i];
    a.q[i] = a.fixed[i] ? qn : 2.0 * y - qn;
  }
  if (i < a.nsys) a.sys_active[i] = 1;
}

// Systems whose status was set outside the Newton bookkeeping (the frame
// evaluation at q_{n+1} of an implicit-midpoint step) count as failed.
__global__ void k_collect_failures(int nsys, const int32_t *sys_status, int32_t *ctrl) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || sys_status[s] == 0) return;
  atomicAdd(&ctrl[1], 1);
  atomicMin(&ctrl[2], s);
}

// Failed step: drop the iterate, the committed state is untouched.
__global__ void k_restore(StepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nd) a.q[i] = a.qn[i];
}

// End of one Newton round inside the round graph: counts the round and
// keeps the graph's while loop going while some system is still active and
// fewer than max_rounds rounds have run (ctrl[0] = systems still active,
// ctrl[4] = rounds of this step), so the loop always ends.
__global__ void k_round_continue(int32_t *ctrl, int max_rounds, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int r = ++ctrl[4];
  cudaGraphSetConditional(h, (ctrl[0] > 0 && r < max_rounds) ? 1u : 0u);
}

// Clears the residual slots of the systems [lo, hi) still iterating before a
// round's row kernels max-reduce into them; a system that has stopped keeps
// the residual of its last evaluated iterate (the value dm_step reports).
__global__ void k_reset_res(int lo, int hi, const int32_t *sys_active,
                            unsigned long long *sys_res) {
  const int s = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (s < hi && sys_active[s]) sys_res[s] = 0ull;
}

// Committed tangents recomputed from q (after a state is set).
__global__ void k_tangents(int ne, const int32_t *edge_a, const int32_t *edge_b,
                           const double *q, double *tn, int32_t *bad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int ia = edge_a[e], ib = edge_b[e];
  const double x = q[ib] - q[ia], y = q[ib + 1] - q[ia + 1], z = q[ib + 2] - q[ia + 2];
  const double l2 = x * x + y * y + z * z;
  if (!(l2 > 0.0)) {
    atomicExch(bad, 1);
    return;
  }
  const double il = rsqrt(l2);
  tn[e] = x * il;
  tn[ne + e] = y * il;
  tn[2 * ne + e] = z * il;
}

}  // namespace dm
