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

// Length-projected Newton guess (an option of the predictor): for each
// single-rod system, every edge of the guess in q is rescaled to its length
// in the committed state q_n, node positions rebuilt outward from the rod's
// first node along the guess's edge directions; a node with a fixed position
// DOF keeps its value.  The stiff stretching part of the guess's error goes,
// the soft bending part stays.  The rebuilt positions are a prefix sum of
// the rescaled edge vectors that restarts at node 0 and at every fixed node
// (a segmented scan): one warp per system, 32 nodes per pass, the running
// position carried from pass to pass (Eq. 1 layout: node k at DOFs 4k..4k+2).
// Implicit midpoint (q holds the midpoint guess y): the projection acts on
// the step's end guess 2y - q_n and y is rebuilt as its mean with q_n.
__global__ void k_project_lengths(int nsys, const int32_t *sys_kind, const int32_t *sys_dof0,
                                  const int32_t *sys_ndof, const uint8_t *fixed,
                                  const double *qn, double *q, int midpoint) {
  const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nsys || sys_kind[s] != SOLVE_ROD_BAND) return;  // warp-uniform
  const unsigned full = 0xffffffffu;
  const int d0 = sys_dof0[s], N = (sys_ndof[s] + 1) / 4;
  // the previous pass's last node: rebuilt position (c) and guess (p)
  double cx = 0.0, cy = 0.0, cz = 0.0, px = 0.0, py = 0.0, pz = 0.0;
  for (int base = 0; base < N; base += 32) {
    const int k = base + lane;
    const bool on = k < N;
    const int o = d0 + 4 * k;
    // guess of node k, and of node k - 1 from the lane before (or the carry)
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (on) {
      gx = q[o];
      gy = q[o + 1];
      gz = q[o + 2];
      if (midpoint) {
        gx = 2.0 * gx - qn[o];
        gy = 2.0 * gy - qn[o + 1];
        gz = 2.0 * gz - qn[o + 2];
      }
    }
    double hx = __shfl_up_sync(full, gx, 1), hy = __shfl_up_sync(full, gy, 1),
           hz = __shfl_up_sync(full, gz, 1);
    if (lane == 0) {
      hx = px;
      hy = py;
      hz = pz;
    }
    // a head restarts the sum at its own (guessed) position; any other node
    // adds its rescaled edge vector from node k - 1
    bool head = true, keep = true;
    double vx = gx, vy = gy, vz = gz;
    if (on) {
      keep = k == 0 || fixed[o] || fixed[o + 1] || fixed[o + 2];
      head = keep;
      if (!keep) {
        const double ex = gx - hx, ey = gy - hy, ez = gz - hz;
        const double lx = qn[o] - qn[o - 4], ly = qn[o + 1] - qn[o - 3], lz = qn[o + 2] - qn[o - 2];
        const double l2 = ex * ex + ey * ey + ez * ez;
        const double sc = l2 > 0.0 ? sqrt((lx * lx + ly * ly + lz * lz) / l2) : 1.0;
        vx = sc * ex;
        vy = sc * ey;
        vz = sc * ez;
      }
    }
    // inclusive segmented scan over the pass
    bool h = head;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double ux = __shfl_up_sync(full, vx, d), uy = __shfl_up_sync(full, vy, d),
                   uz = __shfl_up_sync(full, vz, d);
      const bool uh = __shfl_up_sync(full, (int)h, d) != 0;
      if (lane >= d) {
        if (!h) {
          vx += ux;
          vy += uy;
          vz += uz;
        }
        h = h || uh;
      }
    }
    if (!h) {  // no restart in this pass up to here: continue from the carry
      vx += cx;
      vy += cy;
      vz += cz;
    }
    if (on && !keep) {  // only this lane reads its node's q
      if (midpoint) {
        q[o] = 0.5 * (qn[o] + vx);
        q[o + 1] = 0.5 * (qn[o + 1] + vy);
        q[o + 2] = 0.5 * (qn[o + 2] + vz);
      } else {
        q[o] = vx;
        q[o + 1] = vy;
        q[o + 2] = vz;
      }
    }
    const int last = min(31, N - 1 - base);
    cx = __shfl_sync(full, vx, last);
    cy = __shfl_sync(full, vy, last);
    cz = __shfl_sync(full, vz, last);
    px = __shfl_sync(full, gx, last);
    py = __shfl_sync(full, gy, last);
    pz = __shfl_sync(full, gz, last);
  }
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

// Counts a round run before the graph's while node (the fused first round).
__global__ void k_round_count(int32_t *ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ++ctrl[4];
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
