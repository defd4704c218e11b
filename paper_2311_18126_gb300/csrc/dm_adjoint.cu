// Adjoint of one backward-Euler step of single rods (Sec. III-C, Eq. 15),
// for gradients of a loss L(q_{n+1}, qdot_{n+1}) with respect to the
// natural curvatures of the step and the state (q_n, qdot_n), the committed
// reference frames held fixed.  With f(q_{n+1}; q_n, qdot_n, kappabar) = 0,
// qdot_{n+1} = (q_{n+1} - q_n)/dt and J = df/dq_{n+1} (symmetric for rods):
//   J lambda = gbar,  gbar = dL/dq_{n+1} + dL/dqdot_{n+1} / dt   (free DOFs)
//   dL/dkappabar_c = -lambda . df/dkappabar_c =  EI/V lambda . grad kappa_c
//   dL/dq_n        = -lambda . df/dq_n - dL/dqdot_{n+1} / dt
//                  =  lambda (M/dt^2 + c_damp) - dL/dqdot_{n+1} / dt
//   dL/dqdot_n     = -lambda . df/dqdot_n = lambda M / dt
// Fixed DOFs keep q_{n+1} = q_n: dL/dq_n = dL/dq_{n+1} there, no velocity
// gradient, and they do not enter the solve.
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

__global__ void k_adj_rhs(AdjArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  a.rhs[i] = a.fixed[i] ? 0.0 : a.rhs_sign * (a.gq[i] + a.gv[i] / a.dt);
}

__global__ void k_adj_state(AdjArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  if (a.fixed[i]) {
    a.gq0[i] = a.gq[i];
    a.gv0[i] = 0.0;
    return;
  }
  const double m = a.mass[i], idt = 1.0 / a.dt;
  double g = a.lam[i] * (m * idt * idt + a.damp[i]) - a.gv[i] * idt;
  if (a.nt) {
    // ground friction depends on x - x_n: dL/dx_n += lambda^T J_plane
    // (the in-plane block of -dF/dx, node terms rows 0-1, column c)
    const int c = a.dof_comp[i];
    if (c < 2) {
      const int v = a.dof_node[i], d = a.node_dof[v], NN = a.nn;
      g = fma(a.lam[d], a.nt[(3 + c) * NN + v], g);
      g = fma(a.lam[d + 1], a.nt[(6 + c) * NN + v], g);
    }
  }
  a.gq0[i] = g;
  a.gv0[i] = a.lam[i] * m * idt;
}

__global__ void k_adj_midpoint_in(int nd, const uint8_t *fixed, const double *qn, double *q,
                                  double *gq, double *gv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  q[i] = fixed[i] ? qn[i] : 0.5 * (qn[i] + q[i]);
  gq[i] *= 2.0;
  gv[i] *= 2.0;
}

// gq2, gv2: the doubled loss gradients.  Fixed DOFs: the core passed 2 gq
// through, the step keeps them (gq0 = gq) and gives them no velocity.
__global__ void k_adj_midpoint_out(int nd, const uint8_t *fixed, const double *gq2,
                                   const double *gv2, double *gq0, double *gv0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  gq0[i] -= 0.5 * gq2[i];
  if (!fixed[i]) gv0[i] -= 0.5 * gv2[i];
}

// dst = transposed condensation-path storage: per limb the band
// B'[p][k + 10] = B[p + k][10 - k], C' = R^T, R' = C^T (one thread per entry)
__global__ void k_gen_transpose(SolveGenArgs a, const double *src, double *dst) {
  const int L = blockIdx.y;
  if (L >= a.nlimb || !a.gs_fast[a.lb_gsys[L]]) return;
  const int n = a.lb_n[L], m = a.lb_m[L], nbc = a.lb_nbc[L];
  const double *B = src + a.lb_band[L];
  double *Bt = dst + a.lb_band[L];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * 21; e += gridDim.x * blockDim.x) {
    const int p = e / 21, k = e - p * 21 - 10;
    Bt[e] = (p + k >= 0 && p + k < n) ? B[(size_t)(p + k) * 21 + (10 - k)] : 0.0;
  }
  if (blockIdx.x == 0) {
    const double *C = src + a.lb_C[L], *R = src + a.lb_R[L];
    double *Ct = dst + a.lb_C[L], *Rt = dst + a.lb_R[L];
    for (int e = threadIdx.x; e < m * nbc; e += blockDim.x) {
      const int r = e / nbc, b = e - r * nbc;
      Ct[e] = R[(size_t)b * m + r];
      Rt[(size_t)b * m + r] = C[e];
    }
  }
}

__global__ void k_gen_transpose_border(SolveGenArgs a, const double *src, double *dst) {
  const int w = blockIdx.x;
  if (w >= a.ngen || !a.gs_fast[w]) return;
  const int nB = a.gs_nB[w];
  const double *J = src + a.gs_JBB[w];
  double *Jt = dst + a.gs_JBB[w];
  for (int e = threadIdx.x; e < nB * nB; e += blockDim.x) {
    const int i = e / nB, j = e - i * nB;
    Jt[(size_t)j * nB + i] = J[e];
  }
}

__global__ void k_adj_kbar(AdjArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nslots) return;
  const int k = a.slot2st[t];
  const int NS = a.ns;
  int dof[11];
#pragma unroll
  for (int n = 0; n < 3; ++n)
#pragma unroll
    for (int c = 0; c < 3; ++c) dof[4 * n + c] = a.st_nd[n * NS + k] + c;
  dof[3] = a.st_th[k];
  dof[7] = a.st_th[NS + k];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    double v = 0.0;
#pragma unroll
    for (int p = 0; p < 11; ++p) v = fma(a.lam[dof[p]], a.dk[(size_t)(11 * c + p) * NS + k], v);
    a.gkbar[2 * t + c] = a.st_kb[k] * v;
  }
}



// ---------------------------------------------------------------------------
// Frame chain of a rollout adjoint (the step adjoint holds the committed
// frames fixed; each step's frames come from the earlier tangents by
// time-parallel transport, Sec. III).  A rotation of edge e's committed
// director acts on the energy like a shift of its twist angle, so its
// adjoint is sigma_e = -(gbar_theta - M_theta/dt^2 lambda_theta), which in
// the step adjoint's own quantities is -((gq + gv/dt) - gv0/dt) at theta_e;
// moving a tangent rotates the directors transported from or to it by
// -w . dt with w(a, b) = (a x b)/(1 + a . b), the holonomy of the geodesic
// triangle.  Carried backwards: Phibar_n = Phibar_{n+1} + sigma and
// dL/dt_n = -Phibar_n [w(t_n, t_{n+1}) + w(t_{n-1}, t_n)], taken to the
// node positions through t = e/|e|.  All vectors in the state layout.
//
// Implicit midpoint: the step's energy is taken at y = (q_n + q_{n+1})/2,
// its frames transported from step n's to the tangents t_y of y, while the
// committed frames of step n+1 are transported to t_{n+1}.  In the outputs
// of the midpoint step adjoint (core over h = dt/2 with doubled gradients)
// sigma = -(2 gq + (gv - gv0)/h), and the transport out of t_n splits:
// dL/dt_n = -[Phibar_{n+1} w(t_n, t_{n+1}) + sigma w(t_n, t_y)
//             + Phibar_n w(t_{n-1}, t_n)].

__device__ __forceinline__ void unit_edge(const double *q, int a, double t[3], double &il) {
  const double ex = q[a + 4] - q[a], ey = q[a + 5] - q[a + 1], ez = q[a + 6] - q[a + 2];
  il = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
  t[0] = ex * il;
  t[1] = ey * il;
  t[2] = ez * il;
}

__device__ __forceinline__ void add_holonomy(const double a[3], const double b[3], double w[3]) {
  const double c = 1.0 / (1.0 + a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
  w[0] += (a[1] * b[2] - a[2] * b[1]) * c;
  w[1] += (a[2] * b[0] - a[0] * b[2]) * c;
  w[2] += (a[0] * b[1] - a[1] * b[0]) * c;
}

// per edge: sigma, Phibar, and the tangent term g_e (3 doubles) to add at
// its end node and subtract at its start node
__global__ void k_frame_chain_edges(FrameChainArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  const int x0 = a.edge_lay[e], th = x0 + 3;
  double sigma = 0.0;
  if (!a.fixed[a.layout2dof[th]])
    sigma = a.midpoint ? -(2.0 * a.gq[th] + (a.gv[th] - a.gv0[th]) / a.dt)
                       : -((a.gq[th] + a.gv[th] / a.dt) - a.gv0[th] / a.dt);
  const double phi1 = a.phibar[e], phi = phi1 + sigma;
  a.phibar[e] = phi;
  double t[3], t1[3], il, il1, w[3] = {0.0, 0.0, 0.0};
  unit_edge(a.q, x0, t, il);
  unit_edge(a.q_next, x0, t1, il1);
  if (a.q_prev) {
    double tp[3], ilp;
    unit_edge(a.q_prev, x0, tp, ilp);
    add_holonomy(tp, t, w);
  }
  double gt[3];
  if (a.midpoint) {
    double w1[3] = {0.0, 0.0, 0.0}, wy[3] = {0.0, 0.0, 0.0}, ty[3];
    add_holonomy(t, t1, w1);
    double ey[3], ly = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ey[c] = 0.5 * ((a.q[x0 + 4 + c] + a.q_next[x0 + 4 + c]) - (a.q[x0 + c] + a.q_next[x0 + c]));
      ly += ey[c] * ey[c];
    }
    ly = 1.0 / sqrt(ly);
#pragma unroll
    for (int c = 0; c < 3; ++c) ty[c] = ey[c] * ly;
    add_holonomy(t, ty, wy);
#pragma unroll
    for (int c = 0; c < 3; ++c) gt[c] = -(phi * w[c] + phi1 * w1[c] + sigma * wy[c]);
  } else {
    add_holonomy(t, t1, w);
#pragma unroll
    for (int c = 0; c < 3; ++c) gt[c] = -phi * w[c];
  }
  const double tg = gt[0] * t[0] + gt[1] * t[1] + gt[2] * t[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) a.g[3 * e + c] = (gt[c] - tg * t[c]) * il;
}

// per layout node: + the term of the edge ending there - that of the edge
// starting there (a fixed order: deterministic)
__global__ void k_frame_chain_nodes(FrameChainArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.nlnode) return;
  const int x = a.lnode_lay[k], ein = a.lnode_ein[k], eout = a.lnode_eout[k];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    if (ein >= 0) v += a.g[3 * ein + c];
    if (eout >= 0) v -= a.g[3 * eout + c];
    a.gq0[x + c] += v;
  }
}

// committed directors SoA [3][Ne] <-> caller layout [Ne][3]
__global__ void k_frames_out(int ne, const double *soa, double *aos) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  for (int c = 0; c < 3; ++c) aos[3 * e + c] = soa[c * ne + e];
}
__global__ void k_frames_in(int ne, const double *aos, double *soa) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  for (int c = 0; c < 3; ++c) soa[c * ne + e] = aos[3 * e + c];
}

}  // namespace dm
