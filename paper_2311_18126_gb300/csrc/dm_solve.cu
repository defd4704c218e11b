// Residual, Jacobian assembly and linear solve of the backward-Euler Newton
// iteration (DisMech, arXiv 2311.18126, Sec. III-C, Eq. 15-16), FP64.
//
//  k_rows_rod   -- one thread per DOF row of a single-rod system: gathers the
//                  forces of the stencils/edges that touch the DOF (Eq. 9 plus
//                  gravity and damping), forms the residual
//                  f = M/dt^2 (q - q_n) - M/dt qdot_n - F, its scaled size
//                  |f| / (D l) (max-reduced per system), and the lower band
//                  row of J = M/dt^2 - dF/dq (half bandwidth 10 in the Eq. 1
//                  layout: a bend-twist stencil spans DOFs 4m-4 .. 4m+6).
//  k_solve_rod  -- one thread per rod: convergence decision, banded LDL^T
//                  factorisation (J is symmetric without friction) with a
//                  sliding 11x11 window, two triangular solves and q += dq.
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

template <int n>
__device__ __forceinline__ constexpr int upk(int i, int j) {
  return i * n - i * (i - 1) / 2 + (j - i);
}

__device__ __forceinline__ int ksym(int c, int cp) {  // packed 3x3 (xx,xy,xz,yy,yz,zz)
  int i = c < cp ? c : cp, j = c < cp ? cp : c;
  return 3 + (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

__global__ void __launch_bounds__(256) k_rows_rod(RowArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  const int s = a.dof_sys[i];
  if (!a.sys_active[s]) return;
  const int base = a.sys_dof0[s];
  const int r = i - base;
  const int n = a.sys_ndof[s];
  const int N = (n + 1) >> 2;
  const int node = r >> 2, c = r & 3;
  const int st0 = a.sys_st0[s], e0 = a.sys_edge0[s];
  const int NS = a.ns, NE = a.ne;
  double F = 0.0;
  double brow[11];
#pragma unroll
  for (int d = 0; d < 11; ++d) brow[d] = 0.0;
  // stencils m (interior nodes 1..N-2) with 4m-4 <= r <= 4m+6
  int mlo = (r - 6 + 3) >= 0 ? (r - 6 + 3) / 4 : 0;
  if (mlo < 1) mlo = 1;
  int mhi = (r + 4) / 4;
  if (mhi > N - 2) mhi = N - 2;
  for (int m = mlo; m <= mhi; ++m) {
    const int lr = r - 4 * (m - 1);
    const int st = st0 + m - 1;
    F -= a.sg[lr * NS + st];
#pragma unroll
    for (int d = 0; d < 11; ++d) {
      const int lc = lr - d;
      if (lc >= 0) brow[d] += a.sh[upk<11>(lc, lr) * NS + st];
    }
  }
  const double m_i = a.mass[i];
  const double idt = 1.0 / a.dt;
  if (c < 3) {
    if (node <= N - 2) {  // edge `node` starts here
      const int e = e0 + node;
      F += a.es[c * NE + e];
#pragma unroll
      for (int cp = 0; cp <= 2; ++cp)
        if (cp <= c) brow[c - cp] += a.es[ksym(c, cp) * NE + e];
    }
    if (node >= 1) {  // edge `node-1` ends here
      const int e = e0 + node - 1;
      F -= a.es[c * NE + e];
#pragma unroll
      for (int cp = 0; cp <= 2; ++cp) {
        const double kv = a.es[ksym(c, cp) * NE + e];
        if (cp <= c) brow[c - cp] += kv;
        brow[4 + c - cp] -= kv;
      }
    }
    F += m_i * a.g[c];
    const double cd = a.damp[i];
    F -= cd * (a.q[i] - a.qn[i]);
    brow[0] += cd;
  }
  brow[0] += m_i * idt * idt;
  double f = m_i * idt * idt * (a.q[i] - a.qn[i]) - m_i * idt * a.vn[i] - F;
  if (a.fixed[i]) {
    f = 0.0;
    brow[0] = 1.0;
#pragma unroll
    for (int d = 1; d < 11; ++d) brow[d] = 0.0;
  } else {
#pragma unroll
    for (int d = 1; d < 11; ++d)
      if (r - d < 0 || a.fixed[i - d]) brow[d] = 0.0;
  }
  a.f[i] = f;
#pragma unroll
  for (int d = 0; d < 11; ++d) a.band[(size_t)d * a.nd + i] = brow[d];
  // scaled residual, max-reduced per system (order independent)
  const double rr = fabs(f) * a.rscale[i];
  atomicMax(&a.sys_res[s], (unsigned long long)__double_as_longlong(rr));
}

__global__ void __launch_bounds__(64) k_solve_rod(SolveArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nsys) return;
  const int s = a.order[t];
  if (!a.sys_active[s]) return;
  const double res = __longlong_as_double((long long)a.sys_res[s]);
  int st = a.sys_status[s];
  if (st == 0 && isnan(res)) st = DM_ERR_NONFINITE;
  if (st == 0 && res <= a.tol) {  // converged at this iterate
    a.sys_active[s] = 0;
    return;
  }
  if (st == 0 && a.sys_iters[s] >= a.max_iter) st = DM_ERR_NOT_CONVERGED;
  if (st != 0) {
    a.sys_status[s] = st;
    a.sys_active[s] = 0;
    atomicAdd(&a.ctrl[1], 1);
    atomicMin(&a.ctrl[2], s);
    return;
  }
  const int n = a.sys_ndof[s];
  const int base = a.sys_dof0[s];
  const size_t ND = (size_t)a.nd;
  double *B = a.band;
  // sliding window of the lower band: W[row % 11][d] = J[row][row - d]
  double W[11][11];
  for (int rr = 0; rr < 11 && rr < n; ++rr)
#pragma unroll
    for (int d = 0; d < 11; ++d) W[rr][d] = B[d * ND + base + rr];
  int slot = 0;
  for (int j = 0; j < n; ++j) {
    const double dj = W[slot][0];
    if (!(fabs(dj) > 1e-300)) {
      a.sys_status[s] = DM_ERR_DEGENERATE;
      a.sys_active[s] = 0;
      atomicAdd(&a.ctrl[1], 1);
      atomicMin(&a.ctrl[2], s);
      return;
    }
    const double rj = 1.0 / dj;
    B[base + j] = dj;
    double u[11];
#pragma unroll
    for (int i = 1; i < 11; ++i) {
      int si = slot + i;
      si -= (si >= 11) ? 11 : 0;
      u[i] = (j + i < n) ? W[si][i] : 0.0;
    }
#pragma unroll
    for (int i = 1; i < 11; ++i) {
      int si = slot + i;
      si -= (si >= 11) ? 11 : 0;
      const double li = u[i] * rj;
#pragma unroll
      for (int k = 1; k <= i; ++k) W[si][i - k] = fma(-li, u[k], W[si][i - k]);
      if (j + i < n) B[i * ND + base + j + i] = li;
    }
    // row j + 11 enters the freed slot
    if (j + 11 < n) {
#pragma unroll
      for (int d = 0; d < 11; ++d) W[slot][d] = B[d * ND + base + j + 11];
    }
    slot = (slot == 10) ? 0 : slot + 1;
  }
  // forward L y = -f (y kept in dq), then D, then backward L^T x = z, q += x
  double y[11];
#pragma unroll
  for (int d = 0; d < 11; ++d) y[d] = 0.0;
  slot = 0;
  for (int i = 0; i < n; ++i) {
    double v = -a.f[base + i];
#pragma unroll
    for (int d = 1; d < 11; ++d) {
      int sd = slot - d;
      sd += (sd < 0) ? 11 : 0;
      if (i - d >= 0) v = fma(-B[d * ND + base + i], y[sd], v);
    }
    y[slot] = v;
    a.dq[base + i] = v;
    slot = (slot == 10) ? 0 : slot + 1;
  }
#pragma unroll
  for (int d = 0; d < 11; ++d) y[d] = 0.0;
  slot = 0;
  for (int i = n - 1; i >= 0; --i) {
    double v = a.dq[base + i] / B[base + i];
#pragma unroll
    for (int d = 1; d < 11; ++d) {
      int sd = slot - d;
      sd += (sd < 0) ? 11 : 0;
      if (i + d < n) v = fma(-B[d * ND + base + i + d], y[sd], v);
    }
    y[slot] = v;
    a.q[base + i] += v;
    slot = (slot == 10) ? 0 : slot + 1;
  }
  a.sys_iters[s] += 1;
  atomicAdd(&a.ctrl[0], 1);
}

}  // namespace dm
