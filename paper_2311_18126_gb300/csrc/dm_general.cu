// General systems: rods joined at elastic joints (Sec. III-D) and rods on
// the ground with IMC contact and smooth Coulomb friction (Sec. III-B,
// Eq. 10-13), FP64.
//
//  k_nodes         -- one thread per node: ground contact force along z
//                     (Eq. 10-11 with stiffness k_c) and friction (Eq. 12-13)
//                     with the implicit tangential velocity (x - x_n)/dt, plus
//                     -dF/dx (3x3, not symmetric: friction depends on z
//                     through |F_n|).
//  k_rows_gen      -- one thread per DOF: residual of Eq. 15 from the force
//                     gather lists and its scaled size.
//  k_assemble_gen  -- one thread per matrix entry of the limb bands, the
//                     limb/border coupling blocks and the border block of
//                     the systems that solve this round: the sum of its
//                     element contributions in a fixed order.
//  k_solve_gen     -- one warp per system: banded LU with partial pivoting of
//                     every limb interior (one lane per limb), the Schur complement
//                     on the border DOFs (joint nodes, their neighbours and
//                     the first twist angles) with a dense pivoted LU, and
//                     back-substitution.
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

__device__ __forceinline__ double softplus(double x) {
  return fmax(x, 0.0) + log1p(exp(-fabs(x)));
}

__global__ void k_nodes(NodeArgs a) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nn) return;
  if (!a.sys_active[a.node_sys[v]]) return;
  count_active(a.units);
  const int NN = a.nn;
  const int d = a.node_dof[v];
  const double z = a.q[d + 2] - a.ground_z;
  const double C = a.node_h[v], dl = a.delta, K1 = 15.0 / dl, kc = a.node_kc[v];
  // Eq. 10 and its first two derivatives in D
  double dE = 0.0, d2E = 0.0;
  if (z <= C - dl) {
    dE = -2.0 * (C - z);
    d2E = 2.0;
  } else if (z < C + dl) {
    const double s = K1 * (C - z);
    const double sp = softplus(s);
    const double sg = 1.0 / (1.0 + exp(-s));
    dE = -2.0 * sp * sg / K1;
    d2E = 2.0 * (sg * sg + sp * sg * (1.0 - sg));
  }
  const double Fn = -kc * dE;
  double F[3] = {0.0, 0.0, Fn};
  double J[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, kc * d2E};
  const double mu = a.node_mu[v];
  if (mu > 0.0 && Fn != 0.0) {
    const double K2 = 15.0 / a.slip_nu, idt = 1.0 / a.dt;
    const double ux = (a.q[d] - a.qn[d]) * idt, uy = (a.q[d + 1] - a.qn[d + 1]) * idt;
    const double s = sqrt(ux * ux + uy * uy);
    const double fn = fabs(Fn);
    if (s == 0.0) {
      // limit of -mu |F_n| gamma(|u|) u/|u| at u = 0 (reading C14)
      const double c = mu * fn * 0.5 * K2 * idt;
      J[0] = c;
      J[4] = c;
    } else {
      const double th = tanh(0.5 * K2 * s);   // gamma of Eq. 12
      const double dth = 0.5 * K2 * (1.0 - th * th);
      const double hx = ux / s, hy = uy / s;
      F[0] = -mu * th * hx * fn;
      F[1] = -mu * th * hy * fn;
      // -dF/dx in the plane: mu |F_n| [g/s (I - u u^T) + g' u u^T] / dt
      const double a1 = mu * fn * th / s * idt, a2 = mu * fn * dth * idt;
      J[0] = a1 * (1.0 - hx * hx) + a2 * hx * hx;
      J[1] = (a2 - a1) * hx * hy;
      J[3] = J[1];
      J[4] = a1 * (1.0 - hy * hy) + a2 * hy * hy;
      // -dF/dz: |F_n| = -k_c E'(D) in contact, d|F_n|/dz = -k_c E''
      J[2] = -mu * th * hx * kc * d2E;
      J[5] = -mu * th * hy * kc * d2E;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) a.nt[c * NN + v] = F[c];
#pragma unroll
  for (int k = 0; k < 9; ++k) a.nt[(3 + k) * NN + v] = J[k];
}

__global__ void __launch_bounds__(256) k_rows_gen(RowGenArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  const int s = a.dof_sys[i];
  if (a.sys_kind[s] != SOLVE_GENERAL || !a.sys_active[s]) return;
  count_active(a.units);
  double F = 0.0;
  for (int k = a.gat_ptr[i]; k < a.gat_ptr[i + 1]; ++k) {
    const int code = a.gat_ent[k];
    const int idx = code >> 5;
    if (code & 16) {
      const int slot = code & 15;
      const double v = a.es[(slot % 3) * a.ne + idx];
      F += slot < 3 ? v : -v;
    } else {
      F -= a.sg[(code & 15) * a.ns + idx];
    }
  }
  const int c = a.dof_comp[i];
  const double m = a.mass[i], idt = a.idt;
  if (c < 3) {
    F += m * a.g[c];
    F -= a.damp[i] * (a.q[i] - a.qn[i]);
    if (a.nt) F += a.nt[c * a.nn + a.dof_node[i]];
  }
  double f = m * idt * idt * (a.q[i] - a.qn[i]) - m * idt * a.vn[i] - F;
  if (a.fixed[i]) f = 0.0;
  a.f[i] = f;
  const double rr = fabs(f) * a.rscale[i];
  atomicMax(&a.sys_res[s], (unsigned long long)__double_as_longlong(rr));
}

// Grid (system, chunk of kAsmPerBlock targets): blocks of systems that do
// not solve this round (inactive or backtracking) leave at once; every
// target entry gets the sum of its element contributions in a fixed order.
__global__ void k_assemble_gen(AsmArgs a) {
  const int w = blockIdx.x;
  const int sy = a.gen_sys[w];
  if (!a.sys_active[sy] || (a.ls_action && a.ls_action[sy] == 1)) return;  // no solve
  if (a.units && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(a.units, (unsigned long long)a.sys_ndof[sy]);
  const int t1 = a.t0[w + 1];
#pragma unroll
  for (int u = 0; u < kAsmPerBlock / 256; ++u) {
    const int t = a.t0[w] + (int)blockIdx.y * kAsmPerBlock + u * 256 + (int)threadIdx.x;
    if (t >= t1) break;
    double v = 0.0;
    for (int k = a.ptr[t]; k < a.ptr[t + 1]; ++k) {
      const uint32_t code = a.src[k];
      const uint32_t type = (code >> 29) & 3u, idx = code & 0x1FFFFFFFu;
      double x;
      if (type == SRC_STENCIL) x = a.sh[idx];
      else if (type == SRC_EDGE) x = a.es[idx];
      else if (type == SRC_NODE) x = a.nt[idx];
      else x = a.dconst[idx];
      v += (code & 0x80000000u) ? -x : x;
    }
    a.gen[a.target[t]] = v;
  }
}

// Storage of the systems on the pivoting path that solve this round: it
// holds the last factorisation (in place, with fill), cleared before the
// assembly; one block per system.
__global__ void k_gen_clear_slow(AsmArgs a, const int32_t *gs_fast) {
  const int w = blockIdx.x;
  if (gs_fast[w]) return;
  const int sy = a.gen_sys[w];
  if (!a.sys_active[sy] || (a.ls_action && a.ls_action[sy] == 1)) return;
  for (int64_t i = a.mat0[w] + threadIdx.x; i < a.mat1[w]; i += blockDim.x) a.gen[i] = 0.0;
}

__global__ void k_solve_gen(SolveGenArgs a) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= a.ngen || a.gs_fast[w]) return;  // condensation path systems
  const int s = a.gen_sys[w];
  int st = 0;
  int go = 0;
  if (lane == 0 && a.sys_active[s] && a.ls_action && a.ls_action[s] == 1) {
    atomicAdd(&a.ctrl[0], 1);  // backtracking: no solve this round
  } else if (lane == 0 && a.sys_active[s]) {
    const double res = __longlong_as_double((long long)a.sys_res[s]);
    st = a.sys_status[s];
    if (st == 0 && isnan(res)) st = DM_ERR_NONFINITE;
    if (st == 0 && res <= a.tol) {
      a.sys_active[s] = 0;
    } else {
      if (st == 0 && a.sys_iters[s] >= a.max_iter) st = DM_ERR_NOT_CONVERGED;
      if (st != 0) {
        a.sys_status[s] = st;
        a.sys_active[s] = 0;
        atomicAdd(&a.ctrl[1], 1);
        atomicMin(&a.ctrl[2], s);
      } else {
        go = 1;
      }
    }
  }
  go = __shfl_sync(0xffffffffu, go, 0);
  if (!go) return;
  const int nl = a.gs_nlimb[w], nB = a.gs_nB[w], L0 = a.gs_limb0[w], B0 = a.gs_border0[w];
  double *G = a.gen;
  bool bad = false;
  // 1) limbs: banded LU with partial pivoting (band[d][r] = J[r][r + d - 10],
  //    d in 0..30: 10 subdiagonals, 10 superdiagonals and 10 more for the
  //    fill of row interchanges), then y = J_ii^{-1} (-f_i), Y = J_ii^{-1} C_i
  for (int l = lane; l < nl; l += 32) {
    const int L = L0 + l;
    const int n = a.lb_n[L], ncr = a.lb_ncr[L];
    const int32_t *cr = a.coupled_rows + a.lb_cr0[L];
    double *A = G + a.lb_band[L];
    double *piv = G + a.lb_piv[L];
    double *C = G + a.lb_C[L];
    double *Y = G + a.lb_Y[L];
    double *y = G + a.lb_y[L];
    const int d0 = a.lb_dof0[L];
    for (int j = 0; j < n; ++j) {
      int p = j;
      double best = fabs(A[10 * n + j]);
      for (int i = 1; i <= 10 && j + i < n; ++i) {
        const double v = fabs(A[(10 - i) * n + j + i]);
        if (v > best) {
          best = v;
          p = j + i;
        }
      }
      piv[j] = (double)p;
      if (!(best > 0.0) || !isfinite(best)) {
        bad = true;
        break;
      }
      if (p != j)  // swap rows j and p over columns j .. j + 20
        for (int c = j; c <= j + 20 && c < n; ++c) {
          double *x1 = A + (c - j + 10) * n + j, *x2 = A + (c - p + 10) * n + p;
          const double t = *x1;
          *x1 = *x2;
          *x2 = t;
        }
      const double rp = 1.0 / A[10 * n + j];
      for (int i = 1; i <= 10 && j + i < n; ++i) {
        const double li = A[(10 - i) * n + j + i] * rp;
        A[(10 - i) * n + j + i] = li;
        if (li != 0.0)
          for (int k = 1; k <= 20 && j + k < n; ++k)
            A[(10 + k - i) * n + j + i] = fma(-li, A[(10 + k) * n + j], A[(10 + k - i) * n + j + i]);
      }
    }
    for (int r = 0; r < n; ++r) y[r] = -a.f[d0 + r];
    for (int r = 0; r < n * nB; ++r) Y[r] = 0.0;
    for (int k = 0; k < ncr; ++k)
      for (int b = 0; b < nB; ++b) Y[cr[k] * nB + b] = C[k * nB + b];
    for (int col = -1; col < nB && !bad; ++col) {
      double *v = col < 0 ? y : Y + col;
      const int st2 = col < 0 ? 1 : nB;
      for (int j = 0; j < n; ++j) {
        const int p = (int)piv[j];
        if (p != j) {
          const double t = v[j * st2];
          v[j * st2] = v[p * st2];
          v[p * st2] = t;
        }
        const double vj = v[j * st2];
        if (vj != 0.0)
          for (int i = 1; i <= 10 && j + i < n; ++i)
            v[(j + i) * st2] = fma(-A[(10 - i) * n + j + i], vj, v[(j + i) * st2]);
      }
      for (int j = n - 1; j >= 0; --j) {
        double x = v[j * st2];
        for (int k = 1; k <= 20 && j + k < n; ++k) x = fma(-A[(10 + k) * n + j], v[(j + k) * st2], x);
        v[j * st2] = x / A[10 * n + j];
      }
    }
  }
  __syncwarp();
  bad = __any_sync(0xffffffffu, bad);
  // 2) Schur complement on the border and its right-hand side
  double *S = G + a.gs_S[w], *JBB = G + a.gs_JBB[w], *rB = G + a.gs_rB[w], *xB = G + a.gs_xB[w];
  for (int e = lane; e < nB * nB; e += 32) {
    const int b1 = e / nB, b2 = e - b1 * nB;
    double v = JBB[e];
    for (int l = 0; l < nl; ++l) {
      const int L = L0 + l;
      const int ncr = a.lb_ncr[L];
      const int32_t *cr = a.coupled_rows + a.lb_cr0[L];
      const double *R = G + a.lb_R[L];
      const double *Y = G + a.lb_Y[L];
      for (int k = 0; k < ncr; ++k) v = fma(-R[b1 * ncr + k], Y[cr[k] * nB + b2], v);
    }
    S[e] = v;
  }
  for (int b1 = lane; b1 < nB; b1 += 32) {
    double v = -a.f[a.border_dof[B0 + b1]];
    for (int l = 0; l < nl; ++l) {
      const int L = L0 + l;
      const int ncr = a.lb_ncr[L];
      const int32_t *cr = a.coupled_rows + a.lb_cr0[L];
      const double *R = G + a.lb_R[L];
      const double *y = G + a.lb_y[L];
      for (int k = 0; k < ncr; ++k) v = fma(-R[b1 * ncr + k], y[cr[k]], v);
    }
    rB[b1] = v;
  }
  __syncwarp();
  // 3) dense LU with partial pivoting of the border system (lane 0)
  if (lane == 0 && nB > 0 && !bad) {
    for (int j = 0; j < nB; ++j) {
      int p = j;
      double best = fabs(S[j * nB + j]);
      for (int i = j + 1; i < nB; ++i)
        if (fabs(S[i * nB + j]) > best) {
          best = fabs(S[i * nB + j]);
          p = i;
        }
      if (!(best > 0.0) || !isfinite(best)) {
        bad = true;
        break;
      }
      if (p != j) {
        for (int k = 0; k < nB; ++k) {
          const double t = S[j * nB + k];
          S[j * nB + k] = S[p * nB + k];
          S[p * nB + k] = t;
        }
        const double t = rB[j];
        rB[j] = rB[p];
        rB[p] = t;
      }
      const double rp = 1.0 / S[j * nB + j];
      for (int i = j + 1; i < nB; ++i) {
        const double li = S[i * nB + j] * rp;
        if (li == 0.0) continue;
        for (int k = j + 1; k < nB; ++k) S[i * nB + k] = fma(-li, S[j * nB + k], S[i * nB + k]);
        rB[i] = fma(-li, rB[j], rB[i]);
      }
    }
    if (!bad)
      for (int i = nB - 1; i >= 0; --i) {
        double x = rB[i];
        for (int k = i + 1; k < nB; ++k) x = fma(-S[i * nB + k], xB[k], x);
        xB[i] = x / S[i * nB + i];
      }
  }
  __syncwarp();
  bad = __any_sync(0xffffffffu, bad);
  if (bad) {
    if (lane == 0) {
      a.sys_status[s] = DM_ERR_DEGENERATE;
      a.sys_active[s] = 0;
      atomicAdd(&a.ctrl[1], 1);
      atomicMin(&a.ctrl[2], s);
    }
    return;
  }
  // 4) back-substitution: x_i = y_i - Y_i x_B
  for (int l = lane; l < nl; l += 32) {
    const int L = L0 + l;
    const int n = a.lb_n[L], d0 = a.lb_dof0[L];
    const double *Y = G + a.lb_Y[L];
    const double *y = G + a.lb_y[L];
    for (int r = 0; r < n; ++r) {
      double x = y[r];
      for (int b = 0; b < nB; ++b) x = fma(-Y[r * nB + b], xB[b], x);
      a.q[d0 + r] += x;
    }
  }
  for (int b = lane; b < nB; b += 32) a.q[a.border_dof[B0 + b]] += xB[b];
  __syncwarp();
  if (lane == 0) {
    a.sys_iters[s] += 1;
    if (a.ls_trial) a.ls_trial[s] = 1;
    atomicAdd(&a.ctrl[0], 1);
    if (a.units) {
      int nd = nB;
      for (int l = 0; l < nl; ++l) nd += a.lb_n[L0 + l];
      atomicAdd(a.units, (unsigned long long)nd);
    }
  }
}

}  // namespace dm
