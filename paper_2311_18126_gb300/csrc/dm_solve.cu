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
  const bool act = i < a.nd && a.sys_active[a.dof_sys[i]] &&
                   a.sys_kind[a.dof_sys[i]] != SOLVE_GENERAL;
  count_units(a.units, act);
  if (!act) return;
  const int s = a.dof_sys[i];
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
  if (a.fc) F += a.fc[i];
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

// Banded LDL^T solve of J dq = -f for single rods.
//
// The FP64 pipe of an SM partition retires one warp instruction about every
// 80 cycles whatever the active mask, and a column of the band elimination
// is a short dependency chain, so a 4096-rod batch is latency-bound unless
// every partition holds several warps whose lanes all do useful FP64 work.
// Each rod is therefore factored from both ends at once (a twisted
// factorisation): a top chain eliminates columns 0..m-1 downwards, a bottom
// chain eliminates columns n-1..m+10 upwards, and the 10-row separator left
// in the middle is combined from both windows and solved densely.  Each
// chain is run by four lanes with one uniform instruction stream; the 11x11
// active window and the right-hand side live in shared memory.  Eliminating
// a column costs 10 multipliers, 55 trailing updates and 10 right-hand-side
// updates (forward substitution fused in); lane p owns whole window rows,
// balanced by work (row i carries i + 1 FMAs):
//   lane 0: rows 10, 3, 1   lane 1: rows 9, 5   lane 2: rows 8, 6
//   lane 3: rows 7, 4, 2    -- at most 17 FMAs and 3 multipliers per lane.
// The next pivot is updated first by lane 0, broadcast by a shuffle, and its
// reciprocal (FP32 seed, two FP64 Newton steps) overlaps the other updates.
// Rods are taken from a queue in order of decreasing size, four per warp.
#define SOLVE_WARPS 4
#define SOLVE_RODS_PER_WARP 4
#define SOLVE_CHAIN_STRIDE 133  // doubles per chain: W 121, z 11, spare 1

__device__ __forceinline__ int wrap11(int x) { return x >= 11 ? x - 11 : x; }

// 1/d from an FP32 seed and two Newton steps in FP64 (|d| within FP32 range).
__device__ __forceinline__ double rcp64(double d) {
  double r = (double)__frcp_rn((float)d);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// Task k of lane p: window row i (bits 0-3) and u index q (bits 4-7,
// 0 = right-hand side, 15 = padding); row slot r (bits 8-9) in rows[].
__host__ __device__ constexpr int task_code(int p, int k) {
  // lane rows in order; each row i contributes q = 1..i then q = 0
  int rows[4][3] = {{10, 3, 1}, {9, 5, 0}, {8, 6, 0}, {7, 4, 2}};
  int t = 0;
  for (int r = 0; r < 3; ++r) {
    const int i = rows[p][r];
    if (i == 0) continue;
    for (int q = 1; q <= i + 1; ++q) {
      const int qq = (q == i + 1) ? 0 : q;
      if (t == k) return i | (qq << 4) | (r << 8);
      ++t;
    }
  }
  return 15 << 4;  // padding
}

struct Chain {
  // address maps of one elimination direction
  double *B;
  const double *f;
  double *dq;
  size_t ND, base;
  int n, dir;  // dir = +1 top-down, -1 bottom-up
  __device__ __forceinline__ int orig(int idx) const { return dir > 0 ? idx : n - 1 - idx; }
  // lower-band entry (idx, idx - d) of the chain's matrix
  __device__ __forceinline__ double *entry(int idx, int d) const {
    return B + d * ND + base + (dir > 0 ? idx : n - 1 - idx + d);
  }
  // storage of the multiplier L[c + i][c]
  __device__ __forceinline__ double *lstore(int c, int i) const {
    return B + i * ND + base + (dir > 0 ? c + i : n - 1 - c);
  }
  __device__ __forceinline__ double rhs(int idx) const { return -f[base + orig(idx)]; }
  __device__ __forceinline__ double *zstore(int idx) const { return dq + base + orig(idx); }
};

// Eliminates `ncol` columns of a chain.  On return W/Z hold rows
// ncol..ncol+10 of the partially reduced matrix and right-hand side.
__device__ __forceinline__ bool eliminate(const Chain &c, int ncol, double *W, double *Z,
                                          int p, unsigned cmask, int leader) {
  const int n = c.n;
  int rows[3];
  rows[0] = p == 0 ? 10 : (p == 1 ? 9 : (p == 2 ? 8 : 7));
  rows[1] = p == 0 ? 3 : (p == 1 ? 5 : (p == 2 ? 6 : 4));
  rows[2] = p == 0 ? 1 : (p == 3 ? 2 : 0);
  int code[17];
#pragma unroll
  for (int k = 0; k < 17; ++k)
    code[k] = p == 0 ? task_code(0, k) : (p == 1 ? task_code(1, k) : (p == 2 ? task_code(2, k) : task_code(3, k)));
  for (int e = p; e < 121; e += 4) {
    const int r = e / 11, d = e - 11 * r;
    W[e] = (r < n && d <= r) ? *c.entry(r, d) : 0.0;
  }
  for (int r = p; r < 11; r += 4) Z[r] = (r < n) ? c.rhs(r) : 0.0;
  __syncwarp(cmask);
  double rj = rcp64(W[0]);
  bool bad = false;
  int s0 = 0;
  for (int j = 0; j < ncol; ++j) {
    const bool more = j + 11 < n;
    double pre0 = 0.0, pre1 = 0.0, pre2 = 0.0;
    if (more) {
      pre0 = *c.entry(j + 11, p);
      pre1 = *c.entry(j + 11, p + 4);
      if (p + 8 < 11) pre2 = *c.entry(j + 11, p + 8);
    }
    const double zj = Z[s0];
    if (p == 0) {
      if (!isfinite(rj) || rj == 0.0) bad = true;
      *c.zstore(j) = zj * rj;  // z_j = y_j / D_j for the backward pass
    }
    double l[3], uq[17];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = rows[r];
      const bool ok = i > 0 && j + i < n;
      l[r] = (ok ? W[wrap11(s0 + i) * 11 + i] : 0.0) * rj;
    }
#pragma unroll
    for (int k = 0; k < 17; ++k) {
      const int q = (code[k] >> 4) & 15;
      uq[k] = (q > 0 && q < 15 && j + q < n) ? W[wrap11(s0 + q) * 11 + q] : (q == 0 ? zj : 0.0);
    }
    // next pivot first (lane 0 owns window row 1), broadcast, reciprocal
    double piv = 0.0;
    if (p == 0) piv = (j + 1 < n) ? fma(-l[2], uq[0], W[wrap11(s0 + 1) * 11]) : 1.0;
    piv = __shfl_sync(cmask, piv, leader);
    const double rnext = rcp64(piv);
    __syncwarp(cmask);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = rows[r];
      if (i > 0 && j + i < n) *c.lstore(j, i) = l[r];
    }
#pragma unroll
    for (int k = 0; k < 17; ++k) {
      const int i = code[k] & 15, q = (code[k] >> 4) & 15, r = code[k] >> 8;
      const double lk = r == 0 ? l[0] : (r == 1 ? l[1] : l[2]);
      if (q < 15 && j + i < n) {
        double *dst = (q == 0) ? (Z + wrap11(s0 + i)) : (W + wrap11(s0 + i) * 11 + (i - q));
        *dst = fma(-lk, uq[k], *dst);
      }
    }
    __syncwarp(cmask);
    if (more) {
      W[s0 * 11 + p] = pre0;
      W[s0 * 11 + p + 4] = pre1;
      if (p + 8 < 11) W[s0 * 11 + p + 8] = pre2;
      if (p == 0) Z[s0] = c.rhs(j + 11);
    } else {
#pragma unroll
      for (int d = 0; d < 11; d += 4) if (d + p < 11) W[s0 * 11 + d + p] = 0.0;
      if (p == 0) Z[s0] = 0.0;
    }
    s0 = wrap11(s0 + 1);
    rj = rnext;
    __syncwarp(cmask);
  }
  return bad;
}

// Right-looking backward substitution x_i = z_i - sum_d L[i+d][i] x_{i+d}
// for chain rows kstart-1 .. 0, given x of rows kstart..kstart+9 in xs[].
__device__ __forceinline__ void back_substitute(const Chain &c, int kstart, const double *xs,
                                                double *Z, double *q, int p, unsigned cmask) {
  // Z slot m % 11 holds the running z of chain row m (m < kstart)
  for (int m = kstart - 1 - p; m >= 0 && m >= kstart - 11; m -= 4) Z[m % 11] = *c.zstore(m);
  __syncwarp(cmask);
  for (int k = kstart + 9; k >= 0; --k) {
    if (k >= c.n) continue;
    double xk;
    if (k >= kstart) {
      xk = xs[k - kstart];
    } else {
      xk = Z[k % 11];
      if (p == 0) q[c.base + c.orig(k)] += xk;
    }
    double Lv[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int d = 1 + p + 4 * t;
      Lv[t] = (d <= 10 && k - d >= 0 && k - d < kstart) ? *c.entry(k, d) : 0.0;
    }
    const double znew = (p == 1 && k < kstart && k - 11 >= 0) ? *c.zstore(k - 11) : 0.0;
    __syncwarp(cmask);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int d = 1 + p + 4 * t;
      if (d <= 10 && k - d >= 0 && k - d < kstart) {
        const int slot = (k - d) % 11;
        Z[slot] = fma(-Lv[t], xk, Z[slot]);
      }
    }
    if (p == 1 && k < kstart && k - 11 >= 0) Z[k % 11] = znew;
    __syncwarp(cmask);
  }
}

__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_solve_rod(SolveArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int unit = lane >> 3;          // rod slot in the warp
  const int half = (lane >> 2) & 1;    // 0 = top chain, 1 = bottom chain
  const int p = lane & 3;
  const int rid = (threadIdx.x >> 5) * SOLVE_RODS_PER_WARP + unit;
  double *Wt = smem + (size_t)rid * (2 * SOLVE_CHAIN_STRIDE + 32);
  double *Wb = Wt + SOLVE_CHAIN_STRIDE;
  double *XS = Wb + SOLVE_CHAIN_STRIDE;  // separator solution (10) + scratch
  double *W = half ? Wb : Wt;
  double *Z = W + 121;
  const unsigned umask = 0xFFu << (unit * 8);
  const unsigned cmask = 0xFu << (unit * 8 + half * 4);
  const int leader = unit * 8 + half * 4;

  while (true) {
    int t = 0;
    if ((lane & 7) == 0) t = atomicAdd(&a.ctrl[3], 1);
    t = __shfl_sync(umask, t, unit * 8);
    if (t >= a.nsys) break;
    const int s = a.order[t];
    if (!a.sys_active[s]) continue;
    if (a.ls_action && a.ls_action[s] == 1) {  // backtracking: no solve this round
      if ((lane & 7) == 0) atomicAdd(&a.ctrl[0], 1);
      continue;
    }
    const double res = __longlong_as_double((long long)a.sys_res[s]);
    int st = a.sys_status[s];
    if (st == 0 && isnan(res)) st = DM_ERR_NONFINITE;
    if (st == 0 && res <= a.tol) {  // converged at this iterate
      if ((lane & 7) == 0) a.sys_active[s] = 0;
      continue;
    }
    if (st == 0 && a.sys_iters[s] >= a.max_iter) st = DM_ERR_NOT_CONVERGED;
    if (st != 0) {
      if ((lane & 7) == 0) {
        a.sys_status[s] = st;
        a.sys_active[s] = 0;
        atomicAdd(&a.ctrl[1], 1);
        atomicMin(&a.ctrl[2], s);
      }
      continue;
    }
    const int n = a.sys_ndof[s];
    Chain c{a.band, a.f, a.dq, (size_t)a.nd, (size_t)a.sys_dof0[s], n, half ? -1 : 1};
    // split: top eliminates [0, m), bottom [m + 10, n), separator [m, m + 10)
    const bool twist = n >= 32;
    const int m = twist ? (n - 10) / 2 : n;
    const int ncol = half ? (twist ? n - m - 10 : 0) : m;
    bool bad = false;
    if (!half || twist) bad = eliminate(c, ncol, W, Z, p, cmask, leader);
    bad = __any_sync(umask, bad);
    __syncwarp(umask);
    if (bad) {
      if ((lane & 7) == 0) {
        a.sys_status[s] = DM_ERR_DEGENERATE;
        a.sys_active[s] = 0;
        atomicAdd(&a.ctrl[1], 1);
        atomicMin(&a.ctrl[2], s);
      }
      continue;
    }
    if (twist) {
      // separator: S = top window + bottom window - original, same for the
      // right-hand side; dense LDL^T by one lane (10 x 10)
      if ((lane & 7) == 0) {
        const int nb = n - m - 10;
        double S[10][10], r[10];
        for (int i = 0; i < 10; ++i) {
          for (int j2 = 0; j2 <= i; ++j2) {
            const int d = i - j2;
            const double top = Wt[((m + i) % 11) * 11 + d];
            const double bot = Wb[((nb + 9 - j2) % 11) * 11 + d];
            const double org = a.band[d * (size_t)a.nd + c.base + m + i];
            S[i][j2] = top + bot - org;
          }
          r[i] = Wt[121 + (m + i) % 11] + Wb[121 + (nb + 9 - i) % 11] + a.f[c.base + m + i];
        }
        for (int j2 = 0; j2 < 10; ++j2) {
          const double dinv = 1.0 / S[j2][j2];
          if (!isfinite(dinv)) bad = true;
          // rows in decreasing order: S[k][j2] (k < i) is still unscaled
          for (int i = 9; i > j2; --i) {
            const double li = S[i][j2] * dinv;
            for (int k = j2 + 1; k <= i; ++k) S[i][k] = fma(-li, S[k][j2], S[i][k]);
            r[i] = fma(-li, r[j2], r[i]);
            S[i][j2] = li;
          }
          S[j2][j2] = dinv;
        }
        for (int i = 9; i >= 0; --i) {
          double x = r[i] * S[i][i];
          for (int k = i + 1; k < 10; ++k) x = fma(-S[k][i], XS[k], x);
          XS[i] = x;
          a.q[c.base + m + i] += x;
        }
      }
      bad = __any_sync(umask, bad);
      __syncwarp(umask);
      if (bad) {
        if ((lane & 7) == 0) {
          a.sys_status[s] = DM_ERR_DEGENERATE;
          a.sys_active[s] = 0;
          atomicAdd(&a.ctrl[1], 1);
          atomicMin(&a.ctrl[2], s);
        }
        continue;
      }
      // separator x in chain order for each half (the bottom chain sees the
      // separator rows reversed)
      double xs[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) xs[i] = half ? XS[9 - i] : XS[i];
      const int kstart = half ? n - m - 10 : m;
      back_substitute(c, kstart, xs, Z, a.q, p, cmask);
    } else if (!half) {
      double xs[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) xs[i] = 0.0;
      back_substitute(c, n, xs, Z, a.q, p, cmask);
    }
    __syncwarp(umask);
    if ((lane & 7) == 0) {
      a.sys_iters[s] += 1;
      if (a.ls_trial) a.ls_trial[s] = 1;
      atomicAdd(&a.ctrl[0], 1);
      if (a.units) atomicAdd(a.units, (unsigned long long)n);
    }
  }
}

// Line search (optional): Armijo test on the 2-norm of the scaled residual
// |f_i| / (D_i l_i) of each system (the Newton direction is a descent
// direction for it); a trial point without sufficient decrease is pulled
// halfway back to the last accepted iterate, at most 12 times.
// k_ls_merit: one warp per system, fixed summation order (deterministic).
__global__ void k_ls_merit(LineSearchArgs a) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= a.nsys) return;
  if (!a.sys_active[s]) return;
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s];
  double acc = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double v = a.f[d0 + i] * a.rscale[d0 + i];
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) a.merit[s] = sqrt(acc);
}

__global__ void k_ls_decide(LineSearchArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nsys || !a.sys_active[s]) return;
  const double m = a.merit[s];
  if (a.wstry && a.wstry[s]) {
    // the learned guess is kept only if it lowers the merit below that of
    // the extrapolation; otherwise the iterate returns to the extrapolation
    a.wstry[s] = 0;
    if (!(m <= (1.0 - 1e-4) * a.racc[s])) {
      a.action[s] = 1;
      a.alpha[s] = 0.0;
      a.trial[s] = 0;
      a.nback[s] = 0;
      return;
    }
  }
  if (a.trial[s] && a.nback[s] < 12 && !(m <= (1.0 - 1e-4 * a.alpha[s]) * a.racc[s])) {
    a.action[s] = 1;
    a.alpha[s] *= 0.5;
    a.nback[s] += 1;
  } else {
    a.action[s] = 0;
    a.trial[s] = 0;
    a.nback[s] = 0;
    a.alpha[s] = 1.0;
    a.racc[s] = m;
  }
}

__global__ void k_ls_apply(LineSearchArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  const int s = a.dof_sys[i];
  if (!a.sys_active[s]) return;
  if (a.action[s] == 1) a.q[i] = a.alpha[s] == 0.0 ? a.qacc[i] : 0.5 * (a.q[i] + a.qacc[i]);
  else a.qacc[i] = a.q[i];
}

}  // namespace dm
