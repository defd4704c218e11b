// Partitioned solve of long symmetric banded systems (half bandwidth 10, the
// single-rod Jacobian of Sec. III-C, Eq. 16) that removes the sequential
// chain over the whole rod: the DOFs of a system are cut into interiors of
// m - 10 rows separated by 10-row separators, so that interiors do not
// couple (|i - j| > 10 across a separator).  With B_p the interior blocks,
// C_p their couplings to the neighbouring separators and B_p = L D L^T:
//
//   1. per interior, in parallel: L D L^T of B_p; forward solves
//      Z_p = L^{-1} C_p and z_p = L^{-1} f_p; the Schur contributions
//      Z_p^T D^{-1} Z_p and Z_p^T D^{-1} z_p (symmetry: only forward solves);
//   2. per system: the separators' block-tridiagonal Schur system
//      T x_S = g, T = A_SS - sum_p C_p^T B_p^{-1} C_p, eliminated block by
//      block (10 x 10 Gauss-Jordan, no pivoting: T is symmetric, and
//      positive definite whenever the rod Jacobian is);
//   3. per interior, in parallel: x_p = L^{-T} D^{-1} (z_p - Z_p x_S).
//
// The work per interior is a few times that of the plain band LDL^T, but
// the sequential depth is m rows plus one 10 x 10 elimination per
// separator instead of n rows.  One warp per interior or system; an
// interior keeps its band in shared memory.
#include <string>
#include <vector>

#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

namespace {

constexpr int PW = 10;  // half bandwidth = separator width

// Pivots smaller than this fraction of their row's original diagonal entry
// are treated as zero (DM_ERR_DEGENERATE): without pivoting they would
// amplify rounding errors without bound.
constexpr double kTinyPivot = 1e-13;

__device__ __forceinline__ double pb_recip(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
  double r = (double)__frcp_rn((float)d);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

struct PartArgs {
  int64_t ntot;
  int nparts, nsep;
  const int32_t *p_a, *p_mm, *p_top, *p_bot;  // interior rows [a, a+mm), separator ids or -1
  const int32_t *s_a;                          // separator rows [s_a, s_a + 10)
  const int32_t *sys_sep0, *sys_nsep;          // per system: first separator, count
  const double *band, *rhs;
  double *x;
  double *Lf, *Df, *Zt, *zf;   // [ntot][10], 1/D [ntot], [ntot][10], [ntot]
  double *Zb;                  // [nparts][10][10]: L^{-1} C_bot in the last 10 rows
  double *ct, *cb, *co;        // [nparts][110]: top/bottom contributions (10x10 + 10), top x bottom (10x10)
  double *Xs;                  // [nsep][110]: T'^{-1} [To | g']
  const int32_t *p_sys;        // interior -> system (index into go / bad)
  const int32_t *go;           // per system: solve it (NULL: all)
  int *bad;                    // per system: zero or non-finite pivot
};

// pair t in [0, 55) -> (u, v), 0 <= v <= u < 10
__device__ __forceinline__ void pair_uv(int t, int &u, int &v) {
  u = 0;
  while ((u + 1) * (u + 2) / 2 <= t) ++u;
  v = t - u * (u + 1) / 2;
}

__global__ void __launch_bounds__(32) k_part_factor(PartArgs a) {
  extern __shared__ double sm[];
  const int p = blockIdx.x, lane = threadIdx.x;
  const int sys = a.p_sys[p];
  if (a.go && !a.go[sys]) return;
  const int r0 = a.p_a[p], mm = a.p_mm[p];
  const bool top = a.p_top[p] >= 0, bot = a.p_bot[p] >= 0;
  double *Bs = sm;                     // [mm][11]: band, then multipliers
  double *Zs = a.Zt + (size_t)r0 * PW;  // [mm][10]: L^{-1} C_top (global, L2-resident)
  const int64_t N = a.ntot;
  for (int t = lane; t < mm * 11; t += 32) {
    const int i = t / 11, d = t - i * 11;
    Bs[t] = d <= i ? a.band[(size_t)d * N + r0 + i] : 0.0;
  }
  __syncwarp();
  // band L D L^T of the interior
  for (int j = 0; j < mm; ++j) {
    const double dj = Bs[j * 11];
    if (!(fabs(dj) > 0.0) || !isfinite(dj)) {
      if (lane == 0) atomicExch(a.bad + sys, 1);
      return;  // uniform: every lane read the same pivot
    }
    const double rj = pb_recip(dj);
    if (lane == 0) a.Df[r0 + j] = rj;
    const int i = j + 1 + lane;
    if (lane < PW && i < mm) Bs[i * 11 + (i - j)] *= rj;  // multiplier l_ij
    __syncwarp();
    for (int t = lane; t < 55; t += 32) {
      int u, v;
      pair_uv(t, u, v);
      const int ii = j + 1 + u, kk = j + 1 + v;
      if (ii < mm)
        Bs[ii * 11 + (ii - kk)] -= Bs[ii * 11 + (ii - j)] * dj * Bs[kk * 11 + (kk - j)];
    }
    __syncwarp();
  }
  // a pivot below kTinyPivot times its row's original diagonal entry counts
  // as zero (the Jacobian need not be positive definite); checked here, in
  // parallel, off the sequential chain
  bool tiny = false;
  for (int j = lane; j < mm; j += 32)
    if (fabs(a.band[r0 + j]) * kTinyPivot * fabs(a.Df[r0 + j]) > 1.0) tiny = true;
  if (__any_sync(0xffffffffu, tiny)) {
    if (lane == 0) atomicExch(a.bad + sys, 1);
    return;
  }
  for (int t = lane; t < mm * PW; t += 32) {
    const int i = t / PW, d = t - i * PW + 1;
    a.Lf[(size_t)(r0 + i) * PW + d - 1] = d <= i ? Bs[i * 11 + d] : 0.0;
  }
  // forward solves: lanes 0-9 the top coupling columns, lane 10 the
  // right-hand side, lanes 11-20 the bottom coupling columns (non-zero in
  // the last 10 rows only)
  double win[PW];
#pragma unroll
  for (int k = 0; k < PW; ++k) win[k] = 0.0;
  const int c = lane < PW ? lane : lane - 11;
  const int sa_bot = r0 + mm;  // first row of the bottom separator
  for (int i = 0; i < mm; ++i) {
    double z = 0.0;
    if (lane < PW) {  // C_top[i][c] = A[r0+i][r0-10+c], d = i + 10 - c
      if (top && c >= i) z = a.band[(size_t)(i + PW - c) * N + r0 + i];
    } else if (lane == PW) {
      z = a.rhs[r0 + i];
    } else if (lane < 2 * PW + 1) {  // C_bot[i][c] = A[sa_bot+c][r0+i], d = mm + c - i
      if (bot && i >= mm - PW + c) z = a.band[(size_t)(mm + c - i) * N + sa_bot + c];
    }
#pragma unroll
    for (int k = 1; k <= PW; ++k)
      if (k <= i) z = fma(-Bs[i * 11 + k], win[k - 1], z);
#pragma unroll
    for (int k = PW - 1; k > 0; --k) win[k] = win[k - 1];
    win[0] = z;
    if (lane < PW) {
      Zs[i * PW + c] = z;
    } else if (lane == PW) {
      a.zf[r0 + i] = z;
    } else if (lane < 2 * PW + 1 && i >= mm - PW && mm >= PW) {
      a.Zb[((size_t)p * PW + (i - (mm - PW))) * PW + c] = z;
    }
  }
  __syncwarp();
  // Schur contributions: ct = Zt^T D^{-1} [Zt | zf], cb = Zb^T D^{-1} [Zb | zf]
  // over the last 10 rows, co = Zt^T D^{-1} Zb
  const int lo = mm >= PW ? mm - PW : 0;
  for (int t = lane; t < 110 * 3; t += 32) {
    const int blk = t / 110, e = t - blk * 110;
    const int u = e < 100 ? e / PW : e - 100, v = e < 100 ? e % PW : -1;
    double s = 0.0;
    if (blk == 0) {  // ct
      if (!top) continue;
      for (int i = 0; i < mm; ++i) {
        const double rd = a.Df[r0 + i];
        const double zv = v >= 0 ? Zs[i * PW + v] : a.zf[r0 + i];
        s = fma(Zs[i * PW + u] * rd, zv, s);
      }
      a.ct[(size_t)p * 110 + e] = s;
    } else if (blk == 1) {  // cb
      if (!bot) continue;
      for (int i = lo; i < mm; ++i) {
        const double rd = a.Df[r0 + i];
        const double zu = a.Zb[((size_t)p * PW + (i - lo)) * PW + u];
        const double zv = v >= 0 ? a.Zb[((size_t)p * PW + (i - lo)) * PW + v] : a.zf[r0 + i];
        s = fma(zu * rd, zv, s);
      }
      a.cb[(size_t)p * 110 + e] = s;
    } else {  // co (top row u, bottom column v)
      if (!top || !bot || v < 0) continue;
      for (int i = lo; i < mm; ++i) {
        const double rd = a.Df[r0 + i];
        s = fma(Zs[i * PW + u] * rd, a.Zb[((size_t)p * PW + (i - lo)) * PW + v], s);
      }
      a.co[(size_t)p * 110 + e] = s;
    }
  }
}

// Gauss-Jordan on M [10][21] in shared memory, lane j owning column j:
// M <- [I | M_left^{-1} M_right].  No pivoting: M_left is a Schur complement
// of the symmetric rod Jacobian (positive definite at small steps, where
// M/dt^2 dominates).  Returns false on a zero or non-finite pivot, or one
// below kTinyPivot times the block's starting diagonal entry.
__device__ bool gj10(double (*M)[22], int lane, int ncol) {
  double d0[PW];
#pragma unroll
  for (int k = 0; k < PW; ++k) d0[k] = M[k][k];
  __syncwarp();
  for (int k = 0; k < PW; ++k) {
    const double pk = M[k][k];
    if (!(fabs(pk) > 0.0) || !isfinite(pk) || fabs(pk) < kTinyPivot * fabs(d0[k])) return false;
    const double r = pb_recip(pk);
    double colk[PW];
#pragma unroll
    for (int i = 0; i < PW; ++i) colk[i] = M[i][k];
    __syncwarp();
    if (lane < ncol) {
      const double mk = M[k][lane] * r;
#pragma unroll
      for (int i = 0; i < PW; ++i)
        M[i][lane] = i == k ? mk : fma(-colk[i], mk, M[i][lane]);
    }
    __syncwarp();
  }
  return true;
}

__global__ void __launch_bounds__(32) k_part_separators(PartArgs a) {
  __shared__ double M[PW][22];
  __shared__ double Tp[PW][PW + 1];  // To of the previous separator
  const int sys = blockIdx.x, lane = threadIdx.x;
  const int s0 = a.sys_sep0[sys], ns = a.sys_nsep[sys];
  if (ns == 0 || (a.go && !a.go[sys]) || a.bad[sys]) return;
  const int64_t N = a.ntot;
  // forward elimination: separator s couples to s+1 through interior s+1
  for (int s = 0; s < ns; ++s) {
    const int gs = s0 + s, sa = a.s_a[gs];
    const int pu = gs + sys;      // interior above separator s (its bottom side)
    const int pd = gs + sys + 1;  // interior below (its top side)
    // T_s = A[S,S] - cb[pu] - ct[pd]; g_s = f_S - cb[pu]_g - ct[pd]_g
    for (int t = lane; t < PW * PW + PW; t += 32) {
      if (t < PW * PW) {
        const int i = t / PW, j = t % PW;
        const int hi = i > j ? i : j, lo = i > j ? j : i;
        double v = a.band[(size_t)(hi - lo) * N + sa + hi];
        v -= a.cb[(size_t)pu * 110 + t] + a.ct[(size_t)pd * 110 + t];
        M[i][j] = v;
      } else {
        const int i = t - PW * PW;
        M[i][2 * PW] = a.rhs[sa + i] - a.cb[(size_t)pu * 110 + 100 + i] -
                       a.ct[(size_t)pd * 110 + 100 + i];
      }
    }
    __syncwarp();
    if (s > 0) {  // T'_s = T_s - To^T X_prev, g'_s = g_s - To^T y_prev
      const double *Xp = a.Xs + (size_t)(gs - 1) * 110;
      for (int t = lane; t < PW * PW + PW; t += 32) {
        const int i = t < PW * PW ? t / PW : t - PW * PW;
        const int j = t < PW * PW ? t % PW : -1;
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < PW; ++k)
          v = fma(Tp[k][i], j >= 0 ? Xp[k * PW + j] : Xp[100 + k], v);
        if (j >= 0) M[i][j] -= v;
        else M[i][2 * PW] -= v;
      }
      __syncwarp();
    }
    // To_s = -co[pd] (separator s row, separator s+1 column), if s+1 exists
    for (int t = lane; t < PW * PW; t += 32) {
      const int i = t / PW, j = t % PW;
      const double v = s + 1 < ns ? -a.co[(size_t)pd * 110 + t] : 0.0;
      M[i][PW + j] = v;
      Tp[i][j] = v;
    }
    __syncwarp();
    if (!gj10(M, lane, 2 * PW + 1)) {
      if (lane == 0) atomicExch(a.bad + sys, 1);
      return;
    }
    double *Xo = a.Xs + (size_t)gs * 110;
    for (int t = lane; t < 110; t += 32) {
      const int i = t < 100 ? t / PW : t - 100, j = t < 100 ? PW + t % PW : 2 * PW;
      Xo[t] = M[i][j];
    }
    __syncwarp();
  }
  // back substitution: x_s = y_s - X_s x_{s+1}
  double xn = 0.0;  // lane i < 10: x_{s+1}[i]
  for (int s = ns - 1; s >= 0; --s) {
    const int gs = s0 + s;
    const double *X = a.Xs + (size_t)gs * 110;
    double xv = 0.0;
    if (lane < PW) {
      xv = X[100 + lane];
      if (s + 1 < ns)
        for (int k = 0; k < PW; ++k)
          xv = fma(-X[lane * PW + k], __shfl_sync(0x3ffu, xn, k), xv);
      a.x[a.s_a[gs] + lane] = xv;
    }
    xn = xv;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32) k_part_back(PartArgs a) {
  const int p = blockIdx.x, lane = threadIdx.x;
  if ((a.go && !a.go[a.p_sys[p]]) || a.bad[a.p_sys[p]]) return;
  const int r0 = a.p_a[p], mm = a.p_mm[p];
  const int st = a.p_top[p], sb = a.p_bot[p];
  const int lo = mm - PW;  // interiors have at least 11 rows
  double xt = 0.0, xb = 0.0;  // lane c < 10: separator values
  if (lane < PW) {
    if (st >= 0) xt = a.x[a.s_a[st] + lane];
    if (sb >= 0) xb = a.x[a.s_a[sb] + lane];
  }
  // x_i = (zf_i - (Zt x_top + Zb x_bot)_i) / D_i - sum_{k=1..10} L[i+k][i] x_{i+k},
  // from the bottom row up; lane k < 10 keeps x_{i+1+k} in `mine`
  double mine = 0.0;
  for (int i = mm - 1; i >= 0; --i) {
    double zc = 0.0, lc = 0.0;
    if (lane < PW) {
      if (st >= 0) zc = a.Zt[(size_t)(r0 + i) * PW + lane] * xt;
      if (sb >= 0 && i >= lo) zc = fma(a.Zb[((size_t)p * PW + (i - lo)) * PW + lane], xb, zc);
      const int row = i + 1 + lane;
      if (row < mm) lc = a.Lf[(size_t)(r0 + row) * PW + lane] * mine;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zc += __shfl_xor_sync(0xffffffffu, zc, o);
      lc += __shfl_xor_sync(0xffffffffu, lc, o);
    }
    const double xi = (a.zf[r0 + i] - zc) * a.Df[r0 + i] - lc;
    mine = __shfl_up_sync(0xffffffffu, mine, 1);
    if (lane == 0) {
      mine = xi;
      a.x[r0 + i] = xi;
    }
  }
}

// Newton rounds of long rods (the partitioned path of dm_step): the
// bookkeeping of the rod solver (converged, failed or solving this round),
// the right-hand side -f, and after the solve q += dq.
struct LongArgs {
  int nlong;
  const int32_t *sys;                 // long system -> system index
  const int32_t *sys_dof0, *sys_ndof;  // per system
  double tol;
  int max_iter;
  const double *f;
  double *q, *dq, *rhs;
  int32_t *sys_active, *sys_iters, *sys_status;
  const unsigned long long *sys_res;
  int32_t *ctrl;
  const int32_t *ls_action;
  int32_t *ls_trial;
  int32_t *go;
  int *bad;
};

__global__ void k_long_decide(LongArgs a) {
  __shared__ int go_s;
  const int k = blockIdx.x;
  const int s = a.sys[k];
  if (threadIdx.x == 0) {
    int go = 0;
    a.bad[k] = 0;
    if (a.sys_active[s]) {
      if (a.ls_action && a.ls_action[s] == 1) {  // backtracking: no solve this round
        atomicAdd(&a.ctrl[0], 1);
      } else {
        const double res = __longlong_as_double((long long)a.sys_res[s]);
        int st = a.sys_status[s];
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
    }
    a.go[k] = go;
    go_s = go;
  }
  __syncthreads();
  if (!go_s) return;
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s];
  for (int i = threadIdx.x; i < n; i += blockDim.x) a.rhs[d0 + i] = -a.f[d0 + i];
}

__global__ void k_long_finish(LongArgs a) {
  const int k = blockIdx.x;
  if (!a.go[k]) return;
  const int s = a.sys[k];
  if (a.bad[k]) {
    if (threadIdx.x == 0) {
      a.sys_status[s] = DM_ERR_DEGENERATE;
      a.sys_active[s] = 0;
      atomicAdd(&a.ctrl[1], 1);
      atomicMin(&a.ctrl[2], s);
    }
    return;
  }
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s];
  for (int i = threadIdx.x; i < n; i += blockDim.x) a.q[d0 + i] += a.dq[d0 + i];
  if (threadIdx.x == 0) {
    a.sys_iters[s] += 1;
    if (a.ls_trial) a.ls_trial[s] = 1;
    atomicAdd(&a.ctrl[0], 1);
  }
}

}  // namespace

// Host plan of a partitioned solve: interiors, separators and scratch for
// a fixed set of systems.
struct PartPlan {
  int np = 0, nsep = 0, nsys = 0;
  size_t smem = 0;
  char *scr = nullptr;
  PartArgs A{};
};

static void part_plan_free(PartPlan &P) {
  if (P.scr) cudaFree(P.scr);
  P.scr = nullptr;
}

// layout: interiors [k m, k m + m - 10), separators [k m + m - 10, (k+1) m),
// the last interior [(P-1) m, n) with at least 11 rows
static dm_status part_plan_build(int nsys, const int32_t *sys_dof0, const int32_t *sys_ndof,
                                 int64_t ntot, int m, PartPlan &P, cudaStream_t st) {
  std::vector<int32_t> pa, pmm, ptop, pbot, psys, sa, s0(nsys), nsp(nsys);
  for (int k = 0; k < nsys; ++k) {
    const int n = sys_ndof[k], d0 = sys_dof0[k];
    if (n <= 0 || d0 < 0 || (int64_t)d0 + n > ntot) {
      set_error("partitioned band solve: system outside the vectors");
      return DM_ERR_INVALID_ARG;
    }
    int np = (n - 1) / m + 1;
    while (np > 1 && n - (np - 1) * m < PW + 1) --np;
    s0[k] = (int32_t)sa.size();
    nsp[k] = np - 1;
    for (int p = 0; p < np; ++p) {
      const int a = p * m, b = p + 1 < np ? a + m - PW : n;
      pa.push_back(d0 + a);
      pmm.push_back(b - a);
      psys.push_back(k);
      // the top separator of interior p > 0 is the bottom one of p - 1
      ptop.push_back(p > 0 ? pbot.back() : -1);
      if (p + 1 < np) sa.push_back(d0 + b);
      pbot.push_back(p + 1 < np ? (int32_t)sa.size() - 1 : -1);
    }
  }
  const int np = (int)pa.size(), nsep = (int)sa.size();
  P.np = np;
  P.nsep = nsep;
  P.nsys = nsys;
  size_t bytes = 0;
  auto take = [&](size_t n, size_t elt) {
    const size_t o = bytes;
    bytes += (n * elt + 255) / 256 * 256;
    return o;
  };
  const size_t oL = take((size_t)ntot * PW, 8), oD = take(ntot, 8), oZ = take((size_t)ntot * PW, 8),
               oz = take(ntot, 8), oZb = take((size_t)np * PW * PW, 8), oct = take((size_t)np * 110, 8),
               ocb = take((size_t)np * 110, 8), oco = take((size_t)np * 110, 8),
               oX = take((size_t)std::max(nsep, 1) * 110, 8),
               oI = take(5 * (size_t)np + (size_t)nsep + 3 * (size_t)nsys + 1, 4);
  if (cudaMalloc(&P.scr, bytes) != cudaSuccess) {
    set_error("partitioned band solve: cudaMalloc");
    return DM_ERR_OOM;
  }
  std::vector<int32_t> ints;
  for (auto *v : {&pa, &pmm, &ptop, &pbot, &psys, &sa, &s0, &nsp}) ints.insert(ints.end(), v->begin(), v->end());
  ints.resize(ints.size() + nsys, 0);  // bad flags
  int32_t *ib = reinterpret_cast<int32_t *>(P.scr + oI);
  PartArgs &A = P.A;
  A.ntot = ntot;
  A.nparts = np;
  A.nsep = nsep;
  A.p_a = ib;
  A.p_mm = ib + np;
  A.p_top = ib + 2 * np;
  A.p_bot = ib + 3 * np;
  A.p_sys = ib + 4 * np;
  A.s_a = ib + 5 * np;
  A.sys_sep0 = ib + 5 * np + nsep;
  A.sys_nsep = ib + 5 * np + nsep + nsys;
  A.bad = ib + 5 * np + nsep + 2 * nsys;
  A.Lf = reinterpret_cast<double *>(P.scr + oL);
  A.Df = reinterpret_cast<double *>(P.scr + oD);
  A.Zt = reinterpret_cast<double *>(P.scr + oZ);
  A.zf = reinterpret_cast<double *>(P.scr + oz);
  A.Zb = reinterpret_cast<double *>(P.scr + oZb);
  A.ct = reinterpret_cast<double *>(P.scr + oct);
  A.cb = reinterpret_cast<double *>(P.scr + ocb);
  A.co = reinterpret_cast<double *>(P.scr + oco);
  A.Xs = reinterpret_cast<double *>(P.scr + oX);
  cudaError_t e = cudaMemcpyAsync(ib, ints.data(), ints.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.scr + oct, 0, oX - oct, st);
  int mmax = 0;
  for (int v : pmm) mmax = std::max(mmax, v);
  P.smem = (size_t)mmax * 11 * sizeof(double);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_part_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P.smem);
  if (e != cudaSuccess) {
    part_plan_free(P);
    set_error(std::string("partitioned band solve: ") + cudaGetErrorString(e));
    return DM_ERR_CUDA;
  }
  return DM_OK;
}

static cudaError_t part_launch(const PartPlan &P, const double *band, const double *rhs,
                               double *x, const int32_t *go, cudaStream_t st) {
  PartArgs A = P.A;
  A.band = band;
  A.rhs = rhs;
  A.x = x;
  A.go = go;
  k_part_factor<<<P.np, 32, P.smem, st>>>(A);
  if (P.nsep > 0) k_part_separators<<<P.nsys, 32, 0, st>>>(A);
  k_part_back<<<P.np, 32, 0, st>>>(A);
  return cudaGetLastError();
}

struct LongRods {
  PartPlan plan;
  LongArgs la{};
  std::vector<void *> allocs;
};

dm_status long_rods_create(dm_system *s, const std::vector<int32_t> &sys, int part_rows,
                           LongRods **out) {
  *out = nullptr;
  if (sys.empty()) return DM_OK;
  const HostTopology &T = s->T;
  auto *L = new LongRods();
  const int nl = (int)sys.size();
  std::vector<int32_t> d0(nl), nd(nl);
  for (int k = 0; k < nl; ++k) {
    d0[k] = T.sys_dof0[sys[k]];
    nd[k] = T.sys_ndof[sys[k]];
  }
  dm_status r = part_plan_build(nl, d0.data(), nd.data(), T.n_dofs, part_rows, L->plan, s->stream);
  auto dal = [&](void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    L->allocs.push_back(*p);
    return true;
  };
  int32_t *dsys = nullptr, *dgo = nullptr;
  double *drhs = nullptr;
  if (r == DM_OK && (!dal((void **)&dsys, nl * 4) || !dal((void **)&dgo, nl * 4) ||
                     !dal((void **)&drhs, (size_t)T.n_dofs * 8))) {
    set_error("long rods: cudaMalloc");
    r = DM_ERR_OOM;
  }
  if (r == DM_OK && cudaMemcpy(dsys, sys.data(), nl * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    r = DM_ERR_CUDA;
  if (r != DM_OK) {
    long_rods_free(L);
    return r;
  }
  L->la.nlong = nl;
  L->la.sys = dsys;
  L->la.go = dgo;
  L->la.rhs = drhs;
  L->la.bad = L->plan.A.bad;
  *out = L;
  return DM_OK;
}

void long_rods_free(LongRods *L) {
  if (!L) return;
  part_plan_free(L->plan);
  for (void *p : L->allocs) cudaFree(p);
  delete L;
}

int long_rods_count(const LongRods *L) { return L ? L->la.nlong : 0; }

cudaError_t long_rods_round(LongRods *L, const SolveArgs &v, cudaStream_t st) {
  LongArgs a = L->la;
  a.sys_dof0 = v.sys_dof0;
  a.sys_ndof = v.sys_ndof;
  a.tol = v.tol;
  a.max_iter = v.max_iter;
  a.f = v.f;
  a.q = v.q;
  a.dq = v.dq;
  a.sys_active = v.sys_active;
  a.sys_iters = v.sys_iters;
  a.sys_status = v.sys_status;
  a.sys_res = v.sys_res;
  a.ctrl = v.ctrl;
  a.ls_action = v.ls_action;
  a.ls_trial = v.ls_trial;
  k_long_decide<<<a.nlong, 256, 0, st>>>(a);
  cudaError_t e = part_launch(L->plan, v.band, a.rhs, a.dq, a.go, st);
  if (e != cudaSuccess) return e;
  k_long_finish<<<a.nlong, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dm

namespace dm {
bool check_band_batch(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                      const double *band, const double *rhs, const double *x);
}  // namespace dm

using namespace dm;

extern "C" dm_status dm_solve_band_partitioned(int32_t nsys, const int32_t *sys_dof0,
                                               const int32_t *sys_ndof, int64_t ntot,
                                               const double *band, const double *rhs, double *x,
                                               int32_t part_rows, void *stream) {
  // the same batch rules as dm_solve_band (systems in range, no shared
  // rows, x apart from band and rhs)
  if (!check_band_batch(nsys, sys_dof0, sys_ndof, ntot, band, rhs, x)) return DM_ERR_INVALID_ARG;
  const int m = part_rows > 0 ? part_rows : 512;
  if (m < 2 * PW + 1 || m > 1024) {
    set_error("dm_solve_band_partitioned: part_rows must be in [21, 1024]");
    return DM_ERR_INVALID_ARG;
  }
  if (nsys == 0) return DM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  PartPlan P;
  dm_status r = part_plan_build(nsys, sys_dof0, sys_ndof, ntot, m, P, st);
  if (r != DM_OK) return r;
  cudaError_t e = part_launch(P, band, rhs, x, nullptr, st);
  std::vector<int> bad(nsys, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bad.data(), P.A.bad, nsys * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  part_plan_free(P);
  if (e != cudaSuccess) {
    set_error(std::string("dm_solve_band_partitioned: ") + cudaGetErrorString(e));
    return DM_ERR_CUDA;
  }
  for (int k = 0; k < nsys; ++k)
    if (bad[k]) {
      set_error("dm_solve_band_partitioned: zero or non-finite pivot in system " +
                std::to_string(k));
      return DM_ERR_DEGENERATE;
    }
  return DM_OK;
}
