// Condensation solve of the Newton system J dq = -f for general systems
// whose limbs couple to the border only through the rows at one end (rods
// attached at one end: star robots; single rods on the ground).
//
//   1. k_gen_limb_factor (one warp per limb): banded LU without pivoting of
//      the limb block in its elimination order (from the free end), with the
//      right-hand side eliminated alongside.  What remains is the dense m x m
//      block A_m of the rows next to the border; with it the limb's Schur
//      complement R_m A_m^{-1} C_m and right-hand side R_m A_m^{-1} y_m are
//      subtracted from the border system (atomics on the system's matrix).
//   2. k_gen_border (one warp per system): Newton bookkeeping for the system
//      and the dense LU with partial pivoting of the border system.
//   3. k_gen_limb_back (one warp per limb): the m condensed rows from the
//      border values, then back substitution towards the free end; q += dq.
//
// The Jacobian is that of Sec. III-C (M/dt^2 - dF/dq, with the contact and
// friction terms of Sec. III-B), not symmetric when friction acts, hence LU.
// Band storage of a limb (row-major in elimination order p): entry (p, p+k)
// at [p][k + 10], |k| <= 10.
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

namespace {
constexpr int kRow = 22;        // 21 band entries and the right-hand side
constexpr int kSmall = kFastMaxM * (kFastMaxM + kFastMaxBC + 1);  // condensed block
constexpr unsigned kFull = 0xffffffffu;

// The border kernel's decision for system s, without its side effects.
__device__ __forceinline__ bool wants_solve(const SolveGenArgs &a, int s) {
  if (!a.sys_active[s]) return false;
  if (a.ls_action && a.ls_action[s] == 1) return false;
  if (a.sys_status[s] != 0) return false;
  const double res = __longlong_as_double((long long)a.sys_res[s]);
  if (isnan(res) || res <= a.tol) return false;
  return a.sys_iters[s] < a.max_iter;
}

// B <- A^{-1} B for a dense n x n matrix A (row-major, leading dimension
// lda) and n x nrhs right-hand sides B (leading dimension ldb), both in
// shared memory, by one warp: Gaussian elimination with partial pivoting,
// then back substitution.  A is destroyed.  Returns false (uniformly) on a
// zero or non-finite pivot.
__device__ bool warp_lu_solve(double *A, int n, int lda, double *B, int nrhs, int ldb,
                              int lane) {
  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + lane; i < n; i += 32) {
      const double v = fabs(A[i * lda + j]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(best > 0.0) || !isfinite(best)) return false;
    if (bi != j) {
      for (int c = lane; c < n; c += 32) {
        const double t = A[j * lda + c];
        A[j * lda + c] = A[bi * lda + c];
        A[bi * lda + c] = t;
      }
      for (int c = lane; c < nrhs; c += 32) {
        const double t = B[j * ldb + c];
        B[j * ldb + c] = B[bi * ldb + c];
        B[bi * ldb + c] = t;
      }
    }
    __syncwarp();
    const double rp = 1.0 / A[j * lda + j];
    // each lane updates whole rows: row i reads column j and row j, which no
    // update of this step writes
    for (int i = j + 1 + lane; i < n; i += 32) {
      const double l = A[i * lda + j] * rp;
      double *Ai = A + i * lda;
      const double *Aj = A + j * lda;
      for (int c = j + 1; c < n; ++c) Ai[c] = fma(-l, Aj[c], Ai[c]);
      for (int c = 0; c < nrhs; ++c) B[i * ldb + c] = fma(-l, B[j * ldb + c], B[i * ldb + c]);
    }
    __syncwarp();
  }
  if (nrhs == 1) {
    for (int i = n - 1; i >= 0; --i) {
      double part = 0.0;
      for (int k = i + 1 + lane; k < n; k += 32) part = fma(A[i * lda + k], B[k * ldb], part);
#pragma unroll
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
      if (lane == 0) B[i * ldb] = (B[i * ldb] - part) / A[i * lda + i];
      __syncwarp();
    }
  } else {
    for (int c = lane; c < nrhs; c += 32)
      for (int i = n - 1; i >= 0; --i) {
        double v = B[i * ldb + c];
        for (int k = i + 1; k < n; ++k) v = fma(-A[i * lda + k], B[k * ldb + c], v);
        B[i * ldb + c] = v / A[i * lda + i];
      }
    __syncwarp();
  }
  return true;
}

}  // namespace

__global__ void __launch_bounds__(128) k_gen_limb_factor(SolveGenArgs a) {
  // per warp: the limb band with its right-hand side [n][22], then the
  // condensed block and its right-hand sides
  extern __shared__ double dyn[];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = blockIdx.x * (blockDim.x >> 5) + wi;
  if (L >= a.nlimb) return;
  const int w = a.lb_gsys[L];
  if (!a.gs_fast[w]) return;
  const int s = a.gen_sys[w];
  if (!wants_solve(a, s)) return;
  double *Bs = dyn + (size_t)wi * (a.limb_nmax * kRow + kSmall);
  double *small = Bs + (size_t)a.limb_nmax * kRow;
  const int n = a.lb_n[L], m = a.lb_m[L], nbc = a.lb_nbc[L], dir = a.lb_dir[L];
  const int d0 = a.lb_dof0[L];
  double *G = a.gen;
  double *band = G + a.lb_band[L];
  double *rpv = G + a.lb_piv[L];
  double *y = G + a.lb_y[L];
  // coalesced staging of the contiguous band
  for (int e = lane; e < n * 21; e += 32) {
    const int p = e / 21;
    Bs[p * kRow + (e - p * 21)] = band[e];
  }
  for (int p = lane; p < n; p += 32) Bs[p * kRow + 21] = -a.f[d0 + (dir ? n - 1 - p : p)];
  __syncwarp();
  bool bad = false;
  const int ne = n - m;  // rows eliminated inside the limb
  for (int j = 0; j < ne; ++j) {
    const double *pr = Bs + j * kRow;
    const double piv = pr[10];
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
      bad = true;
      break;
    }
    const double rp = 1.0 / piv;
    // updates of rows j+i (i = 1..10): k = 0 the multiplier and the
    // right-hand side, k = 1..10 the band entry under column j + k
    double val[4], mul[4];
    int tgt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      tgt[u] = -1;
      const int t = lane + 32 * u;
      if (t < 110) {
        const int i = t / 11 + 1, k = t - (i - 1) * 11;
        if (j + i < n) {
          const double *ri = Bs + (j + i) * kRow;
          const double l = ri[10 - i] * rp;
          mul[u] = l;
          if (k == 0) {
            val[u] = fma(-l, pr[21], ri[21]);
            tgt[u] = (j + i) * kRow + 21;
          } else {
            val[u] = fma(-l, pr[10 + k], ri[10 - i + k]);
            tgt[u] = (j + i) * kRow + 10 - i + k;
          }
        }
      }
    }
    if (lane == 0) rpv[j] = rp;
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (tgt[u] >= 0) {
        Bs[tgt[u]] = val[u];
        const int t = lane + 32 * u, i = t / 11 + 1;
        if (t - (i - 1) * 11 == 0) Bs[(j + i) * kRow + 10 - i] = mul[u];
      }
    __syncwarp();
  }
  // factors of the eliminated rows (L multipliers, U rows) and their
  // eliminated right-hand side, for the back substitution
  if (!bad) {
    for (int e = lane; e < ne * 21; e += 32) {
      const int p = e / 21;
      band[e] = Bs[p * kRow + (e - p * 21)];
    }
    for (int p = lane; p < ne; p += 32) y[p] = Bs[p * kRow + 21];
  }
  if (!bad && m > 0) {
    // condensed block A_m and right-hand sides [C_m | y_m]
    double *A = small;
    double *B = A + m * m;
    const int ldb = nbc + 1;
    const double *C = G + a.lb_C[L];
    for (int e = lane; e < m * m; e += 32) {
      const int r = e / m, c = e - r * m;
      A[e] = Bs[(ne + r) * kRow + 10 + c - r];
    }
    for (int e = lane; e < m * ldb; e += 32) {
      const int r = e / ldb, c = e - r * ldb;
      B[e] = c < nbc ? C[r * nbc + c] : Bs[(ne + r) * kRow + 21];
    }
    __syncwarp();
    if (!warp_lu_solve(A, m, m, B, ldb, ldb, lane)) {
      bad = true;
    } else {
      double *Z = G + a.lb_Y[L];
      for (int e = lane; e < m * ldb; e += 32) Z[e] = B[e];
      // Schur complement and right-hand side of the border system
      const double *R = G + a.lb_R[L];
      const int32_t *bc = a.lb_bcols + a.lb_bc0[L];
      const int nB = a.gs_nB[w];
      double *S = G + a.gs_JBB[w];
      double *rB = G + a.gs_rB[w];
      for (int e = lane; e < nbc * ldb; e += 32) {
        const int b1 = e / ldb, b2 = e - b1 * ldb;
        double v = 0.0;
        for (int r = 0; r < m; ++r) v = fma(R[b1 * m + r], B[r * ldb + b2], v);
        if (b2 < nbc) atomicAdd(S + (int64_t)bc[b1] * nB + bc[b2], -v);
        else atomicAdd(rB + bc[b1], -v);
      }
    }
  }
  if (bad && lane == 0) atomicOr(a.gen_bad + w, 1);
}

__global__ void k_gen_border(SolveGenArgs a) {
  extern __shared__ double sm[];
  const int w = blockIdx.x, lane = threadIdx.x;
  if (w >= a.ngen || !a.gs_fast[w]) return;
  const int s = a.gen_sys[w];
  int go = 0, bad = 0;
  if (lane == 0) {
    if (a.sys_active[s] && a.ls_action && a.ls_action[s] == 1) {
      atomicAdd(&a.ctrl[0], 1);  // backtracking: no solve this round
    } else if (a.sys_active[s]) {
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
    if (go) {
      bad = a.gen_bad[w];
      a.gen_bad[w] = 0;
    }
  }
  go = __shfl_sync(kFull, go, 0);
  bad = __shfl_sync(kFull, bad, 0);
  const int nB = a.gs_nB[w];
  if (go && !bad && nB > 0) {
    double *S = sm, *x = sm + nB * nB;
    const double *J = a.gen + a.gs_JBB[w];
    const double *acc = a.gen + a.gs_rB[w];
    const int32_t *bd = a.border_dof + a.gs_border0[w];
    for (int e = lane; e < nB * nB; e += 32) S[e] = J[e];
    for (int b = lane; b < nB; b += 32) x[b] = acc[b] - a.f[bd[b]];
    __syncwarp();
    if (!warp_lu_solve(S, nB, nB, x, 1, 1, lane)) {
      bad = 1;
    } else {
      double *xB = a.gen + a.gs_xB[w];
      for (int b = lane; b < nB; b += 32) {
        xB[b] = x[b];
        a.q[bd[b]] += x[b];
      }
    }
  }
  if (lane == 0) {
    if (go && bad) {
      a.sys_status[s] = DM_ERR_DEGENERATE;
      a.sys_active[s] = 0;
      atomicAdd(&a.ctrl[1], 1);
      atomicMin(&a.ctrl[2], s);
      go = 0;
    }
    a.gen_go[w] = go;
    if (go) {
      a.sys_iters[s] += 1;
      if (a.ls_trial) a.ls_trial[s] = 1;
      atomicAdd(&a.ctrl[0], 1);
      if (a.units) {
        int nd = nB;
        for (int l = 0; l < a.gs_nlimb[w]; ++l) nd += a.lb_n[a.gs_limb0[w] + l];
        atomicAdd(a.units, (unsigned long long)nd);
      }
    }
  }
}

__global__ void __launch_bounds__(128) k_gen_limb_back(SolveGenArgs a) {
  // per warp: U rows (10 off-diagonal entries), eliminated right-hand side
  // and reciprocal pivot [n][12], then a ring of 16 solution values
  extern __shared__ double dyn[];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = blockIdx.x * (blockDim.x >> 5) + wi;
  if (L >= a.nlimb) return;
  const int w = a.lb_gsys[L];
  if (!a.gs_fast[w] || !a.gen_go[w]) return;
  double *Us = dyn + (size_t)wi * (a.limb_nmax * 12 + 16);
  double *xr = Us + (size_t)a.limb_nmax * 12;  // x of rows p .. p + 10 at [p & 15]
  const int n = a.lb_n[L], m = a.lb_m[L], nbc = a.lb_nbc[L], dir = a.lb_dir[L];
  const int d0 = a.lb_dof0[L], ne = n - m;
  const double *G = a.gen;
  const double *band = G + a.lb_band[L];
  const double *rpv = G + a.lb_piv[L];
  const double *y = G + a.lb_y[L];
  auto dof = [&](int p) { return d0 + (dir ? n - 1 - p : p); };
  for (int e = lane; e < ne * 21; e += 32) {
    const int p = e / 21, c = e - p * 21;
    if (c > 10) Us[p * 12 + c - 11] = band[e];
  }
  for (int p = lane; p < ne; p += 32) {
    Us[p * 12 + 10] = y[p];
    Us[p * 12 + 11] = rpv[p];
  }
  if (lane < m) {
    const double *Z = G + a.lb_Y[L] + lane * (nbc + 1);
    const double *xB = G + a.gs_xB[w];
    const int32_t *bc = a.lb_bcols + a.lb_bc0[L];
    double v = Z[nbc];
    for (int b = 0; b < nbc; ++b) v = fma(-Z[b], xB[bc[b]], v);
    xr[(ne + lane) & 15] = v;
    atomicAdd(a.q + dof(ne + lane), v);
  }
  __syncwarp();
  for (int p = ne - 1; p >= 0; --p) {
    const double *u = Us + p * 12;
    double t = (lane >= 1 && lane <= 10 && p + lane < n) ? u[lane - 1] * xr[(p + lane) & 15] : 0.0;
#pragma unroll
    for (int o = 8; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (lane == 0) {
      const double x = (u[10] - t) * u[11];
      xr[p & 15] = x;
      atomicAdd(a.q + dof(p), x);  // a reduction: no load on the recurrence
    }
    __syncwarp();
  }
}

}  // namespace dm
