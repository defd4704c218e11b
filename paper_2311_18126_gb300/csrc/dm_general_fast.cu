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
//   2. k_gen_border (a block per system): Newton bookkeeping for the system
//      and the dense LU of the border system (in order, partial pivoting
//      where a pivot is tiny).
//   3. k_gen_limb_back (one warp per limb): the m condensed rows from the
//      border values, then back substitution towards the free end; q += dq.
//
// Late Newton rounds carry few systems, so a round costs the length of one
// limb's elimination chain; both limb kernels keep that chain short.  Per
// column the factor takes the 10 multipliers in one instruction (a lane
// each, broadcast by shuffles), the 110 updates in four, and the next
// pivot's reciprocal (an FP32 seed and one third-order step, three FP64
// instructions) interleaved with the updates after the one that produces
// it; a pivot outside [2^-126, 2^126) (zero and non-finite included) fails
// the system.  The band, C_m and R_m are staged by asynchronous copies, and
// the condensed block's small LU spreads its work over (row, column)
// pairs.  The back substitution
// is column oriented: lanes 1..10 hold the partial right-hand sides of the
// ten rows above the current one in registers, so a row costs one multiply,
// one update and two shuffles.
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
// condensed block [A_m | C_m | y_m] (leading dimension m + nbc + 1), the
// coupling rows R_m (nbc x m), then the small LU's scratch
constexpr int kSmall = kFastMaxM * (kFastMaxM + kFastMaxBC + 1) + kFastMaxBC * kFastMaxM + 2 * kFastMaxM;
constexpr unsigned kFull = 0xffffffffu;

// Pivots of the border system's elimination in order smaller than this
// fraction of their original diagonal entry send it to partial pivoting.
constexpr double kTinyPivotB = 1e-13;

// 1/d by rcp64 (three FP64 instructions); a division outside its range.
__device__ __forceinline__ double limb_recip(double d) {
  return rcp64_in_range(d) ? rcp64(d) : 1.0 / d;
}

// The border kernel's decision for system s, without its side effects.
__device__ __forceinline__ bool wants_solve(const SolveGenArgs &a, int s) {
  if (!a.sys_active[s]) return false;
  if (a.ls_action && a.ls_action[s] == 1) return false;
  if (a.sys_status[s] != 0) return false;
  const double res = __longlong_as_double((long long)a.sys_res[s]);
  if (isnan(res) || res <= a.tol) return false;
  return a.sys_iters[s] < a.max_iter;
}

// [A | B] <- [U | A^{-1} B] for a dense n x n matrix A with nrhs
// right-hand sides B beside it (row-major, leading dimension ld >= n + nrhs)
// in shared memory, by one warp: Gaussian elimination with partial
// pivoting, reciprocal pivots, the multipliers of a column by one lane per
// row, the trailing update and the back substitution spread over (row,
// column) pairs -- no lane works through a whole row.  lm and dinv: n
// doubles of scratch each.  Returns false (uniformly) on a zero or
// non-finite pivot.
__device__ bool warp_lu_solve(double *M, int n, int ld, int nrhs, double *lm, double *dinv,
                              int lane) {
  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + lane; i < n; i += 32) {
      const double v = fabs(M[i * ld + j]);
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
    if (bi != j)
      for (int c = j + lane; c < n + nrhs; c += 32) {
        const double t = M[j * ld + c];
        M[j * ld + c] = M[bi * ld + c];
        M[bi * ld + c] = t;
      }
    __syncwarp();
    const double rp = limb_recip(M[j * ld + j]);
    if (lane == 0) dinv[j] = rp;
    for (int i = j + 1 + lane; i < n; i += 32) lm[i] = M[i * ld + j] * rp;
    __syncwarp();
    // rows j+1.., columns j+1 .. n+nrhs-1; the row of pair e by a float
    // reciprocal (e < 2^10, so the quotient is exact after rounding down)
    const int wdt = n + nrhs - j - 1, cnt = (n - j - 1) * wdt;
    const float iw = 1.0f / (float)wdt;
    for (int e = lane; e < cnt; e += 32) {
      const int r = (int)(((float)e + 0.5f) * iw);
      const int i = j + 1 + r, c = j + 1 + e - r * wdt;
      M[i * ld + c] = fma(-lm[i], M[j * ld + c], M[i * ld + c]);
    }
    __syncwarp();
  }
  // back substitution, column by column of U: x_i = y_i / u_ii, then
  // y_k -= u_ki x_i for the rows above
  const float ir = 1.0f / (float)nrhs;
  for (int i = n - 1; i >= 0; --i) {
    for (int c = lane; c < nrhs; c += 32) M[i * ld + n + c] *= dinv[i];
    __syncwarp();
    for (int e = lane; e < i * nrhs; e += 32) {
      const int k = (int)(((float)e + 0.5f) * ir), c = e - k * nrhs;
      M[k * ld + n + c] = fma(-M[k * ld + i], M[i * ld + n + c], M[k * ld + n + c]);
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
  const double *band = G + a.lb_band[L];
  double *U = G + a.lb_y[L];  // [ne][12] out: U row, right-hand side, 1/pivot
  // staging of the contiguous band by asynchronous copies (all in flight
  // at once), the right-hand side alongside
  for (int e = lane; e < n * 21; e += 32) {
    const int p = e / 21;
    cp_async8(Bs + p * kRow + (e - p * 21), band + e);
  }
  cp_async_commit();
#pragma unroll 4
  for (int p = lane; p < n; p += 32) Bs[p * kRow + 21] = -a.f[d0 + (dir ? n - 1 - p : p)];
  cp_async_wait_all();
  __syncwarp();
  bool bad = false;
  const int ne = n - m;  // rows eliminated inside the limb
  // update slots of this lane, the same for every column: row j + si
  // (si = 1..10; 0 = no slot) and entry sk (0 = right-hand side, 1..10 =
  // the band entry under column j + sk); the slot (1, 1), which yields the
  // next pivot, is lane 1's first
  int si[4], sk[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = lane + 32 * u;
    si[u] = t < 110 ? t / 11 + 1 : 0;
    sk[u] = t < 110 ? t - (si[u] - 1) * 11 : 0;
  }
  double rp = 1.0;
  if (ne > 0) {
    const double piv = Bs[10];
    if (!rcp64_in_range(piv)) bad = true;
    else rp = rcp64(piv);
  }
  // columns whose ten rows below lie inside the limb: no tests of its end,
  // per-lane offsets from the pivot row, the next pivot's update first
  const int jf = min(ne, n - 10);
  {
    const int mo = lane < 10 ? (lane + 1) * kRow + 9 - lane : kRow + 9;
    int dof[4], sof[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      dof[u] = si[u] > 0 ? si[u] * kRow + (sk[u] ? 10 - si[u] + sk[u] : 21) : 0;
      sof[u] = sk[u] ? 10 + sk[u] : 21;
    }
    const bool s3 = si[3] > 0;
    double *pr = Bs;
    for (int j = 0; j < jf && !bad; ++j, pr += kRow) {
      const double l = pr[mo] * rp;
      if (lane < 10) pr[mo] = l;
      if (lane == 0) pr[10] = rp;  // the pivot is read no more
      const double v0 = fma(-__shfl_sync(kFull, l, si[0] - 1), pr[sof[0]], pr[dof[0]]);
      pr[dof[0]] = v0;
      // the next pivot's reciprocal (seed, e = 1 - d r0, t = e + e^2,
      // r0 + r0 t) interleaved with the other updates, without branches; a
      // pivot outside [2^-126, 2^126) (zero and non-finite included) fails
      const double pn = __shfl_sync(kFull, v0, 1);
      const double r0 = rcp64_seed(pn);
      const double l1 = __shfl_sync(kFull, l, si[1] - 1);
      const double l2 = __shfl_sync(kFull, l, si[2] - 1);
      const double l3 = __shfl_sync(kFull, l, s3 ? si[3] - 1 : 0);
      const double v1 = fma(-l1, pr[sof[1]], pr[dof[1]]);
      const double e = fma(-pn, r0, 1.0);
      const double v2 = fma(-l2, pr[sof[2]], pr[dof[2]]);
      const double t = fma(e, e, e);
      const double v3 = fma(-l3, pr[sof[3]], pr[dof[3]]);
      const double rn = fma(r0, t, r0);
      pr[dof[1]] = v1;
      pr[dof[2]] = v2;
      if (s3) pr[dof[3]] = v3;
      if (j + 1 < ne) {
        if (!rcp64_in_range(pn)) bad = true;
        rp = rn;
      }
      __syncwarp();
    }
  }
  for (int j = max(jf, 0); j < ne && !bad; ++j) {
    const double *pr = Bs + j * kRow;
    // multiplier of row j + 1 + lane, stored in place by the lane that reads it
    double l = 0.0;
    if (lane < 10 && j + lane + 1 < n) {
      double *mp = Bs + (j + lane + 1) * kRow + 9 - lane;
      l = *mp * rp;
      *mp = l;
    }
    if (lane == 0) Bs[j * kRow + 10] = rp;  // the pivot is read no more
    double v0 = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double lu = __shfl_sync(kFull, l, si[u] > 0 ? si[u] - 1 : 0);
      if (si[u] > 0 && j + si[u] < n) {
        double *dst = Bs + (j + si[u]) * kRow + (sk[u] ? 10 - si[u] + sk[u] : 21);
        const double v = fma(-lu, pr[sk[u] ? 10 + sk[u] : 21], *dst);
        *dst = v;
        if (u == 0) v0 = v;
      }
      if (u == 0 && j + 1 < ne) {
        // the next pivot (lane 1's first slot), its reciprocal off the chain
        const double pn = __shfl_sync(kFull, v0, 1);
        if (!rcp64_in_range(pn)) bad = true;
        else rp = rcp64(pn);
      }
    }
    __syncwarp();
  }
  // U rows, eliminated right-hand sides and reciprocal pivots of the
  // eliminated rows, for the back substitution
  if (!bad)
    for (int e = lane; e < ne * 12; e += 32) {
      const int p = e / 12, c = e - p * 12;
      U[e] = Bs[p * kRow + (c < 10 ? 11 + c : (c == 10 ? 21 : 10))];
    }
  if (!bad && m > 0) {
    // condensed block [A_m | C_m | y_m] (leading dimension ld), C_m and the
    // coupling rows R_m by asynchronous copies
    const int ldb = nbc + 1, ld = m + ldb;
    double *M = small;
    double *Rs = small + kFastMaxM * (kFastMaxM + kFastMaxBC + 1);
    double *lm = Rs + kFastMaxBC * kFastMaxM, *dinv = lm + kFastMaxM;
    const double *C = G + a.lb_C[L];
    const double *R = G + a.lb_R[L];
    for (int e = lane; e < m * nbc; e += 32) {
      const int r = e / nbc;
      cp_async8(M + r * ld + m + e - r * nbc, C + e);
    }
    for (int e = lane; e < nbc * m; e += 32) cp_async8(Rs + e, R + e);
    cp_async_commit();
    for (int e = lane; e < m * m; e += 32) {
      const int r = e / m, c = e - r * m;
      M[r * ld + c] = Bs[(ne + r) * kRow + 10 + c - r];
    }
    for (int r = lane; r < m; r += 32) M[r * ld + m + nbc] = Bs[(ne + r) * kRow + 21];
    cp_async_wait_all();
    __syncwarp();
    if (!warp_lu_solve(M, m, ld, ldb, lm, dinv, lane)) {
      bad = true;
    } else {
      // Z = A_m^{-1} [C_m | y_m] for the back substitution
      double *Z = G + a.lb_Y[L];
      for (int e = lane; e < m * ldb; e += 32) {
        const int r = e / ldb;
        Z[e] = M[r * ld + m + e - r * ldb];
      }
      // Schur complement and right-hand side of the border system
      const int32_t *bc = a.lb_bcols + a.lb_bc0[L];
      const int nB = a.gs_nB[w];
      double *S = G + a.gs_JBB[w];
      double *rB = G + a.gs_rB[w];
      for (int e = lane; e < nbc * ldb; e += 32) {
        const int b1 = e / ldb, b2 = e - b1 * ldb;
        double v = 0.0;
        for (int r = 0; r < m; ++r) v = fma(Rs[b1 * m + r], M[r * ld + m + b2], v);
        if (b2 < nbc) atomicAdd(S + (int64_t)bc[b1] * nB + bc[b2], -v);
        else atomicAdd(rB + bc[b1], -v);
      }
    }
  }
  if (bad && lane == 0) atomicOr(a.gen_bad + w, 1);
}

// The border system [S | r] (row-major, leading dimension nB + 1, right-hand
// side in the last column) solved by a block of kGenBorderThreads: Gaussian
// elimination in order, the trailing update spread over all threads (one
// matrix entry per thread and step) and the next pivot's reciprocal taken by
// the thread that updates it, so one barrier per column; a pivot below
// kTinyPivotB of its original diagonal entry restarts the elimination with
// partial pivoting (the pivot search, row swap and multipliers by warp 0).
// Then a column-oriented back substitution by warp 0 with the right-hand
// sides in registers (rows lane, lane + 32, lane + 64).
__global__ void __launch_bounds__(kGenBorderThreads) k_gen_border(SolveGenArgs a) {
  extern __shared__ double sm[];
  __shared__ int flag[4];  // go, bad, -, pivot ok
  const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = blockDim.x;
  if (w >= a.ngen || !a.gs_fast[w]) return;  // block-uniform
  const int s = a.gen_sys[w];
  if (tid == 0) {
    int go = 0, bad = 0;
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
    flag[0] = go;
    flag[1] = bad;
  }
  __syncthreads();
  const int go = flag[0];
  bool bad = flag[1] != 0;
  const int nB = a.gs_nB[w];
  const int ld = nB + 1;
  double *S = sm, *rinv = sm + (size_t)nB * ld, *lm = rinv + nB, *dorig = lm + nB;
  const int32_t *bd = a.border_dof + a.gs_border0[w];
  double *J = a.gen + a.gs_JBB[w];
  double *acc = a.gen + a.gs_rB[w];
  // the border block [S | r] from the assembled block and the limbs' Schur sums
  // (asynchronous copies for the matrix, all in flight at once)
  auto load = [&]() {
    for (int e = tid; e < nB * nB; e += nt) {
      const int r = e / nB;
      cp_async8(S + r * ld + e - r * nB, J + e);
    }
    cp_async_commit();
    for (int b = tid; b < nB; b += nt) S[b * ld + nB] = acc[b] - a.f[bd[b]];
    cp_async_wait_all();
  };
  if (go && !bad && nB > 0) {
    load();
    __syncthreads();
    for (int b = tid; b < nB; b += nt) dorig[b] = fabs(S[b * ld + b]);
    if (tid == 0) flag[3] = 1;
    __syncthreads();
    // first attempt: elimination in order, without pivoting; the thread that
    // updates the next pivot takes its reciprocal (one barrier per column).
    // A pivot below kTinyPivotB of its original diagonal entry, or not
    // finite, abandons it for partial pivoting.
    if (tid == 0) {
      const double v = S[0];
      if (!(fabs(v) > kTinyPivotB * dorig[0]) || !isfinite(v)) flag[3] = 0;
      else rinv[0] = limb_recip(v);
    }
    __syncthreads();
    for (int j = 0; j < nB && flag[3]; ++j) {
      const double rp = rinv[j];
      const int nc = nB - j;
      const float inv = 1.0f / (float)nc;
      for (int e = tid; e < (nB - j - 1) * nc; e += nt) {
        const int r = (int)(((float)e + 0.5f) * inv);
        const int i = j + 1 + r, c = j + 1 + e - r * nc;
        const double v = fma(-(S[i * ld + j] * rp), S[j * ld + c], S[i * ld + c]);
        S[i * ld + c] = v;
        if (r == 0 && c == j + 1) {
          if (!(fabs(v) > kTinyPivotB * dorig[j + 1]) || !isfinite(v)) flag[3] = 0;
          else rinv[j + 1] = limb_recip(v);
        }
      }
      __syncthreads();
    }
    if (!flag[3]) {
      // partial pivoting on a fresh copy
      __syncthreads();
      load();
      __syncthreads();
      for (int j = 0; j < nB; ++j) {
        // warp 0: pivot search, row swap, reciprocal and multipliers
        if (warp == 0) {
          double best = -1.0;
          int bi = j;
          for (int i = j + lane; i < nB; i += 32) {
            const double v = fabs(S[i * ld + j]);
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
          const bool ok = (best > 0.0) && isfinite(best);
          if (ok) {
            if (bi != j)
              for (int c = j + lane; c <= nB; c += 32) {
                const double t = S[j * ld + c];
                S[j * ld + c] = S[bi * ld + c];
                S[bi * ld + c] = t;
              }
            __syncwarp();
            const double rp = limb_recip(S[j * ld + j]);
            if (lane == 0) rinv[j] = rp;
            for (int i = j + 1 + lane; i < nB; i += 32) lm[i] = S[i * ld + j] * rp;
          }
          if (lane == 0) flag[3] = ok;
        }
        __syncthreads();
        if (!flag[3]) {
          bad = true;
          break;  // uniform
        }
        // rows j+1.., columns j+1..nB (the right-hand side included); the row
        // of entry e by a float reciprocal: the quotient is below 96 and at
        // least 0.5/96 from an integer, its float error below 2e-5
        const int nc = nB - j;
        const float inv = 1.0f / (float)nc;
        for (int e = tid; e < (nB - j - 1) * nc; e += nt) {
          const int r = (int)(((float)e + 0.5f) * inv);
          const int i = j + 1 + r, c = j + 1 + e - r * nc;
          S[i * ld + c] = fma(-lm[i], S[j * ld + c], S[i * ld + c]);
        }
        __syncthreads();
      }
    }
    if (!bad && warp == 0) {
      double b0 = lane < nB ? S[lane * ld + nB] : 0.0;
      double b1 = lane + 32 < nB ? S[(lane + 32) * ld + nB] : 0.0;
      double b2 = lane + 64 < nB ? S[(lane + 64) * ld + nB] : 0.0;
      for (int i = nB - 1; i >= 0; --i) {
        const int hi = i >> 5;
        const double src = hi == 0 ? b0 : (hi == 1 ? b1 : b2);
        const double xi = __shfl_sync(kFull, src, i & 31) * rinv[i];
        if (lane == 0) lm[i] = xi;
        if (lane < i) b0 = fma(-S[lane * ld + i], xi, b0);
        if (lane + 32 < i) b1 = fma(-S[(lane + 32) * ld + i], xi, b1);
        if (lane + 64 < i) b2 = fma(-S[(lane + 64) * ld + i], xi, b2);
      }
    }
    __syncthreads();
    if (!bad) {
      double *xB = a.gen + a.gs_xB[w];
      for (int b = tid; b < nB; b += nt) {
        xB[b] = lm[b];
        a.q[bd[b]] += lm[b];
      }
    }
  }
  if (go && nB > 0) {
    // the border block and the limbs' Schur sums, left zero for the next
    // round's assembly and atomics (the limb factors ran: go)
    for (int e = tid; e < nB * nB; e += nt) J[e] = 0.0;
    for (int b = tid; b < nB; b += nt) acc[b] = 0.0;
  }
  if (tid == 0) {
    int g = go;
    if (g && bad) {
      a.sys_status[s] = DM_ERR_DEGENERATE;
      a.sys_active[s] = 0;
      atomicAdd(&a.ctrl[1], 1);
      atomicMin(&a.ctrl[2], s);
      g = 0;
    }
    a.gen_go[w] = g;
    if (g) {
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
  // and reciprocal pivot [n][12], then the m condensed rows' values
  extern __shared__ double dyn[];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = blockIdx.x * (blockDim.x >> 5) + wi;
  if (L >= a.nlimb) return;
  const int w = a.lb_gsys[L];
  if (!a.gs_fast[w] || !a.gen_go[w]) return;
  double *Us = dyn + (size_t)wi * (a.limb_nmax * 12 + 16);
  double *xr = Us + (size_t)a.limb_nmax * 12;  // x of rows ne .. n - 1
  const int n = a.lb_n[L], m = a.lb_m[L], nbc = a.lb_nbc[L], dir = a.lb_dir[L];
  const int d0 = a.lb_dof0[L], ne = n - m;
  const double *G = a.gen;
  const double *Ug = G + a.lb_y[L];
  auto dof = [&](int p) { return d0 + (dir ? n - 1 - p : p); };
  // the U rows by asynchronous copies, in flight while the condensed rows
  // are formed
  for (int e = lane; e < ne * 12; e += 32) cp_async8(Us + e, Ug + e);
  cp_async_commit();
  // the condensed rows ne..n-1 from the border values: the nbc values this
  // limb couples to fetched one per lane (one round trip), then broadcast
  {
    const double *xB = G + a.gs_xB[w];
    const int32_t *bc = a.lb_bcols + a.lb_bc0[L];
    const double xbv = lane < nbc ? xB[bc[lane]] : 0.0;
    const double *Z = G + a.lb_Y[L] + (lane < m ? lane : 0) * (nbc + 1);
    double v = lane < m ? Z[nbc] : 0.0;
#pragma unroll
    for (int b = 0; b < kFastMaxBC; ++b) {
      const double xb = __shfl_sync(kFull, xbv, b);
      if (lane < m && b < nbc) v = fma(-Z[b], xb, v);
    }
    if (lane < m) {
      xr[lane] = v;
      atomicAdd(a.q + dof(ne + lane), v);
    }
  }
  cp_async_wait_all();
  __syncwarp();
  // lane i (0..10) holds the right-hand side of row p - i less the terms of
  // the solved rows; lane 11 brings in row p - 11 untouched
  auto U = [&](int r, int k) { return Us[r * 12 + k - 1]; };  // entry (r, r + k)
  double acc = 0.0;
  {
    const int r = ne - 1 - lane;
    if (lane <= 11 && r >= 0) {
      acc = Us[r * 12 + 10];
      if (lane <= 10)
        for (int c = ne; c < n && c <= r + 10; ++c) acc = fma(-U(r, c - r), xr[c - ne], acc);
    }
  }
  for (int p = ne - 1; p >= 0; --p) {
    const double x = __shfl_sync(kFull, acc * Us[p * 12 + 11], 0);
    if (lane == 0) atomicAdd(a.q + dof(p), x);  // a reduction: no load on the recurrence
    if (lane >= 1 && lane <= 10 && p - lane >= 0) acc = fma(-U(p - lane, lane), x, acc);
    // row p - 1 - i to lane i; lane 11 takes row p - 12
    acc = __shfl_down_sync(kFull, acc, 1);
    if (lane == 11) acc = p - 12 >= 0 ? Us[(p - 12) * 12 + 10] : 0.0;
  }
}

}  // namespace dm
