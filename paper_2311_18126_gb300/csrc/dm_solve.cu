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

// The band pass runs for a system only if the solver will factor its
// Jacobian this round (the test of the Hessian pass of the stencils).
__device__ __forceinline__ bool band_due(const RowArgs &a, int s) {
  if (a.sys_status[s] != 0) return false;
  if (a.ls_action && a.ls_action[s] == 1) return false;
  return !(__longlong_as_double((long long)a.sys_res[s]) <= a.tol);
}

// One DOF row (the work of one thread); returns early when inactive.
// MODE 0: residual and band row; 1: residual only (the residual pass of a
// round); 2: band row of the systems the solver will factor (the Jacobian
// pass).
template <int MODE>
__device__ __forceinline__ void k_rows_rod_one(RowArgs a, const int i) {
  bool act = i < a.nd && a.sys_active[a.dof_sys[i]] &&
             a.sys_kind[a.dof_sys[i]] != SOLVE_GENERAL;
  if (MODE == 2 && act) act = band_due(a, a.dof_sys[i]);
  count_units(a.units, act);
  if (!act) return;
  const int s = a.dof_sys[i];
  const int rod = a.dof_rod[i];
  const int base = a.rod_dof0[rod];
  const int r = i - base;
  const int n = a.rod_ndof[rod];
  const int N = (n + 1) >> 2;
  const int node = r >> 2, c = r & 3;
  const int st0 = a.rod_st0[rod], e0 = a.rod_edge0[rod];
  const int NS = a.ns, NE = a.ne;
  // G = minus the sum of the forces on DOF i (the residual adds it), so
  // that the sums start from their first term, not from an add to zero
  double G = 0.0;
  double brow[11];
  // stencils m (interior nodes 1..N-2) with 4m-4 <= r <= 4m+6
  int mlo = (r - 6 + 3) >= 0 ? (r - 6 + 3) / 4 : 0;
  if (mlo < 1) mlo = 1;
  int mhi = (r + 4) / 4;
  if (mhi > N - 2) mhi = N - 2;
  {
    const bool any = mlo <= mhi;
    const int lr = r - 4 * (mlo - 1);
    const int st = st0 + mlo - 1;
    if (MODE != 2 && any) G = a.sg[lr * NS + st];
#pragma unroll
    for (int d = 0; d < 11; ++d) {
      const int lc = lr - d;
      brow[d] = (MODE != 1 && any && lc >= 0) ? a.sh[upk<11>(lc, lr) * NS + st] : 0.0;
    }
  }
  for (int m = mlo + 1; m <= mhi; ++m) {
    const int lr = r - 4 * (m - 1);
    const int st = st0 + m - 1;
    if (MODE != 2) G += a.sg[lr * NS + st];
    if (MODE != 1) {
#pragma unroll
      for (int d = 0; d < 11; ++d) {
        const int lc = lr - d;
        if (lc >= 0) brow[d] += a.sh[upk<11>(lc, lr) * NS + st];
      }
    }
  }
  const double m_i = a.mass[i];
  const double idt = a.idt;
  if (c < 3) {
    // one copy per component, so that every index of brow is a constant
    // (brow stays in registers)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      if (cc != c) continue;
      if (node <= N - 2) {  // edge `node` starts here
        const int e = e0 + node;
        if (MODE != 2) G -= a.es[cc * NE + e];
        if (MODE != 1) {
#pragma unroll
          for (int cp = 0; cp <= cc; ++cp) brow[cc - cp] += a.es[ksym(cc, cp) * NE + e];
        }
      }
      if (node >= 1) {  // edge `node-1` ends here
        const int e = e0 + node - 1;
        if (MODE != 2) G += a.es[cc * NE + e];
        if (MODE != 1) {
#pragma unroll
          for (int cp = 0; cp <= 2; ++cp) {
            const double kv = a.es[ksym(cc, cp) * NE + e];
            if (cp <= cc) brow[cc - cp] += kv;
            brow[4 + cc - cp] -= kv;
          }
        }
      }
    }
    const double cd = a.damp[i];
    if (MODE != 2) {
      G = fma(-m_i, a.g[c], G);
      G = fma(cd, a.q[i] - a.qn[i], G);
    }
    brow[0] += cd;
  }
  if (MODE != 1) {
    brow[0] += m_i * idt * idt;
    if (a.fixed[i]) {
      brow[0] = 1.0;
#pragma unroll
      for (int d = 1; d < 11; ++d) brow[d] = 0.0;
    } else {
#pragma unroll
      for (int d = 1; d < 11; ++d)
        if (r - d < 0 || a.fixed[i - d]) brow[d] = 0.0;
    }
#pragma unroll
    for (int d = 0; d < 11; ++d) a.band[(size_t)d * a.nd + i] = brow[d];
  }
  if (MODE != 2) {
    if (a.fc) G -= a.fc[i];
    double f = m_i * idt * idt * (a.q[i] - a.qn[i]) - m_i * idt * a.vn[i] + G;
    if (a.fixed[i]) f = 0.0;
    a.f[i] = f;
    // scaled residual, max-reduced per system (order independent)
    const double rr = fabs(f) * a.rscale[i];
    atomicMax(&a.sys_res[s], (unsigned long long)__double_as_longlong(rr));
  }
}

// block-uniform grid-stride loops (count_units synchronises the block)
__global__ void __launch_bounds__(256) k_rows_rod(RowArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.nd; b0 += gridDim.x * blockDim.x)
    k_rows_rod_one<0>(a, b0 + threadIdx.x);
}
__global__ void __launch_bounds__(256) k_rows_rod_res(RowArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.nd; b0 += gridDim.x * blockDim.x)
    k_rows_rod_one<1>(a, b0 + threadIdx.x);
}
__global__ void __launch_bounds__(256) k_rows_rod_band(RowArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.nd; b0 += gridDim.x * blockDim.x)
    k_rows_rod_one<2>(a, b0 + threadIdx.x);
}

// Banded LDL^T solve of J dq = -f for single rods.
//
// The FP64 pipe of an SM partition retires one warp instruction about every
// 64 cycles whatever the active mask, and a column of the band elimination
// is a short dependency chain, so the solve is bound by the chain of
// dependent column steps of the largest rods unless every lane does useful
// FP64 work and every column step is short.  Each rod is therefore factored
// from both ends at once (a twisted factorisation): a top chain eliminates
// columns 0..m-1 downwards, a bottom chain eliminates columns n-1..m+10
// upwards, and the 10-row separator left in the middle is combined from both
// windows and solved densely.  Each chain is run by eight lanes with one
// uniform instruction stream; the 11x11 active window and the right-hand
// side live in shared memory.  Eliminating a column costs 10 multipliers,
// 55 trailing updates and 10 right-hand-side updates (forward substitution
// fused in); the 65 update tasks are split over the eight lanes, rows 9 and
// 10 across two lanes each (q = column in the window, r = right-hand side):
//   lane 0: row 8            lane 1: row 7          lane 2: rows 1, 6
//   lane 3: rows 5, 2        lane 4: rows 4, 3      lane 5: row 10 q1-7
//   lane 6: row 10 q8-10,r; row 9 q1-3              lane 7: row 9 q4-9,r
// -- at most 9 FMAs and 2 multipliers per lane.  Lane 2's first update is
// the next pivot (row 1), broadcast by a shuffle; its reciprocal overlaps
// the other updates.  Lane 0 computes z_j = y_j / D_j in the instruction of
// the second multipliers, which it does not use, and the tiny-pivot test
// runs on the integer pipe, so that a column costs 14 FP64 warp
// instructions (2 multiplier products, 9 update FMAs, 3 for the reciprocal).
// A warp holds two rods (four chains); rods are taken from a queue in order
// of decreasing size, two per warp.
#define SOLVE_WARPS 4
#define SOLVE_RODS_PER_WARP kSolveRodsPerWarp
#define SOLVE_LANES 8  // lanes per chain
static_assert(SOLVE_RODS_PER_WARP * 2 * SOLVE_LANES == 32, "two chains per rod fill a warp");
// Window of a chain in shared memory: matrix rows in order, 12 doubles per
// row (the 11 lower-band diagonals J[r][r-d], d = 0..10, then the
// right-hand side), SOLVE_WROWS rows; the pivot row walks down the buffer
// and the last 11 rows are moved back to the top every 11 columns.
#define SOLVE_WROWS 22
#define SOLVE_CHAIN_STRIDE (SOLVE_WROWS * 12 + 2)  // window + final base + spare
static_assert(SOLVE_CHAIN_STRIDE * 2 + 32 == kSolveRodDoubles, "rod smem layout");


// Task k of lane p: window row i (bits 0-3) and u index q (bits 4-7,
// 0 = right-hand side, 15 = padding); row slot (bits 8-9) among the lane's
// two multipliers.
__host__ __device__ constexpr int task_code(int p, int k) {
  // (row, first q, last q) segments of each lane; q = i + 1 stands for the
  // right-hand side
  const int seg[8][2][3] = {{{8, 1, 9}, {0, 0, -1}},  {{7, 1, 8}, {0, 0, -1}},
                            {{1, 1, 2}, {6, 1, 7}},   {{5, 1, 6}, {2, 1, 3}},
                            {{4, 1, 5}, {3, 1, 4}},   {{10, 1, 7}, {0, 0, -1}},
                            {{10, 8, 11}, {9, 1, 3}}, {{9, 4, 10}, {0, 0, -1}}};
  int t = 0;
  for (int r = 0; r < 2; ++r) {
    const int i = seg[p][r][0];
    for (int q = seg[p][r][1]; q <= seg[p][r][2]; ++q) {
      const int qq = (q == i + 1) ? 0 : q;
      if (t == k) return i | (qq << 4) | (r << 8);
      ++t;
    }
  }
  return 15 << 4;  // padding
}
// window row of the lane's multiplier slot r (0 = none)
__host__ __device__ constexpr int lane_row(int p, int r) {
  return r == 0 ? (p == 0 ? 8 : p == 1 ? 7 : p == 2 ? 1 : p == 3 ? 5 : p == 4 ? 4 : p == 5 ? 10
                                                                       : p == 6 ? 10 : 9)
                : (p == 2 ? 6 : p == 3 ? 2 : p == 4 ? 3 : p == 6 ? 9 : 0);
}
// the lane that stores the multiplier of slot r (rows 9 and 10 live on two lanes)
__host__ __device__ constexpr bool lane_stores(int p, int r) {
  return lane_row(p, r) > 0 && !(p == 6 && r == 0) && !(p == 7 && r == 0);
}
#define SOLVE_TASKS 9
#define SOLVE_PIVOT_LANE 2  // owns row 1, its first task: the next pivot
// Every update task (row i = 1..10, column q = 1..i or the right-hand side)
// appears exactly once over the lanes' task lists; every task's row is its
// lane's multiplier row of the slot it names; the multipliers of rows
// 1..10 are stored by exactly one lane each.
__host__ __device__ constexpr bool solve_tasks_cover() {
  int seen[11][12] = {};
  for (int p = 0; p < SOLVE_LANES; ++p)
    for (int k = 0; k < SOLVE_TASKS; ++k) {
      const int code = task_code(p, k);
      const int i = code & 15, q = (code >> 4) & 15, r = code >> 8;
      if (q == 15) continue;
      if (i < 1 || i > 10 || q > i || lane_row(p, r) != i) return false;
      ++seen[i][q];
    }
  for (int i = 1; i <= 10; ++i)
    for (int q = 0; q <= i; ++q)
      if (seen[i][q] != 1) return false;
  int stored[11] = {};
  for (int p = 0; p < SOLVE_LANES; ++p)
    for (int r = 0; r < 2; ++r)
      if (lane_stores(p, r)) ++stored[lane_row(p, r)];
  for (int i = 1; i <= 10; ++i)
    if (stored[i] != 1) return false;
  return true;
}
static_assert(solve_tasks_cover(), "rod solver task tables");
static_assert(task_code(SOLVE_PIVOT_LANE, 0) == (1 | (1 << 4)), "the pivot lane's first task");

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

// A pivot smaller than 2^-43 (1.1e-13) times the original diagonal entry of
// its row counts as zero: J = M/dt^2 - dF/dq need not be positive definite
// (large steps, compressed or buckling rods), and without pivoting such a
// pivot would amplify rounding errors without bound.  So do pivots outside
// [2^-126, 2^126) (the reciprocal's range; physical Jacobians stay many
// decades inside), infinite or NaN ones.  The test compares the upper 32
// bits of |D| (exponent and 20 leading mantissa bits, whose integer order is
// the order of the magnitudes) with a per-row threshold: the upper word of
// |J_jj| with 43 subtracted from its exponent field, at least that of
// 2^-126.  Exact but for ties in those 32 bits.
constexpr int kTinyPivotExp = 43;
constexpr int kPivotFloorHi = (1023 - 126) << 20;  // upper word of 2^-126
constexpr int kPivotCeilHi = (1023 + 126) << 20;   // upper word of 2^126
__device__ __forceinline__ int pivot_threshold(double jjj) {
  return max((__double2hiint(jjj) & 0x7FFFFFFF) - (kTinyPivotExp << 20), kPivotFloorHi);
}
__device__ __forceinline__ bool pivot_bad(int dhi, int thr) {
  const int h = dhi & 0x7FFFFFFF;
  return h < thr || h >= kPivotCeilHi;
}

// Eliminates `ncol` columns of a chain.  On return the window rows
// W[(b + i) * 12 + .] (b = the final base, also stored at W[SOLVE_WROWS * 12])
// hold rows ncol..ncol+10 of the partially reduced matrix and right-hand side.
//
// The window stores each matrix row by absolute diagonal, so the slide from
// column j to j+1 moves no data: the update of window entry (i, q) (row
// j+i, column j+q) is always at offset 12 i + (i - q) from the pivot row,
// its column entry a_q at 13 q, the multiplier source at 13 i, and the
// right-hand side at 12 i + 11; every lane holds its 9 offsets in
// registers.  Rows beyond the end are zero, so no update needs a bound test.
//
// All four chains of a warp run the same number of iterations (`nwarp`,
// the warp's largest ncol); a chain past its own ncol changes nothing, so
// every synchronisation is warp-wide and the warp never diverges.
//
// Dg (lane 0 of the chain only): an 11-slot ring of the pivot-test
// thresholds of the rows in the window, from the original diagonal entries
// that the loads bringing the rows in deliver; Dg[11..21] is scratch.
//
// The first `nfast` columns (a multiple of 11 that every solving chain of
// the warp eliminates with rows j + 11 in its rod: no tests of the rod's
// end) run an unrolled loop over the window's 11-column period: every
// shared-memory address is a per-lane constant plus an immediate, and the
// lanes without a task (pads, the second row load of lanes 4-7, the ring
// writes of lanes 1-7) store into scratch instead of branching -- the
// window row two below the new one, which the next column's row load
// overwrites, or the word after the last row.  A chain without columns
// (its rod does not solve this round) runs along on rows 0..nfast + 10 of
// the batch's arrays (which exist: a solving rod of the warp has that many
// rows) with its global stores off; its window is not used afterwards.
__device__ __forceinline__ double pick(double a, double b, unsigned m) {  // m ? b : a, m = 0 or ~0
  const unsigned alo = (unsigned)__double2loint(a), ahi = (unsigned)__double2hiint(a);
  const unsigned blo = (unsigned)__double2loint(b), bhi = (unsigned)__double2hiint(b);
  return __hiloint2double((int)((ahi & ~m) | (bhi & m)), (int)((alo & ~m) | (blo & m)));
}

__device__ __forceinline__ bool eliminate(const Chain &c, int ncol, int nwarp, int nfast, double *W,
                                          int p, int pivot_lane, int *Dg) {
  const int n = c.n;
  int toff[SOLVE_TASKS], uoff[SOLVE_TASKS], rsel[SOLVE_TASKS];
#pragma unroll
  for (int k = 0; k < SOLVE_TASKS; ++k) {
    int code = 0;
#pragma unroll
    for (int pp = 0; pp < SOLVE_LANES; ++pp)
      if (p == pp) code = task_code(pp, k);
    const int i = code & 15, q = (code >> 4) & 15;
    rsel[k] = q == 15 ? 2 : (code >> 8);
    toff[k] = q == 15 ? 0 : (q == 0 ? 12 * i + 11 : 12 * i + (i - q));
    uoff[k] = q == 15 ? 0 : (q == 0 ? 11 : 13 * q);
  }
  int row0 = 0, row1 = 0;
  bool st0 = false, st1 = false;
#pragma unroll
  for (int pp = 0; pp < SOLVE_LANES; ++pp)
    if (p == pp) {
      row0 = lane_row(pp, 0);
      row1 = lane_row(pp, 1);
      st0 = lane_stores(pp, 0);
      st1 = lane_stores(pp, 1);
    }
  // the second multiplier's source; lane 0 (one row) takes the pivot row's
  // right-hand side there, which makes its product z_j = y_j / D_j
  const int loff0 = 13 * row0, loff1 = row1 > 0 ? 13 * row1 : 11;
  // rows 0..10 of the chain; diagonals reaching before row 0 are zero
  if (ncol > 0)
    for (int e = p; e < 11 * 12; e += SOLVE_LANES) {
      const int r = e / 12, d = e - 12 * r;
      double v = 0.0;
      if (r < n) v = d == 11 ? c.rhs(r) : (d <= r ? *c.entry(r, d) : 0.0);
      W[e] = v;
    }
  __syncwarp();
  if (ncol > 0 && p == 0)
    for (int r = 0; r < 11; ++r) Dg[r] = pivot_threshold(W[12 * r]);
  double rj = ncol > 0 ? rcp64(W[0]) : 1.0;
  int dhi = __double2hiint(W[0]);  // upper word of the pivot D_j
  bool bad = false;
  int b = 0, jr = 0;  // jr = j mod 11, the ring slot of row j
  const ptrdiff_t step = c.dir;
  if (nfast > 0) {
    __syncwarp();  // the ring, read by every lane below
    double *tg[SOLVE_TASKS];
    const double *sr[SOLVE_TASKS];
    unsigned sm[SOLVE_TASKS];
#pragma unroll
    for (int k = 0; k < SOLVE_TASKS; ++k) {
      tg[k] = W + (rsel[k] == 2 ? 144 : toff[k]);  // pads: scratch row
      sr[k] = W + uoff[k];
      sm[k] = rsel[k] == 1 ? ~0u : 0u;
    }
    const double *ls0 = W + loff0, *ls1 = W + loff1;
    // the new row: diagonal p by every lane, then diagonals 8-10 (lanes
    // 0-2), the right-hand side -f (lane 3, sign flipped on the upper word)
    // or scratch (lanes 4-7)
    double *nw1 = W + (p < 3 ? 140 + p : p == 3 ? 143 : 144);
    const unsigned neg = p == 3 ? 0x80000000u : 0u;
    const bool live = ncol > 0;
    Chain cf = c;
    if (!live) cf.base = 0, cf.dir = 1;
    const ptrdiff_t fstep = cf.dir;
    const double *qe0 = cf.entry(11, p);
    const double *qe1 = p < 3 ? cf.entry(11, p + 8) : p == 3 ? cf.f + cf.base + cf.orig(11) : qe0;
    int *ringw = Dg + (p == 0 ? 0 : 11);
    // lane 0 stores z_j through its second multiplier slot
    double *ql0 = cf.lstore(0, row0);
    double *ql1 = p == 0 ? cf.dq + cf.base + cf.orig(0) : cf.lstore(0, row1);
    const bool w0 = st0 && live, w1 = (st1 || p == 0) && live;
    for (int j0 = 0; j0 < nfast; j0 += 11) {
#pragma unroll
      for (int u = 0; u < 11; ++u) {
        const double pre0 = *qe0;
        const double pre1 = *qe1;
        qe0 += fstep;
        qe1 += fstep;
        if (pivot_bad(dhi, Dg[u])) bad = true;
        ringw[u] = pivot_threshold(pre0);
        const double l0 = ls0[12 * u] * rj;
        const double l1 = ls1[12 * u] * rj;
        double uq[SOLVE_TASKS], dv[SOLVE_TASKS], v[SOLVE_TASKS];
#pragma unroll
        for (int k = 0; k < SOLVE_TASKS; ++k) {
          uq[k] = sr[k][12 * u];
          dv[k] = tg[k][12 * u];
        }
#pragma unroll
        for (int k = 0; k < SOLVE_TASKS; ++k) v[k] = fma(-pick(l0, l1, sm[k]), uq[k], dv[k]);
        const double piv = __shfl_sync(0xffffffffu, v[0], pivot_lane);
        rj = rcp64(piv);
        dhi = __double2hiint(piv);
        if (w0) *ql0 = l0;
        if (w1) *ql1 = l1;
        ql0 += fstep;
        ql1 += fstep;
#pragma unroll
        for (int k = 0; k < SOLVE_TASKS; ++k) tg[k][12 * u] = v[k];
        W[12 * u + 132 + p] = pre0;
        nw1[12 * u] = __hiloint2double(__double2hiint(pre1) ^ (int)neg, __double2loint(pre1));
        __syncwarp();
      }
      // rows 11..21 (the next window) to the top of the buffer
#pragma unroll
      for (int e = 0; e < 132; e += SOLVE_LANES)
        if (e + p < 132) W[e + p] = W[132 + e + p];
      __syncwarp();
    }
  }
  // running addresses (one element per column in the chain's direction) of
  // row j + 11's diagonals p and p + 8 and right-hand side, of z_j, and of
  // the lane's multipliers L[j + row][j]
  const double *pe0 = c.entry(nfast + 11, p), *pe1 = c.entry(nfast + 11, p + 8 < 11 ? p + 8 : p);
  const double *pfz = c.f + c.base + c.orig(nfast + 11);
  double *pz = c.dq + c.base + c.orig(nfast);
  double *pl0 = c.lstore(nfast, row0), *pl1 = c.lstore(nfast, row1);
  for (int j = nfast; j < nwarp; ++j) {
    const bool act = j < ncol;
    // prefetch of row j + 11 (diagonals p and p + 8; the right-hand side)
    const bool more = act && j + 11 < n;
    double pre0 = 0.0, pre1 = 0.0, prz = 0.0;
    if (more) {
      pre0 = *pe0;
      if (p + 8 < 11) pre1 = *pe1;
      if (p == 3) prz = -*pfz;
    }
    pe0 += step;
    pe1 += step;
    pfz += step;
    double *Wb = W + 12 * b;
    if (act && p == 0) {
      if (pivot_bad(dhi, Dg[jr])) bad = true;
      Dg[jr] = pivot_threshold(pre0);  // row j + 11 takes the slot (0 past the end)
      jr = jr == 10 ? 0 : jr + 1;
    }
    const double l0 = Wb[loff0] * rj;
    const double l1 = Wb[loff1] * rj;  // lane 0: z_j for the backward pass
    if (act && p == 0) *pz = l1;
    pz += step;
    double uq[SOLVE_TASKS], dv[SOLVE_TASKS];
#pragma unroll
    for (int k = 0; k < SOLVE_TASKS; ++k) {
      uq[k] = Wb[uoff[k]];
      dv[k] = Wb[toff[k]];
    }
    // the updates; the pivot lane's first one is the next pivot D_{j+1}
    // (row 1; zero, and unused, past a short rod's last column), broadcast
    // for the reciprocal, which overlaps the other updates
    double v[SOLVE_TASKS];
#pragma unroll
    for (int k = 0; k < SOLVE_TASKS; ++k) v[k] = fma(-(rsel[k] == 1 ? l1 : l0), uq[k], dv[k]);
    const double piv = __shfl_sync(0xffffffffu, v[0], pivot_lane);
    // no barrier here: every update target is read only by its own lane
    const double rnext = act ? rcp64(piv) : rj;
    if (act) {
      if (st0 && j + row0 < n) *pl0 = l0;
      if (st1 && j + row1 < n) *pl1 = l1;
#pragma unroll
      for (int k = 0; k < SOLVE_TASKS; ++k)
        if (rsel[k] < 2) Wb[toff[k]] = v[k];
      // the new row j + 11 (zeros past the end)
      double *Wn = Wb + 12 * 11;
      Wn[p] = pre0;
      if (p + 8 < 11) Wn[p + 8] = pre1;
      if (p == 3) Wn[11] = prz;
    }
    const bool wrap = act && b + 1 == SOLVE_WROWS - 11;
    // move rows b+1..b+11 (the next window) to the top of the buffer; the
    // extra barriers only in the columns where some chain of the warp wraps
    if (__any_sync(0xffffffffu, wrap)) {
      double t[17];
      if (wrap) {
#pragma unroll
        for (int u = 0; u < 17; ++u)
          if (p + SOLVE_LANES * u < 132) t[u] = Wb[12 + p + SOLVE_LANES * u];
      }
      __syncwarp();
      if (wrap) {
#pragma unroll
        for (int u = 0; u < 17; ++u)
          if (p + SOLVE_LANES * u < 132) W[p + SOLVE_LANES * u] = t[u];
      }
      __syncwarp();
    } else {
      __syncwarp();
    }
    pl0 += step;
    pl1 += step;
    if (act) {
      b = wrap ? 0 : b + 1;
      rj = rnext;
      dhi = __double2hiint(piv);
    }
  }
  if (p == 0) W[SOLVE_WROWS * 12] = (double)b;
  __syncwarp();
  return bad;
}

__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Back substitution x_i = z_i - sum_d L[i+d][i] x_{i+d} of a chain, rows
// kstart + 9 .. 0 (the separator rows kstart..kstart+9, whose x is known,
// only contribute), in blocks of 11 rows from k0 = kstart + 9 - 11 g down.
// Z = W + 242 holds the running values in a sliding linear buffer: at the
// start of a block, Z[i] is row k0 - i (i = 0..10); the step of row
// k = k0 - u takes x_k = Z[u], subtracts L[k][k-d] x_k from Z[u + d]
// (d = 1..10) and brings z_{k-11} into Z[u + 11]; at the end of the block
// Z[11..21] moves to Z[0..10].  So each row step has one warp barrier.  The
// block's multipliers L(k, d) (d = 1..10) and z_{k-11} (d = 0) for
// k = k0 - u sit in cur[11 u + d], staged one block ahead by asynchronous
// copies into two buffers (W[0..120], W[121..241]).

// Stages block k0 of a chain with the tests of the rod's ends: entries that
// do not exist or are not used are zero.  (The z of row kk - 11 is staged
// for rows kk past the rod's end too: a rod too short to twist has
// kstart = n, and its first block's steps beyond the end bring in its last
// rows.)
__device__ __forceinline__ void stage_block(const Chain &c, bool on, int k0, int kstart,
                                            double *buf, int p) {
  for (int e = p; e < 121; e += SOLVE_LANES) {
    const int u = e / 11, d = e - 11 * u;
    const int kk = k0 - u;
    bool ok = on && kk >= 0;
    const double *src = nullptr;
    if (ok) {
      if (d == 0) {
        ok = kk - 11 >= 0 && kk - 11 < kstart;
        if (ok) src = c.zstore(kk - 11);
      } else {
        ok = kk < c.n && kk - d >= 0 && kk - d < kstart;
        if (ok) src = c.entry(kk, d);
      }
    }
    if (ok) cp_async8(buf + e, src);
    else buf[e] = 0.0;
  }
}

// Stages a block whose rows k0 - 10 .. k0 all lie in [11, kstart): every
// entry exists.  Lane p copies diagonal 1 + p of the 11 rows, lanes 0-1
// diagonals 9-10, lane 2 the z values.
__device__ __forceinline__ void stage_block_full(const Chain &c, int k0, double *buf, int p) {
  const ptrdiff_t dn = -(ptrdiff_t)c.dir;  // address step from row k to row k - 1
  const double *s1 = c.entry(k0, 1 + p);
#pragma unroll
  for (int u = 0; u < 11; ++u) cp_async8(buf + 11 * u + 1 + p, s1 + dn * u);
  if (p < 3) {
    const double *s2 = p < 2 ? c.entry(k0, 9 + p) : c.zstore(k0 - 11);
    double *b2 = buf + (p < 2 ? 9 + p : 0);
#pragma unroll
    for (int u = 0; u < 11; ++u) cp_async8(b2 + 11 * u, s2 + dn * u);
  }
}

// xs = x of the separator rows kstart..kstart+9 (zero for a rod without
// one); `nblk` = the warp's largest block count, blocks [1, gfast) run the
// unrolled step (every row of them in [11, kstart) for every chain of the
// warp that solves; the others run along on their own scratch).
__device__ __forceinline__ void back_substitute(const Chain &c, bool on, int kstart, int nblk,
                                                int gfast, const double *xs, double *W, double *q,
                                                int p) {
  double *Z = W + 242;
  // block 0: the separator's x at Z[0..9] (rows kstart+9..kstart), z of row
  // kstart - 1 at Z[10]
  if (p == 0) {
#pragma unroll
    for (int i = 0; i < 10; ++i) Z[i] = xs[9 - i];
    Z[10] = (on && kstart - 1 >= 0) ? *c.zstore(kstart - 1) : 0.0;
  }
  stage_block(c, on, kstart + 9, kstart, W, p);
  cp_async_commit();
  // lane 0 adds x_k into q (rows below the separator), running address
  double *qk = q + c.base + c.orig(kstart + 9);
  const ptrdiff_t dn = -(ptrdiff_t)c.dir;
  for (int g = 0; g < nblk; ++g) {
    const int k0 = kstart + 9 - 11 * g;
    double *cur = W + 121 * (g & 1);
    double *nxt = W + 121 * ((g + 1) & 1);
    if (g + 1 < nblk) {
      if (g + 1 < gfast) stage_block_full(c, k0 - 11, nxt, p);
      else stage_block(c, on, k0 - 11, kstart, nxt, p);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    if (g >= 1 && g < gfast) {
      // every row of the block is below the separator and at least 11
      double *z1 = Z + 1 + p, *z2 = Z + 9 + (p & 1);
      const double *c1 = cur + 1 + p, *c2 = cur + 9 + (p & 1);
#pragma unroll
      for (int u = 0; u < 11; ++u) {
        const double xk = Z[u];
        if (p == 0 && on) atomicAdd(qk, xk);
        qk += dn;
        z1[u] = fma(-c1[11 * u], xk, z1[u]);
        if (p < 2) z2[u] = fma(-c2[11 * u], xk, z2[u]);
        if (p == 2) Z[u + 11] = cur[11 * u];
        __syncwarp();
      }
    } else {
      for (int u = 0; u < 11; ++u) {
        const int k = k0 - u;
        const bool act = on && k >= 0 && k < c.n;
        const double xk = Z[u];
        if (act && p == 0 && k < kstart) atomicAdd(qk, xk);
        qk += dn;
        if (act) {
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int d = 1 + p + SOLVE_LANES * t;
            if (d <= 10 && k - d >= 0 && k - d < kstart) Z[u + d] = fma(-cur[11 * u + d], xk, Z[u + d]);
          }
        }
        if (on && p == 2 && k - 11 >= 0 && k - 11 < kstart) Z[u + 11] = cur[11 * u];
        __syncwarp();
      }
    }
    // rows k0 - 11 .. k0 - 21 to the top of the buffer
    Z[p] = Z[11 + p];
    if (p < 3) Z[8 + p] = Z[19 + p];
    __syncwarp();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncwarp();
}

__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_solve_rod(SolveArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int unit = lane >> 4;                      // rod slot in the warp
  const int half = (lane >> 3) & 1;                // 0 = top chain, 1 = bottom chain
  const int p = lane & (SOLVE_LANES - 1);
  const int rid = (threadIdx.x >> 5) * SOLVE_RODS_PER_WARP + unit;
  double *Wt = smem + (size_t)rid * (2 * SOLVE_CHAIN_STRIDE + 32);
  double *Wb = Wt + SOLVE_CHAIN_STRIDE;
  double *XS = Wb + SOLVE_CHAIN_STRIDE;  // separator solution (10), diagonal rings (2 x 11)
  double *W = half ? Wb : Wt;
  const unsigned full = 0xffffffffu;
  const int pivot_lane = unit * 16 + half * SOLVE_LANES + SOLVE_PIVOT_LANE;
  const bool head = (lane & 15) == 0;     // bookkeeping lane of the rod
  const unsigned rod_mask = 0xFFFFu << (unit * 16);

  // The warp takes two consecutive rods of the size-sorted queue at a time
  // and factors them in lockstep.
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&a.ctrl[3], SOLVE_RODS_PER_WARP);
    t = __shfl_sync(full, t, 0);
    if (t >= a.nsys) break;
    const int my = t + unit;
    const int s = my < a.nsys ? a.order[my] : -1;
    // Newton bookkeeping of this rod: go = a solve is due this round
    bool go = false;
    if (s >= 0 && a.sys_active[s]) {
      if (a.ls_action && a.ls_action[s] == 1) {  // backtracking: no solve this round
        if (head) atomicAdd(&a.ctrl[0], 1);
      } else {
        const double res = __longlong_as_double((long long)a.sys_res[s]);
        int st = a.sys_status[s];
        if (st == 0 && isnan(res)) st = DM_ERR_NONFINITE;
        if (st == 0 && res <= a.tol) {  // converged at this iterate
          if (head) a.sys_active[s] = 0;
        } else {
          if (st == 0 && a.sys_iters[s] >= a.max_iter) st = DM_ERR_NOT_CONVERGED;
          if (st != 0) {
            if (head) {
              a.sys_status[s] = st;
              a.sys_active[s] = 0;
              atomicAdd(&a.ctrl[1], 1);
              atomicMin(&a.ctrl[2], s);
            }
          } else {
            go = true;
          }
        }
      }
    }
    __syncwarp();
    const int n = go ? a.sys_ndof[s] : 0;
    Chain c{a.band, a.f, a.dq, (size_t)a.nd, go ? (size_t)a.sys_dof0[s] : 0, n, half ? -1 : 1};
    // split: top eliminates [0, m), bottom [m + 10, n), separator [m, m + 10)
    const bool twist = n >= 32;
    const int m = twist ? (n - 10) / 2 : n;
    const int ncol = !go ? 0 : (half ? (twist ? n - m - 10 : 0) : m);
    const int nwarp = __reduce_max_sync(full, ncol);
    // the unrolled columns: whole 11-column blocks that every solving chain
    // of the warp eliminates, none if a solving rod is too short to twist
    const unsigned fmin = __reduce_min_sync(full, go ? (twist ? (unsigned)ncol : 0u) : ~0u);
    const int nfast = nwarp > 0 ? 11 * (int)(fmin / 11) : 0;
    // the rod's scratch past the separator solution: one diagonal ring per chain
    bool bad = eliminate(c, ncol, nwarp, nfast, W, p, pivot_lane,
                         reinterpret_cast<int *>(XS + 10 + 11 * half));
    // a rod is bad if either of its chains met a zero pivot
    bad = (__ballot_sync(full, bad) & rod_mask) != 0;
    if (bad && go) {
      if (head) {
        a.sys_status[s] = DM_ERR_DEGENERATE;
        a.sys_active[s] = 0;
        atomicAdd(&a.ctrl[1], 1);
        atomicMin(&a.ctrl[2], s);
      }
      go = false;
    }
    // separator: S = top window + bottom window - original (10 x 10, lower),
    // right-hand side likewise; dense LDL^T by the rod's top-chain lanes (one
    // row of the trailing update each, rows 8 and 9 by lanes 0 and 1), staged
    // in the top window after it has been read
    const bool sep = go && twist && half == 0;
    const int r8 = p;
    double sv[14];
    if (sep) {
      const int bt = (int)Wt[SOLVE_WROWS * 12], bb = (int)Wb[SOLVE_WROWS * 12];
#pragma unroll
      for (int u = 0; u < 14; ++u) {
        const int e = r8 + 8 * u;  // 0..54 lower entries, 55..64 right-hand side
        double v = 0.0;
        if (e < 55) {
          int i = 0;
          while ((i + 1) * (i + 2) / 2 <= e) ++i;
          const int j2 = e - i * (i + 1) / 2, d = i - j2;
          v = Wt[(bt + i) * 12 + d] + Wb[(bb + 9 - j2) * 12 + d] -
              a.band[d * (size_t)a.nd + c.base + m + i];
        } else if (e < 65) {
          const int i = e - 55;
          v = Wt[(bt + i) * 12 + 11] + Wb[(bb + 9 - i) * 12 + 11] + a.f[c.base + m + i];
        }
        sv[u] = v;
      }
    }
    __syncwarp();
    double *S = Wt;          // S[i * 10 + k], k <= i
    double *rs = Wt + 100;   // right-hand side
    if (sep) {
#pragma unroll
      for (int u = 0; u < 14; ++u) {
        const int e = r8 + 8 * u;
        if (e < 55) {
          int i = 0;
          while ((i + 1) * (i + 2) / 2 <= e) ++i;
          S[i * 10 + (e - i * (i + 1) / 2)] = sv[u];
        } else if (e < 65) {
          rs[e - 55] = sv[u];
        }
      }
    }
    __syncwarp();
    bool sbad = false;
    for (int j2 = 0; j2 < 10; ++j2) {
      double dinv = 1.0, li[2] = {0.0, 0.0};
      int ri[2] = {-1, -1};
      if (sep) {
        dinv = 1.0 / S[j2 * 10 + j2];
        if (!isfinite(dinv)) sbad = true;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int i = j2 + 1 + r8 + 8 * h2;
          if (i < 10) {
            ri[h2] = i;
            li[h2] = S[i * 10 + j2] * dinv;
          }
        }
      }
      __syncwarp();
      if (sep) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int i = ri[h2];
          if (i < 0) continue;
          for (int k = j2 + 1; k <= i; ++k) S[i * 10 + k] = fma(-li[h2], S[k * 10 + j2], S[i * 10 + k]);
          rs[i] = fma(-li[h2], rs[j2], rs[i]);
        }
      }
      __syncwarp();
      if (sep) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
          if (ri[h2] >= 0) S[ri[h2] * 10 + j2] = li[h2];
        if (r8 == 0) S[j2 * 10 + j2] = dinv;
      }
      __syncwarp();
    }
    if (sep && head) {
      for (int i = 9; i >= 0; --i) {
        double x = rs[i] * S[i * 10 + i];
        for (int k = i + 1; k < 10; ++k) x = fma(-S[k * 10 + i], XS[k], x);
        XS[i] = x;
        atomicAdd(a.q + c.base + m + i, x);
      }
    }
    if ((__ballot_sync(full, sbad) & rod_mask) != 0 && go) {
      if (head) {
        a.sys_status[s] = DM_ERR_DEGENERATE;
        a.sys_active[s] = 0;
        atomicAdd(&a.ctrl[1], 1);
        atomicMin(&a.ctrl[2], s);
      }
      go = false;
    }
    __syncwarp();
    // separator x in chain order for each half (the bottom chain sees the
    // separator rows reversed); a short rod is one top chain with no separator
    double xs[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) xs[i] = (go && twist) ? (half ? XS[9 - i] : XS[i]) : 0.0;
    const bool on = go && (twist || !half);
    const int kstart = !on ? 0 : (twist ? (half ? n - m - 10 : m) : n);
    // blocks of 11 rows from kstart + 9 down to row 0; the unrolled ones have
    // all rows in [11, kstart) for every chain that solves; a chain that does
    // not runs along on rows of the batch's arrays (the largest kstart's)
    const int nblk = (int)__reduce_max_sync(full, on ? (unsigned)((kstart + 20) / 11) : 0u);
    const unsigned gf = __reduce_min_sync(
        full, on ? (kstart >= 12 ? (unsigned)((kstart - 12) / 11 + 1) : 1u) : ~0u);
    const int gfast = nblk > 0 ? (int)min(gf, (unsigned)nblk) : 0;
    const int kmax = (int)__reduce_max_sync(full, on ? (unsigned)kstart : 0u);
    Chain cb = c;
    int kb = kstart;
    if (!on) cb.base = 0, cb.dir = 1, cb.n = a.nd, kb = kmax;
    back_substitute(cb, on, kb, nblk, gfast, xs, W, a.q, p);
    if (go && head) {
      a.sys_iters[s] += 1;
      if (a.ls_trial) a.ls_trial[s] = 1;
      atomicAdd(&a.ctrl[0], 1);
      if (a.units) atomicAdd(a.units, (unsigned long long)n);
    }
    __syncwarp();
  }
}

// Line search (optional): Armijo test on the 2-norm of the scaled residual
// |f_i| / (D_i l_i) of each system (the Newton direction is a descent
// direction for it); a trial point without sufficient decrease is pulled
// halfway back to the last accepted iterate, at most 12 times.  One block
// of kLineSearchThreads per system: the merit in a fixed summation order
// (per-thread strided sums, then a fixed tree: deterministic), the decision
// by thread 0, then the move (or the new accepted iterate) over the
// system's DOFs.
__global__ void __launch_bounds__(kLineSearchThreads) k_line_search(LineSearchArgs a) {
  __shared__ double part[kLineSearchThreads / 32];
  __shared__ int s_action;
  __shared__ double s_alpha;
  const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (s >= a.nsys || !a.sys_active[s]) return;  // block-uniform
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s];
  double acc = 0.0;
  for (int i = tid; i < n; i += kLineSearchThreads) {
    const double v = a.f[d0 + i] * a.rscale[d0 + i];
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kLineSearchThreads / 32; ++w) tot += part[w];
    const double m = sqrt(tot);
    a.merit[s] = m;
    int action = 0;
    double alpha = 1.0;
    bool done = false;
    if (a.wstry && a.wstry[s]) {
      // the learned guess is kept only if it lowers the merit below that of
      // the extrapolation; otherwise the iterate returns to the extrapolation
      a.wstry[s] = 0;
      if (!(m <= (1.0 - 1e-4) * a.racc[s])) {
        action = 1;
        alpha = 0.0;
        a.trial[s] = 0;
        a.nback[s] = 0;
        done = true;
      }
    }
    if (!done) {
      if (a.trial[s] && a.nback[s] < 12 && !(m <= (1.0 - 1e-4 * a.alpha[s]) * a.racc[s])) {
        action = 1;
        alpha = 0.5 * a.alpha[s];
        a.nback[s] += 1;
      } else {
        a.trial[s] = 0;
        a.nback[s] = 0;
        a.racc[s] = m;
      }
    }
    a.action[s] = action;
    a.alpha[s] = alpha;
    s_action = action;
    s_alpha = alpha;
  }
  __syncthreads();
  const int action = s_action;
  const double alpha = s_alpha;
  for (int i = d0 + tid; i < d0 + n; i += kLineSearchThreads) {
    if (action == 1) a.q[i] = alpha == 0.0 ? a.qacc[i] : 0.5 * (a.q[i] + a.qacc[i]);
    else a.qacc[i] = a.q[i];
  }
}

}  // namespace dm
