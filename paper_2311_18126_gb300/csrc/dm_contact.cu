// Edge-edge contact within a rod (DisMech, arXiv 2311.18126, Sec. III-B,
// Eq. 10-11) and the linear solve of systems that carry it.
//
//  k_cc_cells / k_cc_fill  -- uniform grid over edge midpoints, hashed into a
//                             table; cell size >= longest edge + C + delta,
//                             so two edges closer than C + delta lie in
//                             neighbouring cells.
//  k_cc_pairs              -- one thread per edge: the edges of the 27
//                             neighbouring cells, minus the excluded pairs
//                             (sharing a node or at most two edges apart
//                             along the rod), whose segment distance D is
//                             below C + delta (C = sum of the radii).
//  k_cc_terms              -- one thread per active pair: D and its first
//                             and second derivatives with respect to the 12
//                             node coordinates (second-order forward-mode
//                             dual numbers through the closest-point
//                             computation), k_c E(D) of Eq. 10 by the chain
//                             rule; -grad into the contact force vector,
//                             the Hessian into the system's dense matrix.
//  k_cc_band               -- adds the rod's own band (11 lower diagonals of
//                             the symmetric Jacobian) to the dense matrix.
//  k_lu_* / k_cc_subst     -- blocked LU without pivoting restricted to the
//                             current bandwidth (the rod band widened by the
//                             contacts) over all SMs, then the solve, q += dq.
#include <cmath>

#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

namespace {

constexpr int kNH = 78;  // packed upper 12x12

__device__ __forceinline__ int hidx(int i, int j) {  // i <= j
  return i * 12 - i * (i - 1) / 2 + (j - i);
}

// Second-order dual number in the 12 coordinates of a pair: value,
// gradient and Hessian (packed upper triangle).
struct HD {
  double v;
  double g[12];
  double h[kNH];
};

__device__ void hd_zero(HD &o, double v) {
  o.v = v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = 0.0;
#pragma unroll
  for (int i = 0; i < kNH; ++i) o.h[i] = 0.0;
}

// o = a * b (o may alias neither)
__device__ void hd_mul(const HD &a, const HD &b, HD &o) {
  o.v = a.v * b.v;
  for (int i = 0; i < 12; ++i) o.g[i] = a.v * b.g[i] + b.v * a.g[i];
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j) {
      const int k = hidx(i, j);
      o.h[k] = a.v * b.h[k] + b.v * a.h[k] + a.g[i] * b.g[j] + a.g[j] * b.g[i];
    }
}

// o = ca * a + cb * b (o may alias a or b)
__device__ void hd_axpby(double ca, const HD &a, double cb, const HD &b, HD &o) {
  o.v = ca * a.v + cb * b.v;
  for (int i = 0; i < 12; ++i) o.g[i] = ca * a.g[i] + cb * b.g[i];
  for (int i = 0; i < kNH; ++i) o.h[i] = ca * a.h[i] + cb * b.h[i];
}

// o = f(a) for a scalar function with f(a.v) = f0, f' = f1, f'' = f2
// (o may alias a)
__device__ void hd_apply(const HD &a, double f0, double f1, double f2, HD &o) {
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j) {
      const int k = hidx(i, j);
      o.h[k] = f1 * a.h[k] + f2 * a.g[i] * a.g[j];
    }
  for (int i = 0; i < 12; ++i) o.g[i] = f1 * a.g[i];
  o.v = f0;
}

// o = a / b
__device__ void hd_div(const HD &a, const HD &b, HD &tmp, HD &o) {
  const double r = 1.0 / b.v;
  hd_apply(b, r, -r * r, 2.0 * r * r * r, tmp);
  hd_mul(a, tmp, o);
}

// First-order dual number in the 12 coordinates of a pair (value and
// gradient), for the friction force whose Jacobian is not a Hessian.
struct D1 {
  double v;
  double g[12];
};
__device__ __forceinline__ D1 d1_of(const HD &a) {
  D1 o;
  o.v = a.v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = a.g[i];
  return o;
}
__device__ __forceinline__ D1 d1_const(double v) {
  D1 o;
  o.v = v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = 0.0;
  return o;
}
__device__ __forceinline__ D1 d1_var(double v, int k) {
  D1 o = d1_const(v);
  o.g[k] = 1.0;
  return o;
}
__device__ __forceinline__ D1 operator+(const D1 &a, const D1 &b) {
  D1 o;
  o.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = a.g[i] + b.g[i];
  return o;
}
__device__ __forceinline__ D1 operator-(const D1 &a, const D1 &b) {
  D1 o;
  o.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = a.g[i] - b.g[i];
  return o;
}
__device__ __forceinline__ D1 operator*(const D1 &a, const D1 &b) {
  D1 o;
  o.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = fma(a.v, b.g[i], b.v * a.g[i]);
  return o;
}
__device__ __forceinline__ D1 operator*(double c, const D1 &a) {
  D1 o;
  o.v = c * a.v;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = c * a.g[i];
  return o;
}
// f(a) with f(a.v) = f0, f'(a.v) = f1
__device__ __forceinline__ D1 d1_apply(const D1 &a, double f0, double f1) {
  D1 o;
  o.v = f0;
#pragma unroll
  for (int i = 0; i < 12; ++i) o.g[i] = f1 * a.g[i];
  return o;
}

// Coordinates of a pair: x[0..2] = p0, x[3..5] = p1, x[6..8] = q0,
// x[9..11] = q1.  The vectors a = p1 - p0, b = q1 - q0, r = p0 - q0 are
// linear in x: component c is +1 at variable P + c and -1 at N + c.
struct Lin {
  double v[3];
  int P, N;
};

// o = u . w for linear vectors
__device__ void hd_lindot(const Lin &u, const Lin &w, HD &o) {
  hd_zero(o, u.v[0] * w.v[0] + u.v[1] * w.v[1] + u.v[2] * w.v[2]);
  for (int c = 0; c < 3; ++c) {
    o.g[u.P + c] += w.v[c];
    o.g[u.N + c] -= w.v[c];
    o.g[w.P + c] += u.v[c];
    o.g[w.N + c] -= u.v[c];
    const int ui[2] = {u.P + c, u.N + c}, wi[2] = {w.P + c, w.N + c};
    const double sg[2] = {1.0, -1.0};
    for (int x = 0; x < 2; ++x)
      for (int y = 0; y < 2; ++y) {
        const int i = ui[x], j = wi[y];
        const double val = sg[x] * sg[y];
        if (i == j) o.h[hidx(i, i)] += 2.0 * val;
        else o.h[hidx(min(i, j), max(i, j))] += val;
      }
  }
}

// o += s * L_c (scalar dual times component c of a linear vector)
__device__ void hd_add_scaled_lin(const HD &s, const Lin &L, int c, double sign, HD &o) {
  const double lv = L.v[c];
  o.v += sign * s.v * lv;
  for (int i = 0; i < 12; ++i) o.g[i] += sign * lv * s.g[i];
  o.g[L.P + c] += sign * s.v;
  o.g[L.N + c] -= sign * s.v;
  for (int k = 0; k < kNH; ++k) o.h[k] += sign * lv * s.h[k];
  // cross terms s.g (x) dL + dL (x) s.g
  const int li[2] = {L.P + c, L.N + c};
  const double ls[2] = {sign, -sign};
  for (int x = 0; x < 2; ++x) {
    const int j = li[x];
    for (int i = 0; i < 12; ++i) {
      const double val = ls[x] * s.g[i];
      if (i == j) o.h[hidx(i, i)] += 2.0 * val;
      else o.h[hidx(min(i, j), max(i, j))] += val;
    }
  }
}

// clamp to [0, 1]: outside the interval the result is a constant
__device__ void hd_clamp01(HD &a) {
  if (a.v < 0.0) hd_zero(a, 0.0);
  else if (a.v > 1.0) hd_zero(a, 1.0);
}

// Segment distance with its derivatives, by the same closest-point rule
// as the definition it follows: s from the unconstrained minimiser clamped
// to [0, 1] (s = 0 for near-parallel segments), t for that s clamped, then s
// again for the clamped t, clamped.
struct DistWork {
  HD A, B, Cc, Dd, Ee, den, s, t, u, w, tmp, d[3];
};

__device__ void segment_distance_hd(const double *x, DistWork &W, HD &D) {
  Lin a, b, r;
  for (int c = 0; c < 3; ++c) {
    a.v[c] = x[3 + c] - x[c];
    b.v[c] = x[9 + c] - x[6 + c];
    r.v[c] = x[c] - x[6 + c];
  }
  a.P = 3; a.N = 0;
  b.P = 9; b.N = 6;
  r.P = 0; r.N = 6;
  hd_lindot(a, a, W.A);
  hd_lindot(a, b, W.B);
  hd_lindot(b, b, W.Cc);
  hd_lindot(a, r, W.Dd);
  hd_lindot(b, r, W.Ee);
  // den = A Cc - B^2
  hd_mul(W.A, W.Cc, W.u);
  hd_mul(W.B, W.B, W.w);
  hd_axpby(1.0, W.u, -1.0, W.w, W.den);
  const bool par = W.den.v < 1e-12 * W.A.v * W.Cc.v;
  if (par) {
    hd_zero(W.s, 0.0);
  } else {
    hd_mul(W.B, W.Ee, W.u);
    hd_mul(W.Cc, W.Dd, W.w);
    hd_axpby(1.0, W.u, -1.0, W.w, W.u);
    hd_div(W.u, W.den, W.tmp, W.s);
    hd_clamp01(W.s);
  }
  // t = clamp((B s + Ee) / Cc)
  hd_mul(W.B, W.s, W.u);
  hd_axpby(1.0, W.u, 1.0, W.Ee, W.u);
  hd_div(W.u, W.Cc, W.tmp, W.t);
  hd_clamp01(W.t);
  // s = clamp((B t - Dd) / A)
  hd_mul(W.B, W.t, W.u);
  hd_axpby(1.0, W.u, -1.0, W.Dd, W.u);
  hd_div(W.u, W.A, W.tmp, W.s);
  hd_clamp01(W.s);
  // d = r + s a - t b; D = |d|
  for (int c = 0; c < 3; ++c) {
    hd_zero(W.d[c], r.v[c]);
    W.d[c].g[r.P + c] = 1.0;
    W.d[c].g[r.N + c] = -1.0;
    hd_add_scaled_lin(W.s, a, c, 1.0, W.d[c]);
    hd_add_scaled_lin(W.t, b, c, -1.0, W.d[c]);
  }
  hd_mul(W.d[0], W.d[0], W.u);
  hd_mul(W.d[1], W.d[1], W.w);
  hd_axpby(1.0, W.u, 1.0, W.w, W.u);
  hd_mul(W.d[2], W.d[2], W.w);
  hd_axpby(1.0, W.u, 1.0, W.w, W.u);
  const double sq = sqrt(W.u.v);
  hd_apply(W.u, sq, 0.5 / sq, -0.25 / (sq * W.u.v), D);
}

// Plain segment distance (same rule), for the candidate filter.
__device__ double segment_distance(const double *x) {
  double a[3], b[3], r[3];
  for (int c = 0; c < 3; ++c) {
    a[c] = x[3 + c] - x[c];
    b[c] = x[9 + c] - x[6 + c];
    r[c] = x[c] - x[6 + c];
  }
  const double A = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const double B = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const double Cc = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const double Dd = a[0] * r[0] + a[1] * r[1] + a[2] * r[2];
  const double Ee = b[0] * r[0] + b[1] * r[1] + b[2] * r[2];
  const double den = A * Cc - B * B;
  double s = den < 1e-12 * A * Cc ? 0.0 : fmin(fmax((B * Ee - Cc * Dd) / den, 0.0), 1.0);
  const double t = fmin(fmax((B * s + Ee) / Cc, 0.0), 1.0);
  s = fmin(fmax((B * t - Dd) / A, 0.0), 1.0);
  double dd = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double d = r[c] + s * a[c] - t * b[c];
    dd += d * d;
  }
  return sqrt(dd);
}

// Eq. 10 with K1 = 15/delta: value and the first two derivatives in D.
__device__ void imc(double D, double C, double delta, double &e0, double &e1, double &e2) {
  if (D <= C - delta) {
    e0 = (C - D) * (C - D);
    e1 = -2.0 * (C - D);
    e2 = 2.0;
  } else if (D < C + delta) {
    const double K1 = 15.0 / delta;
    const double u = K1 * (C - D);
    const double sp = fmax(u, 0.0) + log1p(exp(-fabs(u)));
    const double sg = 1.0 / (1.0 + exp(-u));
    e0 = (sp / K1) * (sp / K1);
    e1 = -2.0 * sp * sg / K1;
    e2 = 2.0 * (sg * sg + sp * sg * (1.0 - sg));
  } else {
    e0 = e1 = e2 = 0.0;
  }
}

__device__ __forceinline__ unsigned long long cell_key(int cx, int cy, int cz) {
  return ((unsigned long long)(cx & 0x1fffff) << 42) | ((unsigned long long)(cy & 0x1fffff) << 21) |
         (unsigned long long)(cz & 0x1fffff);
}

__device__ __forceinline__ unsigned hash_key(unsigned long long k, unsigned mask) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (unsigned)k & mask;
}

__device__ __forceinline__ void edge_cell(const ContactArgs &a, int e, int c[3]) {
  const int ia = a.edge_a[e], ib = a.edge_b[e];
  for (int k = 0; k < 3; ++k) c[k] = (int)floor(0.5 * (a.q[ia + k] + a.q[ib + k]) * a.inv_cell);
}

}  // namespace

__global__ void k_cc_cells(ContactArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  if (!a.sys_active[a.edge_sys[e]] || a.sys_kind[a.edge_sys[e]] != SOLVE_CONTACT) return;
  int c[3];
  edge_cell(a, e, c);
  const unsigned long long k = cell_key(c[0], c[1], c[2]);
  a.edge_key[e] = k;
  atomicAdd(a.bucket_count + hash_key(k, a.table_mask), 1);
}

// exclusive prefix sum of the bucket counts (one block)
__global__ void k_cc_scan(ContactArgs a) {
  __shared__ int part[1024];
  const int T = a.table_mask + 1, tid = threadIdx.x;
  const int per = (T + blockDim.x - 1) / blockDim.x;
  const int b0 = tid * per, b1 = min(T, b0 + per);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += a.bucket_count[b];
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const int v = part[k];
      part[k] = run;
      run += v;
    }
    a.bucket_start[T] = run;
  }
  __syncthreads();
  int run = part[tid];
  for (int b = b0; b < b1; ++b) {
    a.bucket_start[b] = run;
    a.bucket_fill[b] = run;
    run += a.bucket_count[b];
  }
}

__global__ void k_cc_fill(ContactArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  if (!a.sys_active[a.edge_sys[e]] || a.sys_kind[a.edge_sys[e]] != SOLVE_CONTACT) return;
  const unsigned h = hash_key(a.edge_key[e], a.table_mask);
  a.bucket_edges[atomicAdd(a.bucket_fill + h, 1)] = e;
}

__global__ void k_cc_pairs(ContactArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ne) return;
  const int s = a.edge_sys[e];
  if (!a.sys_active[s] || a.sys_kind[s] != SOLVE_CONTACT) return;
  int c[3];
  edge_cell(a, e, c);
  double x[12];
  const int ia = a.edge_a[e], ib = a.edge_b[e];
  for (int k = 0; k < 3; ++k) {
    x[k] = a.q[ia + k];
    x[3 + k] = a.q[ib + k];
  }
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const unsigned long long key = cell_key(c[0] + dx, c[1] + dy, c[2] + dz);
        const unsigned h = hash_key(key, a.table_mask);
        for (int k = a.bucket_start[h]; k < a.bucket_start[h + 1]; ++k) {
          const int f = a.bucket_edges[k];
          if (f <= e || a.edge_key[f] != key || a.edge_sys[f] != s) continue;
          if (abs(a.edge_idx[f] - a.edge_idx[e]) <= 2) continue;  // excluded pairs
          const int ja = a.edge_a[f], jb = a.edge_b[f];
          for (int k2 = 0; k2 < 3; ++k2) {
            x[6 + k2] = a.q[ja + k2];
            x[9 + k2] = a.q[jb + k2];
          }
          const double C = a.edge_h[e] + a.edge_h[f];
          const double D = segment_distance(x);
          if (!(D > 0.0)) {  // Eq. 10 undefined: interpenetration
            atomicCAS(a.sys_status + s, 0, (int)DM_ERR_PENETRATION);
            continue;
          }
          if (D < C + a.delta) {
            const int p = atomicAdd(a.npairs, 1);
            if (p < a.pair_cap) {
              a.pairs[2 * p] = e;
              a.pairs[2 * p + 1] = f;
            } else {
              atomicCAS(a.sys_status + s, 0, (int)DM_ERR_DEGENERATE);
            }
          }
        }
      }
}

__global__ void __launch_bounds__(64) k_cc_terms(ContactArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = min(*a.npairs, a.pair_cap);
  if (p >= np) return;
  const int e = a.pairs[2 * p], f = a.pairs[2 * p + 1];
  const int s = a.edge_sys[e];
  int dof[12];
  const int nodes[4] = {a.edge_a[e], a.edge_b[e], a.edge_a[f], a.edge_b[f]};
  double x[12];
  for (int n = 0; n < 4; ++n)
    for (int k = 0; k < 3; ++k) {
      dof[3 * n + k] = nodes[n] + k;
      x[3 * n + k] = a.q[nodes[n] + k];
    }
  DistWork W;
  HD D;
  segment_distance_hd(x, W, D);
  const double C = a.edge_h[e] + a.edge_h[f];
  double e0, e1, e2;
  imc(D.v, C, a.delta, e0, e1, e2);
  const double kc = a.kc;
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s];
  double *M = a.dense + a.sys_dense0[s];
  int bw = 0;
  for (int i = 0; i < 12; ++i) {
    if (a.fixed[dof[i]]) continue;
    atomicAdd(a.fc + dof[i], -kc * e1 * D.g[i]);  // F = -dE/dq (Eq. 11)
    for (int j = 0; j < 12; ++j) {
      if (a.fixed[dof[j]]) continue;
      const int lo = min(i, j), hi = max(i, j);
      const double hv = kc * (e1 * D.h[hidx(lo, hi)] + e2 * D.g[i] * D.g[j]);
      const int r = dof[i] - d0, c = dof[j] - d0;
      atomicAdd(M + (size_t)r * n + c, hv);
      bw = max(bw, abs(r - c));
    }
  }
  atomicMax(a.sys_bw + s, bw);
  if (a.mu == 0.0) return;
  // Friction at the closest points (Eq. 12-13): u = tangential relative
  // velocity of the closest points with the implicit velocities
  // (x - x_n)/dt; F_a = -mu gamma(|u|) u/|u| |F_con| on edge a, -F_a on
  // edge b, spread by the closest-point weights; |F_con| = k_c |dE/dD|.
  // Derivatives by first-order dual numbers; at |u| = 0 the limit
  // gamma/|u| -> K2/2 of the smooth law.
  const D1 sD = d1_of(W.s), tD = d1_of(W.t), Dd = d1_of(D);
  D1 nrm[3];
  const D1 iD = d1_apply(Dd, 1.0 / Dd.v, -1.0 / (Dd.v * Dd.v));
#pragma unroll
  for (int c = 0; c < 3; ++c) nrm[c] = d1_of(W.d[c]) * iD;
  const double idt = 1.0 / a.dt;
  D1 ur[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const D1 v0 = idt * (d1_var(x[c], c) - d1_const(a.qn[dof[c]]));
    const D1 v1 = idt * (d1_var(x[3 + c], 3 + c) - d1_const(a.qn[dof[3 + c]]));
    const D1 v2 = idt * (d1_var(x[6 + c], 6 + c) - d1_const(a.qn[dof[6 + c]]));
    const D1 v3 = idt * (d1_var(x[9 + c], 9 + c) - d1_const(a.qn[dof[9 + c]]));
    const D1 one = d1_const(1.0);
    ur[c] = ((one - sD) * v0 + sD * v1) - ((one - tD) * v2 + tD * v3);
  }
  const D1 vn = ur[0] * nrm[0] + ur[1] * nrm[1] + ur[2] * nrm[2];
  D1 u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = ur[c] - vn * nrm[c];
  const D1 s2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  // |F_con| = -k_c e1 (e1 <= 0 in contact), derivative -k_c e2 grad D
  const D1 fn = d1_apply(Dd, -kc * e1, -kc * e2);
  D1 coef;
  if (s2.v > 0.0) {
    const double sg = sqrt(s2.v);
    const D1 sig = d1_apply(s2, sg, 0.5 / sg);
    const double ex = exp(-a.K2 * sg);
    const double gam = 2.0 / (1.0 + ex) - 1.0;
    const double dgam = 2.0 * a.K2 * ex / ((1.0 + ex) * (1.0 + ex));
    // gamma(sigma) / sigma
    const D1 gs = d1_apply(sig, gam / sg, (dgam * sg - gam) / (sg * sg));
    coef = (-a.mu) * (fn * gs);
  } else {
    coef = (-0.5 * a.mu * a.K2) * fn;
  }
  D1 Fa[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) Fa[c] = coef * u[c];
  const D1 one = d1_const(1.0);
  const D1 wgt[4] = {one - sD, sD, tD - one, d1_const(0.0) - tD};
#pragma unroll
  for (int nd = 0; nd < 4; ++nd)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int i = 3 * nd + c;
      if (a.fixed[dof[i]]) continue;
      const D1 F = wgt[nd] * Fa[c];
      atomicAdd(a.fc + dof[i], F.v);
      for (int j = 0; j < 12; ++j) {
        if (a.fixed[dof[j]] || F.g[j] == 0.0) continue;
        const int r = dof[i] - d0, cc = dof[j] - d0;
        atomicAdd(M + (size_t)r * n + cc, -F.g[j]);  // J = -dF/dq
      }
    }
}

// Ground contact and friction of the nodes of contact systems (Eq. 10-13,
// the node terms of k_nodes: force F and -dF/dx, nonsymmetric with friction)
// into their contact force and dense matrix, one thread per node; after
// k_cc_terms in stream order (no concurrent writer to these entries).
__global__ void k_cc_ground(ContactArgs a, const int32_t *node_dof, const int32_t *node_sys,
                            const double *nt) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nn) return;
  const int s = node_sys[v];
  // residual phase of the round: the line search has not decided yet (an
  // earlier round's backtracking decision must not drop the force)
  if (!a.sys_active[s] || a.sys_kind[s] != SOLVE_CONTACT) return;
  const int d = node_dof[v], d0 = a.sys_dof0[s], n = a.sys_ndof[s], NN = a.nn;
  double *M = a.dense + a.sys_dense0[s];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (a.fixed[d + r]) continue;
    a.fc[d + r] += nt[r * NN + v];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (!a.fixed[d + c]) M[(size_t)(d + r - d0) * n + (d + c - d0)] += nt[(3 + 3 * r + c) * NN + v];
  }
}

// The rod's band (lower, symmetric) into the dense matrix of each contact
// system, one thread per DOF row.
__global__ void k_cc_band(ContactArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nd) return;
  const int s = a.dof_sys[i];
  if (!a.sys_active[s] || a.sys_kind[s] != SOLVE_CONTACT) return;
  if (a.ls_action && a.ls_action[s] == 1) return;
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s], r = i - d0;
  double *M = a.dense + a.sys_dense0[s];
  for (int d = 0; d <= 10 && d <= r; ++d) {
    const double v = a.band[(size_t)d * a.nd + i];
    M[(size_t)r * n + (r - d)] += v;
    if (d > 0) M[(size_t)(r - d) * n + r] += v;
  }
}

// Clears the band (of the last bandwidth) of each active contact system.
// A warp per matrix row, lanes striding along it (coalesced stores).
__global__ void k_cc_clear(ContactArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t >> 5), lane = (int)(t & 31);
  if (i >= a.nd) return;
  const int s = a.dof_sys[i];
  if (a.sys_kind[s] != SOLVE_CONTACT) return;
  const int d0 = a.sys_dof0[s], n = a.sys_ndof[s], r = i - d0;
  const int bw = max(10, a.sys_bw[s]);
  double *M = a.dense + a.sys_dense0[s] + (size_t)r * n;
  for (int c = max(0, r - bw) + lane; c <= min(n - 1, r + bw); c += 32) M[c] = 0.0;
}

__global__ void k_cc_reset_bw(ContactArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < a.nsys) a.sys_bw[s] = 10;
}

// --- blocked LU of a contact system (no pivoting), spread over the GPU ---
//
// The rod's Jacobian widened by the contact blocks, within its current
// bandwidth bw, is factored in panels of kNB columns: the kNB x kNB
// diagonal block by one block (k_lu_diag), the panel's L (rows below) and
// U (columns right) by triangular solves with one thread per row or column
// (k_lu_trsm), and the trailing update A22 -= L21 U12 by 64 x 64 FP64 tiles
// over all SMs (k_lu_gemm).  Nothing outside |i - j| <= bw is touched: the
// LU of a band matrix without pivoting has no fill outside the band.
// k_cc_decide takes the Newton decision of each contact system first;
// k_cc_subst solves with the factors (blocked forward and backward
// substitution) and updates q.

__global__ void k_cc_decide(ContactArgs a, SolveArgs v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_contact) return;
  const int s = a.contact_sys[c];
  int go = 0;
  if (v.sys_active[s] && v.ls_action && v.ls_action[s] == 1) {
    atomicAdd(&v.ctrl[0], 1);  // backtracking: no solve this round
  } else if (v.sys_active[s]) {
    const double res = __longlong_as_double((long long)v.sys_res[s]);
    int st = v.sys_status[s];
    if (st == 0 && isnan(res)) st = DM_ERR_NONFINITE;
    if (st == 0 && res <= v.tol) {
      v.sys_active[s] = 0;
    } else {
      if (st == 0 && v.sys_iters[s] >= v.max_iter) st = DM_ERR_NOT_CONVERGED;
      if (st != 0) {
        v.sys_status[s] = st;
        v.sys_active[s] = 0;
        atomicAdd(&v.ctrl[1], 1);
        atomicMin(&v.ctrl[2], s);
      } else {
        go = 1;
      }
    }
  }
  a.cgo[c] = go;
  a.cbad[c] = 0;
}

// 1/d from an FP32 seed and two FP64 Newton steps (relative error at the
// FP64 rounding level) where |d| is well inside the FP32 range, else by
// division: the panel kernels take many reciprocals, and an FP64 division
// costs tens of FP64 instructions.
__device__ __forceinline__ double lu_recip(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
  double r = (double)__frcp_rn((float)d);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

__global__ void __launch_bounds__(256) k_lu_diag(ContactArgs a, int c, int k) {
  if (!a.cgo[c] || a.cbad[c]) return;
  const int s = a.contact_sys[c];
  const int n = a.sys_ndof[s];
  const int nb = min(kNB, n - k);
  double *A = a.dense + a.sys_dense0[s];
  __shared__ double D[kNB][kNB + 1];
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    D[i][j] = A[(size_t)(k + i) * n + k + j];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const double piv = D[j][j];
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
      if (threadIdx.x == 0) a.cbad[c] = 1;
      return;  // uniform: every thread read the same pivot
    }
    // only the threads that scale the column take the reciprocal
    if (j + 1 + (int)threadIdx.x < nb) {
      const double rp = lu_recip(piv);
      for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) D[i][j] *= rp;
    }
    __syncthreads();
    const int m = nb - 1 - j;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = j + 1 + t / m, cc = j + 1 + t % m;
      D[i][cc] = fma(-D[i][j], D[j][cc], D[i][cc]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    A[(size_t)(k + i) * n + k + j] = D[i][j];
  }
}

// Rows [k+nb, rend): L21 = A21 U11^{-1}; columns [k+nb, cend): U12 = L11^{-1} A12.
// A thread per row or column, launched in small blocks so that the FP64 work
// spreads over many SMs; the diagonal block and the reciprocals of its
// pivots are staged in shared memory, the thread's row or column in
// registers (loops fully unrolled, zero-padded past nb).
__global__ void __launch_bounds__(128) k_lu_trsm(ContactArgs a, int c, int k) {
  if (!a.cgo[c] || a.cbad[c]) return;
  const int s = a.contact_sys[c];
  const int n = a.sys_ndof[s];
  const int nb = min(kNB, n - k);
  const int bw = max(10, a.sys_bw[s]);
  const int lo = k + nb, hi = min(n, k + nb + bw);
  const int cnt = hi - lo;
  if (cnt <= 0 || blockIdx.x * blockDim.x >= 2 * cnt) return;
  double *A = a.dense + a.sys_dense0[s];
  __shared__ double D[kNB][kNB + 1];
  __shared__ double R[kNB];
  for (int t = threadIdx.x; t < kNB * kNB; t += blockDim.x) {
    const int i = t / kNB, j = t - i * kNB;
    D[i][j] = (i < nb && j < nb) ? A[(size_t)(k + i) * n + k + j] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kNB; j += blockDim.x) R[j] = lu_recip(D[j][j]);
  __syncthreads();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  double x[kNB];
  if (g < cnt) {  // a row of L21: x U11 = a
    double *row = A + (size_t)(lo + g) * n + k;
#pragma unroll
    for (int j = 0; j < kNB; ++j) x[j] = j < nb ? row[j] : 0.0;
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
      double v = x[j];
#pragma unroll
      for (int m = 0; m < j; ++m) v = fma(-x[m], D[m][j], v);
      x[j] = v * R[j];
    }
#pragma unroll
    for (int j = 0; j < kNB; ++j)
      if (j < nb) row[j] = x[j];
  } else if (g < 2 * cnt) {  // a column of U12: L11 x = a (unit lower)
    const int col = lo + (g - cnt);
#pragma unroll
    for (int j = 0; j < kNB; ++j) x[j] = j < nb ? A[(size_t)(k + j) * n + col] : 0.0;
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
      double v = x[j];
#pragma unroll
      for (int m = 0; m < j; ++m) v = fma(-D[j][m], x[m], v);
      x[j] = v;
    }
#pragma unroll
    for (int j = 0; j < kNB; ++j)
      if (j < nb) A[(size_t)(k + j) * n + col] = x[j];
  }
}

// A22 -= L21 U12 over [k+nb, k+nb+bw)^2 in 64 x 64 tiles, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_lu_gemm(ContactArgs a, int c, int k) {
  if (!a.cgo[c] || a.cbad[c]) return;
  const int s = a.contact_sys[c];
  const int n = a.sys_ndof[s];
  const int nb = min(kNB, n - k);
  const int bw = max(10, a.sys_bw[s]);
  const int lo = k + nb, hi = min(n, k + nb + bw);
  const int r0 = lo + blockIdx.y * 64, c0 = lo + blockIdx.x * 64;
  if (r0 >= hi || c0 >= hi) return;
  if (a.lu_flops && threadIdx.x == 0)
    atomicAdd(a.lu_flops, 2ull * (unsigned long long)(min(64, hi - r0) * min(64, hi - c0) * nb));
  double *A = a.dense + a.sys_dense0[s];
  __shared__ double Ls[64][kNB + 1];
  __shared__ double Us[kNB][64 + 1];
  for (int t = threadIdx.x; t < 64 * kNB; t += blockDim.x) {
    const int i = t / kNB, m = t - i * kNB;
    Ls[i][m] = (r0 + i < hi && m < nb) ? A[(size_t)(r0 + i) * n + k + m] : 0.0;
  }
  for (int t = threadIdx.x; t < kNB * 64; t += blockDim.x) {
    const int m = t / 64, j = t - m * 64;
    Us[m][j] = (c0 + j < hi && m < nb) ? A[(size_t)(k + m) * n + c0 + j] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[u][w] = 0.0;
  for (int m = 0; m < nb; ++m) {
    double lv[4], uv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) lv[u] = Ls[ty + 16 * u][m];
#pragma unroll
    for (int w = 0; w < 4; ++w) uv[w] = Us[m][tx + 16 * w];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] = fma(lv[u], uv[w], acc[u][w]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = r0 + ty + 16 * u;
    if (i >= hi) continue;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int j = c0 + tx + 16 * w;
      if (j < hi) A[(size_t)i * n + j] -= acc[u][w];
    }
  }
}

// In-place transpose of a contact system's matrix within its bandwidth
// (for the adjoint's J^T solve): one thread per (row, offset) pair.
__global__ void k_cc_transpose(ContactArgs a, int c) {
  const int s = a.contact_sys[c];
  const int n = a.sys_ndof[s];
  const int bw = max(10, a.sys_bw[s]);
  double *A = a.dense + a.sys_dense0[s];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * bw) return;
  const int i = (int)(t / bw), j = i + 1 + (int)(t - (int64_t)i * bw);
  if (j >= n) return;
  const double x = A[(size_t)i * n + j];
  A[(size_t)i * n + j] = A[(size_t)j * n + i];
  A[(size_t)j * n + i] = x;
}

// Blocked substitution with the factors (L unit lower, U upper), q += x.
__global__ void __launch_bounds__(1024) k_cc_subst(ContactArgs a, SolveArgs v) {
  const int c = blockIdx.x;
  const int s = a.contact_sys[c];
  if (!a.cgo[c]) return;
  if (a.cbad[c]) {
    if (threadIdx.x == 0) {
      v.sys_status[s] = DM_ERR_DEGENERATE;
      v.sys_active[s] = 0;
      atomicAdd(&v.ctrl[1], 1);
      atomicMin(&v.ctrl[2], s);
    }
    return;
  }
  const int d0 = v.sys_dof0[s], n = v.sys_ndof[s];
  const int bw = max(10, a.sys_bw[s]);
  const double *A = a.dense + a.sys_dense0[s];
  double *y = v.dq + d0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = -v.f[d0 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // forward: L y = -f
  for (int k = 0; k < n; k += kNB) {
    const int nb = min(kNB, n - k);
    if (warp == 0) {
      double yv = lane < nb ? y[k + lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        const double yj = __shfl_sync(0xffffffffu, yv, j);
        if (lane > j && lane < nb) yv = fma(-A[(size_t)(k + lane) * n + k + j], yj, yv);
      }
      if (lane < nb) y[k + lane] = yv;
    }
    __syncthreads();
    for (int i = k + nb + threadIdx.x; i < min(n, k + nb + bw); i += blockDim.x) {
      double v2 = y[i];
      for (int m = 0; m < nb; ++m) v2 = fma(-A[(size_t)i * n + k + m], y[k + m], v2);
      y[i] = v2;
    }
    __syncthreads();
  }
  // backward: U x = y
  for (int k = ((n - 1) / kNB) * kNB; k >= 0; k -= kNB) {
    const int nb = min(kNB, n - k);
    if (warp == 0) {
      double xv = lane < nb ? y[k + lane] : 0.0;
      // the panel's pivot reciprocals, one per lane, off the sequential chain
      const double rj = lane < nb ? lu_recip(A[(size_t)(k + lane) * n + k + lane]) : 1.0;
      for (int j = nb - 1; j >= 0; --j) {
        double xj = __shfl_sync(0xffffffffu, xv, j) * __shfl_sync(0xffffffffu, rj, j);
        if (lane == j) xv = xj;
        if (lane < j) xv = fma(-A[(size_t)(k + lane) * n + k + j], xj, xv);
      }
      if (lane < nb) {
        y[k + lane] = xv;
        atomicAdd(v.q + d0 + k + lane, xv);
      }
    }
    __syncthreads();
    for (int i = max(0, k - bw) + threadIdx.x; i < k; i += blockDim.x) {
      double v2 = y[i];
      for (int m = 0; m < nb; ++m) v2 = fma(-A[(size_t)i * n + k + m], y[k + m], v2);
      y[i] = v2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    v.sys_iters[s] += 1;
    if (v.ls_trial) v.ls_trial[s] = 1;
    atomicAdd(&v.ctrl[0], 1);
    if (v.units) atomicAdd(v.units, (unsigned long long)n);
  }
}

}  // namespace dm
