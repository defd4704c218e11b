// Elastic forces and Hessians of the implicit DER step, FP64, sm_103a.
//
//  k_edge     -- one thread per edge: tangent, time-parallel reference frame
//                (Sec. III), material frame, stretching force and Hessian
//                (Sec. III-A, Eq. 2-3).
//  k_stencil  -- one thread per bend-twist stencil: curvature binormal
//                (Eq. 4), material curvatures (Eq. 5), reference twist and
//                twist (Eq. 7), and the gradient and Hessian of
//                1/2 EI/V |kappa - kappabar|^2 + 1/2 GJ/V (tau - taubar)^2
//                (Eq. 6, 8) in closed form: first in the at-point gauge
//                (reference frames carried by parallel transport from the
//                current iterate), then corrected by the holonomy of the
//                time-parallel transport so that they are the exact
//                derivatives of the energy whose frames are carried from the
//                committed step.
//
// The GB300 FP64 pipe is narrow (about 1 TFLOP/s) and charges a full warp
// slot for every FP64 instruction whatever its active mask, so each thread
// owns one whole edge or stencil and all 32 lanes do useful FP64 work.
#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

// One edge (the work of one thread); returns early when inactive.
__device__ __forceinline__ void k_edge_one(EdgeArgs a, const int e) {
  const bool act = e < a.ne && a.sys_active[a.edge_sys[e]];
  count_units(a.units, act);
  if (!act) return;
  const int s = a.edge_sys[e];
  const int ia = a.edge_a[e], ib = a.edge_b[e];
  const double ex = a.q[ib] - a.q[ia];
  const double ey = a.q[ib + 1] - a.q[ia + 1];
  const double ez = a.q[ib + 2] - a.q[ia + 2];
  const double l2 = ex * ex + ey * ey + ez * ez;
  if (!(l2 > 0.0)) {
    atomicMax(&a.sys_status[s], (int)DM_ERR_DEGENERATE);
    return;
  }
  const double il = rsqrt(l2);
  const double l = l2 * il;
  const double tx = ex * il, ty = ey * il, tz = ez * il;
  const int NE = a.ne;
  const double nx = a.tn[e], ny = a.tn[NE + e], nz = a.tn[2 * NE + e];
  const double c = 1.0 + nx * tx + ny * ty + nz * tz;
  if (!(c > 1e-12)) {  // edge reversed within one step: transport undefined
    atomicMax(&a.sys_status[s], (int)DM_ERR_DEGENERATE);
    return;
  }
  // time-parallel transport of d1 from t_n to t (d1 normal to t_n)
  const double px = a.d1n[e], py = a.d1n[NE + e], pz = a.d1n[2 * NE + e];
  const double k = (px * tx + py * ty + pz * tz) * rcp64(c);  // c in (1e-12, 2]
  const double d1x = px - k * (nx + tx), d1y = py - k * (ny + ty), d1z = pz - k * (nz + tz);
  const double d2x = ty * d1z - tz * d1y, d2y = tz * d1x - tx * d1z, d2z = tx * d1y - ty * d1x;
  double sn, cs;
  sincos(a.q[a.edge_th[e]], &sn, &cs);
  double *o = a.ef;
  o[0 * NE + e] = tx;
  o[1 * NE + e] = ty;
  o[2 * NE + e] = tz;
  o[3 * NE + e] = il;
  o[4 * NE + e] = d1x;
  o[5 * NE + e] = d1y;
  o[6 * NE + e] = d1z;
  o[7 * NE + e] = cs * d1x + sn * d2x;   // m1
  o[8 * NE + e] = cs * d1y + sn * d2y;
  o[9 * NE + e] = cs * d1z + sn * d2z;
  o[10 * NE + e] = -sn * d1x + cs * d2x; // m2
  o[11 * NE + e] = -sn * d1y + cs * d2y;
  o[12 * NE + e] = -sn * d1z + cs * d2z;
  // stretching: dE/dx_b = EA (l/lbar - 1) t,
  // Hessian block K = EA/l t t^T + EA (1/lbar - 1/l) I
  const double EA = a.edge_EA[e], ilb = a.edge_ilbar[e];
  const double fm = EA * (l * ilb - 1.0);
  const double al = EA * (ilb - il), be = EA * il;
  double *w = a.es;
  w[0 * NE + e] = fm * tx;
  w[1 * NE + e] = fm * ty;
  w[2 * NE + e] = fm * tz;
  w[3 * NE + e] = fma(be * tx, tx, al);
  w[4 * NE + e] = be * tx * ty;
  w[5 * NE + e] = be * tx * tz;
  w[6 * NE + e] = fma(be * ty, ty, al);
  w[7 * NE + e] = be * ty * tz;
  w[8 * NE + e] = fma(be * tz, tz, al);
}

__global__ void k_edge(EdgeArgs a) {
  // block-uniform grid-stride loop (count_units synchronises the block)
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.ne; b0 += gridDim.x * blockDim.x)
    k_edge_one(a, b0 + threadIdx.x);
}

// ---------------------------------------------------------------------------
// small vector helpers (FP64)
// ---------------------------------------------------------------------------
struct v3 {
  double x, y, z;
};
__device__ __forceinline__ v3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ v3 operator+(v3 a, v3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ v3 operator-(v3 a, v3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ v3 operator*(double s, v3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(v3 a, v3 b) { return fma(a.x, b.x, fma(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ v3 cross(v3 a, v3 b) {
  return {fma(a.y, b.z, -a.z * b.y), fma(a.z, b.x, -a.x * b.z), fma(a.x, b.y, -a.y * b.x)};
}
__device__ __forceinline__ v3 axpy(double s, v3 x, v3 y) {  // s x + y
  return {fma(s, x.x, y.x), fma(s, x.y, y.y), fma(s, x.z, y.z)};
}
// component access by compile-time index
__device__ __forceinline__ double cmp(const v3 &a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
// P_perp(t) v = v - (t.v) t
__device__ __forceinline__ v3 perp(v3 t, v3 v) { return axpy(-dot(t, v), t, v); }

// packed upper-triangle index of an n x n symmetric matrix (i <= j)
template <int n>
__host__ __device__ constexpr int up(int i, int j) {
  return i * n - i * (i - 1) / 2 + (j - i);
}

// H8[blk] += s * (x y^T + y x^T) on a 3x3 diagonal block starting at o
__device__ __forceinline__ void add_sym(double *h, int o, double s, v3 x, v3 y) {
  const v3 sx = s * x;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      h[up<8>(o + i, o + j)] = fma(cmp(sx, i), cmp(y, j), fma(cmp(y, i), cmp(sx, j), h[up<8>(o + i, o + j)]));
}

// s x for s = +-1 given as a sign word (0 or 0x80000000): the sign bit
// flipped on the integer pipe, the same value as the FP64 product
__device__ __forceinline__ double sgnmul(unsigned sw, double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)sw, __double2loint(x));
}
__device__ __forceinline__ unsigned sign_word(int s) { return s < 0 ? 0x80000000u : 0u; }
__device__ __forceinline__ v3 sgn3(int s, v3 v) {
  const unsigned sw = sign_word(s);
  return mk(sgnmul(sw, v.x), sgnmul(sw, v.y), sgnmul(sw, v.z));
}

__device__ __forceinline__ void load_edge(const double *ef, int NE, int e, int sgn,
                                          v3 &t, double &il, v3 &d1, v3 &m1, v3 &m2) {
  const unsigned sw = sign_word(sgn);
  t = mk(sgnmul(sw, ef[e]), sgnmul(sw, ef[NE + e]), sgnmul(sw, ef[2 * NE + e]));
  il = ef[3 * NE + e];
  d1 = mk(ef[4 * NE + e], ef[5 * NE + e], ef[6 * NE + e]);
  m1 = mk(ef[7 * NE + e], ef[8 * NE + e], ef[9 * NE + e]);
  m2 = mk(sgnmul(sw, ef[10 * NE + e]), sgnmul(sw, ef[11 * NE + e]), sgnmul(sw, ef[12 * NE + e]));
}

// Slot p of the 11 DOFs [x0 (0-2), th_a (3), x1 (4-6), th_b (7), x2 (8-10)]
// as a combination of the 8-space (e_a 0-2, e_b 3-5, A 6, B 7): x0 = -e_a,
// x1 = e_a - e_b, x2 = e_b, th_a = sa A, th_b = sb B.  Term t (0, 1) of
// slot p: its 8-space index (-1: none) and weight (1: +1, -1: -1, 2: sa,
// 3: sb).
__host__ __device__ constexpr int slot_index(int p, int t) {
  return p == 3 ? (t == 0 ? 6 : -1)
       : p == 7 ? (t == 0 ? 7 : -1)
       : p < 3  ? (t == 0 ? p : -1)
       : p < 7  ? (t == 0 ? p - 4 : p - 1)
                : (t == 0 ? p - 5 : -1);
}
__host__ __device__ constexpr int slot_weight(int p, int t) {
  return p == 3 ? 2 : p == 7 ? 3 : p < 3 ? -1 : p < 7 ? (t == 0 ? 1 : -1) : 1;
}

// Gradient of one stencil in its 11 DOFs: (e_a, e_b, A, B) -> [x0, th_a,
// x1, th_b, x2] with x0 = -e_a, x1 = e_a - e_b, x2 = e_b, A = sa th_a,
// B = sb th_b.
__device__ __forceinline__ void write_gradient(const StencilArgs &a, int k, const double *g8,
                                               int sa, int sb) {
  double *G = a.sg;
  const int NS = a.ns;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    G[(0 + c) * NS + k] = -g8[c];
    G[(4 + c) * NS + k] = g8[c] - g8[3 + c];
    G[(8 + c) * NS + k] = g8[3 + c];
  }
  G[3 * NS + k] = sgnmul(sign_word(sa), g8[6]);
  G[7 * NS + k] = sgnmul(sign_word(sb), g8[7]);
}

// The Hessian pass runs for a system only if the solver will factor its
// Jacobian this round: it is still iterating, its residual is above the
// tolerance (the solver's own convergence test on the same value), it has
// not failed, and the line search is not backtracking it.
__device__ __forceinline__ bool hess_due(const StencilArgs &a, int s) {
  if (a.sys_status[s] != 0) return false;
  if (a.ls_action && a.ls_action[s] == 1) return false;
  return !(__longlong_as_double((long long)a.sys_res[s]) <= a.tol);
}

// One bend-twist stencil (the work of one thread); returns early when
// inactive.  MODE 0: gradient and Hessian; 1: reference twist and gradient
// (the residual pass of a round); 2: Hessian of the systems the solver will
// factor, with the reference twist the gradient pass wrote (the Jacobian
// pass of a round).
template <int MODE>
__device__ __forceinline__ void k_stencil_one(StencilArgs a, const int k) {
  bool act = k < a.ns && a.sys_active[a.st_sys[k]];
  if (MODE == 2 && act) act = hess_due(a, a.st_sys[k]);
  count_units(a.units, act);
  if (!act) return;
  const int sys = a.st_sys[k];
  const int NS = a.ns, NE = a.ne;
  const int sg = a.st_sg[k];
  const int sa = (sg & 1) ? -1 : 1, sb = (sg & 2) ? -1 : 1;
  v3 ta, d1a, m1a, m2a, tb, d1b, m1b, m2b;
  double ila, ilb;
  load_edge(a.ef, NE, a.st_ed[k], sa, ta, ila, d1a, m1a, m2a);
  load_edge(a.ef, NE, a.st_ed[NS + k], sb, tb, ilb, d1b, m1b, m2b);

  // Eq. 4: curvature binormal
  const double chi = 1.0 + dot(ta, tb);
  if (!(chi > 1e-12)) {
    if (MODE != 2) atomicMax(&a.sys_status[sys], (int)DM_ERR_DEGENERATE);
    return;
  }
  const double ichi = rcp64(chi);  // chi in (1e-12, 2]
  const v3 kb = (2.0 * ichi) * cross(ta, tb);
  const v3 M1 = m1a + m1b, M2 = m2a + m2b;
  // Eq. 5: material curvatures
  const double k1 = 0.5 * dot(kb, M2);
  const double k2 = -0.5 * dot(kb, M1);
  // Eq. 7: reference twist, continued from the committed value
  const v3 s_ab = ta + tb;
  double beta;
  if (MODE == 2) {
    beta = a.beta_it[k];
  } else {
    const v3 u = axpy(-dot(d1a, tb) * ichi, s_ab, d1a);
    const double ang = atan2(dot(tb, cross(u, d1b)), dot(u, d1b));
    const double bn = a.beta_n[k];
    double dd = ang - bn;
    dd -= 6.283185307179586 * rint(dd * 0.15915494309189535);
    beta = bn + dd;
    a.beta_it[k] = beta;
    if (a.frames_only) return;
  }
  const double tha = a.q[a.st_th[k]], thb = a.q[a.st_th[NS + k]];
  const double tau = sgnmul(sign_word(sb), thb) - sgnmul(sign_word(sa), tha) + beta;
  const double kbs = a.st_kb[k], kts = a.st_kt[k];
  const double c1 = kbs * (k1 - a.kbar[k]);
  const double c2 = kbs * (k2 - a.kbar[NS + k]);
  const double c3 = kts * (tau - a.taubar[k]);

  // gradients of kappa1, kappa2, tau in (e_a, e_b, theta_a, theta_b)
  const v3 tt = ichi * s_ab, mt1 = ichi * M1, mt2 = ichi * M2;
  double g1[8], g2[8], g3[8];
  {
    v3 x;
    x = ila * (cross(tb, mt2) - k1 * tt);
    g1[0] = x.x; g1[1] = x.y; g1[2] = x.z;
    x = ilb * ((-k1) * tt - cross(ta, mt2));
    g1[3] = x.x; g1[4] = x.y; g1[5] = x.z;
    g1[6] = -0.5 * dot(kb, m1a);
    g1[7] = -0.5 * dot(kb, m1b);
    x = ila * ((-k2) * tt - cross(tb, mt1));
    g2[0] = x.x; g2[1] = x.y; g2[2] = x.z;
    x = ilb * (cross(ta, mt1) - k2 * tt);
    g2[3] = x.x; g2[4] = x.y; g2[5] = x.z;
    g2[6] = -0.5 * dot(kb, m2a);
    g2[7] = -0.5 * dot(kb, m2b);
    g3[0] = 0.5 * ila * kb.x; g3[1] = 0.5 * ila * kb.y; g3[2] = 0.5 * ila * kb.z;
    g3[3] = 0.5 * ilb * kb.x; g3[4] = 0.5 * ilb * kb.y; g3[5] = 0.5 * ilb * kb.z;
    g3[6] = -1.0;
    g3[7] = 1.0;
  }
  // energy gradient (8-space) and its outer-product Hessian part
  double g8[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) g8[i] = fma(c1, g1[i], fma(c2, g2[i], c3 * g3[i]));
  if (MODE == 1) {
    // the holonomy correction of the gradient (see the Hessian block below)
    const v3 tna = sgn3(sa, mk(a.tn[a.st_ed[k]], a.tn[NE + a.st_ed[k]], a.tn[2 * NE + a.st_ed[k]]));
    const v3 tnb = sgn3(sb, mk(a.tn[a.st_ed[NS + k]], a.tn[NE + a.st_ed[NS + k]],
                                   a.tn[2 * NE + a.st_ed[NS + k]]));
    const v3 ga = ila * (rcp64(1.0 + dot(tna, ta)) * cross(tna, ta));
    const v3 gb = ilb * (rcp64(1.0 + dot(tnb, tb)) * cross(tnb, tb));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g8[i] -= g8[6] * cmp(ga, i);
      g8[3 + i] -= g8[7] * cmp(gb, i);
    }
    write_gradient(a, k, g8, sa, sb);
    return;
  }
  double h[36];
  {
    // gradients pre-scaled by the stiffnesses: three FP64 instructions an entry
    double a1[8], a2[8], a3[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      a1[i] = kbs * g1[i];
      a2[i] = kbs * g2[i];
      a3[i] = kts * g3[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = i; j < 8; ++j) h[up<8>(i, j)] = fma(a1[i], g1[j], fma(a2[i], g2[j], a3[i] * g3[j]));
  }

  // second-derivative part, first in tangent space then projected
  const v3 w = c1 * M2 - c2 * M1;
  const double kw = dot(kb, w);
  const double ichi2 = ichi * ichi;
  const v3 pb = perp(ta, tb);   // P_a t_b
  const v3 pa = perp(tb, ta);   // P_b t_a
  // t-space gradient of E (the extension of the energy off the sphere)
  const v3 tbxw = cross(tb, w), wxta = cross(w, ta);
  const v3 gta = axpy(ichi, tbxw, axpy(-0.5 * kw * ichi, tb, (0.5 * c3) * kb));
  const v3 gtb = axpy(ichi, wxta, axpy(-0.5 * kw * ichi, ta, (0.5 * c3) * kb));
  const double tga = 0.5 * kw * ichi;  // t_a . g_ta == t_b . g_tb
  const v3 hga = perp(ta, gta), hgb = perp(tb, gtb);
  const v3 Pa = c1 * m2a - c2 * m1a, Pb = c1 * m2b - c2 * m1b;
  const v3 Ra = c1 * m1a + c2 * m2a, Rb = c1 * m1b + c2 * m2b;
  // aa block
  {
    const double s2 = ila * ila;
    const v3 Xa = axpy(-ichi2, perp(ta, tbxw), axpy(0.5 * kw * ichi2, pb, (-0.25 * c3 * ichi) * kb));
    add_sym(h, 0, s2, Xa, pb);
    add_sym(h, 0, 0.25 * s2, perp(ta, Pa), kb);
    add_sym(h, 0, -s2, ta, hga);
    {
      // - s2 tga (I - t_a t_a^T)
      const double c = s2 * tga;
      const v3 ct = c * ta;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
          h[up<8>(i, j)] = fma(cmp(ct, i), cmp(ta, j), i == j ? h[up<8>(i, j)] - c : h[up<8>(i, j)]);
    }
  }
  // bb block
  {
    const double s2 = ilb * ilb;
    const v3 Xb = axpy(-ichi2, perp(tb, wxta), axpy(0.5 * kw * ichi2, pa, (-0.25 * c3 * ichi) * kb));
    add_sym(h, 3, s2, Xb, pa);
    add_sym(h, 3, 0.25 * s2, perp(tb, Pb), kb);
    add_sym(h, 3, -s2, tb, hgb);
    {
      const double c = s2 * tga;
      const v3 ct = c * tb;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
          h[up<8>(3 + i, 3 + j)] =
              fma(cmp(ct, i), cmp(tb, j), i == j ? h[up<8>(3 + i, 3 + j)] - c : h[up<8>(3 + i, 3 + j)]);
    }
  }
  // ab block: M = -ichi [w]x - ichi^2 (alpha_a t_a^T + t_b alpha_b^T)
  //               + (kw ichi^2) t_b t_a^T - kw ichi/2 I
  //               + c3 ichi [t_a]x - c3 ichi/2 kb t_a^T,  then P_a M P_b
  {
    double Mab[3][3];
    const double ca = -0.5 * kw * ichi;
    // the rank-one parts as Ev t_a^T + Bv wxta^T
    const v3 Ev = axpy(-ichi2, tbxw, axpy(kw * ichi2, tb, (-0.5 * c3 * ichi) * kb));
    const v3 Bv = (-ichi2) * tb;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double v = fma(cmp(Ev, i), cmp(ta, j), cmp(Bv, i) * cmp(wxta, j));
        Mab[i][j] = i == j ? v + ca : v;
      }
    // skew parts: -ichi [w]x + c3 ichi [t_a]x = [z]x with z = ichi (c3 t_a - w)
    const v3 z = ichi * axpy(c3, ta, (-1.0) * w);
    Mab[0][1] -= z.z; Mab[0][2] += z.y;
    Mab[1][0] += z.z; Mab[1][2] -= z.x;
    Mab[2][0] -= z.y; Mab[2][1] += z.x;
    // P_a M P_b
    double r[3], cc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) r[j] = ta.x * Mab[0][j] + ta.y * Mab[1][j] + ta.z * Mab[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i) cc[i] = Mab[i][0] * tb.x + Mab[i][1] * tb.y + Mab[i][2] * tb.z;
    const double sc = r[0] * tb.x + r[1] * tb.y + r[2] * tb.z;
    const double s2 = ila * ilb;
    // M - t_a r^T - cc t_b^T + sc t_a t_b^T = M - t_a (r - sc t_b)^T - cc t_b^T
#pragma unroll
    for (int j = 0; j < 3; ++j) r[j] = fma(-sc, cmp(tb, j), r[j]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double v = fma(-cmp(ta, i), r[j], fma(-cc[i], cmp(tb, j), Mab[i][j]));
        h[up<8>(i, 3 + j)] = fma(s2, v, h[up<8>(i, 3 + j)]);
      }
  }
  // theta cross blocks: -1/2 P ga(R), ga(v) = 2 ichi (t_b x v) - (kb.v) ichi t_b,
  //                                     gb(v) = 2 ichi (v x t_a) - (kb.v) ichi t_a
  {
    const double kRa = dot(kb, Ra), kRb = dot(kb, Rb);
    v3 x;
    x = (-0.5 * ila) * axpy(2.0 * ichi, perp(ta, cross(tb, Ra)), (-kRa * ichi) * pb);
    h[up<8>(0, 6)] += x.x; h[up<8>(1, 6)] += x.y; h[up<8>(2, 6)] += x.z;
    x = (-0.5 * ilb) * axpy(2.0 * ichi, perp(tb, cross(Ra, ta)), (-kRa * ichi) * pa);
    h[up<8>(3, 6)] += x.x; h[up<8>(4, 6)] += x.y; h[up<8>(5, 6)] += x.z;
    x = (-0.5 * ila) * axpy(2.0 * ichi, perp(ta, cross(tb, Rb)), (-kRb * ichi) * pb);
    h[up<8>(0, 7)] += x.x; h[up<8>(1, 7)] += x.y; h[up<8>(2, 7)] += x.z;
    x = (-0.5 * ilb) * axpy(2.0 * ichi, perp(tb, cross(Rb, ta)), (-kRb * ichi) * pa);
    h[up<8>(3, 7)] += x.x; h[up<8>(4, 7)] += x.y; h[up<8>(5, 7)] += x.z;
    h[up<8>(6, 6)] += -0.5 * dot(kb, Pa);
    h[up<8>(7, 7)] += -0.5 * dot(kb, Pb);
  }

  // Exact derivatives of the energy with the reference frames carried from
  // the committed step by time-parallel transport (Eq. 9): moving the edge
  // tangent t also rotates its time-transported director about t by the
  // holonomy chi of the geodesic triangle (t_n, t, t'), which acts like a
  // twist-angle shift.  With Phi the at-point energy above:
  //   grad E = grad Phi - sum_x E_x grad chi_x
  //   hess E = H - sum_x sym(H[:, x], grad chi_x) + sum_xy H[x, y] grad chi_x grad chi_y^T
  //            - sum_x E_x hess chi_x,      x in {A, B} (effective angles)
  // grad_e chi = w / l with w = (t_n x t)/(1 + t_n.t), and
  // hess_e chi = -[ (n s^T + s n^T) / (2 c^2) + w t^T + t w^T ] / l^2,
  // n = t_n x t, c = 1 + t_n.t, s = t_n - (t_n.t) t.
  {
    const v3 tna = sgn3(sa, mk(a.tn[a.st_ed[k]], a.tn[NE + a.st_ed[k]], a.tn[2 * NE + a.st_ed[k]]));
    const v3 tnb = sgn3(sb, mk(a.tn[a.st_ed[NS + k]], a.tn[NE + a.st_ed[NS + k]],
                                   a.tn[2 * NE + a.st_ed[NS + k]]));
    v3 ga, gb;
    double Ha[6], Hb[6];
    {
      const double c = 1.0 + dot(tna, ta), ic = rcp64(c);
      const v3 n = cross(tna, ta), w = ic * n;
      const v3 sp = axpy(-dot(tna, ta), ta, tna);
      ga = ila * w;
      const double f1 = -0.5 * ic * ic * ila * ila, f2 = -ila * ila;
      const v3 fn = f1 * n, fw = f2 * w;
      int e = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j, ++e)
          Ha[e] = fma(cmp(fn, i), cmp(sp, j),
                      fma(cmp(sp, i), cmp(fn, j), fma(cmp(fw, i), cmp(ta, j), cmp(ta, i) * cmp(fw, j))));
    }
    {
      const double c = 1.0 + dot(tnb, tb), ic = rcp64(c);
      const v3 n = cross(tnb, tb), w = ic * n;
      const v3 sp = axpy(-dot(tnb, tb), tb, tnb);
      gb = ilb * w;
      const double f1 = -0.5 * ic * ic * ilb * ilb, f2 = -ilb * ilb;
      const v3 fn = f1 * n, fw = f2 * w;
      int e = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j, ++e)
          Hb[e] = fma(cmp(fn, i), cmp(sp, j),
                      fma(cmp(sp, i), cmp(fn, j), fma(cmp(fw, i), cmp(tb, j), cmp(tb, i) * cmp(fw, j))));
    }
    double colA[8], colB[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      colA[i] = i <= 6 ? h[up<8>(i, 6)] : h[up<8>(6, i)];
      colB[i] = h[up<8>(i < 7 ? i : 7, 7)];
    }
    const double EA = g8[6], EB = g8[7];
    const double HAA = h[up<8>(6, 6)], HBB = h[up<8>(7, 7)], HAB = h[up<8>(6, 7)];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g8[i] -= EA * cmp(ga, i);
      g8[3 + i] -= EB * cmp(gb, i);
    }
    // grad chi_A lives on entries 0-2, grad chi_B on 3-5: only the terms
    // whose factors are not structurally zero are formed (a product with a
    // literal zero is not dropped by an IEEE-conforming compiler)
    v3 hga_a = HAA * ga, hab_a = HAB * ga, hgb_b = HBB * gb;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = i; j < 8; ++j) {
        const bool ai = i < 3, aj = j < 3, bi = i >= 3 && i < 6, bj = j >= 3 && j < 6;
        if (!ai && !bi) continue;  // i, j >= 6: no correction
        double v = h[up<8>(i, j)];
        if (aj) v = fma(-colA[i], cmp(ga, j), v);
        if (ai) v = fma(-cmp(ga, i), colA[j], v);
        if (bj) v = fma(-colB[i], cmp(gb, j - 3), v);
        if (bi) v = fma(-cmp(gb, i - 3), colB[j], v);
        if (ai && aj) v = fma(cmp(hga_a, i), cmp(ga, j), fma(-EA, Ha[up<3>(i, j)], v));
        if (ai && bj) v = fma(cmp(hab_a, i), cmp(gb, j - 3), v);
        if (bi && bj) v = fma(cmp(hgb_b, i - 3), cmp(gb, j - 3), fma(-EB, Hb[up<3>(i - 3, j - 3)], v));
        h[up<8>(i, j)] = v;
      }
    if (a.dk) {
      // gradients of kappa1 and kappa2 as functions of the 11 DOFs (the
      // same holonomy correction as the energy gradient), for the adjoint:
      // d(grad E)/d(kappabar_c) = -EI/V grad kappa_c
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double *gc = c == 0 ? g1 : g2;
        double e8[8];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          e8[i] = gc[i] - gc[6] * cmp(ga, i);
          e8[3 + i] = gc[3 + i] - gc[7] * cmp(gb, i);
        }
        e8[6] = gc[6];
        e8[7] = gc[7];
        double *o = a.dk + (size_t)(11 * c) * NS + k;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          o[(size_t)i * NS] = -e8[i];
          o[(size_t)(4 + i) * NS] = e8[i] - e8[3 + i];
          o[(size_t)(8 + i) * NS] = e8[3 + i];
        }
        o[(size_t)3 * NS] = sgnmul(sign_word(sa), e8[6]);
        o[(size_t)7 * NS] = sgnmul(sign_word(sb), e8[7]);
      }
    }
  }

  if (MODE == 0) write_gradient(a, k, g8, sa, sb);

  // H11 = T^T H8 T written as packed upper triangle
  auto H8 = [&](int i, int j) -> double { return i <= j ? h[up<8>(i, j)] : h[up<8>(j, i)]; };
  // each entry a signed sum of H8 entries, from its first term (no add of
  // a zero), the signs sa, sb applied on the integer pipe
  double *Ho = a.sh;
  const unsigned swa = sign_word(sa), swb = sign_word(sb);
#pragma unroll
  for (int p = 0; p < 11; ++p)
#pragma unroll
    for (int q = p; q < 11; ++q) {
      double v = 0.0;
      bool first = true;
#pragma unroll
      for (int tp = 0; tp < 2; ++tp)
#pragma unroll
        for (int tq = 0; tq < 2; ++tq) {
          const int ip = slot_index(p, tp), iq = slot_index(q, tq);
          if (ip < 0 || iq < 0) continue;
          const int wp = slot_weight(p, tp), wq = slot_weight(q, tq);
          const bool neg = (wp == -1) != (wq == -1);
          const unsigned sw = (wp == 2 ? swa : wp == 3 ? swb : 0u) ^ (wq == 2 ? swa : wq == 3 ? swb : 0u);
          if (first) {
            v = sgnmul(sw ^ (neg ? 0x80000000u : 0u), H8(ip, iq));
            first = false;
          } else {
            const double x = sgnmul(sw, H8(ip, iq));
            v = neg ? v - x : v + x;
          }
        }
      Ho[up<11>(p, q) * NS + k] = v;
    }
}

// block-uniform grid-stride loops (count_units synchronises the block)
__global__ void __launch_bounds__(128) k_stencil(StencilArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.ns; b0 += gridDim.x * blockDim.x)
    k_stencil_one<0>(a, b0 + threadIdx.x);
}
__global__ void __launch_bounds__(128) k_stencil_grad(StencilArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.ns; b0 += gridDim.x * blockDim.x)
    k_stencil_one<1>(a, b0 + threadIdx.x);
}
__global__ void __launch_bounds__(128) k_stencil_hess(StencilArgs a) {
  for (int b0 = blockIdx.x * blockDim.x; b0 < a.ns; b0 += gridDim.x * blockDim.x)
    k_stencil_one<2>(a, b0 + threadIdx.x);
}

}  // namespace dm
