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
//      block (10 x 10, Gauss-Jordan with partial pivoting);
//   3. per interior, in parallel: x_p = L^{-T} D^{-1} (z_p - Z_p x_S).
//
// The work per interior is a few times that of the plain band LDL^T, but
// the sequential depth is m rows plus one 10 x 10 elimination per
// separator instead of n rows.  One warp per interior or system; an
// interior keeps its band and its top coupling solve in shared memory.
#include <vector>

#include "dm_internal.h"

namespace dm {

namespace {

constexpr int PW = 10;  // half bandwidth = separator width

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
  int *bad;
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
  const int r0 = a.p_a[p], mm = a.p_mm[p];
  const bool top = a.p_top[p] >= 0, bot = a.p_bot[p] >= 0;
  double *Bs = sm;                     // [mm][11]: band, then multipliers
  double *Zs = sm + (size_t)mm * 11;   // [mm][10]: L^{-1} C_top
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
      if (lane == 0) atomicExch(a.bad, 1);
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
      a.Zt[(size_t)(r0 + i) * PW + c] = z;
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

// Gauss-Jordan with partial pivoting on M [10][21] in shared memory, lane j
// owning column j: M <- [I | M_left^{-1} M_right].  Returns false on a zero
// or non-finite pivot.
__device__ bool gj10(double (*M)[22], int lane, int ncol) {
  for (int k = 0; k < PW; ++k) {
    int piv = k;
    if (lane == 0) {
      double best = fabs(M[k][k]);
      for (int i = k + 1; i < PW; ++i)
        if (fabs(M[i][k]) > best) {
          best = fabs(M[i][k]);
          piv = i;
        }
    }
    piv = __shfl_sync(0xffffffffu, piv, 0);
    __syncwarp();
    if (lane < ncol && piv != k) {
      const double tmp = M[k][lane];
      M[k][lane] = M[piv][lane];
      M[piv][lane] = tmp;
    }
    __syncwarp();
    const double pk = M[k][k];
    if (!(fabs(pk) > 0.0) || !isfinite(pk)) return false;
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
  if (ns == 0) return;
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
      if (lane == 0) atomicExch(a.bad, 1);
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

}  // namespace

}  // namespace dm

using namespace dm;

extern "C" dm_status dm_solve_band_partitioned(int32_t nsys, const int32_t *sys_dof0,
                                               const int32_t *sys_ndof, int64_t ntot,
                                               const double *band, const double *rhs, double *x,
                                               int32_t part_rows, void *stream) {
  if (nsys < 0 || (nsys > 0 && (!sys_dof0 || !sys_ndof || !band || !rhs || !x)) || ntot < 0) {
    set_error("dm_solve_band_partitioned: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  const int m = part_rows > 0 ? part_rows : 512;
  if (m < 2 * PW + 1 || m > 1024) {
    set_error("dm_solve_band_partitioned: part_rows must be in [21, 1024]");
    return DM_ERR_INVALID_ARG;
  }
  // layout: interiors [k m, k m + m - 10), separators [k m + m - 10, (k+1) m),
  // the last interior [(P-1) m, n) with at least 11 rows
  std::vector<int32_t> pa, pmm, ptop, pbot, sa, s0(nsys), nsp(nsys);
  for (int k = 0; k < nsys; ++k) {
    const int n = sys_ndof[k], d0 = sys_dof0[k];
    if (n <= 0 || d0 < 0 || (int64_t)d0 + n > ntot) {
      set_error("dm_solve_band_partitioned: system outside the vectors");
      return DM_ERR_INVALID_ARG;
    }
    int P = (n - 1) / m + 1;
    while (P > 1 && n - (P - 1) * m < PW + 1) --P;
    s0[k] = (int32_t)sa.size();
    nsp[k] = P - 1;
    for (int p = 0; p < P; ++p) {
      const int a = p * m, b = p + 1 < P ? a + m - PW : n;
      pa.push_back(d0 + a);
      pmm.push_back(b - a);
      // the top separator of interior p > 0 is the bottom one of p - 1
      ptop.push_back(p > 0 ? pbot.back() : -1);
      if (p + 1 < P) sa.push_back(d0 + b);
      pbot.push_back(p + 1 < P ? (int32_t)sa.size() - 1 : -1);
    }
  }
  const int np = (int)pa.size(), nsep = (int)sa.size();
  if (np == 0) return DM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // scratch
  size_t bytes = 0;
  auto take = [&](size_t n) {
    const size_t o = bytes;
    bytes += (n * sizeof(double) + 255) / 256 * 256;
    return o;
  };
  const size_t oL = take((size_t)ntot * PW), oD = take(ntot), oZ = take((size_t)ntot * PW),
               oz = take(ntot), oZb = take((size_t)np * PW * PW), oct = take((size_t)np * 110),
               ocb = take((size_t)np * 110), oco = take((size_t)np * 110),
               oX = take((size_t)std::max(nsep, 1) * 110), oI = take((4 * (size_t)np + 3 * nsys +
                                                                      (size_t)nsep + 8) / 2 + 1);
  char *scr = nullptr;
  if (cudaMalloc(&scr, bytes) != cudaSuccess) {
    set_error("dm_solve_band_partitioned: cudaMalloc");
    return DM_ERR_OOM;
  }
  int32_t *ib = reinterpret_cast<int32_t *>(scr + oI);
  std::vector<int32_t> ints;
  ints.insert(ints.end(), pa.begin(), pa.end());
  ints.insert(ints.end(), pmm.begin(), pmm.end());
  ints.insert(ints.end(), ptop.begin(), ptop.end());
  ints.insert(ints.end(), pbot.begin(), pbot.end());
  ints.insert(ints.end(), sa.begin(), sa.end());
  ints.insert(ints.end(), s0.begin(), s0.end());
  ints.insert(ints.end(), nsp.begin(), nsp.end());
  ints.push_back(0);  // bad flag
  PartArgs A{};
  A.ntot = ntot;
  A.nparts = np;
  A.nsep = nsep;
  A.p_a = ib;
  A.p_mm = ib + np;
  A.p_top = ib + 2 * np;
  A.p_bot = ib + 3 * np;
  A.s_a = ib + 4 * np;
  A.sys_sep0 = ib + 4 * np + nsep;
  A.sys_nsep = ib + 4 * np + nsep + nsys;
  A.bad = ib + 4 * np + nsep + 2 * nsys;
  A.band = band;
  A.rhs = rhs;
  A.x = x;
  A.Lf = reinterpret_cast<double *>(scr + oL);
  A.Df = reinterpret_cast<double *>(scr + oD);
  A.Zt = reinterpret_cast<double *>(scr + oZ);
  A.zf = reinterpret_cast<double *>(scr + oz);
  A.Zb = reinterpret_cast<double *>(scr + oZb);
  A.ct = reinterpret_cast<double *>(scr + oct);
  A.cb = reinterpret_cast<double *>(scr + ocb);
  A.co = reinterpret_cast<double *>(scr + oco);
  A.Xs = reinterpret_cast<double *>(scr + oX);
  cudaError_t e = cudaMemcpyAsync(ib, ints.data(), ints.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(scr + oct, 0, oX - oct, st);
  int mmax = 0;
  for (int v : pmm) mmax = std::max(mmax, v);
  const size_t smem = (size_t)mmax * (11 + PW) * sizeof(double);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_part_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e == cudaSuccess) {
    k_part_factor<<<np, 32, smem, st>>>(A);
    if (nsep > 0) k_part_separators<<<nsys, 32, 0, st>>>(A);
    k_part_back<<<np, 32, 0, st>>>(A);
    e = cudaGetLastError();
  }
  int bad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, A.bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(scr);
  if (e != cudaSuccess) {
    set_error(std::string("dm_solve_band_partitioned: ") + cudaGetErrorString(e));
    return DM_ERR_CUDA;
  }
  if (bad) {
    set_error("dm_solve_band_partitioned: zero or non-finite pivot");
    return DM_ERR_DEGENERATE;
  }
  return DM_OK;
}
