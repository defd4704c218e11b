// Learned warm start of the Newton iteration (no counterpart in the paper).
//
// One "segment" per rod node i >= 1 with the edge i-1 that ends at it.  From
// the committed state (q_n, qdot_n, frames, natural curvature) a feature
// vector is built in the local frame of edge i-1 at t_n; the network
// (dm_mlp.cu, tensor cores) predicts the correction of node i and of the
// twist angle of edge i-1 over the extrapolation q_n + dt qdot_n, which then
// seeds Newton.  Newton still runs to the same residual, so the physics is
// unchanged; only the number of iterations can change.
//
// Features (64, the last 7 zero), local frame {t, d1, d2} of edge i-1, edge
// rest length l:
//   0..29  nodes i-2..i+2: (x_j - x_i)/l and dt qdot_j / l (local), zero if absent
//   30..34 presence flags of those nodes
//   35..37 dt thetadot of edges i-2, i-1, i;  38..39 theta_{i-2,i} - theta_{i-1}
//   40..45 natural curvature (kappabar1, kappabar2) at nodes i-1, i, i+1
//   46..48 gravity dt^2 / l (local);  49 (z_i - z_ground)/h;  50 mu (ground on)
//   51..54 static: log10 E, log10(h/l), log10 rho, log10(dt^2 EA/(m l))
//   55..58 the previous step's correction dt (qdot_n - qdot_{n-1}) of node i
//          (local, / l: p) and of the twist of edge i-1 (p_theta), divided by
//          the segment's scales sigma = max(|p|, |g| dt^2 / l) and
//          sigma_theta = max(|p_theta|, 1e-9) (p = 0 after a state is set or
//          when the warm start is enabled)
//   59..60 log10 sigma, log10 sigma_theta
// Targets: local (x_i^{n+1} - x_i^pred)/(l sigma) and
// (theta^{n+1} - theta^pred)/sigma_theta, where x^{n+1} - x^pred =
// dt (qdot_{n+1} - qdot_n): the correction relative to the last one, so
// that the network's error is relative to each segment's own correction
// (corrections differ by orders of magnitude between stiff and soft rods).
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <vector>

#include "dm_internal.h"

namespace dm {
float *mlp_forward_async(dm_mlp *m, const void *X, int M, cudaStream_t st, int *err);
}

using namespace dm;

namespace dm {

struct WarmStart {
  int64_t nseg = 0, mpad = 0;
  int32_t *seg_i = nullptr;  // [16][nseg]
  float *seg_f = nullptr;    // [6][nseg]
  double *basis = nullptr;   // [12][nseg]: t, d1, d2, l, sigma, sigma_theta
  double *pred = nullptr;    // [4][nseg]
  uint16_t *X = nullptr;     // [mpad][64] bf16
  double *ql = nullptr;      // learned guess [n_dofs] (line-search trial)
  double *vprev = nullptr;   // qdot_{n-1} [n_dofs]
  int32_t *learned_sys = nullptr;  // [n_systems] 1: this step's guess came from the network
  int32_t *wstry = nullptr;  // [n_systems]
  float *norm = nullptr;     // in_mean[64], in_std[64], out_scale[4]
  int *err = nullptr;
  dm_mlp *net = nullptr;
  std::vector<void *> allocs;
};

namespace {

struct FeatArgs {
  int64_t nseg, nd, ns, ne, nn;
  double dt, g[3], ground_z;
  int ground;
  const int32_t *seg_i;
  const float *seg_f;
  const double *qn, *vn, *vprev, *tn, *d1n, *kbar, *node_h, *node_mu;
  const int32_t *dof_node;
  double *basis, *pred;
  float *raw;          // mode 0: raw features [nseg][64]
  uint16_t *X;         // mode 1: normalised bf16 [mpad][64]
  const float *norm;   // mode 1
};

__device__ __forceinline__ uint16_t f2bf(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t *>(&b);
}

__global__ void k_ws_features(FeatArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nseg) return;
  const int64_t S = a.nseg;
  auto I = [&](int k) { return a.seg_i[k * S + s]; };
  const int nd = I(0), th = I(1), e = I(2);
  const int64_t NE = a.ne;
  const double t[3] = {a.tn[e], a.tn[NE + e], a.tn[2 * NE + e]};
  const double d1[3] = {a.d1n[e], a.d1n[NE + e], a.d1n[2 * NE + e]};
  const double d2[3] = {t[1] * d1[2] - t[2] * d1[1], t[2] * d1[0] - t[0] * d1[2],
                        t[0] * d1[1] - t[1] * d1[0]};
  const double l = (double)a.seg_f[5 * S + s];
  const double il = 1.0 / l, dt = a.dt;
  float f[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) f[k] = 0.0f;
  auto local = [&](double x, double y, double z, float *o, double sc) {
    o[0] = (float)(sc * (x * t[0] + y * t[1] + z * t[2]));
    o[1] = (float)(sc * (x * d1[0] + y * d1[1] + z * d1[2]));
    o[2] = (float)(sc * (x * d2[0] + y * d2[1] + z * d2[2]));
  };
  const double xi = a.qn[nd], yi = a.qn[nd + 1], zi = a.qn[nd + 2];
#pragma unroll
  for (int w = 0; w < 5; ++w) {
    const int j = I(3 + w);
    if (j >= 0) {
      local(a.qn[j] - xi, a.qn[j + 1] - yi, a.qn[j + 2] - zi, f + 6 * w, il);
      local(dt * a.vn[j], dt * a.vn[j + 1], dt * a.vn[j + 2], f + 6 * w + 3, il);
      f[30 + w] = 1.0f;
    }
  }
  const double thm = a.qn[th];
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    const int d = I(8 + w);
    if (d >= 0) {
      f[35 + w] = (float)(dt * a.vn[d]);
      if (w != 1) f[38 + (w == 2)] = (float)(a.qn[d] - thm);
    }
  }
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    const int st = I(11 + w);
    if (st >= 0) {
      f[40 + 2 * w] = (float)a.kbar[st];
      f[41 + 2 * w] = (float)a.kbar[a.ns + st];
    }
  }
  local(a.g[0] * dt * dt, a.g[1] * dt * dt, a.g[2] * dt * dt, f + 46, il);
  if (a.ground) {
    const int v = a.dof_node[nd];
    f[49] = (float)fmin(fmax((zi - a.ground_z) / a.node_h[v], -5.0), 20.0);
    f[50] = (float)a.node_mu[v];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) f[51 + k] = a.seg_f[k * S + s];
  {
    double pc[3];
    const double px = dt * (a.vn[nd] - a.vprev[nd]), py = dt * (a.vn[nd + 1] - a.vprev[nd + 1]),
                 pz = dt * (a.vn[nd + 2] - a.vprev[nd + 2]);
    pc[0] = il * (px * t[0] + py * t[1] + pz * t[2]);
    pc[1] = il * (px * d1[0] + py * d1[1] + pz * d1[2]);
    pc[2] = il * (px * d2[0] + py * d2[1] + pz * d2[2]);
    const double gn = sqrt(a.g[0] * a.g[0] + a.g[1] * a.g[1] + a.g[2] * a.g[2]);
    const double sig = fmax(sqrt(pc[0] * pc[0] + pc[1] * pc[1] + pc[2] * pc[2]),
                            fmax(gn * dt * dt * il, 1e-30));
    const double pth = dt * (a.vn[th] - a.vprev[th]);
    const double sth = fmax(fabs(pth), 1e-9);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[55 + c] = (float)(pc[c] / sig);
    f[58] = (float)(pth / sth);
    f[59] = (float)log10(sig);
    f[60] = (float)log10(sth);
    a.basis[10 * S + s] = sig;
    a.basis[11 * S + s] = sth;
  }
  // local basis and the extrapolation this segment corrects
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.basis[c * S + s] = t[c];
    a.basis[(3 + c) * S + s] = d1[c];
    a.basis[(6 + c) * S + s] = d2[c];
    a.pred[c * S + s] = a.qn[nd + c] + dt * a.vn[nd + c];
  }
  a.basis[9 * S + s] = l;
  a.pred[3 * S + s] = a.qn[th] + dt * a.vn[th];
  if (a.raw) {
#pragma unroll
    for (int k = 0; k < 64; ++k) a.raw[s * 64 + k] = f[k];
  }
  if (a.X) {
#pragma unroll
    for (int k = 0; k < 64; ++k)
      a.X[s * 64 + k] = f2bf((f[k] - a.norm[k]) / a.norm[64 + k]);
  }
}

__global__ void k_ws_apply(int64_t nseg, const int32_t *seg_i, const double *basis,
                           const float *Y, const float *norm, double *q,
                           const int32_t *dof_sys, int32_t *learned_sys) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int64_t S = nseg;
  const int nd = seg_i[s], th = seg_i[S + s], flags = seg_i[14 * S + s];
  if (learned_sys && flags) learned_sys[dof_sys[nd]] = 1;
  const float *o = norm + 128;
  const double y0 = Y[s * 64] * o[0], y1 = Y[s * 64 + 1] * o[1], y2 = Y[s * 64 + 2] * o[2];
  const double l = basis[9 * S + s] * basis[10 * S + s];
  if (flags & 1)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      q[nd + c] += l * (y0 * basis[c * S + s] + y1 * basis[(3 + c) * S + s] +
                        y2 * basis[(6 + c) * S + s]);
  if (flags & 2) q[th] += (double)Y[s * 64 + 3] * o[3] * basis[11 * S + s];
}

// Fallback to the extrapolation: a system whose Newton run from the learned
// guess has taken kWsRestart iterations without converging starts over from
// q_n + dt qdot_n (fixed DOFs keep q_n); the iteration count carries on, so
// this happens once per step.
constexpr int kWsRestart = 6;
__global__ void k_ws_fallback(int32_t nd, double dt, const int32_t *dof_sys,
                              const int32_t *learned_sys, const int32_t *sys_active,
                              const int32_t *sys_iters, const uint8_t *fixed, const double *qn,
                              const double *vn, double *q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const int s = dof_sys[i];
  if (!learned_sys[s] || !sys_active[s] || sys_iters[s] != kWsRestart) return;
  q[i] = fixed[i] ? qn[i] : fma(dt, vn[i], qn[i]);
}

__global__ void k_ws_targets(int64_t nseg, const int32_t *seg_i, const double *basis,
                             const double *pred, const double *qn, float *tgt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int64_t S = nseg;
  const int nd = seg_i[s], th = seg_i[S + s];
  double dx[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dx[c] = qn[nd + c] - pred[c * S + s];
  const double il = 1.0 / (basis[9 * S + s] * basis[10 * S + s]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) v += dx[c] * basis[(3 * k + c) * S + s];
    tgt[s * 4 + k] = (float)(v * il);
  }
  tgt[s * 4 + 3] = (float)((qn[th] - pred[3 * S + s]) / basis[11 * S + s]);
}

__global__ void k_ws_gather(int32_t M, const float *feat, const float *tgt, const int64_t *idx,
                            const float *norm, uint16_t *X, float *Y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * 64) return;
  const int64_t r = t / 64;
  const int k = (int)(t - r * 64);
  const int64_t src = idx[r];
  X[t] = f2bf((feat[src * 64 + k] - norm[k]) / norm[64 + k]);
  if (k < 4) Y[r * 4 + k] = tgt[src * 4 + k] / norm[128 + k];
}

// Column sums and sums of squares: each block takes a chunk of rows, thread t
// column t % cols, rows strided by blockDim / cols; one double atomic per
// thread and moment.
__global__ void k_col_partial(int64_t rows, int32_t cols, int64_t chunk, const float *data,
                              double *acc) {
  const int c = threadIdx.x % cols, r0 = threadIdx.x / cols, rs = blockDim.x / cols;
  if (r0 >= rs) return;
  const int64_t b = (int64_t)blockIdx.x * chunk, e = min(rows, b + chunk);
  double s = 0.0, s2 = 0.0;
  for (int64_t r = b + r0; r < e; r += rs) {
    const double v = data[r * cols + c];
    s += v;
    s2 += v * v;
  }
  atomicAdd(acc + c, s);
  atomicAdd(acc + cols + c, s2);
}

__global__ void k_col_final(int64_t rows, int32_t cols, const double *acc, float *stats) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const double m = acc[c] / (double)rows;
  const double var = acc[cols + c] / (double)rows - m * m;
  stats[c] = (float)m;
  stats[cols + c] = (float)(var > 1e-24 ? sqrt(var) : 1.0);
}

inline int nb(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// Builds the segment tables from the topology.
dm_status ws_build(dm_system *s, WarmStart *w) {
  const HostTopology &T = s->T;
  std::vector<int32_t> st_of_slot;
  int64_t nslots = 0;
  std::vector<int64_t> kslot0(T.n_rods + 1, 0);
  for (int r = 0; r < T.n_rods; ++r) kslot0[r + 1] = kslot0[r] + (T.npr[r] - 2);
  nslots = kslot0[T.n_rods];
  st_of_slot.assign(std::max<int64_t>(nslots, 1), -1);
  for (int64_t k = 0; k < T.n_stencils; ++k)
    if (T.st_rod_slot[k] >= 0) st_of_slot[T.st_rod_slot[k]] = (int32_t)k;
  std::vector<std::vector<int32_t>> I(16);
  std::vector<std::vector<float>> F(6);
  std::vector<char> owned(T.n_nodes, 0);
  const double dt = s->p.dt;
  for (int r = 0; r < T.n_rods; ++r) {
    const int N = T.npr[r];
    auto node_of = [&](int i) { return T.flat2node[T.rod_node0[r] + i]; };
    for (int i = 1; i < N; ++i) {
      const int64_t v = node_of(i);
      const int64_t e = T.rod_edge0[r] + i - 1;
      const int32_t nd = T.node_dof[v], th = T.edge_thdof[e];
      I[0].push_back(nd);
      I[1].push_back(th);
      I[2].push_back((int32_t)e);
      for (int o = -2; o <= 2; ++o) {
        const int j = i + o;
        I[5 + o].push_back((j >= 0 && j < N) ? T.node_dof[node_of(j)] : -1);
      }
      for (int o = -2; o <= 0; ++o) {
        const int ee = i - 1 + o + 1;  // edges i-2, i-1, i
        I[10 + o].push_back((ee >= 0 && ee <= N - 2) ? T.edge_thdof[T.rod_edge0[r] + ee] : -1);
      }
      for (int o = -1; o <= 1; ++o) {
        const int m = i + o;
        I[12 + o].push_back((m >= 1 && m <= N - 2) ? st_of_slot[kslot0[r] + m - 1] : -1);
      }
      int flags = 0;
      if (!owned[v] && !T.dof_fixed[nd] && !T.dof_fixed[nd + 1] && !T.dof_fixed[nd + 2]) {
        flags |= 1;
        owned[v] = 1;
      }
      if (!T.dof_fixed[th]) flags |= 2;
      I[14].push_back(flags);
      I[15].push_back(r);
      const double h = T.edge_h[e], A = M_PI * h * h;
      const double E = T.edge_EA[e] / A, rho = T.edge_rhoA[e] / A, l = T.edge_lbar[e];
      const double m = T.node_mass[v];
      F[0].push_back((float)std::log10(E));
      F[1].push_back((float)std::log10(h / l));
      F[2].push_back((float)std::log10(rho));
      F[3].push_back((float)std::log10(dt * dt * T.edge_EA[e] / (m * l)));
      F[4].push_back(0.0f);
      F[5].push_back((float)l);
    }
  }
  w->nseg = (int64_t)I[0].size();
  w->mpad = (w->nseg + 127) / 128 * 128;
  const int64_t S = w->nseg;
  std::vector<int32_t> ii(16 * S);
  std::vector<float> ff(6 * S);
  for (int k = 0; k < 16; ++k) std::copy(I[k].begin(), I[k].end(), ii.begin() + k * S);
  for (int k = 0; k < 6; ++k) std::copy(F[k].begin(), F[k].end(), ff.begin() + k * S);
  auto dal = [&](void **p, size_t bytes) {
    if (cudaMalloc(p, bytes + 16) != cudaSuccess) return false;
    cudaMemset(*p, 0, bytes + 16);
    w->allocs.push_back(*p);
    return true;
  };
  if (!dal((void **)&w->seg_i, ii.size() * 4) || !dal((void **)&w->seg_f, ff.size() * 4) ||
      !dal((void **)&w->basis, 12 * S * 8) || !dal((void **)&w->pred, 4 * S * 8) ||
      !dal((void **)&w->X, w->mpad * 64 * 2) || !dal((void **)&w->norm, 132 * 4) ||
      !dal((void **)&w->err, 4) || !dal((void **)&w->ql, T.n_dofs * 8) ||
      !dal((void **)&w->vprev, T.n_dofs * 8) || !dal((void **)&w->learned_sys, T.n_systems * 4) ||
      !dal((void **)&w->wstry, T.n_systems * 4)) {
    set_error("warm start: cudaMalloc failed");
    return DM_ERR_OOM;
  }
  cudaMemcpy(w->seg_i, ii.data(), ii.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(w->seg_f, ff.data(), ff.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(w->vprev, s->d.vn, T.n_dofs * 8, cudaMemcpyDeviceToDevice);
  return cudaDeviceSynchronize() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

static FeatArgs feat_args(dm_system *s, WarmStart *w) {
  const HostTopology &T = s->T;
  FeatArgs a{};
  a.nseg = w->nseg;
  a.nd = T.n_dofs;
  a.ns = T.n_stencils;
  a.ne = T.n_edges;
  a.nn = T.n_nodes;
  a.dt = s->p.dt;
  for (int c = 0; c < 3; ++c) a.g[c] = s->p.g[c];
  a.ground_z = s->prm.ground_z;
  a.ground = T.ground ? 1 : 0;
  a.seg_i = w->seg_i;
  a.seg_f = w->seg_f;
  a.qn = s->d.qn;
  a.vn = s->d.vn;
  a.vprev = w->vprev;
  a.tn = s->d.tn;
  a.d1n = s->d.d1n;
  a.kbar = s->d.kbar;
  a.node_h = s->d.node_h;
  a.node_mu = s->d.node_mu;
  a.dof_node = s->d.dof_node;
  a.basis = w->basis;
  a.pred = w->pred;
  return a;
}

bool ws_active(const dm_system *s) { return s->ws && s->ws->net && s->ws->nseg > 0; }

cudaError_t ws_keep_velocity(dm_system *s, cudaStream_t st) {
  if (!s->ws || !s->ws->vprev) return cudaSuccess;
  return cudaMemcpyAsync(s->ws->vprev, s->d.vn, s->T.n_dofs * sizeof(double),
                         cudaMemcpyDeviceToDevice, st);
}

int32_t *ws_trial_flags(dm_system *s) { return s->ws ? s->ws->wstry : nullptr; }

cudaError_t ws_predict(dm_system *s, cudaStream_t st, bool defer, const int32_t *dof_sys) {
  WarmStart *w = s->ws;
  if (!ws_active(s)) return cudaSuccess;
  if (!defer) cudaMemsetAsync(w->learned_sys, 0, s->T.n_systems * sizeof(int32_t), st);
  FeatArgs a = feat_args(s, w);
  a.X = w->X;
  a.norm = w->norm;
  k_ws_features<<<nb(w->nseg, 128), 128, 0, st>>>(a);
  float *Y = mlp_forward_async(w->net, w->X, (int)w->mpad, st, w->err);
  if (!Y) return cudaErrorUnknown;
  double *dst = s->d.q;
  if (defer) {
    cudaMemcpyAsync(w->ql, s->d.q, s->T.n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, st);
    dst = w->ql;
  }
  k_ws_apply<<<nb(w->nseg, 128), 128, 0, st>>>(w->nseg, w->seg_i, w->basis, Y, w->norm, dst,
                                                dof_sys, defer ? nullptr : w->learned_sys);
  return cudaGetLastError();
}

cudaError_t ws_fallback(dm_system *s, cudaStream_t st, const int32_t *dof_sys) {
  WarmStart *w = s->ws;
  if (!ws_active(s)) return cudaSuccess;
  const int nd = (int)s->T.n_dofs;
  k_ws_fallback<<<nb(nd, 256), 256, 0, st>>>(nd, s->p.dt, dof_sys, w->learned_sys,
                                             s->d.sys_active, s->d.sys_iters, s->d.fixed,
                                             s->d.qn, s->d.vn, s->d.q);
  return cudaGetLastError();
}

namespace {
__global__ void k_ws_inject(int32_t nsys, const int32_t *sys_active, int32_t *action,
                            int32_t *trial, int32_t *wstry) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || !sys_active[s]) return;
  action[s] = 1;  // no Newton solve in this round
  trial[s] = 1;
  wstry[s] = 1;
}
}  // namespace

cudaError_t ws_inject(dm_system *s, cudaStream_t st, int32_t *ls_action, int32_t *ls_trial) {
  WarmStart *w = s->ws;
  // every system is still active after the first round (nothing has been
  // solved yet), so the whole vector is replaced
  cudaMemcpyAsync(s->d.q, w->ql, s->T.n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, st);
  const int S = s->T.n_systems;
  k_ws_inject<<<nb(S, 128), 128, 0, st>>>(S, s->d.sys_active, ls_action, ls_trial, w->wstry);
  return cudaGetLastError();
}

void ws_free(WarmStart *w) {
  if (!w) return;
  for (void *p : w->allocs) cudaFree(p);
  delete w;
}

}  // namespace dm

extern "C" {

dm_status dm_ws_enable(dm_system *s) {
  if (!s) return DM_ERR_INVALID_ARG;
  if (s->ws) return DM_OK;
  if (!s->d.node_h) {
    // the feature kernel reads node radii/friction (allocated for general
    // systems only): allocate them here for rod batches
    std::vector<double> h = s->T.node_h, mu = s->T.node_mu;
    if (cudaMalloc(&s->d.node_h, h.size() * 8 + 8) || cudaMalloc(&s->d.node_mu, mu.size() * 8 + 8))
      return DM_ERR_OOM;
    s->allocations.push_back(s->d.node_h);
    s->allocations.push_back(s->d.node_mu);
    cudaMemcpy(s->d.node_h, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(s->d.node_mu, mu.data(), mu.size() * 8, cudaMemcpyHostToDevice);
  }
  WarmStart *w = new WarmStart();
  dm_status st = ws_build(s, w);
  if (st != DM_OK) {
    ws_free(w);
    return st;
  }
  s->ws = w;
  return DM_OK;
}

int64_t dm_ws_num_segments(const dm_system *s) { return (s && s->ws) ? s->ws->nseg : 0; }

dm_status dm_ws_capture_features(dm_system *s, float *feat) {
  if (!s || !s->ws || !feat) {
    set_error("dm_ws_capture_features: call dm_ws_enable first");
    return DM_ERR_INVALID_ARG;
  }
  FeatArgs a = feat_args(s, s->ws);
  a.raw = feat;
  k_ws_features<<<nb(s->ws->nseg, 128), 128, 0, s->stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_ws_capture_targets(dm_system *s, float *tgt) {
  if (!s || !s->ws || !tgt) return DM_ERR_INVALID_ARG;
  WarmStart *w = s->ws;
  k_ws_targets<<<nb(w->nseg, 128), 128, 0, s->stream>>>(w->nseg, w->seg_i, w->basis, w->pred,
                                                        s->d.qn, tgt);
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_ws_set_model(dm_system *s, dm_mlp *net, const float *norm) {
  if (!s || !s->ws) {
    set_error("dm_ws_set_model: call dm_ws_enable first");
    return DM_ERR_INVALID_ARG;
  }
  if (net && !norm) return DM_ERR_INVALID_ARG;
  if (norm) cudaMemcpy(s->ws->norm, norm, 132 * 4, cudaMemcpyHostToDevice);
  s->ws->net = net;
  return DM_OK;
}

dm_status dm_ws_prepare_batch(const float *feat, const float *tgt, const int64_t *idx,
                              int32_t M, const float *norm, void *X, float *Y, void *stream) {
  if (!feat || !tgt || !idx || !norm || !X || !Y || M <= 0) return DM_ERR_INVALID_ARG;
  k_ws_gather<<<nb((int64_t)M * 64, 256), 256, 0, (cudaStream_t)stream>>>(
      M, feat, tgt, idx, norm, (uint16_t *)X, Y);
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_ws_column_stats(const float *data, int64_t rows, int32_t cols, float *stats,
                             void *stream) {
  if (!data || !stats || rows <= 0 || cols <= 0 || cols > 256) {
    set_error("dm_ws_column_stats: bad arguments (1 <= cols <= 256)");
    return DM_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *acc = nullptr;
  if (cudaMallocAsync((void **)&acc, 2 * cols * sizeof(double), st) != cudaSuccess)
    return DM_ERR_OOM;
  cudaMemsetAsync(acc, 0, 2 * cols * sizeof(double), st);
  const int64_t chunk = 1 << 14;
  k_col_partial<<<nb(rows, (int)chunk), 256, 0, st>>>(rows, cols, chunk, data, acc);
  k_col_final<<<nb(cols, 64), 64, 0, st>>>(rows, cols, acc, stats);
  cudaFreeAsync(acc, st);
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

}  // extern "C"
