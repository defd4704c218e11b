// C ABI of the GB300 implicit DER library (include/dismech.h).
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dm_internal.h"
#include "dm_kernels.cuh"

namespace dm {

static thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }

}  // namespace dm

using namespace dm;

namespace {

#define DM_CK(call)                                                             \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #call); \
      return e_ == cudaErrorMemoryAllocation ? DM_ERR_OOM : DM_ERR_CUDA;        \
    }                                                                           \
  } while (0)

template <class T>
dm_status dalloc(dm_system *s, T **p, size_t n) {
  void *v = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&v, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return DM_ERR_OOM;
  }
  s->allocations.push_back(v);
  *p = (T *)v;
  return DM_OK;
}

template <class T>
dm_status upload(dm_system *s, T **p, const std::vector<T> &h) {
  dm_status st = dalloc(s, p, h.size());
  if (st != DM_OK) return st;
  if (!h.empty()) DM_CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DM_OK;
}

#define DM_TRY(x)                 \
  do {                            \
    dm_status st_ = (x);          \
    if (st_ != DM_OK) return st_; \
  } while (0)

inline int blocks(int64_t n, int b) { return (int)((n + b - 1) / b); }

__global__ void k_gather_layout(int n, const int32_t *map, const double *src, double *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[map[i]];
}
__global__ void k_scatter_layout(int n, const int32_t *map, const double *src, double *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[map[i]] = src[i];
}
// layout -> DOF order summing the copies of a shared (joint) node
__global__ void k_scatter_add_layout(int n, const int32_t *map, const double *src, double *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(dst + map[i], src[i]);
}
// DOF -> layout order with a shared node's value in its first copy only
__global__ void k_gather_layout_first(int n, const int32_t *map, const uint8_t *first,
                                      const double *src, double *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = first[i] ? src[map[i]] : 0.0;
}
__global__ void k_scatter_kbar(int n, const int32_t *slot2st, int slot0, int ns,
                               const double *in, double *kbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int st = slot2st[slot0 + i];
  kbar[st] = in[2 * i];
  kbar[ns + st] = in[2 * i + 1];
}

enum {
  K_EDGE = 0, K_STENCIL = 1, K_ROWS = 2, K_SOLVE = 3, K_BEGIN = 4, K_COMMIT = 5,
  K_NODES = 6, K_ROWS_GEN = 7, K_ASM_GEN = 8, K_SOLVE_GEN = 9, K_WARM = 10,
  K_CONTACT = 11, K_SOLVE_CONTACT = 12, K_HESS = 13, K_BAND = 14, K_FUSED = 15,
  K_ROWS_FUSED = 16
};
const char *kKernelNames[DM_NUM_KERNELS] = {
    "edge_frames_stretch", "bend_twist_gradient", "residual_rows", "band_ldlt_solve",
    "step_begin",          "step_commit",        "ground_contact_friction", "residual_rows_general",
    "assemble_general",    "limb_schur_solve",   "learned_warm_start",
    "edge_contact_pairs",  "contact_band_lu",    "bend_twist_hessian", "jacobian_band_rows",
    "bend_twist_fused",    "residual_jacobian_rows"};

struct Extra {
  bool prof = false;
  cudaEvent_t ev[2 * DM_NUM_KERNELS] = {};
  bool ev_used[DM_NUM_KERNELS] = {};
  int64_t launches[DM_NUM_KERNELS] = {};
  double ms[DM_NUM_KERNELS] = {};
  unsigned long long *d_units = nullptr;
  int32_t *d_bad = nullptr;
  int32_t *d_sys_kind = nullptr;
  int32_t *ls_action = nullptr, *ls_trial = nullptr, *ls_nback = nullptr;
  double *ls_alpha = nullptr, *ls_racc = nullptr, *ls_qacc = nullptr, *ls_merit = nullptr;
  int n_rod_sys = 0;
  struct {
    int table = 0, pair_cap = 0, n_contact = 0;
    double inv_cell = 0.0;
    double *edge_h = nullptr, *fc = nullptr, *dense = nullptr;
    int32_t *edge_idx = nullptr, *contact_sys = nullptr, *sys_bw = nullptr;
    int32_t *bucket_count = nullptr, *bucket_start = nullptr, *bucket_fill = nullptr,
            *bucket_edges = nullptr, *pairs = nullptr, *npairs = nullptr;
    int32_t *cgo = nullptr, *cbad = nullptr;
    int64_t *sys_dense0 = nullptr;
    unsigned long long *edge_key = nullptr;
  } cc;  // edge-edge contact
  struct {
    double *buf = nullptr;   // [6][nd]: lambda, rhs, gq, gv, gq0, gv0 (DOF order)
    double *dk = nullptr;    // [22][Ns] curvature gradients
    double *gk = nullptr;    // [2][slots]
    double *stage = nullptr; // [n] layout staging
    char *scratch = nullptr; // banded-solve scratch
    double *gen2 = nullptr;  // transposed general-path storage
    uint8_t *first = nullptr; // first copy of each DOF in the layout
    int32_t *ints = nullptr; // bookkeeping of the transposed solve
    unsigned long long *res = nullptr;
  } adj;  // step adjoint (allocated on first use)
  struct {
    int nlnode = 0;
    int32_t *edge_lay = nullptr, *lnode_lay = nullptr, *lnode_ein = nullptr,
            *lnode_eout = nullptr, *layout2dof = nullptr;
    double *g = nullptr;
  } fchain;  // frame chain of rollout adjoints (allocated on first use)
  int n_fast = 0, n_slow = 0;   // general systems on the condensation / Schur path
  size_t border_smem = 0;
  int limb_nmax = 0, wpb_factor = 1, wpb_back = 1;  // limb kernels: rows, warps per block
  int asm_chunks = 0;  // assembly blocks per system (the largest system's targets)
  size_t smem_factor = 0, smem_back = 0;
  int solve_blocks = 1;
  size_t solve_smem = 0;
  int sms = 1;
  int wpb_factor_max = 1, wpb_back_max = 1;
  // launch shapes (dm_autotune): threads per block and work per thread of
  // the edge, stencil and row kernels; warps per block and blocks per SM of
  // the persistent rod solver
  struct {
    int edge_threads = 256, stencil_threads = 128, stencil_per_thread = 1, rows_threads = 256;
    int solve_warps = 4, solve_bps = 1;
  } tune;
  // Newton rounds as one CUDA graph: a device-side while loop over rounds
  bool graphs = true;
  bool fused_first = true;  // first round of a step: fused gradient+Hessian passes
  cudaStream_t cap_stream = nullptr;
  // a side branch of a round (the ground-contact node terms, independent of
  // the edge and stencil kernels), forked and joined by events
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t round_graph = nullptr;
  cudaGraphExec_t first_graph = nullptr;            // the fused first round of a step
  int64_t first_launches[DM_NUM_KERNELS] = {};
  bool graph_ws = false;  // learned warm start on when the graph was captured
  bool midpoint = false;  // implicit midpoint (p.dt holds dt/2)
  LongRods *longr = nullptr;  // single rods on the partitioned solve
  int64_t round_launches[DM_NUM_KERNELS] = {};  // launches of one captured round
  std::vector<int32_t> slot2st;
  int32_t *d_slot2st = nullptr;
  int32_t *d_dof_sys = nullptr;
  // rod tables of the row kernel: DOF -> rod (-1 on general systems), and
  // per rod its first DOF, DOF count, first stencil and first edge
  int32_t *d_dof_rod = nullptr, *d_rod_dof0 = nullptr, *d_rod_ndof = nullptr,
          *d_rod_st0 = nullptr, *d_rod_edge0 = nullptr;
  double *d_damp = nullptr;
  double *d_scratch = nullptr;  // layout-sized staging for state copies
  size_t scratch_n = 0;
};

}  // namespace

// Extra per-handle data lives next to the handle.
struct dm_system_ext : dm_system {
  Extra x;
};

// Persistent rod solver shape: `warps` warps of two rods each per block,
// `bps` blocks per SM, no more blocks than the batch needs.
static void set_solve_shape(dm_system_ext *s, int warps, int bps) {
  s->x.tune.solve_warps = warps;
  s->x.tune.solve_bps = bps;
  s->x.solve_smem = (size_t)warps * kSolveRodsPerWarp * kSolveRodDoubles * sizeof(double);
  const int rods_per_block = kSolveRodsPerWarp * warps;
  const int want = (s->x.n_rod_sys + rods_per_block - 1) / rods_per_block;
  s->x.solve_blocks = std::max(1, std::min(want, bps * s->x.sms));
}

static dm_status create_impl(const dm_system_desc *desc, const dm_params *prm,
                             dm_system_ext *s) {
  HostTopology &T = s->T;
  // implicit midpoint: every step-size-dependent quantity (inertia M/dt^2,
  // damping, friction velocity, residual scale, predictor) is built for the
  // backward-Euler solve over dt/2 in the midpoint configuration
  dm_params half;
  if (prm->integrator == 1) {
    half = *prm;
    half.dt = 0.5 * prm->dt;
    prm = &half;
    s->x.midpoint = true;
  } else if (prm->integrator != 0) {
    set_error("integrator must be 0 (backward Euler) or 1 (implicit midpoint)");
    return DM_ERR_INVALID_ARG;
  }
  if (prm->predictor != 0 && prm->predictor != 1) {
    set_error("predictor must be 0 (extrapolated) or 1 (length-projected)");
    return DM_ERR_INVALID_ARG;
  }
  if (!build_topology(desc, prm, T)) return DM_ERR_INVALID_ARG;
  if (prm->self_contact) {
    // edge-edge contact within single rods and contact groups (no joints),
    // on the ground or not
    if (prm->pair_mu < 0.0 || (prm->pair_mu > 0.0 && !(prm->slip_nu > 0.0))) {
      set_error("edge-edge friction needs pair_mu >= 0 and slip_nu > 0");
      return DM_ERR_INVALID_ARG;
    }
    if (!(prm->pair_kc > 0 && prm->delta > 0)) {
      set_error("edge-edge contact needs pair_kc > 0 and delta > 0");
      return DM_ERR_INVALID_ARG;
    }
    double dense = 0.0;
    for (int k = 0; k < T.n_systems; ++k) {
      if (T.sys_kind[k] != SOLVE_ROD_BAND && T.sys_kind[k] != SOLVE_CONTACT) {
        set_error("edge-edge contact is supported on single rods and contact groups of "
                  "rods without joints (system " + std::to_string(k) + " has joints)");
        return DM_ERR_INVALID_ARG;
      }
      T.sys_kind[k] = SOLVE_CONTACT;
      dense += (double)T.sys_ndof[k] * T.sys_ndof[k];
    }
    if (dense * 8.0 > 8e9) {
      set_error("edge-edge contact: the per-system matrices would exceed 8 GB");
      return DM_ERR_INVALID_ARG;
    }
  }
  if (prm->ground && !(prm->delta > 0 && prm->slip_nu > 0)) {
    set_error("ground contact needs delta > 0 and slip_nu > 0");
    return DM_ERR_INVALID_ARG;
  }
  s->prm = *prm;
  s->stream = (cudaStream_t)prm->stream;
  s->p.dt = prm->dt;
  s->p.tol = prm->newton_tol;
  s->p.max_iter = prm->max_iter;
  for (int c = 0; c < 3; ++c) s->p.g[c] = prm->gravity[c];
  s->p.eta = prm->damping;

  const int64_t nd = T.n_dofs, ne = T.n_edges, ns = T.n_stencils;
  const int S = T.n_systems;
  DevArrays &d = s->d;
  // DOF vectors
  DM_TRY(upload(s, &d.q, T.q0));
  DM_TRY(upload(s, &d.qn, T.q0));
  DM_TRY(upload(s, &d.vn, T.v0));
  DM_TRY(dalloc(s, &d.f, nd));
  DM_TRY(upload(s, &d.mass, T.dof_mass));
  DM_TRY(upload(s, &d.rscale, T.dof_rscale));
  DM_TRY(upload(s, &d.fixed, T.dof_fixed));
  std::vector<int32_t> dof_sys(nd);
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < T.sys_ndof[k]; ++i) dof_sys[T.sys_dof0[k] + i] = k;
  DM_TRY(upload(s, &s->x.d_dof_sys, dof_sys));
  std::vector<double> damp(nd, 0.0);
  for (int64_t v = 0; v < T.n_nodes; ++v)
    for (int c = 0; c < 3; ++c) damp[T.node_dof[v] + c] = prm->damping * T.node_vor[v] / prm->dt;
  DM_TRY(upload(s, &s->x.d_damp, damp));
  // edges
  std::vector<int32_t> ea(ne), eb(ne);
  for (int64_t e = 0; e < ne; ++e) {
    ea[e] = T.node_dof[T.edge_a[e]];
    eb[e] = T.node_dof[T.edge_b[e]];
  }
  DM_TRY(upload(s, &d.edge_a, ea));
  DM_TRY(upload(s, &d.edge_b, eb));
  DM_TRY(upload(s, &d.edge_th, T.edge_thdof));
  DM_TRY(upload(s, &d.edge_sys, T.edge_sys));
  {
    std::vector<double> il(T.edge_lbar.size());
    for (size_t e = 0; e < il.size(); ++e) il[e] = 1.0 / T.edge_lbar[e];
    DM_TRY(upload(s, &d.edge_ilbar, il));
  }
  DM_TRY(upload(s, &d.edge_EA, T.edge_EA));
  std::vector<double> soa(3 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 3; ++c) soa[c * ne + e] = T.d1_init[3 * e + c];
  DM_TRY(upload(s, &d.d1n, soa));
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 3; ++c) soa[c * ne + e] = T.t_init[3 * e + c];
  DM_TRY(upload(s, &d.tn, soa));
  DM_TRY(dalloc(s, &d.ef, 13 * ne));
  DM_TRY(dalloc(s, &d.es, 9 * ne));
  // stencils
  std::vector<int32_t> sted(2 * ns), stth(2 * ns), stsg(ns);
  for (int64_t k = 0; k < ns; ++k) {
    sted[k] = T.st_edge[0][k];
    sted[ns + k] = T.st_edge[1][k];
    stth[k] = T.edge_thdof[T.st_edge[0][k]];
    stth[ns + k] = T.edge_thdof[T.st_edge[1][k]];
    stsg[k] = (T.st_sign[0][k] < 0 ? 1 : 0) | (T.st_sign[1][k] < 0 ? 2 : 0);
  }
  {
    std::vector<int32_t> stnd(3 * ns);
    for (int64_t k = 0; k < ns; ++k)
      for (int n3 = 0; n3 < 3; ++n3) stnd[n3 * ns + k] = T.node_dof[T.st_node[n3][k]];
    DM_TRY(upload(s, &d.st_nd, stnd));
  }
  DM_TRY(upload(s, &d.st_ed, sted));
  DM_TRY(upload(s, &d.st_th, stth));
  DM_TRY(upload(s, &d.st_sg, stsg));
  DM_TRY(upload(s, &d.st_sys, T.st_sys));
  DM_TRY(upload(s, &d.st_kb, T.st_kb));
  DM_TRY(upload(s, &d.st_kt, T.st_kt));
  std::vector<double> kb2(2 * ns);
  for (int64_t k = 0; k < ns; ++k) {
    kb2[k] = T.st_kbar1[k];
    kb2[ns + k] = T.st_kbar2[k];
  }
  DM_TRY(upload(s, &d.kbar, kb2));
  DM_TRY(upload(s, &d.taubar, T.st_taubar));
  DM_TRY(upload(s, &d.beta_n, T.st_beta0));
  DM_TRY(dalloc(s, &d.beta_it, ns));
  DM_TRY(dalloc(s, &d.sg, 11 * ns));
  DM_TRY(dalloc(s, &d.sh, 66 * ns));
  // systems
  DM_TRY(upload(s, &d.sys_dof0, T.sys_dof0));
  DM_TRY(upload(s, &d.sys_ndof, T.sys_ndof));
  DM_TRY(upload(s, &d.sys_st0, T.sys_st0));
  DM_TRY(upload(s, &d.sys_edge0, T.sys_edge0));
  DM_TRY(dalloc(s, &d.sys_active, S));
  DM_TRY(dalloc(s, &d.sys_iters, S));
  DM_TRY(dalloc(s, &d.sys_status, S));
  DM_TRY(dalloc(s, &d.sys_res, S));
  DM_TRY(dalloc(s, &d.ctrl, 8));  // [4] = Newton rounds of the step
  DM_TRY(dalloc(s, &d.band, 11 * nd));
  DM_TRY(dalloc(s, &d.dq, nd));
  std::vector<int32_t> order, longsys;
  const int long_min = prm->long_rod_dofs == 0 ? 2048 : prm->long_rod_dofs;
  for (int k = 0; k < S; ++k)
    if (T.sys_kind[k] == SOLVE_ROD_BAND) {
      if (long_min > 0 && T.sys_ndof[k] >= long_min) longsys.push_back(k);
      else order.push_back(k);
    }
  DM_TRY(long_rods_create(s, longsys, 512, &s->x.longr));
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return T.sys_ndof[a] > T.sys_ndof[b]; });
  s->x.n_rod_sys = (int)order.size();
  DM_TRY(upload(s, &d.solve_order, order));
  DM_TRY(upload(s, &s->x.d_sys_kind, T.sys_kind));
  if (prm->self_contact) {
    auto &c = s->x.cc;
    std::vector<int32_t> eidx(ne), csys;
    // edge index with a gap of three between rods, so that |eidx_e - eidx_f|
    // <= 2 holds exactly for two edges of one rod at most two apart (the
    // excluded pairs of reading C16); edges of different rods never match
    for (int r = 0; r < T.n_rods; ++r)
      for (int64_t e = T.rod_edge0[r]; e < T.rod_edge0[r + 1]; ++e) eidx[e] = (int32_t)(e + 3 * r);
    std::vector<int64_t> dense0(S, 0);
    int64_t tot = 0;
    for (int k = 0; k < S; ++k) {
      dense0[k] = tot;
      tot += (int64_t)T.sys_ndof[k] * T.sys_ndof[k];
      csys.push_back(k);
    }
    double lmax = 0.0, hmax = 0.0;
    for (int64_t e = 0; e < ne; ++e) {
      lmax = std::max(lmax, T.edge_lbar[e]);
      hmax = std::max(hmax, T.edge_h[e]);
    }
    int tsize = 1024;
    while (tsize < 2 * ne && tsize < (1 << 22)) tsize <<= 1;
    c.table = tsize;
    c.pair_cap = (int)std::min<int64_t>(64 * std::max<int64_t>(ne, 16), 1 << 24);
    c.inv_cell = 1.0 / (1.5 * lmax + 2.0 * hmax + prm->delta);
    c.n_contact = S;
    DM_TRY(upload(s, &c.edge_h, T.edge_h));
    DM_TRY(upload(s, &c.edge_idx, eidx));
    DM_TRY(upload(s, &c.contact_sys, csys));
    DM_TRY(upload(s, &c.sys_dense0, dense0));
    DM_TRY(dalloc(s, &c.edge_key, ne));
    DM_TRY(dalloc(s, &c.bucket_count, tsize));
    DM_TRY(dalloc(s, &c.bucket_start, tsize + 1));
    DM_TRY(dalloc(s, &c.bucket_fill, tsize));
    DM_TRY(dalloc(s, &c.bucket_edges, ne));
    DM_TRY(dalloc(s, &c.pairs, 2 * (int64_t)c.pair_cap));
    DM_TRY(dalloc(s, &c.npairs, 1));
    DM_TRY(dalloc(s, &c.fc, nd));
    DM_TRY(dalloc(s, &c.dense, tot));
    DM_TRY(dalloc(s, &c.sys_bw, S));
    DM_TRY(dalloc(s, &c.cgo, S));
    DM_TRY(dalloc(s, &c.cbad, S));
    DM_CK(cudaMemset(c.dense, 0, tot * sizeof(double)));
    DM_CK(cudaMemset(c.npairs, 0, sizeof(int32_t)));
    std::vector<int32_t> bw10(S, 10);
    DM_CK(cudaMemcpy(c.sys_bw, bw10.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  if (prm->line_search) {
    DM_TRY(dalloc(s, &s->x.ls_action, S));
    DM_TRY(dalloc(s, &s->x.ls_trial, S));
    DM_TRY(dalloc(s, &s->x.ls_nback, S));
    DM_TRY(dalloc(s, &s->x.ls_alpha, S));
    DM_TRY(dalloc(s, &s->x.ls_racc, S));
    DM_TRY(dalloc(s, &s->x.ls_merit, S));
    DM_TRY(dalloc(s, &s->x.ls_qacc, nd));
  }
  // general path
  DM_TRY(upload(s, &d.dof_node, T.dof_node));
  DM_TRY(upload(s, &d.dof_comp, T.dof_comp));
  {
    std::vector<double> dc(nd);
    for (int64_t i = 0; i < nd; ++i)
      dc[i] = T.dof_fixed[i] ? 1.0 : T.dof_mass[i] / (prm->dt * prm->dt) + damp[i];
    DM_TRY(upload(s, &d.dconst, dc));
  }
  if (T.any_general || T.ground) {
    // node tables and node terms (ground contact and friction, k_nodes)
    std::vector<int32_t> ndof_arr(T.n_nodes);
    for (int64_t v = 0; v < T.n_nodes; ++v) ndof_arr[v] = T.node_dof[v];
    DM_TRY(upload(s, &d.node_dof_arr, ndof_arr));
    DM_TRY(upload(s, &d.node_sys, T.node_sys));
    DM_TRY(upload(s, &d.node_h, T.node_h));
    DM_TRY(upload(s, &d.node_mu, T.node_mu));
    DM_TRY(upload(s, &d.node_kc, T.node_kc));
    DM_TRY(dalloc(s, &d.nt, 12 * T.n_nodes));
    DM_CK(cudaMemset(d.nt, 0, 12 * T.n_nodes * sizeof(double)));
  }
  if (T.any_general) {
    DM_TRY(dalloc(s, &d.gen, T.gen_doubles));
    // entries no assembly targets stay zero: the condensation path factors
    // out of place (the other path's systems are cleared every round)
    DM_CK(cudaMemset(d.gen, 0, std::max<int64_t>(T.gen_doubles, 1) * sizeof(double)));
    DM_TRY(upload(s, &d.gen_sys, T.gen_sys));
    DM_TRY(upload(s, &d.gs_limb0, T.gs_limb0));
    DM_TRY(upload(s, &d.gs_nlimb, T.gs_nlimb));
    DM_TRY(upload(s, &d.gs_nB, T.gs_nB));
    DM_TRY(upload(s, &d.gs_border0, T.gs_border0));
    DM_TRY(upload(s, &d.gs_JBB, T.gs_JBB));
    DM_TRY(upload(s, &d.gs_rB, T.gs_rB));
    DM_TRY(upload(s, &d.gs_S, T.gs_S));
    DM_TRY(upload(s, &d.gs_xB, T.gs_xB));
    DM_TRY(upload(s, &d.gs_mat0, T.gs_mat0));
    DM_TRY(upload(s, &d.gs_mat1, T.gs_mat1));
    DM_TRY(upload(s, &d.lb_dof0, T.lb_dof0));
    DM_TRY(upload(s, &d.lb_n, T.lb_n));
    DM_TRY(upload(s, &d.lb_ncr, T.lb_ncr));
    DM_TRY(upload(s, &d.lb_cr0, T.lb_cr0));
    DM_TRY(upload(s, &d.lb_band, T.lb_band));
    DM_TRY(upload(s, &d.lb_piv, T.lb_piv));
    DM_TRY(upload(s, &d.lb_C, T.lb_C));
    DM_TRY(upload(s, &d.lb_R, T.lb_R));
    DM_TRY(upload(s, &d.lb_Y, T.lb_Y));
    DM_TRY(upload(s, &d.lb_y, T.lb_y));
    DM_TRY(upload(s, &d.border_dof, T.border_dof));
    DM_TRY(upload(s, &d.coupled_rows, T.coupled_rows));
    DM_TRY(upload(s, &d.gs_fast, T.gs_fast));
    DM_TRY(upload(s, &d.lb_gsys, T.lb_gsys));
    DM_TRY(upload(s, &d.lb_dir, T.lb_dir));
    DM_TRY(upload(s, &d.lb_m, T.lb_m));
    DM_TRY(upload(s, &d.lb_nbc, T.lb_nbc));
    DM_TRY(upload(s, &d.lb_bc0, T.lb_bc0));
    DM_TRY(upload(s, &d.lb_bcols, T.lb_bcols));
    DM_TRY(dalloc(s, &d.gen_go, T.gen_sys.size()));
    DM_TRY(dalloc(s, &d.gen_bad, T.gen_sys.size()));
    DM_CK(cudaMemset(d.gen_bad, 0, T.gen_sys.size() * sizeof(int32_t)));
    for (size_t w = 0; w < T.gen_sys.size(); ++w) {
      if (T.gs_fast[w]) {
        s->x.n_fast++;
        s->x.border_smem = std::max<size_t>(
            s->x.border_smem, (size_t)(T.gs_nB[w] * (T.gs_nB[w] + 4)) * sizeof(double));
      } else {
        s->x.n_slow++;
      }
    }
    if (s->x.border_smem > 48 * 1024)
      DM_CK(cudaFuncSetAttribute(k_gen_border, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s->x.border_smem));
    for (size_t L = 0; L < T.lb_n.size(); ++L)
      if (T.gs_fast[T.lb_gsys[L]]) s->x.limb_nmax = std::max(s->x.limb_nmax, T.lb_n[L]);
    {
      // warps per block: up to 4, within 200 KB of shared memory per block
      const size_t pf = gen_factor_smem(s->x.limb_nmax) * sizeof(double);
      const size_t pb = gen_back_smem(s->x.limb_nmax) * sizeof(double);
      s->x.wpb_factor = (int)std::max<size_t>(1, std::min<size_t>(4, (200 << 10) / pf));
      s->x.wpb_back = (int)std::max<size_t>(1, std::min<size_t>(4, (200 << 10) / pb));
      s->x.wpb_factor_max = s->x.wpb_factor;
      s->x.wpb_back_max = s->x.wpb_back;
      s->x.smem_factor = pf * s->x.wpb_factor;
      s->x.smem_back = pb * s->x.wpb_back;
      DM_CK(cudaFuncSetAttribute(k_gen_limb_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s->x.smem_factor));
      DM_CK(cudaFuncSetAttribute(k_gen_limb_back, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s->x.smem_back));
    }
    DM_TRY(upload(s, &d.asm_target, T.asm_target));
    DM_TRY(upload(s, &d.asm_sys, T.asm_sys));
    DM_TRY(upload(s, &d.asm_t0, T.asm_t0));
    for (size_t w = 0; w + 1 < T.asm_t0.size(); ++w)
      s->x.asm_chunks = std::max(s->x.asm_chunks, (T.asm_t0[w + 1] - T.asm_t0[w] + kAsmPerBlock - 1) /
                                                      kAsmPerBlock);
    DM_TRY(upload(s, &d.asm_ptr, T.asm_ptr));
    DM_TRY(upload(s, &d.asm_src, T.asm_src));
    DM_TRY(upload(s, &d.gat_ptr, T.gat_ptr));
    DM_TRY(upload(s, &d.gat_ent, T.gat_ent));
  }
  DM_TRY(upload(s, &d.layout2dof, T.layout2dof));
  // natural-curvature slots -> stencils
  int64_t nslots = 0;
  for (int r = 0; r < T.n_rods; ++r) nslots += T.npr[r] - 2;
  s->x.slot2st.assign(std::max<int64_t>(nslots, 1), 0);
  for (int64_t k = 0; k < ns; ++k)
    if (T.st_rod_slot[k] >= 0) s->x.slot2st[T.st_rod_slot[k]] = (int32_t)k;
  DM_TRY(upload(s, &s->x.d_slot2st, s->x.slot2st));
  {
    const int R = T.n_rods;
    std::vector<int32_t> dof_rod(std::max<int64_t>(T.n_dofs, 1), -1), rd0(R), rnd(R), rst0(R),
        re0(R);
    int64_t k0 = 0;
    for (int r = 0; r < R; ++r) {
      const int N = T.npr[r];
      rd0[r] = T.node_dof[T.flat2node[T.rod_node0[r]]];
      rnd[r] = 4 * N - 1;
      rst0[r] = N > 2 ? s->x.slot2st[k0] : 0;
      re0[r] = (int32_t)T.rod_edge0[r];
      k0 += N - 2;
      const int sys = T.edge_sys[T.rod_edge0[r]];
      if (T.sys_kind[sys] != SOLVE_GENERAL)
        for (int k = 0; k < 4 * N - 1; ++k) dof_rod[rd0[r] + k] = r;
    }
    DM_TRY(upload(s, &s->x.d_dof_rod, dof_rod));
    DM_TRY(upload(s, &s->x.d_rod_dof0, rd0));
    DM_TRY(upload(s, &s->x.d_rod_ndof, rnd));
    DM_TRY(upload(s, &s->x.d_rod_st0, rst0));
    DM_TRY(upload(s, &s->x.d_rod_edge0, re0));
  }
  // staging of q and qdot together (state copies), or of natural curvatures
  s->x.scratch_n = std::max<size_t>({2 * (size_t)T.layout2dof.size(), (size_t)(2 * nslots), (size_t)1});
  DM_TRY(dalloc(s, &s->x.d_scratch, s->x.scratch_n));
  DM_TRY(dalloc(s, &s->x.d_units, DM_NUM_KERNELS));
  DM_CK(cudaMemset(s->x.d_units, 0, DM_NUM_KERNELS * sizeof(unsigned long long)));
  DM_TRY(dalloc(s, &s->x.d_bad, 1));
  for (int k = 0; k < 2 * DM_NUM_KERNELS; ++k) DM_CK(cudaEventCreate(&s->x.ev[k]));
  DM_CK(cudaMallocHost(&s->h_ctrl, 8 * sizeof(int32_t)));
  // persistent banded solver: 8 rods per 128-thread block, enough blocks
  // to cover the batch but no more than fit at once
  s->x.solve_smem = 4 * kSolveRodsPerWarp * kSolveRodDoubles * sizeof(double);  // 4 warps
  DM_CK(cudaFuncSetAttribute(k_solve_rod, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s->x.solve_smem));
  {
    int dev = 0, sms = 0, per_sm = 0;
    DM_CK(cudaGetDevice(&dev));
    DM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_rod, 128,
                                                        s->x.solve_smem));
    // persistent: one block of four warps per SM, so that each SM partition
    // runs one warp; the warps take rod pairs from the size-sorted queue
    // (largest first), which balances the FP64 work across partitions
    s->x.sms = sms;
    set_solve_shape(s, 4, 1);
  }
  DM_CK(cudaDeviceSynchronize());
  return DM_OK;
}

// Event bracket around one kernel launch when profiling is on.
struct Timed {
  dm_system_ext *s;
  int id;
  cudaStream_t st;
  Timed(dm_system_ext *s_, int id_, cudaStream_t st_) : s(s_), id(id_), st(st_) {
    s->x.launches[id]++;
    if (s->x.prof) cudaEventRecord(s->x.ev[2 * id], st);
  }
  ~Timed() {
    if (s->x.prof) {
      cudaEventRecord(s->x.ev[2 * id + 1], st);
      s->x.ev_used[id] = true;
    }
  }
};

// Adds the elapsed time of the event pairs recorded since the last call
// (the stream has been synchronised).
static void harvest(dm_system_ext *s) {
  if (!s->x.prof) return;
  for (int k = 0; k < DM_NUM_KERNELS; ++k)
    if (s->x.ev_used[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s->x.ev[2 * k], s->x.ev[2 * k + 1]) == cudaSuccess)
        s->x.ms[k] += ms;
      s->x.ev_used[k] = false;
    }
}

extern "C" {

const char *dm_last_error(void) { return dm::g_err.c_str(); }

dm_status dm_create_system(const dm_system_desc *desc, const dm_params *params,
                           dm_system **out) {
  if (!out) {
    set_error("out is NULL");
    return DM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  set_error("");
  dm_system_ext *s = new (std::nothrow) dm_system_ext();
  if (!s) {
    set_error("host allocation failed");
    return DM_ERR_OOM;
  }
  dm_status st;
  try {
    st = create_impl(desc, params, s);
  } catch (const std::exception &ex) {
    set_error(std::string("host exception: ") + ex.what());
    st = DM_ERR_OOM;
  }
  if (st != DM_OK) {
    std::string keep = dm::g_err;
    dm_destroy(s);
    set_error(keep);
    return st;
  }
  *out = s;
  return DM_OK;
}

void dm_destroy(dm_system *sys) {
  if (!sys) return;
  for (void *p : sys->allocations) cudaFree(p);
  auto *sx = static_cast<dm_system_ext *>(sys);
  for (int k = 0; k < 2 * DM_NUM_KERNELS; ++k)
    if (sx->x.ev[k]) cudaEventDestroy(sx->x.ev[k]);
  if (sys->h_ctrl) cudaFreeHost(sys->h_ctrl);
  if (sx->x.round_graph) cudaGraphExecDestroy(sx->x.round_graph);
  if (sx->x.first_graph) cudaGraphExecDestroy(sx->x.first_graph);
  long_rods_free(sx->x.longr);
  if (sx->x.cap_stream) cudaStreamDestroy(sx->x.cap_stream);
  if (sx->x.side_stream) cudaStreamDestroy(sx->x.side_stream);
  if (sx->x.ev_fork) cudaEventDestroy(sx->x.ev_fork);
  if (sx->x.ev_join) cudaEventDestroy(sx->x.ev_join);
  dm::ws_free(sys->ws);
  delete static_cast<dm_system_ext *>(sys);
}

int64_t dm_state_size(const dm_system *s) { return s ? (int64_t)s->T.layout2dof.size() : 0; }
int32_t dm_num_systems(const dm_system *s) { return s ? s->T.n_systems : 0; }
int64_t dm_num_stencils(const dm_system *s) { return s ? s->T.n_stencils : 0; }
int64_t dm_num_edges(const dm_system *s) { return s ? s->T.n_edges : 0; }

dm_status dm_set_natural_curvature(dm_system *sys, int32_t rod_begin, int32_t rod_end,
                                   const double *kbar, int32_t is_device) {
  if (!sys || !kbar || rod_begin < 0 || rod_end > sys->T.n_rods || rod_begin > rod_end) {
    set_error("dm_set_natural_curvature: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  const HostTopology &T = s->T;
  int64_t slot0 = 0, n = 0;
  for (int r = 0; r < rod_begin; ++r) slot0 += T.npr[r] - 2;
  for (int r = rod_begin; r < rod_end; ++r) n += T.npr[r] - 2;
  if (n == 0) return DM_OK;
  const double *src = kbar;
  if (!is_device) {
    DM_CK(cudaMemcpyAsync(s->x.d_scratch, kbar, 2 * n * sizeof(double),
                          cudaMemcpyHostToDevice, s->stream));
    src = s->x.d_scratch;
  }
  k_scatter_kbar<<<blocks(n, 256), 256, 0, s->stream>>>((int)n, s->x.d_slot2st, (int)slot0,
                                                        (int)T.n_stencils, src, s->d.kbar);
  DM_CK(cudaGetLastError());
  if (!is_device) DM_CK(cudaStreamSynchronize(s->stream));  // host buffer reusable
  return DM_OK;
}

dm_status dm_step(dm_system *sys, int32_t nsteps, dm_step_stats *stats) {
  if (!sys || nsteps < 0) {
    set_error("dm_step: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  const HostTopology &T = s->T;
  DevArrays &d = s->d;
  cudaStream_t st = s->stream;
  const int nd = (int)T.n_dofs, ne = (int)T.n_edges, ns = (int)T.n_stencils, S = T.n_systems;
  StepArgs sa{nd, ne, ns, S, s->p.dt, d.q, d.qn, d.vn, d.d1n, d.tn, d.beta_n, d.ef, d.beta_it,
              d.fixed, d.sys_active, d.sys_iters, d.sys_status, d.sys_res};
  EdgeArgs ea{ne, d.q, d.edge_a, d.edge_b, d.edge_th, d.edge_sys, d.edge_EA, d.edge_ilbar,
              d.tn, d.d1n, d.sys_active, d.sys_status, d.ef, d.es,
              s->x.prof ? s->x.d_units + K_EDGE : nullptr};
  StencilArgs ka{ns, ne, d.q, d.ef, d.tn, d.st_ed, d.st_th, d.st_sg, d.st_sys, d.st_kb, d.st_kt,
                 d.kbar, d.taubar, d.beta_n, d.sys_active, d.sys_status, d.beta_it, d.sg, d.sh,
                 s->x.prof ? s->x.d_units + K_STENCIL : nullptr};
  const bool contact_on = s->x.cc.n_contact > 0;
  ContactArgs ca{};
  if (contact_on) {
    auto &c = s->x.cc;
    ca.ne = ne; ca.nd = nd; ca.nsys = S; ca.table_mask = c.table - 1; ca.pair_cap = c.pair_cap;
    ca.inv_cell = c.inv_cell; ca.delta = s->prm.delta; ca.kc = s->prm.pair_kc;
    ca.mu = s->prm.pair_mu; ca.K2 = s->prm.pair_mu > 0 ? 15.0 / s->prm.slip_nu : 0.0;
    ca.dt = s->p.dt;
    ca.q = d.q; ca.qn = d.qn; ca.edge_h = c.edge_h; ca.band = d.band;
    ca.edge_a = d.edge_a; ca.edge_b = d.edge_b; ca.edge_sys = d.edge_sys; ca.edge_idx = c.edge_idx;
    ca.sys_kind = s->x.d_sys_kind; ca.sys_active = d.sys_active; ca.dof_sys = s->x.d_dof_sys;
    ca.sys_dof0 = d.sys_dof0; ca.sys_ndof = d.sys_ndof; ca.contact_sys = c.contact_sys;
    ca.ls_action = s->prm.line_search ? s->x.ls_action : nullptr;
    ca.fixed = d.fixed; ca.sys_dense0 = c.sys_dense0; ca.sys_status = d.sys_status;
    ca.sys_bw = c.sys_bw; ca.edge_key = c.edge_key; ca.bucket_count = c.bucket_count;
    ca.bucket_start = c.bucket_start; ca.bucket_fill = c.bucket_fill;
    ca.bucket_edges = c.bucket_edges; ca.pairs = c.pairs; ca.npairs = c.npairs;
    ca.fc = c.fc; ca.dense = c.dense;
    ca.n_contact = c.n_contact; ca.cgo = c.cgo; ca.cbad = c.cbad;
    ca.nn = (int)T.n_nodes;
    ca.lu_flops = s->x.prof ? s->x.d_units + K_SOLVE_CONTACT : nullptr;
  }
  // the Jacobian passes test convergence as the solvers do
  const int32_t *ls_act = s->prm.line_search ? s->x.ls_action : nullptr;
  ka.sys_res = d.sys_res;
  ka.tol = s->p.tol;
  ka.ls_action = ls_act;
  RowArgs ra{};
  ra.sys_status = d.sys_status;
  ra.tol = s->p.tol;
  ra.ls_action = ls_act;
  ra.fc = contact_on ? s->x.cc.fc : nullptr;
  ra.nd = nd; ra.ns = ns; ra.ne = ne; ra.dt = s->p.dt; ra.idt = 1.0 / s->p.dt;
  for (int c = 0; c < 3; ++c) ra.g[c] = s->p.g[c];
  ra.eta = s->p.eta;
  ra.q = d.q; ra.qn = d.qn; ra.vn = d.vn; ra.mass = d.mass; ra.rscale = d.rscale;
  ra.damp = s->x.d_damp; ra.fixed = d.fixed; ra.dof_sys = s->x.d_dof_sys;
  ra.dof_rod = s->x.d_dof_rod; ra.rod_dof0 = s->x.d_rod_dof0; ra.rod_ndof = s->x.d_rod_ndof;
  ra.rod_st0 = s->x.d_rod_st0; ra.rod_edge0 = s->x.d_rod_edge0;
  ra.sys_active = d.sys_active; ra.sys_kind = s->x.d_sys_kind;
  ra.sg = d.sg; ra.sh = d.sh; ra.es = d.es; ra.f = d.f; ra.band = d.band; ra.sys_res = d.sys_res;
  ra.units = s->x.prof ? s->x.d_units + K_ROWS : nullptr;
  SolveArgs va{s->x.n_rod_sys, nd, s->p.tol, s->p.max_iter, d.solve_order, d.sys_dof0, d.sys_ndof, d.fixed, d.f,
               d.band, d.q, d.dq, d.sys_active, d.sys_iters, d.sys_status, d.sys_res, d.ctrl,
               s->x.prof ? s->x.d_units + K_SOLVE : nullptr, s->x.ls_action, s->x.ls_trial};
  const int nn = (int)T.n_nodes;
  NodeArgs na{nn, s->p.dt, s->prm.ground_z, s->prm.delta, s->prm.slip_nu, d.q, d.qn,
              d.node_dof_arr, d.node_sys, d.node_h, d.node_mu, d.node_kc, d.sys_active, d.nt,
              s->x.prof ? s->x.d_units + K_NODES : nullptr};
  RowGenArgs rg{};
  rg.units = s->x.prof ? s->x.d_units + K_ROWS_GEN : nullptr;
  rg.nd = nd; rg.ns = ns; rg.ne = ne; rg.nn = nn; rg.dt = s->p.dt; rg.idt = 1.0 / s->p.dt;
  for (int c = 0; c < 3; ++c) rg.g[c] = s->p.g[c];
  rg.q = d.q; rg.qn = d.qn; rg.vn = d.vn; rg.mass = d.mass; rg.rscale = d.rscale;
  rg.damp = s->x.d_damp; rg.fixed = d.fixed; rg.dof_sys = s->x.d_dof_sys; rg.dof_node = d.dof_node;
  rg.dof_comp = d.dof_comp; rg.sys_kind = s->x.d_sys_kind; rg.sys_active = d.sys_active;
  rg.gat_ptr = d.gat_ptr; rg.gat_ent = d.gat_ent; rg.sg = d.sg; rg.es = d.es;
  rg.nt = T.ground ? d.nt : nullptr; rg.f = d.f; rg.sys_res = d.sys_res;
  const bool ls_on = s->prm.line_search != 0;
  AsmArgs aa{(int)T.asm_target.size(), d.asm_target, d.asm_ptr, d.asm_src, d.sh, d.es, d.nt,
             d.dconst, d.gen, d.asm_sys, d.sys_active, ls_on ? s->x.ls_action : nullptr,
             (int)T.gen_sys.size(), d.gen_sys, d.asm_t0, d.gs_mat0, d.gs_mat1, d.sys_ndof,
             s->x.prof ? s->x.d_units + K_ASM_GEN : nullptr};
  SolveGenArgs ga{};
  ga.ngen = (int)T.gen_sys.size(); ga.max_iter = s->p.max_iter; ga.tol = s->p.tol;
  ga.gen_sys = d.gen_sys; ga.gs_limb0 = d.gs_limb0; ga.gs_nlimb = d.gs_nlimb; ga.gs_nB = d.gs_nB;
  ga.gs_border0 = d.gs_border0; ga.gs_JBB = d.gs_JBB; ga.gs_rB = d.gs_rB; ga.gs_S = d.gs_S;
  ga.gs_xB = d.gs_xB; ga.lb_dof0 = d.lb_dof0; ga.lb_n = d.lb_n; ga.lb_ncr = d.lb_ncr;
  ga.lb_cr0 = d.lb_cr0; ga.lb_band = d.lb_band; ga.lb_piv = d.lb_piv; ga.lb_C = d.lb_C; ga.lb_R = d.lb_R;
  ga.lb_Y = d.lb_Y; ga.lb_y = d.lb_y; ga.border_dof = d.border_dof;
  ga.coupled_rows = d.coupled_rows; ga.f = d.f; ga.gen = d.gen; ga.q = d.q;
  ga.sys_active = d.sys_active; ga.sys_iters = d.sys_iters; ga.sys_status = d.sys_status;
  ga.sys_res = d.sys_res; ga.ctrl = d.ctrl;
  ga.units = s->x.prof ? s->x.d_units + K_SOLVE_GEN : nullptr;
  ga.ls_action = s->x.ls_action;
  ga.ls_trial = s->x.ls_trial;
  ga.nlimb = (int)T.lb_n.size();
  ga.limb_nmax = s->x.limb_nmax;
  ga.gs_fast = d.gs_fast; ga.lb_gsys = d.lb_gsys; ga.lb_dir = d.lb_dir; ga.lb_m = d.lb_m;
  ga.lb_nbc = d.lb_nbc; ga.lb_bc0 = d.lb_bc0; ga.lb_bcols = d.lb_bcols;
  ga.gen_go = d.gen_go; ga.gen_bad = d.gen_bad;
  LineSearchArgs la{S, nd, d.sys_active, s->x.d_dof_sys, d.sys_dof0, d.sys_ndof, d.f, d.rscale,
                    s->x.ls_action, s->x.ls_trial, s->x.ls_nback, s->x.ls_alpha, s->x.ls_racc,
                    s->x.ls_merit, d.q, s->x.ls_qacc, nullptr};
  // learned initial guess: with the line search it is tried against the
  // extrapolation (first round evaluates the extrapolation, the second the
  // learned guess, which is kept only if it lowers the merit)
  const bool ws_on = ws_active(s);
  const bool ws_trial = ws_on && ls_on;
  if (ws_trial) la.wstry = ws_trial_flags(s);
  const int max_rounds = ls_on ? 13 * (s->p.max_iter + 1) : s->p.max_iter + 1;
  const bool gen_on = T.any_general, rod_on = s->x.n_rod_sys > 0;
  const bool long_on = long_rods_count(s->x.longr) > 0;
  if (stats) {
    stats->first_failed = -1;
    stats->steps_done = 0;
    stats->sum_iterations = 0;
    stats->max_iterations = 0;
  }
  std::vector<int32_t> iters;
  // residual and Jacobian passes apart, except with rod networks; the first
  // round of a step, whose guess essentially never meets the tolerance, runs
  // the fused passes (without a learned guess, whose trial round may be
  // rejected)
  const bool split = !gen_on;
  const bool fuse_first = split && !ws_on && s->x.fused_first;
  // the node terms run beside the edge and stencil kernels (not while
  // profiling, whose events time each kernel alone)
  const bool fork_nodes = T.ground && !s->x.prof;
  if (fork_nodes && !s->x.side_stream) {
    DM_CK(cudaStreamCreateWithFlags(&s->x.side_stream, cudaStreamNonBlocking));
    DM_CK(cudaEventCreateWithFlags(&s->x.ev_fork, cudaEventDisableTiming));
    DM_CK(cudaEventCreateWithFlags(&s->x.ev_join, cudaEventDisableTiming));
  }
  // One Newton round: every phase's launches, in stream order on rs.
  auto round = [&](cudaStream_t rs, int it, bool first) -> dm_status {
    const bool sp = split && !first;
    k_reset_res<<<blocks(S, 256), 256, 0, rs>>>(0, S, d.sys_active, d.sys_res);
    s->x.launches[K_BEGIN]++;
    DM_CK(cudaMemsetAsync(d.ctrl, 0, sizeof(int32_t), rs));
    DM_CK(cudaMemsetAsync(d.ctrl + 3, 0, sizeof(int32_t), rs));
    if (fork_nodes) {
      DM_CK(cudaEventRecord(s->x.ev_fork, rs));
      DM_CK(cudaStreamWaitEvent(s->x.side_stream, s->x.ev_fork, 0));
      k_nodes<<<blocks(nn, 256), 256, 0, s->x.side_stream>>>(na);
      s->x.launches[K_NODES]++;
      DM_CK(cudaEventRecord(s->x.ev_join, s->x.side_stream));
    }
    {
      Timed t(s, K_EDGE, rs);
      const int tb = s->x.tune.edge_threads;
      k_edge<<<blocks(ne, tb), tb, 0, rs>>>(ea);
    }
    if (T.ground && !fork_nodes) {
      Timed t(s, K_NODES, rs);
      k_nodes<<<blocks(nn, 256), 256, 0, rs>>>(na);
    }
    // residual pass: reference twist and gradients, then the residual rows;
    // the Jacobian pass (stencil Hessians, band rows) below runs only for
    // systems whose residual is still above the tolerance.  Batches with rod
    // networks keep one fused pass: most of their many rounds carry systems
    // that iterate on, for which the split would only add work.
    const int st_tb = s->x.tune.stencil_threads;
    const int st_grid = blocks(ns, (int64_t)st_tb * s->x.tune.stencil_per_thread);
    if (ns > 0 && sp) {
      Timed t(s, K_STENCIL, rs);
      k_stencil_grad<<<st_grid, st_tb, 0, rs>>>(ka);
    } else if (ns > 0) {
      Timed t(s, K_FUSED, rs);
      StencilArgs kf = ka;
      kf.units = s->x.prof ? s->x.d_units + K_FUSED : nullptr;
      k_stencil<<<st_grid, st_tb, 0, rs>>>(kf);
    }
    if (fork_nodes) DM_CK(cudaStreamWaitEvent(rs, s->x.ev_join, 0));  // the node terms are in
    if (contact_on) {
      Timed t(s, K_CONTACT, rs);
      const auto &c = s->x.cc;
      DM_CK(cudaMemsetAsync(c.fc, 0, nd * sizeof(double), rs));
      DM_CK(cudaMemsetAsync(c.npairs, 0, sizeof(int32_t), rs));
      DM_CK(cudaMemsetAsync(c.bucket_count, 0, c.table * sizeof(int32_t), rs));
      k_cc_clear<<<blocks((int64_t)nd * 32, 256), 256, 0, rs>>>(ca);
      k_cc_reset_bw<<<blocks(S, 256), 256, 0, rs>>>(ca);
      k_cc_cells<<<blocks(ne, 256), 256, 0, rs>>>(ca);
      k_cc_scan<<<1, 1024, 0, rs>>>(ca);
      k_cc_fill<<<blocks(ne, 256), 256, 0, rs>>>(ca);
      k_cc_pairs<<<blocks(ne, 128), 128, 0, rs>>>(ca);
      k_cc_terms<<<blocks(c.pair_cap, 64), 64, 0, rs>>>(ca);
      if (T.ground) k_cc_ground<<<blocks(nn, 128), 128, 0, rs>>>(ca, na.node_dof, d.node_sys, d.nt);
    }
    const bool rows_on = rod_on || contact_on || long_on;
    if (rows_on && sp) {
      Timed t(s, K_ROWS, rs);
      const int tb = s->x.tune.rows_threads;
      k_rows_rod_res<<<blocks(nd, tb), tb, 0, rs>>>(ra);
    } else if (rows_on) {
      Timed t(s, K_ROWS_FUSED, rs);
      const int tb = s->x.tune.rows_threads;
      RowArgs rf = ra;
      rf.units = s->x.prof ? s->x.d_units + K_ROWS_FUSED : nullptr;
      k_rows_rod<<<blocks(nd, tb), tb, 0, rs>>>(rf);
    }
    if (gen_on) {
      Timed t(s, K_ROWS_GEN, rs);
      k_rows_gen<<<blocks(nd, 256), 256, 0, rs>>>(rg);
    }
    if (ls_on) {
      k_line_search<<<S, kLineSearchThreads, 0, rs>>>(la);
      if (ws_trial && it == 0) DM_CK(ws_inject(s, rs, s->x.ls_action, s->x.ls_trial));
    }
    if (sp && ns > 0) {
      Timed t(s, K_HESS, rs);
      StencilArgs kh = ka;
      kh.units = s->x.prof ? s->x.d_units + K_HESS : nullptr;
      k_stencil_hess<<<st_grid, st_tb, 0, rs>>>(kh);
    }
    if (sp && rows_on) {
      Timed t(s, K_BAND, rs);
      const int tb = s->x.tune.rows_threads;
      RowArgs rb = ra;
      rb.units = s->x.prof ? s->x.d_units + K_BAND : nullptr;
      k_rows_rod_band<<<blocks(nd, tb), tb, 0, rs>>>(rb);
    }
    if (rod_on) {
      {
        Timed t(s, K_SOLVE, rs);
        k_solve_rod<<<s->x.solve_blocks, 32 * s->x.tune.solve_warps, s->x.solve_smem, rs>>>(va);
      }
    }
    if (long_on) {
      Timed t(s, K_SOLVE, rs);
      DM_CK(long_rods_round(s->x.longr, va, rs));
    }
    if (contact_on) {
      Timed t(s, K_SOLVE_CONTACT, rs);
      k_cc_band<<<blocks(nd, 256), 256, 0, rs>>>(ca);
      const int nc = s->x.cc.n_contact;
      k_cc_decide<<<blocks(nc, 128), 128, 0, rs>>>(ca, va);
      for (int c = 0; c < nc; ++c) {
        const int n = T.sys_ndof[c];  // contact systems are systems 0..nc-1 in order
        for (int k = 0; k < n; k += kNB) {
          const int rest = n - k - std::min(kNB, n - k);
          k_lu_diag<<<1, 256, 0, rs>>>(ca, c, k);
          if (rest > 0) {
            k_lu_trsm<<<blocks(2 * rest, 32), 32, 0, rs>>>(ca, c, k);
            const int t = (rest + 63) / 64;
            k_lu_gemm<<<dim3(t, t), 256, 0, rs>>>(ca, c, k);
          }
        }
      }
      k_cc_subst<<<nc, 1024, 0, rs>>>(ca, va);
    }
    if (gen_on) {
      {
        Timed t(s, K_ASM_GEN, rs);
        if (s->x.n_slow) k_gen_clear_slow<<<aa.ngen, 256, 0, rs>>>(aa, d.gs_fast);
        if (s->x.asm_chunks > 0)
          k_assemble_gen<<<dim3(aa.ngen, s->x.asm_chunks), 256, 0, rs>>>(aa);
      }
      {
        Timed t(s, K_SOLVE_GEN, rs);
        if (s->x.n_fast) {
          const int wf = s->x.wpb_factor, wb = s->x.wpb_back;
          const size_t sf = s->x.smem_factor / s->x.wpb_factor_max * wf;
          const size_t sb = s->x.smem_back / s->x.wpb_back_max * wb;
          if (ga.nlimb)
            k_gen_limb_factor<<<(ga.nlimb + wf - 1) / wf, 32 * wf, sf, rs>>>(ga);
          k_gen_border<<<ga.ngen, kGenBorderThreads, s->x.border_smem, rs>>>(ga);
          if (ga.nlimb)
            k_gen_limb_back<<<(ga.nlimb + wb - 1) / wb, 32 * wb, sb, rs>>>(ga);
        }
        if (s->x.n_slow)
          k_solve_gen<<<blocks((int64_t)ga.ngen * 32, 128), 128, 0, rs>>>(ga);
      }
    }
    if (ws_on && !ws_trial) DM_CK(ws_fallback(s, rs, s->x.d_dof_sys));
    DM_CK(cudaGetLastError());
    return DM_OK;
  };
  // Rounds as a CUDA graph (no host round trip between rounds): one while
  // node whose body is a round followed by k_round_continue.  The learned
  // guess's trial round (the first, with the injection) runs before the
  // graph; per-kernel profiling uses the host-driven loop.
  const bool graph_mode = s->x.graphs && !s->x.prof;
  if (s->x.round_graph && s->x.graph_ws != ws_on) {  // the round's kernels changed
    cudaGraphExecDestroy(s->x.round_graph);
    s->x.round_graph = nullptr;
    if (s->x.first_graph) cudaGraphExecDestroy(s->x.first_graph);
    s->x.first_graph = nullptr;
  }
  if (graph_mode && !s->x.round_graph) {
    s->x.graph_ws = ws_on;
    if (!s->x.cap_stream) DM_CK(cudaStreamCreateWithFlags(&s->x.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    DM_CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(s->x.cap_stream, cp.conditional.phGraph_out[0], nullptr,
                                        nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      set_error(std::string("CUDA: round graph: ") + cudaGetErrorString(e));
      return DM_ERR_CUDA;
    }
    int64_t before[DM_NUM_KERNELS];
    std::copy(s->x.launches, s->x.launches + DM_NUM_KERNELS, before);
    dm_status rst = round(s->x.cap_stream, 1, false);
    if (rst == DM_OK) k_round_continue<<<1, 32, 0, s->x.cap_stream>>>(d.ctrl, max_rounds, h);
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(s->x.cap_stream, &body);
    for (int k = 0; k < DM_NUM_KERNELS; ++k) {
      s->x.round_launches[k] = s->x.launches[k] - before[k];
      s->x.launches[k] = before[k];
    }
    s->x.round_launches[K_BEGIN] += 1;  // k_round_continue
    if (rst == DM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->x.round_graph, g, 0);
    cudaGraphDestroy(g);
    if (rst != DM_OK) return rst;
    if (e != cudaSuccess) {
      s->x.round_graph = nullptr;
      set_error(std::string("CUDA: round graph: ") + cudaGetErrorString(e));
      return DM_ERR_CUDA;
    }
  }
  if (graph_mode && fuse_first && !s->x.first_graph) {
    // the first round (fused passes), counted as a round of the step
    cudaError_t e = cudaStreamBeginCapture(s->x.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_error(std::string("CUDA: first-round graph: ") + cudaGetErrorString(e));
      return DM_ERR_CUDA;
    }
    int64_t before[DM_NUM_KERNELS];
    std::copy(s->x.launches, s->x.launches + DM_NUM_KERNELS, before);
    dm_status rst = round(s->x.cap_stream, 0, true);
    if (rst == DM_OK) k_round_count<<<1, 32, 0, s->x.cap_stream>>>(d.ctrl);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->x.cap_stream, &g);
    for (int k = 0; k < DM_NUM_KERNELS; ++k) {
      s->x.first_launches[k] = s->x.launches[k] - before[k];
      s->x.launches[k] = before[k];
    }
    s->x.first_launches[K_BEGIN] += 1;  // k_round_count
    if (rst == DM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->x.first_graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rst != DM_OK) return rst;
    if (e != cudaSuccess) {
      s->x.first_graph = nullptr;
      set_error(std::string("CUDA: first-round graph: ") + cudaGetErrorString(e));
      return DM_ERR_CUDA;
    }
  }
  for (int step = 0; step < nsteps; ++step) {
    int32_t init[8] = {0, 0, INT_MAX, 0, 0, 0, 0, 0};  // active, failed, first failed, queue, rounds
    DM_CK(cudaMemcpyAsync(d.ctrl, init, sizeof(init), cudaMemcpyHostToDevice, st));
    {
      Timed t(s, K_BEGIN, st);
      k_begin_step<<<blocks(std::max(nd, S), 256), 256, 0, st>>>(sa);
    }
    if (ws_on) {
      Timed t(s, K_WARM, st);
      DM_CK(ws_predict(s, st, ws_trial, s->x.d_dof_sys));
    }
    if (s->prm.predictor == 1) {
      k_project_lengths<<<blocks((int64_t)S * 32, 128), 128, 0, st>>>(
          S, s->x.d_sys_kind, d.sys_dof0, d.sys_ndof, d.fixed, d.qn, d.q, s->x.midpoint ? 1 : 0);
      s->x.launches[K_BEGIN]++;
    }
    if (ls_on) {
      DM_CK(cudaMemsetAsync(s->x.ls_trial, 0, S * sizeof(int32_t), st));
      DM_CK(cudaMemsetAsync(s->x.ls_nback, 0, S * sizeof(int32_t), st));
      if (ws_trial) DM_CK(cudaMemsetAsync(la.wstry, 0, S * sizeof(int32_t), st));
    }
    if (graph_mode) {
      // an extra round after convergence (the graph body runs at least once)
      // finds no active system and changes nothing
      if (ws_trial) DM_TRY(round(st, 0, false));
      if (fuse_first) DM_CK(cudaGraphLaunch(s->x.first_graph, st));
      DM_CK(cudaGraphLaunch(s->x.round_graph, st));
      DM_CK(cudaMemcpyAsync(s->h_ctrl, d.ctrl, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      DM_CK(cudaStreamSynchronize(st));
      const int64_t loop_rounds = s->h_ctrl[4] - (fuse_first ? 1 : 0);
      for (int k = 0; k < DM_NUM_KERNELS; ++k)
        s->x.launches[k] += loop_rounds * s->x.round_launches[k] +
                            (fuse_first ? s->x.first_launches[k] : 0);
    } else {
      for (int it = 0; it < max_rounds; ++it) {
        DM_TRY(round(st, it, fuse_first && it == 0));
        DM_CK(cudaMemcpyAsync(s->h_ctrl, d.ctrl, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        DM_CK(cudaStreamSynchronize(st));
        harvest(s);
        if (s->h_ctrl[0] == 0) break;
      }
    }
    if (s->x.midpoint && s->h_ctrl[1] == 0) {
      // q_{n+1} = 2y - q_n, the staged velocity, and the frames and reference
      // twist at q_{n+1}; a degenerate edge there fails the step
      k_midpoint_finish<<<blocks(std::max(nd, S), 256), 256, 0, st>>>(sa, d.dq);
      EdgeArgs ef_args = ea;
      ef_args.units = nullptr;
      k_edge<<<blocks(ne, 256), 256, 0, st>>>(ef_args);
      if (ns > 0) {
        StencilArgs kf = ka;
        kf.units = nullptr;
        kf.frames_only = 1;
        k_stencil<<<blocks(ns, 128), 128, 0, st>>>(kf);
      }
      k_collect_failures<<<blocks(S, 256), 256, 0, st>>>(S, d.sys_status, d.ctrl);
      DM_CK(cudaGetLastError());
      DM_CK(cudaMemcpyAsync(s->h_ctrl, d.ctrl, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      DM_CK(cudaStreamSynchronize(st));
      sa.vnew = d.dq;
    }
    if (stats || s->h_ctrl[1] > 0) {
      iters.resize(S);
      DM_CK(cudaMemcpyAsync(iters.data(), d.sys_iters, S * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      DM_CK(cudaStreamSynchronize(st));
    }
    if (s->h_ctrl[1] > 0) {
      if (stats) {
        const int nsys = std::min(stats->capacity, S);
        if (stats->iterations && nsys > 0)
          DM_CK(cudaMemcpyAsync(stats->iterations, d.sys_iters, nsys * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
        if (stats->residual && nsys > 0)
          DM_CK(cudaMemcpyAsync(stats->residual, d.sys_res, nsys * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
        DM_CK(cudaStreamSynchronize(st));
      }
      k_restore<<<blocks(nd, 256), 256, 0, st>>>(sa);
      int32_t first = s->h_ctrl[2], code = 0;
      DM_CK(cudaMemcpyAsync(&code, d.sys_status + first, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      DM_CK(cudaStreamSynchronize(st));
      if (stats) stats->first_failed = first;
      set_error("step " + std::to_string(step) + ": system " + std::to_string(first) +
                " failed with status " + std::to_string(code));
      return (dm_status)code;
    }
    DM_CK(ws_keep_velocity(s, st));
    {
      Timed t(s, K_COMMIT, st);
      k_commit<<<blocks(std::max({nd, ne, ns}), 256), 256, 0, st>>>(sa);
    }
    DM_CK(cudaGetLastError());
    if (stats) {
      stats->steps_done = step + 1;
      for (int k = 0; k < S; ++k) {
        stats->sum_iterations += iters[k];
        stats->max_iterations = std::max(stats->max_iterations, iters[k]);
      }
    }
  }
  if (stats) {
    int n = std::min(stats->capacity, S);
    if (stats->iterations && n > 0) std::copy(iters.begin(), iters.begin() + n, stats->iterations);
    if (stats->residual && n > 0) {
      std::vector<unsigned long long> rb(S);
      DM_CK(cudaMemcpyAsync(rb.data(), d.sys_res, S * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
      DM_CK(cudaStreamSynchronize(st));
      for (int k = 0; k < n; ++k) {
        double v;
        std::memcpy(&v, &rb[k], sizeof(double));
        stats->residual[k] = v;
      }
    }
  }
  return DM_OK;
}

dm_status dm_get_state(dm_system *sys, double *q, double *qdot, size_t cap, int32_t is_device) {
  if (!sys || !q) {
    set_error("dm_get_state: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  const size_t n = s->T.layout2dof.size();
  if (cap < n) {
    set_error("dm_get_state: capacity " + std::to_string(cap) + " < " + std::to_string(n));
    return DM_ERR_INVALID_ARG;
  }
  cudaStream_t st = s->stream;
  // both arrays staged side by side, copied, then one synchronisation
  for (int k = 0; k < 2; ++k) {
    double *dst = k == 0 ? q : qdot;
    if (!dst) continue;
    double *stage = is_device ? dst : s->x.d_scratch + k * n;
    k_gather_layout<<<blocks(n, 256), 256, 0, st>>>((int)n, s->d.layout2dof,
                                                    k == 0 ? s->d.qn : s->d.vn, stage);
    DM_CK(cudaGetLastError());
    if (!is_device)
      DM_CK(cudaMemcpyAsync(dst, stage, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (!is_device) DM_CK(cudaStreamSynchronize(st));
  return DM_OK;
}

dm_status dm_set_state(dm_system *sys, const double *q, const double *qdot, size_t cap,
                       int32_t is_device) {
  if (!sys || !q || !qdot) {
    set_error("dm_set_state: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  const size_t n = s->T.layout2dof.size();
  if (cap < n) {
    set_error("dm_set_state: capacity too small");
    return DM_ERR_INVALID_ARG;
  }
  cudaStream_t st = s->stream;
  // scatter in reverse rod order so that the lowest rod's joint copy wins
  // both arrays staged side by side: one synchronisation for the whole call
  for (int k = 0; k < 2; ++k) {
    const double *src = k == 0 ? q : qdot;
    const double *stage = src;
    if (!is_device) {
      DM_CK(cudaMemcpyAsync(s->x.d_scratch + k * n, src, n * sizeof(double),
                            cudaMemcpyHostToDevice, st));
      stage = s->x.d_scratch + k * n;
    }
    k_scatter_layout<<<blocks(n, 256), 256, 0, st>>>((int)n, s->d.layout2dof, stage,
                                                     k == 0 ? s->d.qn : s->d.vn);
    DM_CK(cudaGetLastError());
  }
  DM_CK(cudaMemcpyAsync(s->d.q, s->d.qn, s->T.n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DM_CK(ws_keep_velocity(s, st));  // no velocity history for a state set from outside
  // committed tangents from the new positions
  DM_CK(cudaMemsetAsync(s->x.d_bad, 0, sizeof(int32_t), st));
  k_tangents<<<blocks(s->T.n_edges, 256), 256, 0, st>>>((int)s->T.n_edges, s->d.edge_a,
                                                       s->d.edge_b, s->d.qn, s->d.tn, s->x.d_bad);
  DM_CK(cudaGetLastError());
  int32_t bad = 0;
  DM_CK(cudaMemcpyAsync(&bad, s->x.d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DM_CK(cudaStreamSynchronize(st));
  if (bad) {
    set_error("dm_set_state: zero-length edge");
    return DM_ERR_DEGENERATE;
  }
  return DM_OK;
}

dm_status dm_get_frames(dm_system *sys, double *d1, double *beta, int32_t is_device) {
  if (!sys) {
    set_error("dm_get_frames: NULL handle");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = sys->T;
  cudaStream_t st = sys->stream;
  const int ne = (int)T.n_edges;
  if (is_device) {
    if (d1 && ne > 0) {
      k_frames_out<<<blocks(ne, 256), 256, 0, st>>>(ne, sys->d.d1n, d1);
      DM_CK(cudaGetLastError());
    }
    if (beta && T.n_stencils > 0)
      DM_CK(cudaMemcpyAsync(beta, sys->d.beta_n, T.n_stencils * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    return DM_OK;
  }
  if (d1) {
    std::vector<double> soa(3 * T.n_edges);
    DM_CK(cudaMemcpyAsync(soa.data(), sys->d.d1n, soa.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, st));
    DM_CK(cudaStreamSynchronize(st));
    for (int64_t e = 0; e < T.n_edges; ++e)
      for (int c = 0; c < 3; ++c) d1[3 * e + c] = soa[c * T.n_edges + e];
  }
  if (beta) {
    DM_CK(cudaMemcpyAsync(beta, sys->d.beta_n, T.n_stencils * sizeof(double),
                          cudaMemcpyDeviceToHost, st));
    DM_CK(cudaStreamSynchronize(st));
  }
  return DM_OK;
}

dm_status dm_set_frames(dm_system *sys, const double *d1, const double *beta,
                        int32_t is_device) {
  if (!sys) {
    set_error("dm_set_frames: NULL handle");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = sys->T;
  cudaStream_t st = sys->stream;
  const int ne = (int)T.n_edges;
  if (is_device) {
    if (d1 && ne > 0) {
      k_frames_in<<<blocks(ne, 256), 256, 0, st>>>(ne, d1, sys->d.d1n);
      DM_CK(cudaGetLastError());
    }
    if (beta && T.n_stencils > 0)
      DM_CK(cudaMemcpyAsync(sys->d.beta_n, beta, T.n_stencils * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    return DM_OK;
  }
  DM_CK(cudaStreamSynchronize(st));
  if (d1) {
    std::vector<double> soa(3 * T.n_edges);
    for (int64_t e = 0; e < T.n_edges; ++e)
      for (int c = 0; c < 3; ++c) soa[c * T.n_edges + e] = d1[3 * e + c];
    DM_CK(cudaMemcpy(sys->d.d1n, soa.data(), soa.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (beta)
    DM_CK(cudaMemcpy(sys->d.beta_n, beta, T.n_stencils * sizeof(double), cudaMemcpyHostToDevice));
  return DM_OK;
}

dm_status dm_adjoint_frame_chain(dm_system *sys, const double *q_prev, const double *q,
                                 const double *q_next, const double *gq, const double *gv,
                                 const double *gv0, double *phibar, double *gq0) {
  auto *s = static_cast<dm_system_ext *>(sys);
  if (!s || !q || !q_next || !gq || !gv || !gv0 || !phibar || !gq0) {
    set_error("dm_adjoint_frame_chain: NULL argument");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = s->T;
  auto &F = s->x.fchain;
  if (!F.g) {
    // layout tables: each edge's start node, each layout node's incident edges
    std::vector<int32_t> edge_lay(T.n_edges), lay, ein, eout;
    for (int r = 0; r < T.n_rods; ++r) {
      const int N = T.npr[r];
      for (int i = 0; i < N; ++i) {
        const int64_t x = T.rod_layout0[r] + 4 * (int64_t)i;
        const int64_t e = T.rod_edge0[r] + i;
        lay.push_back((int32_t)x);
        ein.push_back(i > 0 ? (int32_t)(e - 1) : -1);
        eout.push_back(i + 1 < N ? (int32_t)e : -1);
        if (i + 1 < N) edge_lay[e] = (int32_t)x;
      }
    }
    F.nlnode = (int)lay.size();
    DM_TRY(upload(s, &F.edge_lay, edge_lay));
    DM_TRY(upload(s, &F.lnode_lay, lay));
    DM_TRY(upload(s, &F.lnode_ein, ein));
    DM_TRY(upload(s, &F.lnode_eout, eout));
    DM_TRY(upload(s, &F.layout2dof, T.layout2dof));
    DM_TRY(dalloc(s, &F.g, 3 * std::max<size_t>(1, (size_t)T.n_edges)));
  }
  FrameChainArgs fa{(int)T.n_edges, F.nlnode, s->p.dt, s->x.midpoint ? 1 : 0, F.edge_lay, F.lnode_lay, F.lnode_ein,
                    F.lnode_eout, F.layout2dof, s->d.fixed, q_prev, q, q_next, gq, gv, gv0,
                    phibar, gq0, F.g};
  cudaStream_t st = s->stream;
  if (fa.ne > 0) {
    k_frame_chain_edges<<<blocks(fa.ne, 128), 128, 0, st>>>(fa);
    DM_CK(cudaGetLastError());
    k_frame_chain_nodes<<<blocks(fa.nlnode, 128), 128, 0, st>>>(fa);
    DM_CK(cudaGetLastError());
  }
  return DM_OK;
}

dm_status dm_set_tuning(dm_system *sys, const dm_tuning *t) {
  auto *s = static_cast<dm_system_ext *>(sys);
  if (!s || !t) {
    set_error("dm_set_tuning: NULL argument");
    return DM_ERR_INVALID_ARG;
  }
  auto in = [](int v, std::initializer_list<int> set) {
    for (int x : set)
      if (v == x) return true;
    return false;
  };
  int per_sm = 0;
  const bool solve_ok =
      in(t->solve_warps, {1, 2, 4}) && t->solve_blocks_per_sm >= 1 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, k_solve_rod, 32 * t->solve_warps,
          (size_t)t->solve_warps * kSolveRodsPerWarp * kSolveRodDoubles * 8) == cudaSuccess &&
      per_sm >= t->solve_blocks_per_sm;
  // limb shapes beyond this system's shared-memory limit matter only if it
  // has condensation-path limbs
  const bool limb_ok = in(t->limb_factor_warps, {1, 2, 4}) && in(t->limb_back_warps, {1, 2, 4}) &&
                       (s->x.n_fast == 0 || (t->limb_factor_warps <= s->x.wpb_factor_max &&
                                             t->limb_back_warps <= s->x.wpb_back_max));
  if (!in(t->edge_threads, {128, 256, 512}) || !in(t->stencil_threads, {32, 64, 128}) ||
      !in(t->stencil_per_thread, {1, 2}) || !in(t->rows_threads, {64, 128, 256}) || !solve_ok ||
      !limb_ok) {
    set_error("dm_set_tuning: launch shape outside the autotuner's candidates");
    return DM_ERR_INVALID_ARG;
  }
  auto &tu = s->x.tune;
  tu.edge_threads = t->edge_threads;
  tu.stencil_threads = t->stencil_threads;
  tu.stencil_per_thread = t->stencil_per_thread;
  tu.rows_threads = t->rows_threads;
  set_solve_shape(s, t->solve_warps, t->solve_blocks_per_sm);
  if (s->x.n_fast) {
    s->x.wpb_factor = t->limb_factor_warps;
    s->x.wpb_back = t->limb_back_warps;
  }
  if (s->x.first_graph) {  // launch shapes are baked into the graphs
    cudaGraphExecDestroy(s->x.first_graph);
    s->x.first_graph = nullptr;
  }
  if (s->x.round_graph) {
    cudaGraphExecDestroy(s->x.round_graph);
    s->x.round_graph = nullptr;
  }
  return DM_OK;
}

dm_status dm_autotune(dm_system *sys, int32_t steps, dm_tuning *out) {
  if (!sys || steps < 1) {
    set_error("dm_autotune: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  if (s->ws) {
    set_error("dm_autotune: run it before dm_ws_enable (the warm start keeps a state history)");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = s->T;
  DevArrays &d = s->d;
  cudaStream_t st = s->stream;
  const size_t nd = T.n_dofs, ne = T.n_edges, ns = T.n_stencils;
  // the committed state, restored before every trial and at the end
  double *save = nullptr;
  const size_t nsave = 2 * nd + 6 * ne + ns;
  DM_CK(cudaMalloc(&save, std::max<size_t>(nsave, 1) * sizeof(double)));
  struct Part { double *p; size_t n; };
  const Part parts[] = {{d.qn, nd}, {d.vn, nd}, {d.d1n, 3 * ne}, {d.tn, 3 * ne}, {d.beta_n, ns}};
  auto copy_state = [&](bool to_save) -> cudaError_t {
    size_t off = 0;
    for (const Part &pt : parts) {
      if (pt.n) {
        cudaError_t e = to_save ? cudaMemcpyAsync(save + off, pt.p, pt.n * 8, cudaMemcpyDeviceToDevice, st)
                                : cudaMemcpyAsync(pt.p, save + off, pt.n * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
      }
      off += pt.n;
    }
    return cudaSuccess;
  };
  const bool prof_was = s->x.prof;
  dm_status result = DM_OK;
  // per-launch time of kernel id over `steps` steps from the saved state
  // (a failed trial, or a kernel that did not run, gives +inf)
  auto trial = [&](int id) -> double {
    if (copy_state(false) != cudaSuccess) return INFINITY;
    s->x.prof = true;
    for (int k = 0; k < DM_NUM_KERNELS; ++k) {
      s->x.launches[k] = 0;
      s->x.ms[k] = 0.0;
      s->x.ev_used[k] = false;
    }
    if (dm_step(sys, steps, nullptr) != DM_OK) return INFINITY;
    if (cudaStreamSynchronize(st) != cudaSuccess) return INFINITY;
    // the residual, Jacobian and fused passes of the stencils (of the rows)
    // share one launch shape: all are timed
    double ms = s->x.ms[id];
    int64_t nl = s->x.launches[id];
    if (id == K_STENCIL) {
      ms += s->x.ms[K_HESS] + s->x.ms[K_FUSED];
      nl += s->x.launches[K_FUSED];
    }
    if (id == K_ROWS) {
      ms += s->x.ms[K_BAND] + s->x.ms[K_ROWS_FUSED];
      nl += s->x.launches[K_ROWS_FUSED];
    }
    if (!nl) return INFINITY;
    return ms / (double)nl;
  };
  // coordinate search: the phases run one after another, so each kernel's
  // shape is chosen on its own time, keeping the default unless another
  // shape is faster by more than 2 %
  auto pick = [&](int id, int ncand, auto apply) -> double {
    apply(0);
    double best = trial(id);
    int arg = 0;
    for (int c = 1; c < ncand; ++c) {
      if (!apply(c)) continue;
      const double t = trial(id);
      if (t < 0.98 * best) {
        best = t;
        arg = c;
      }
    }
    apply(arg);
    return best;
  };
  double us[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (copy_state(true) != cudaSuccess) result = DM_ERR_CUDA;
  if (result == DM_OK) trial(K_EDGE);  // warm-up
  if (result == DM_OK) {
    auto &tu = s->x.tune;
    const int e_thr[] = {256, 128, 512};
    us[0] = 1e3 * pick(K_EDGE, 3, [&](int c) { tu.edge_threads = e_thr[c]; return true; });
    if (ns > 0) {
      const int s_thr[] = {128, 64, 128, 64, 32};
      const int s_per[] = {1, 1, 2, 2, 1};
      us[1] = 1e3 * pick(K_STENCIL, 5, [&](int c) {
        tu.stencil_threads = s_thr[c];
        tu.stencil_per_thread = s_per[c];
        return true;
      });
    }
    if (s->x.n_rod_sys > 0 || s->x.cc.n_contact > 0) {
      const int r_thr[] = {256, 128, 64};
      us[2] = 1e3 * pick(K_ROWS, 3, [&](int c) { tu.rows_threads = r_thr[c]; return true; });
    }
    if (s->x.n_rod_sys > 0) {
      const int w[] = {4, 2, 1, 4, 2, 4};
      const int b[] = {1, 2, 4, 2, 1, 3};
      us[3] = 1e3 * pick(K_SOLVE, 6, [&](int c) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_solve_rod, 32 * w[c],
                (size_t)w[c] * kSolveRodsPerWarp * kSolveRodDoubles * 8) !=
                cudaSuccess ||
            per_sm < b[c])
          return false;
        set_solve_shape(s, w[c], b[c]);
        return true;
      });
    }
    if (s->x.n_fast > 0 && !T.lb_n.empty()) {
      // the factor and back-substitution kernels are timed together
      const int wf[] = {s->x.wpb_factor_max, 1, 2, 4};
      us[4] = 1e3 * pick(K_SOLVE_GEN, 4, [&](int c) {
        if (wf[c] > s->x.wpb_factor_max) return false;
        s->x.wpb_factor = wf[c];
        return true;
      });
      const int wb[] = {s->x.wpb_back_max, 1, 2, 4};
      us[5] = 1e3 * pick(K_SOLVE_GEN, 4, [&](int c) {
        if (wb[c] > s->x.wpb_back_max) return false;
        s->x.wpb_back = wb[c];
        return true;
      });
    }
  }
  // leave the state, the counters and the profiling switch as they were
  if (copy_state(false) != cudaSuccess) result = DM_ERR_CUDA;
  cudaStreamSynchronize(st);
  cudaFree(save);
  s->x.prof = prof_was;
  for (int k = 0; k < DM_NUM_KERNELS; ++k) {
    s->x.launches[k] = 0;
    s->x.ms[k] = 0.0;
    s->x.ev_used[k] = false;
  }
  cudaMemset(s->x.d_units, 0, DM_NUM_KERNELS * sizeof(unsigned long long));
  if (s->x.first_graph) {  // launch shapes are baked into the graphs
    cudaGraphExecDestroy(s->x.first_graph);
    s->x.first_graph = nullptr;
  }
  if (s->x.round_graph) {
    cudaGraphExecDestroy(s->x.round_graph);
    s->x.round_graph = nullptr;
  }
  if (out) {
    const auto &tu = s->x.tune;
    out->edge_threads = tu.edge_threads;
    out->stencil_threads = tu.stencil_threads;
    out->stencil_per_thread = tu.stencil_per_thread;
    out->rows_threads = tu.rows_threads;
    out->solve_warps = tu.solve_warps;
    out->solve_blocks_per_sm = tu.solve_bps;
    out->limb_factor_warps = s->x.wpb_factor;
    out->limb_back_warps = s->x.wpb_back;
    for (int k = 0; k < 8; ++k) out->us_per_launch[k] = us[k];
  }
  if (result != DM_OK) set_error("dm_autotune: CUDA error while saving or restoring the state");
  return result;
}

dm_status dm_set_graphs(dm_system *sys, int32_t enable) {
  if (!sys) {
    set_error("dm_set_graphs: NULL handle");
    return DM_ERR_INVALID_ARG;
  }
  static_cast<dm_system_ext *>(sys)->x.graphs = enable != 0;
  return DM_OK;
}

dm_status dm_set_fused_first(dm_system *sys, int32_t enable) {
  if (!sys) {
    set_error("dm_set_fused_first: NULL handle");
    return DM_ERR_INVALID_ARG;
  }
  static_cast<dm_system_ext *>(sys)->x.fused_first = enable != 0;
  return DM_OK;
}

dm_status dm_set_profiling(dm_system *sys, int32_t enable) {
  if (!sys) {
    set_error("dm_set_profiling: NULL handle");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  DM_CK(cudaStreamSynchronize(s->stream));
  s->x.prof = enable != 0;
  for (int k = 0; k < DM_NUM_KERNELS; ++k) {
    s->x.launches[k] = 0;
    s->x.ms[k] = 0.0;
    s->x.ev_used[k] = false;
  }
  DM_CK(cudaMemset(s->x.d_units, 0, DM_NUM_KERNELS * sizeof(unsigned long long)));
  return DM_OK;
}

dm_status dm_get_profile(dm_system *sys, dm_profile *out) {
  if (!sys || !out) {
    set_error("dm_get_profile: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  auto *s = static_cast<dm_system_ext *>(sys);
  DM_CK(cudaStreamSynchronize(s->stream));
  harvest(s);
  unsigned long long u[DM_NUM_KERNELS];
  DM_CK(cudaMemcpy(u, s->x.d_units, sizeof(u), cudaMemcpyDeviceToHost));
  for (int k = 0; k < DM_NUM_KERNELS; ++k) {
    out->launches[k] = s->x.launches[k];
    out->ms[k] = s->x.ms[k];
    out->units[k] = (int64_t)u[k];
  }
  return DM_OK;
}

dm_status dm_debug_copy(dm_system *sys, const char *name, double *out, int64_t n) {
  if (!sys || !name || !out) {
    set_error("dm_debug_copy: bad arguments");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = sys->T;
  const DevArrays &d = sys->d;
  const std::string k(name);
  const double *src = nullptr;
  int64_t len = 0;
  if (k == "gen") { src = d.gen; len = T.gen_doubles; }
  else if (k == "f") { src = d.f; len = T.n_dofs; }
  else if (k == "q") { src = d.q; len = T.n_dofs; }
  else if (k == "nt") { src = d.nt; len = T.any_general ? 12 * T.n_nodes : 0; }
  else if (k == "sg") { src = d.sg; len = 11 * T.n_stencils; }
  else if (k == "sh") { src = d.sh; len = 66 * T.n_stencils; }
  else if (k == "es") { src = d.es; len = 9 * T.n_edges; }
  else if (k == "ef") { src = d.ef; len = 13 * T.n_edges; }
  else {
    set_error("dm_debug_copy: unknown buffer " + k);
    return DM_ERR_INVALID_ARG;
  }
  if (n < len || !src) {
    set_error("dm_debug_copy: buffer " + k + " needs " + std::to_string(len) + " doubles");
    return DM_ERR_INVALID_ARG;
  }
  DM_CK(cudaStreamSynchronize(sys->stream));
  DM_CK(cudaMemcpy(out, src, len * sizeof(double), cudaMemcpyDeviceToHost));
  return DM_OK;
}

dm_status dm_step_adjoint(dm_system *sys, const double *q_next, const double *gq,
                          const double *gv, double *gkbar, double *gq0, double *gv0,
                          int32_t is_device) {
  auto *s = static_cast<dm_system_ext *>(sys);
  if (!s || !q_next || !gq || !gv || !gkbar || !gq0 || !gv0) {
    set_error("dm_step_adjoint: NULL argument");
    return DM_ERR_INVALID_ARG;
  }
  const HostTopology &T = s->T;
  std::vector<int32_t> rod_d0, rod_n;
  for (int k = 0; k < T.n_systems; ++k) {
    if (T.sys_kind[k] == SOLVE_ROD_BAND) {
      rod_d0.push_back(T.sys_dof0[k]);
      rod_n.push_back(T.sys_ndof[k]);
    } else if (T.sys_kind[k] == SOLVE_CONTACT && s->prm.pair_mu != 0.0) {
      set_error("dm_step_adjoint: edge-edge friction (pair_mu != 0) is not supported");
      return DM_ERR_INVALID_ARG;
    }
  }
  const bool contact_on = s->x.cc.n_contact > 0;
  for (size_t w = 0; w < T.gen_sys.size(); ++w)
    if (!T.gs_fast[w]) {
      set_error("dm_step_adjoint: general system " + std::to_string(T.gen_sys[w]) +
                " is not on the condensation path (a limb jointed at both ends)");
      return DM_ERR_INVALID_ARG;
    }
  DevArrays &d = s->d;
  cudaStream_t st = s->stream;
  const int nd = (int)T.n_dofs, ne = (int)T.n_edges, ns = (int)T.n_stencils, S = T.n_systems;
  const int nn = (int)T.n_nodes, ngen = (int)T.gen_sys.size();
  const int n = (int)T.layout2dof.size();
  int nslots = 0;
  for (int r = 0; r < T.n_rods; ++r) nslots += T.npr[r] - 2;
  auto &A = s->x.adj;
  if (!A.buf) {
    DM_TRY(dalloc(s, &A.buf, 7 * (size_t)nd));
    DM_TRY(dalloc(s, &A.dk, 22 * (size_t)std::max(ns, 1)));
    DM_TRY(dalloc(s, &A.gk, 2 * (size_t)std::max(nslots, 1)));
    DM_TRY(dalloc(s, &A.stage, 3 * (size_t)n));
    if (!rod_d0.empty())
      DM_TRY(dalloc(s, &A.scratch, band_scratch_bytes((int32_t)rod_d0.size(), nd)));
    if (ngen > 0) {
      DM_TRY(dalloc(s, &A.gen2, (size_t)T.gen_doubles));
      DM_TRY(dalloc(s, &A.ints, 6 * (size_t)S + 2 * (size_t)ngen + 8));
      DM_TRY(dalloc(s, &A.res, (size_t)S));
    }
  }
  double *lam = A.buf, *rhs = A.buf + nd, *bgq = A.buf + 2 * nd, *bgv = A.buf + 3 * nd;
  double *bgq0 = A.buf + 4 * nd, *bgv0 = A.buf + 5 * nd, *nrhs = A.buf + 6 * nd;
  if (!A.first) {
    std::vector<uint8_t> first(n, 0), seen(nd, 0);
    for (int i = 0; i < n; ++i)
      if (!seen[T.layout2dof[i]]) {
        first[i] = 1;
        seen[T.layout2dof[i]] = 1;
      }
    DM_TRY(upload(s, &A.first, first));
  }
  // inputs in layout order -> DOF order (loss gradients summed over the
  // copies of a shared node)
  const double *src[3] = {q_next, gq, gv};
  double *dst[3] = {d.q, bgq, bgv};
  DM_CK(cudaMemsetAsync(bgq, 0, 2 * (size_t)nd * sizeof(double), st));
  for (int k = 0; k < 3; ++k) {
    const double *in = src[k];
    if (!is_device) {
      DM_CK(cudaMemcpyAsync(A.stage + (size_t)k * n, in, n * sizeof(double),
                            cudaMemcpyHostToDevice, st));
      in = A.stage + (size_t)k * n;
    }
    if (k == 0)
      k_scatter_layout<<<blocks(n, 256), 256, 0, st>>>(n, d.layout2dof, in, dst[k]);
    else
      k_scatter_add_layout<<<blocks(n, 256), 256, 0, st>>>(n, d.layout2dof, in, dst[k]);
  }
  // implicit midpoint: the backward-Euler adjoint over dt/2 at the midpoint
  // configuration, with the loss gradients doubled
  if (s->x.midpoint)
    k_adj_midpoint_in<<<blocks(nd, 256), 256, 0, st>>>(nd, d.fixed, d.qn, d.q, bgq, bgv);
  // every system active; J and the curvature gradients at q_next (at the
  // midpoint configuration for implicit midpoint)
  std::vector<int32_t> ones(S, 1);
  DM_CK(cudaMemcpyAsync(d.sys_active, ones.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  DM_CK(cudaMemsetAsync(d.sys_status, 0, S * sizeof(int32_t), st));
  DM_CK(cudaMemsetAsync(d.sys_res, 0, S * sizeof(unsigned long long), st));
  EdgeArgs ea{ne, d.q, d.edge_a, d.edge_b, d.edge_th, d.edge_sys, d.edge_EA, d.edge_ilbar,
              d.tn, d.d1n, d.sys_active, d.sys_status, d.ef, d.es, nullptr};
  StencilArgs ka{ns, ne, d.q, d.ef, d.tn, d.st_ed, d.st_th, d.st_sg, d.st_sys, d.st_kb, d.st_kt,
                 d.kbar, d.taubar, d.beta_n, d.sys_active, d.sys_status, d.beta_it, d.sg, d.sh,
                 nullptr, A.dk};
  k_edge<<<blocks(ne, 256), 256, 0, st>>>(ea);
  if (T.ground) {
    NodeArgs na{nn, s->p.dt, s->prm.ground_z, s->prm.delta, s->prm.slip_nu, d.q, d.qn,
                d.node_dof_arr, d.node_sys, d.node_h, d.node_mu, d.node_kc, d.sys_active, d.nt};
    k_nodes<<<blocks(nn, 256), 256, 0, st>>>(na);
  }
  if (ns > 0) k_stencil<<<blocks(ns, 128), 128, 0, st>>>(ka);
  ContactArgs ca{};
  if (contact_on) {
    auto &c = s->x.cc;
    ca.ne = ne; ca.nd = nd; ca.nsys = S; ca.table_mask = c.table - 1; ca.pair_cap = c.pair_cap;
    ca.inv_cell = c.inv_cell; ca.delta = s->prm.delta; ca.kc = s->prm.pair_kc;
    ca.mu = 0.0; ca.K2 = 0.0; ca.dt = s->p.dt;
    ca.q = d.q; ca.qn = d.qn; ca.edge_h = c.edge_h; ca.band = d.band;
    ca.edge_a = d.edge_a; ca.edge_b = d.edge_b; ca.edge_sys = d.edge_sys; ca.edge_idx = c.edge_idx;
    ca.sys_kind = s->x.d_sys_kind; ca.sys_active = d.sys_active; ca.dof_sys = s->x.d_dof_sys;
    ca.sys_dof0 = d.sys_dof0; ca.sys_ndof = d.sys_ndof; ca.contact_sys = c.contact_sys;
    ca.ls_action = nullptr; ca.fixed = d.fixed; ca.sys_dense0 = c.sys_dense0;
    ca.sys_status = d.sys_status; ca.sys_bw = c.sys_bw; ca.edge_key = c.edge_key;
    ca.bucket_count = c.bucket_count; ca.bucket_start = c.bucket_start;
    ca.bucket_fill = c.bucket_fill; ca.bucket_edges = c.bucket_edges; ca.pairs = c.pairs;
    ca.npairs = c.npairs; ca.fc = c.fc; ca.dense = c.dense;
    ca.n_contact = c.n_contact; ca.cgo = c.cgo; ca.cbad = c.cbad;
    ca.nn = (int)T.n_nodes;
    DM_CK(cudaMemsetAsync(c.fc, 0, nd * sizeof(double), st));
    DM_CK(cudaMemsetAsync(c.npairs, 0, sizeof(int32_t), st));
    DM_CK(cudaMemsetAsync(c.bucket_count, 0, c.table * sizeof(int32_t), st));
    k_cc_clear<<<blocks((int64_t)nd * 32, 256), 256, 0, st>>>(ca);
    k_cc_reset_bw<<<blocks(S, 256), 256, 0, st>>>(ca);
    k_cc_cells<<<blocks(ne, 256), 256, 0, st>>>(ca);
    k_cc_scan<<<1, 1024, 0, st>>>(ca);
    k_cc_fill<<<blocks(ne, 256), 256, 0, st>>>(ca);
    k_cc_pairs<<<blocks(ne, 128), 128, 0, st>>>(ca);
    k_cc_terms<<<blocks(c.pair_cap, 64), 64, 0, st>>>(ca);
    if (T.ground) k_cc_ground<<<blocks(nn, 128), 128, 0, st>>>(ca, d.node_dof_arr, d.node_sys, d.nt);
  }
  if (!rod_d0.empty() || contact_on) {
    RowArgs ra{};
    ra.fc = contact_on ? s->x.cc.fc : nullptr;
    ra.nd = nd; ra.ns = ns; ra.ne = ne; ra.dt = s->p.dt; ra.idt = 1.0 / s->p.dt;
    for (int c = 0; c < 3; ++c) ra.g[c] = s->p.g[c];
    ra.eta = s->p.eta;
    ra.q = d.q; ra.qn = d.qn; ra.vn = d.vn; ra.mass = d.mass; ra.rscale = d.rscale;
    ra.damp = s->x.d_damp; ra.fixed = d.fixed; ra.dof_sys = s->x.d_dof_sys;
    ra.dof_rod = s->x.d_dof_rod; ra.rod_dof0 = s->x.d_rod_dof0; ra.rod_ndof = s->x.d_rod_ndof;
    ra.rod_st0 = s->x.d_rod_st0; ra.rod_edge0 = s->x.d_rod_edge0;
    ra.sys_active = d.sys_active; ra.sys_kind = s->x.d_sys_kind;
    ra.sg = d.sg; ra.sh = d.sh; ra.es = d.es; ra.f = d.f; ra.band = d.band; ra.sys_res = d.sys_res;
    k_rows_rod<<<blocks(nd, 256), 256, 0, st>>>(ra);
  }
  if (ngen > 0) {
    AsmArgs aa{(int)T.asm_target.size(), d.asm_target, d.asm_ptr, d.asm_src, d.sh, d.es, d.nt,
               d.dconst, d.gen, d.asm_sys, d.sys_active, nullptr,
               (int)T.gen_sys.size(), d.gen_sys, d.asm_t0, d.gs_mat0, d.gs_mat1, d.sys_ndof,
               nullptr};
    if (s->x.n_slow) k_gen_clear_slow<<<aa.ngen, 256, 0, st>>>(aa, d.gs_fast);
    if (s->x.asm_chunks > 0) k_assemble_gen<<<dim3(aa.ngen, s->x.asm_chunks), 256, 0, st>>>(aa);
  }
  AdjArgs aa{nd, ns, nslots, s->p.dt, lam, bgq, bgv, d.mass, s->x.d_damp, A.dk, d.st_kb,
             d.fixed, d.st_nd, d.st_th, s->x.d_slot2st, rhs, bgq0, bgv0, A.gk,
             nn, T.ground ? d.nt : nullptr, d.dof_node, d.dof_comp, d.node_dof_arr, 1.0};
  k_adj_rhs<<<blocks(nd, 256), 256, 0, st>>>(aa);
  DM_CK(cudaGetLastError());
  dm_status bs = DM_OK;
  if (!rod_d0.empty()) {
    // rods: J lambda = gbar by the banded LDL^T (J symmetric); zeroes lambda
    bs = run_band_solve((int32_t)rod_d0.size(), rod_d0.data(), rod_n.data(), nd, d.band, rhs,
                        lam, A.scratch, st);
  } else {
    DM_CK(cudaMemsetAsync(lam, 0, nd * sizeof(double), st));
  }
  if (bs == DM_OK && ngen > 0) {
    // networks: J^T lambda = gbar by the condensation kernels on the
    // transposed storage (they solve J dq = -f and add dq to q)
    AdjArgs an = aa;
    an.rhs = nrhs;
    an.rhs_sign = -1.0;
    k_adj_rhs<<<blocks(nd, 256), 256, 0, st>>>(an);
    int32_t *act = A.ints, *its = act + S, *sts = its + S, *ctl = sts + S;
    int32_t *go = ctl + 8, *bad = go + ngen;
    DM_CK(cudaMemcpyAsync(act, ones.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    DM_CK(cudaMemsetAsync(its, 0, 2 * S * sizeof(int32_t), st));
    const int32_t c0[4] = {0, 0, INT_MAX, 0};
    DM_CK(cudaMemcpyAsync(ctl, c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    DM_CK(cudaMemsetAsync(go, 0, 2 * ngen * sizeof(int32_t), st));
    DM_CK(cudaMemsetAsync(A.res, 0x7f, S * sizeof(unsigned long long), st));  // huge: never converged
    DM_CK(cudaMemsetAsync(A.gen2, 0, T.gen_doubles * sizeof(double), st));
    SolveGenArgs ga{};
    ga.ngen = ngen; ga.max_iter = 1; ga.tol = 0.0;
    ga.gen_sys = d.gen_sys; ga.gs_limb0 = d.gs_limb0; ga.gs_nlimb = d.gs_nlimb; ga.gs_nB = d.gs_nB;
    ga.gs_border0 = d.gs_border0; ga.gs_JBB = d.gs_JBB; ga.gs_rB = d.gs_rB; ga.gs_S = d.gs_S;
    ga.gs_xB = d.gs_xB; ga.lb_dof0 = d.lb_dof0; ga.lb_n = d.lb_n; ga.lb_ncr = d.lb_ncr;
    ga.lb_cr0 = d.lb_cr0; ga.lb_band = d.lb_band; ga.lb_piv = d.lb_piv; ga.lb_C = d.lb_C;
    ga.lb_R = d.lb_R; ga.lb_Y = d.lb_Y; ga.lb_y = d.lb_y; ga.border_dof = d.border_dof;
    ga.coupled_rows = d.coupled_rows; ga.f = nrhs; ga.gen = A.gen2; ga.q = lam;
    ga.sys_active = act; ga.sys_iters = its; ga.sys_status = sts;
    ga.sys_res = A.res; ga.ctrl = ctl; ga.units = nullptr; ga.ls_action = nullptr;
    ga.ls_trial = nullptr;
    ga.nlimb = (int)T.lb_n.size();
    ga.limb_nmax = s->x.limb_nmax;
    ga.gs_fast = d.gs_fast; ga.lb_gsys = d.lb_gsys; ga.lb_dir = d.lb_dir; ga.lb_m = d.lb_m;
    ga.lb_nbc = d.lb_nbc; ga.lb_bc0 = d.lb_bc0; ga.lb_bcols = d.lb_bcols;
    ga.gen_go = go; ga.gen_bad = bad;
    if (ga.nlimb > 0)
      k_gen_transpose<<<dim3(4, ga.nlimb), 256, 0, st>>>(ga, d.gen, A.gen2);
    k_gen_transpose_border<<<ngen, 256, 0, st>>>(ga, d.gen, A.gen2);
    const int wf = s->x.wpb_factor, wb = s->x.wpb_back;
    if (ga.nlimb)
      k_gen_limb_factor<<<(ga.nlimb + wf - 1) / wf, 32 * wf, s->x.smem_factor, st>>>(ga);
    k_gen_border<<<ngen, kGenBorderThreads, s->x.border_smem, st>>>(ga);
    if (ga.nlimb)
      k_gen_limb_back<<<(ga.nlimb + wb - 1) / wb, 32 * wb, s->x.smem_back, st>>>(ga);
    DM_CK(cudaGetLastError());
    int32_t h[4] = {0, 0, 0, 0};
    DM_CK(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
    DM_CK(cudaStreamSynchronize(st));
    if (h[1] > 0) {
      set_error("dm_step_adjoint: zero or non-finite pivot in the transposed solve");
      bs = DM_ERR_DEGENERATE;
    }
  }
  if (bs == DM_OK && contact_on) {
    // contact rods: J^T lambda = gbar with the blocked LU of the transposed
    // dense matrix (the contact kernels solve J dq = -f and add dq to q)
    const int nc = s->x.cc.n_contact;
    k_cc_band<<<blocks(nd, 256), 256, 0, st>>>(ca);
    AdjArgs an = aa;
    an.rhs = nrhs;
    an.rhs_sign = -1.0;
    k_adj_rhs<<<blocks(nd, 256), 256, 0, st>>>(an);
    if (rod_d0.empty() && ngen == 0) DM_CK(cudaMemsetAsync(lam, 0, nd * sizeof(double), st));
    std::vector<int32_t> onec(nc, 1);
    DM_CK(cudaMemcpyAsync(ca.cgo, onec.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    DM_CK(cudaMemsetAsync(ca.cbad, 0, nc * sizeof(int32_t), st));
    for (int c = 0; c < nc; ++c) {
      const int nc_n = T.sys_ndof[c];
      k_cc_transpose<<<blocks((int64_t)nc_n * std::max(10, nc_n), 256), 256, 0, st>>>(ca, c);
      for (int k = 0; k < nc_n; k += kNB) {
        const int rest = nc_n - k - std::min(kNB, nc_n - k);
        k_lu_diag<<<1, 256, 0, st>>>(ca, c, k);
        if (rest > 0) {
          k_lu_trsm<<<blocks(2 * rest, 32), 32, 0, st>>>(ca, c, k);
          const int t = (rest + 63) / 64;
          k_lu_gemm<<<dim3(t, t), 256, 0, st>>>(ca, c, k);
        }
      }
    }
    if (!A.ints) DM_TRY(dalloc(s, &A.ints, 6 * (size_t)S + 2 * (size_t)std::max(ngen, 1) + 8));
    int32_t *its = A.ints, *sts = its + S, *ctl = sts + S;
    DM_CK(cudaMemsetAsync(its, 0, 2 * S * sizeof(int32_t), st));
    const int32_t c0[4] = {0, 0, INT_MAX, 0};
    DM_CK(cudaMemcpyAsync(ctl, c0, sizeof(c0), cudaMemcpyHostToDevice, st));
    SolveArgs vs{};
    vs.nd = nd; vs.sys_dof0 = d.sys_dof0; vs.sys_ndof = d.sys_ndof; vs.f = nrhs;
    vs.q = lam; vs.dq = d.dq; vs.sys_active = d.sys_active; vs.sys_iters = its;
    vs.sys_status = sts; vs.ctrl = ctl;
    k_cc_subst<<<nc, 1024, 0, st>>>(ca, vs);
    DM_CK(cudaGetLastError());
    int32_t h[4] = {0, 0, 0, 0};
    DM_CK(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
    DM_CK(cudaStreamSynchronize(st));
    if (h[1] > 0) {
      set_error("dm_step_adjoint: zero or non-finite pivot in the transposed contact solve");
      bs = DM_ERR_DEGENERATE;
    }
  }
  // the system stays at step n whatever happened
  DM_CK(cudaMemcpyAsync(d.q, d.qn, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (bs != DM_OK) return bs;
  k_adj_state<<<blocks(nd, 256), 256, 0, st>>>(aa);
  if (s->x.midpoint)
    k_adj_midpoint_out<<<blocks(nd, 256), 256, 0, st>>>(nd, d.fixed, bgq, bgv, bgq0, bgv0);
  if (nslots > 0) k_adj_kbar<<<blocks(nslots, 128), 128, 0, st>>>(aa);
  // outputs: state gradients in layout order, curvature gradients by slot
  double *outs[2] = {gq0, gv0};
  const double *ins[2] = {bgq0, bgv0};
  for (int k = 0; k < 2; ++k) {
    double *o = is_device ? outs[k] : A.stage + (size_t)k * n;
    k_gather_layout_first<<<blocks(n, 256), 256, 0, st>>>(n, d.layout2dof, A.first, ins[k], o);
    if (!is_device)
      DM_CK(cudaMemcpyAsync(outs[k], o, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (nslots > 0)
    DM_CK(cudaMemcpyAsync(gkbar, A.gk, 2 * (size_t)nslots * sizeof(double),
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  DM_CK(cudaGetLastError());
  DM_CK(cudaStreamSynchronize(st));
  return DM_OK;
}

int64_t dm_contact_pairs(dm_system *sys) {
  auto *s = static_cast<dm_system_ext *>(sys);
  if (!s || !s->x.cc.npairs) return 0;
  int32_t n = 0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return -1;
  if (cudaMemcpy(&n, s->x.cc.npairs, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -1;
  return n;
}

const char *dm_kernel_name(int32_t id) {
  if (id < 0 || id >= DM_NUM_KERNELS || !kKernelNames[id]) return "";
  return kKernelNames[id];
}

}  // extern "C"

namespace {
// Register-resident DFMA chains: 8 independent chains per thread.
__global__ void k_fp64_probe(double *out, int iters) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-9 * (threadIdx.x + c);
  const double m = 0.999999999, k = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, k);
  }
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) r += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
}  // namespace

extern "C" double dm_fp64_peak_gflops(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  const int threads = 256, nblk = sms * 4, iters = 4096;
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads * nblk) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    k_fp64_probe<<<nblk, threads>>>(buf, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return -1.0;
  const double flops = 2.0 * 8.0 * iters * (double)threads * nblk;
  return flops / (best * 1e-3) / 1e9;
}
