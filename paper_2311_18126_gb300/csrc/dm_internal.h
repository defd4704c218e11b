// Internal declarations of the GB300 implicit DER library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dismech.h"

namespace dm {

// Per-thread last error message (dm_last_error).
void set_error(const std::string &msg);

// ---------------------------------------------------------------------------
// Host-side topology (built once by dm_create_system from the descriptor)
// ---------------------------------------------------------------------------
enum SolverKind : int32_t {
  SOLVE_ROD_BAND = 0,  // one rod, Eq. 1 layout, symmetric, half bandwidth 10
  SOLVE_GENERAL = 1,   // limbs (banded interiors) + dense border (joints,
                       // ground contact/friction: possibly nonsymmetric)
  SOLVE_CONTACT = 2,   // one rod with edge-edge contact: band widened by the
                       // contact blocks, LU in a dense per-system matrix
};

// Gather-map source codes for the general assembly (see dm_general.cu).
// Limits of the condensation path of general systems.
constexpr int kFastMaxM = 10;        // coupled rows at one limb end
constexpr int kFastMaxBC = 16;       // border columns one limb couples to
constexpr int kFastMaxBorder = 96;   // border DOFs of one system
constexpr int kGenBorderThreads = 128;  // block of the border solve
constexpr int kFastMaxRows = 1200;   // rows of one limb (shared-memory staging)

enum SrcType : uint32_t { SRC_STENCIL = 0, SRC_EDGE = 1, SRC_NODE = 2, SRC_DIAG = 3 };
inline uint32_t src_code(uint32_t type, uint32_t index, bool neg) {
  return (neg ? 0x80000000u : 0u) | (type << 29) | index;
}

struct HostTopology {
  int32_t n_rods = 0;
  std::vector<int32_t> npr;      // nodes per rod
  std::vector<int64_t> rod_node0, rod_edge0, rod_layout0; // flat offsets
  // global nodes (joint members merged)
  int64_t n_nodes = 0, n_edges = 0, n_stencils = 0, n_dofs = 0;
  std::vector<int64_t> flat2node;      // (rod,node) flat -> node
  std::vector<int32_t> node_dof;       // DOF index of x of each node
  std::vector<int32_t> node_sys;
  std::vector<double> node_mass, node_vor, node_h, node_mu, node_kc;
  // edges (descriptor order)
  std::vector<int32_t> edge_a, edge_b, edge_rod, edge_sys, edge_thdof;
  std::vector<double> edge_lbar, edge_EA, edge_EI, edge_GJ, edge_rhoA, edge_h;
  std::vector<double> d1_init, t_init;  // [Ne][3]
  // stencils (node order, then incident edge pairs)
  std::vector<int32_t> st_node[3], st_edge[2], st_sign[2], st_sys;
  std::vector<int32_t> st_rod_slot; // -1 for joint stencils, else flat index
                                     // into the per-rod interior-node list
  std::vector<double> st_kb, st_kt, st_beta0, st_kbar1, st_kbar2, st_taubar;
  // systems
  int32_t n_systems = 0;
  std::vector<int32_t> sys_kind, sys_dof0, sys_ndof;
  std::vector<int32_t> sys_rod0, sys_nrods;
  std::vector<int32_t> sys_st0, sys_nst, sys_edge0, sys_nedge;
  // per-DOF data
  std::vector<double> dof_mass, dof_rscale, q0, v0;
  std::vector<uint8_t> dof_fixed;
  // per-rod layout (Eq. 1) -> DOF index
  std::vector<int32_t> layout2dof;
  // force gather CSR: for each DOF, entries (element, local slot)
  std::vector<int32_t> gat_ptr, gat_ent;
  // per-DOF node (-1 for twist angles) and component (0..2, 3 = angle)
  std::vector<int32_t> dof_node, dof_comp;
  // general systems: limbs (banded interiors) and border
  std::vector<int32_t> gen_sys;            // general system ids
  std::vector<int32_t> gs_limb0, gs_nlimb, gs_nB, gs_border0;
  std::vector<int64_t> gs_JBB, gs_rB, gs_S, gs_xB, gs_mat0, gs_mat1;
  std::vector<int32_t> lb_dof0, lb_n, lb_ncr, lb_cr0;
  std::vector<int64_t> lb_band, lb_piv, lb_C, lb_R, lb_Y, lb_y;
  // condensation path (systems whose limbs attach at one end): per system
  // flag; per limb its system, elimination direction (1 = from the last
  // row), trailing block size m and coupled border columns
  std::vector<int32_t> gs_fast, lb_gsys, lb_dir, lb_m, lb_nbc, lb_bc0, lb_bcols;
  std::vector<int32_t> border_dof;         // global DOF of each border entry
  std::vector<int32_t> coupled_rows;       // limb-local rows coupled to border
  int64_t gen_doubles = 0;                 // size of the general scratch
  // gather map for the general assembly: target (offset into the general
  // scratch) <- sum of sources
  std::vector<int64_t> asm_target;
  std::vector<int32_t> asm_sys;            // system of each target
  std::vector<int32_t> asm_t0;             // first target of each general system
  std::vector<int32_t> asm_ptr;
  std::vector<uint32_t> asm_src;
  bool any_general = false, ground = false;
};

// Builds the topology; returns false with set_error() on invalid input.
bool build_topology(const dm_system_desc *desc, const dm_params *prm,
                    HostTopology &T);

// ---------------------------------------------------------------------------
// Device-side state
// ---------------------------------------------------------------------------
struct DevArrays {
  // DOF vectors
  double *q = nullptr, *qn = nullptr, *vn = nullptr, *f = nullptr;
  double *mass = nullptr, *rscale = nullptr;
  uint8_t *fixed = nullptr;
  // nodes
  int32_t *node_dof = nullptr;
  double *node_mass = nullptr, *node_vor = nullptr;
  // edges
  int32_t *edge_a = nullptr, *edge_b = nullptr, *edge_th = nullptr,
          *edge_sys = nullptr;
  double *edge_ilbar = nullptr, *edge_EA = nullptr;  // 1 / rest length, EA
  double *d1n = nullptr, *tn = nullptr;  // committed frames, SoA [3][Ne]
  // per-iteration edge outputs (SoA): t[3], len, d1[3], m1[3], m2[3]
  double *ef = nullptr;                  // [13][Ne]
  double *es = nullptr;                  // stretch: f[3], K[6]  [9][Ne]
  // stencils
  int32_t *st_nd = nullptr;   // [3][Ns] node DOF bases
  int32_t *st_ed = nullptr;   // [2][Ns] edge ids
  int32_t *st_th = nullptr;   // [2][Ns] theta DOF
  int32_t *st_sg = nullptr;   // [Ns] sign bits: bit0 = a reversed, bit1 = b
  int32_t *st_sys = nullptr;
  double *st_kb = nullptr, *st_kt = nullptr, *kbar = nullptr /*[2][Ns]*/,
         *taubar = nullptr, *beta_n = nullptr, *beta_it = nullptr;
  double *sg = nullptr;       // stencil gradient [11][Ns]
  double *sh = nullptr;       // stencil Hessian, packed upper [66][Ns]
  // systems
  int32_t *sys_dof0 = nullptr, *sys_ndof = nullptr, *sys_st0 = nullptr,
          *sys_edge0 = nullptr;
  int32_t *sys_active = nullptr;   // 1 while Newton runs on the system
  int32_t *sys_iters = nullptr;
  int32_t *sys_status = nullptr;
  unsigned long long *sys_res = nullptr; // max scaled residual (double bits)
  int32_t *ctrl = nullptr;         // [0] = number of active systems
  // gather CSR
  int32_t *gat_ptr = nullptr, *gat_ent = nullptr;
  // band workspace for the rod solver: L factors [11][n_dofs]
  double *band = nullptr;
  double *dq = nullptr;
  int32_t *layout2dof = nullptr;
  // rod-solver ordering (systems sorted by size)
  int32_t *solve_order = nullptr;
  // general path
  int32_t *dof_node = nullptr, *dof_comp = nullptr;
  double *nt = nullptr;          // node terms [12][Nn]: force (3), -dF/dx (9)
  double *dconst = nullptr;      // per-DOF M/dt^2 + damping
  int32_t *node_dof_arr = nullptr, *node_sys = nullptr;
  double *node_h = nullptr, *node_mu = nullptr, *node_kc = nullptr;
  double *gen = nullptr;
  int32_t *gen_sys = nullptr, *gs_limb0 = nullptr, *gs_nlimb = nullptr, *gs_nB = nullptr,
          *gs_border0 = nullptr;
  int64_t *gs_JBB = nullptr, *gs_rB = nullptr, *gs_S = nullptr, *gs_xB = nullptr;
  int64_t *gs_mat0 = nullptr, *gs_mat1 = nullptr;  // each system's storage range
  int32_t *lb_dof0 = nullptr, *lb_n = nullptr, *lb_ncr = nullptr, *lb_cr0 = nullptr;
  int64_t *lb_band = nullptr, *lb_piv = nullptr, *lb_C = nullptr, *lb_R = nullptr, *lb_Y = nullptr, *lb_y = nullptr;
  int32_t *border_dof = nullptr, *coupled_rows = nullptr;
  int32_t *gs_fast = nullptr, *lb_gsys = nullptr, *lb_dir = nullptr, *lb_m = nullptr,
          *lb_nbc = nullptr, *lb_bc0 = nullptr, *lb_bcols = nullptr;
  int32_t *gen_go = nullptr, *gen_bad = nullptr;  // per general system
  int64_t *asm_target = nullptr;
  int32_t *asm_sys = nullptr, *asm_t0 = nullptr;
  int32_t *asm_ptr = nullptr;
  uint32_t *asm_src = nullptr;
};

struct Params {
  double dt, tol;
  int32_t max_iter;
  double g[3];
  double eta;
};

// Learned warm start (dm_warmstart.cu).
struct WarmStart;
void ws_free(WarmStart *w);
// Batched banded solve (dm_band_solve.cu): scratch size and the solve with
// host arrays of system offsets/sizes.
size_t band_scratch_bytes(int32_t nsys, int64_t ntot);
dm_status run_band_solve(int32_t nsys, const int32_t *dof0, const int32_t *ndof, int64_t ntot,
                         const double *band, const double *rhs, double *x, char *scr,
                         cudaStream_t st);

bool ws_active(const dm_system *s);  // a network is attached
// Evaluates the network on the committed state.  defer = false: the guess
// replaces the extrapolation in q (and the systems it reached are marked for
// ws_fallback); defer = true: it is kept for ws_inject.
cudaError_t ws_predict(dm_system *s, cudaStream_t st, bool defer, const int32_t *dof_sys);
// After a round's solves (no line search): systems started from the learned
// guess that have not converged in a few iterations restart from the
// extrapolation.
cudaError_t ws_fallback(dm_system *s, cudaStream_t st, const int32_t *dof_sys);
// After the first line-search round: q <- learned guess for every active
// system, marked as a trial (no solve this round).
cudaError_t ws_inject(dm_system *s, cudaStream_t st, int32_t *ls_action, int32_t *ls_trial);
int32_t *ws_trial_flags(dm_system *s);
// qdot_{n-1} of the previous-correction features <- the current qdot_n
// (before a commit overwrites it, and after a state is set).
cudaError_t ws_keep_velocity(dm_system *s, cudaStream_t st);

// Long rods (dm_band_partitioned.cu): the systems `sys` are solved in the
// Newton rounds by the partitioned band solve (interiors of part_rows - 10
// rows).  long_rods_round is declared with the kernel arguments.
struct LongRods;
dm_status long_rods_create(dm_system *s, const std::vector<int32_t> &sys, int part_rows,
                           LongRods **out);
void long_rods_free(LongRods *L);
int long_rods_count(const LongRods *L);

}  // namespace dm

struct dm_system {
  dm::HostTopology T;
  dm::DevArrays d;
  dm::Params p;
  dm_params prm;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocations;
  int32_t *h_ctrl = nullptr;  // pinned
  dm::WarmStart *ws = nullptr;
};

