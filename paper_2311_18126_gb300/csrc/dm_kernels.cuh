// Kernel argument blocks and declarations (internal).
#pragma once
#include "dm_internal.h"

namespace dm {

struct EdgeArgs {
  int ne;
  const double *q;
  const int32_t *edge_a, *edge_b, *edge_th, *edge_sys;
  const double *edge_EA, *edge_ilbar, *tn, *d1n;  // edge_ilbar: 1 / rest length
  const int32_t *sys_active;
  int32_t *sys_status;
  double *ef, *es;
  unsigned long long *units;
};

struct StencilArgs {
  int ns, ne;
  const double *q, *ef, *tn;
  const int32_t *st_ed, *st_th, *st_sg, *st_sys;
  const double *st_kb, *st_kt, *kbar, *taubar, *beta_n;
  const int32_t *sys_active;
  int32_t *sys_status;
  double *beta_it, *sg, *sh;
  unsigned long long *units;
  double *dk;  // NULL, or [22][Ns]: gradients of kappa1, kappa2 (11 stencil DOFs each)
  int frames_only;  // 1: reference twist only (the commit of an implicit-midpoint step)
  // Hessian pass (k_stencil_hess): the solver's convergence test
  const unsigned long long *sys_res;
  double tol;
  const int32_t *ls_action;  // NULL without line search
};

struct RowArgs {
  const double *fc;  // edge-edge contact force per DOF (NULL without contact)
  int nd, ns, ne;
  double dt, g[3], eta;
  double idt;  // 1 / dt
  const double *q, *qn, *vn, *mass, *rscale, *damp;
  const uint8_t *fixed;
  const int32_t *dof_sys;
  // per rod (rows are rod-local; a contact group holds several rods)
  const int32_t *dof_rod, *rod_dof0, *rod_ndof, *rod_st0, *rod_edge0;
  const int32_t *sys_active, *sys_kind;
  const double *sg, *sh, *es;
  double *f, *band;
  unsigned long long *sys_res;
  unsigned long long *units;
  // band pass (k_rows_rod_band): the solver's convergence test
  const int32_t *sys_status;
  double tol;
  const int32_t *ls_action;  // NULL without line search
};

struct SolveArgs {
  int nsys, nd;
  double tol;
  int max_iter;
  const int32_t *order;
  const int32_t *sys_dof0, *sys_ndof;
  const uint8_t *fixed;
  const double *f;
  double *band, *q, *dq;
  int32_t *sys_active, *sys_iters, *sys_status;
  const unsigned long long *sys_res;
  int32_t *ctrl;
  unsigned long long *units;
  const int32_t *ls_action;  // NULL without line search; 1 = backtracking
  int32_t *ls_trial;
};

// shared memory (doubles) per rod of k_solve_rod: two chain windows and the
// separator scratch
constexpr int kSolveRodDoubles = 2 * (22 * 12 + 2) + 32;
// rods per warp of k_solve_rod (two chains of eight lanes each per rod)
constexpr int kSolveRodsPerWarp = 2;

struct NodeArgs {
  int nn;
  double dt, ground_z, delta, slip_nu;
  const double *q, *qn;
  const int32_t *node_dof, *node_sys;
  const double *node_h, *node_mu, *node_kc;
  const int32_t *sys_active;
  double *nt;
  unsigned long long *units;  // profiling: nodes evaluated (or NULL)
};

struct RowGenArgs {
  int nd, ns, ne, nn;
  double dt, g[3];
  double idt;  // 1 / dt
  const double *q, *qn, *vn, *mass, *rscale, *damp;
  const uint8_t *fixed;
  const int32_t *dof_sys, *dof_node, *dof_comp, *sys_kind, *sys_active;
  const int32_t *gat_ptr, *gat_ent;
  const double *sg, *es, *nt;
  double *f;
  unsigned long long *sys_res;
  unsigned long long *units;  // profiling: DOF rows evaluated (or NULL)
};

struct AsmArgs {
  int ntarget;
  const int64_t *target;
  const int32_t *ptr;
  const uint32_t *src;
  const double *sh, *es, *nt, *dconst;
  double *gen;
  const int32_t *tsys;       // system of each target
  const int32_t *sys_active, *ls_action;
  // per general system: its system index, first target, storage range
  int ngen;
  const int32_t *gen_sys, *t0;
  const int64_t *mat0, *mat1;
  const int32_t *sys_ndof;
  unsigned long long *units;  // profiling: DOFs of the systems assembled (or NULL)
};
// Profiling: counts the calling warp's active threads into *units (one
// atomic per warp).
// 1/d for 2^-126 <= |d| < 2^126 (callers test the range first).  The
// leading 23 bits of d become an FP32 number by integer operations (the
// exponent field rebiased by 1023 - 127 = 896: 0x38000000 in the upper word),
// its approximate FP32 reciprocal (relative error ~2^-22) returns the same
// way, and one third-order step of the iteration for 1/d,
// r <- r (1 + e + e^2) with e = 1 - d r (the truncated series of
// r / (1 - e)), leaves a relative error of about e^3 ~ 2^-66, below FP64
// rounding: three FP64 instructions, no FP32/FP64 conversions.
__device__ __forceinline__ double rcp64_seed(double d) {  // the FP32 seed, as FP64
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned fb = (hi & 0x80000000u) | (((hi & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo >> 29);
  float sf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sf) : "f"(__uint_as_float(fb)));
  const unsigned sb = __float_as_uint(sf);
  return __hiloint2double((int)((sb & 0x80000000u) | (((sb & 0x7FFFFFFFu) >> 3) + 0x38000000u)),
                          (int)(sb << 29));
}
__device__ __forceinline__ double rcp64(double d) {
  const double r = rcp64_seed(d);
  const double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Asynchronous 8-byte copy global -> shared (both 8-byte aligned), and the
// group commit / wait for all of this thread's copies.
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Upper word of |d| against the range of rcp64: true for 2^-126 <= |d| < 2^126.
__device__ __forceinline__ bool rcp64_in_range(double d) {
  const unsigned h = (unsigned)__double2hiint(d) & 0x7FFFFFFFu;
  return h >= ((1023u - 126u) << 20) && h < ((1023u + 126u) << 20);
}

// d == 0 or not finite, by integer tests on its words (off the FP64 pipe).
__device__ __forceinline__ bool zero_or_nonfinite(double d) {
  const unsigned h = (unsigned)__double2hiint(d) & 0x7FFFFFFFu;
  return (h | (unsigned)__double2loint(d)) == 0u || h >= 0x7FF00000u;
}

__device__ __forceinline__ void count_active(unsigned long long *units) {
  if (units == nullptr) return;
  const unsigned m = __activemask();
  if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(units, (unsigned long long)__popc(m));
}

struct SolveGenArgs {
  int ngen, max_iter;
  double tol;
  const int32_t *gen_sys, *gs_limb0, *gs_nlimb, *gs_nB, *gs_border0;
  const int64_t *gs_JBB, *gs_rB, *gs_S, *gs_xB;
  const int32_t *lb_dof0, *lb_n, *lb_ncr, *lb_cr0;
  const int64_t *lb_band, *lb_piv, *lb_C, *lb_R, *lb_Y, *lb_y;
  const int32_t *border_dof, *coupled_rows;
  const double *f;
  double *gen, *q;
  int32_t *sys_active, *sys_iters, *sys_status;
  const unsigned long long *sys_res;
  int32_t *ctrl;
  unsigned long long *units;
  const int32_t *ls_action;
  int32_t *ls_trial;
  // condensation path
  int nlimb, limb_nmax;  // limbs; most rows of a condensation-path limb
  const int32_t *gs_fast, *lb_gsys, *lb_dir, *lb_m, *lb_nbc, *lb_bc0, *lb_bcols;
  int32_t *gen_go, *gen_bad;
};

// shared memory (doubles) per warp of the condensation-path limb kernels:
// the factor's limb band, its condensed block [A_m | C_m | y_m], the
// coupling rows R_m and the small LU's scratch
__host__ __device__ constexpr size_t gen_factor_smem(int nmax) {
  return (size_t)nmax * 22 + kFastMaxM * (kFastMaxM + kFastMaxBC + 1) + kFastMaxBC * kFastMaxM +
         2 * kFastMaxM;
}
__host__ __device__ constexpr size_t gen_back_smem(int nmax) { return (size_t)nmax * 12 + 16; }

struct LineSearchArgs {
  int nsys, nd;
  const int32_t *sys_active, *dof_sys, *sys_dof0, *sys_ndof;
  const double *f, *rscale;
  int32_t *action, *trial, *nback;
  double *alpha, *racc, *merit, *q, *qacc;
  int32_t *wstry;  // NULL, or 1 while the trial is the learned initial guess
};
struct ContactArgs {
  int ne, nd, nsys, table_mask, pair_cap;
  double inv_cell, delta, kc;
  double mu, K2, dt;  // edge-edge friction (mu = 0: none)
  const double *q, *qn, *edge_h, *band;
  const int32_t *edge_a, *edge_b, *edge_sys, *edge_idx, *sys_kind, *sys_active, *dof_sys;
  const int32_t *sys_dof0, *sys_ndof, *contact_sys, *ls_action;
  const uint8_t *fixed;
  const int64_t *sys_dense0;
  int32_t *sys_status, *sys_bw;
  unsigned long long *edge_key;
  int32_t *bucket_count, *bucket_start, *bucket_fill, *bucket_edges;
  int32_t *pairs, *npairs;
  double *fc, *dense;
  int n_contact;
  int32_t *cgo, *cbad;  // per contact system: solve this round, zero pivot met
  int nn;  // nodes (ground terms of contact systems)
  unsigned long long *lu_flops;  // profiling: FP64 flops of the LU's trailing updates (or NULL)
};
constexpr int kNB = 32;  // panel width of the contact-system LU
__global__ void k_cc_cells(ContactArgs a);
__global__ void k_cc_scan(ContactArgs a);
__global__ void k_cc_fill(ContactArgs a);
__global__ void k_cc_pairs(ContactArgs a);
__global__ void k_cc_terms(ContactArgs a);
__global__ void k_cc_band(ContactArgs a);
__global__ void k_cc_ground(ContactArgs a, const int32_t *node_dof, const int32_t *node_sys,
                            const double *nt);
__global__ void k_cc_clear(ContactArgs a);
__global__ void k_cc_reset_bw(ContactArgs a);
__global__ void k_cc_decide(ContactArgs a, SolveArgs v);
__global__ void k_lu_diag(ContactArgs a, int c, int k);
__global__ void k_lu_trsm(ContactArgs a, int c, int k);
__global__ void k_lu_gemm(ContactArgs a, int c, int k);
__global__ void k_cc_subst(ContactArgs a, SolveArgs v);
__global__ void k_cc_transpose(ContactArgs a, int c);

// Adjoint of one implicit step (single rods): right-hand side, state and
// natural-curvature gradients.
struct AdjArgs {
  int nd, ns, nslots;
  double dt;
  const double *lam, *gq, *gv, *mass, *damp, *dk, *st_kb;
  const uint8_t *fixed;
  const int32_t *st_nd, *st_th, *slot2st;
  double *rhs, *gq0, *gv0, *gkbar;
  // ground friction (general systems): node terms [12][nn] and DOF maps
  int nn;
  const double *nt;
  const int32_t *dof_node, *dof_comp, *node_dof;
  double rhs_sign;  // +1: rhs = gbar; -1: rhs = -gbar (the solve kernels take -f)
};
// Transposed copy of the condensation-path storage of general systems
// (limb bands, couplings swapped, border block transposed).
__global__ void k_gen_transpose(SolveGenArgs a, const double *src, double *dst);
__global__ void k_gen_transpose_border(SolveGenArgs a, const double *src, double *dst);
__global__ void k_adj_rhs(AdjArgs a);
__global__ void k_adj_state(AdjArgs a);
__global__ void k_adj_kbar(AdjArgs a);
// Implicit midpoint as the backward-Euler adjoint over h = dt/2 at the
// midpoint configuration y: in, y = (q_n + q_{n+1})/2 and the loss
// gradients doubled; out, the terms of q_{n+1} = 2y - q_n and
// qdot_{n+1} = 2 (y - q_n)/h - qdot_n taken explicitly.
__global__ void k_adj_midpoint_in(int nd, const uint8_t *fixed, const double *qn, double *q,
                                  double *gq, double *gv);
__global__ void k_adj_midpoint_out(int nd, const uint8_t *fixed, const double *gq2,
                                   const double *gv2, double *gq0, double *gv0);

constexpr int kLineSearchThreads = 128;
__global__ void k_line_search(LineSearchArgs a);  // one block per system

__global__ void k_nodes(NodeArgs a);
__global__ void k_rows_gen(RowGenArgs a);
constexpr int kAsmPerBlock = 1024;  // assembly targets per block (256 threads)
__global__ void k_assemble_gen(AsmArgs a);  // grid (systems, chunks), 256 threads
__global__ void k_gen_clear_slow(AsmArgs a, const int32_t *gs_fast);
__global__ void k_solve_gen(SolveGenArgs a);
__global__ void k_gen_limb_factor(SolveGenArgs a);
__global__ void k_gen_border(SolveGenArgs a);
__global__ void k_gen_limb_back(SolveGenArgs a);

__global__ void k_edge(EdgeArgs a);
__global__ void k_stencil(StencilArgs a);       // gradient and Hessian
__global__ void k_stencil_grad(StencilArgs a);  // reference twist and gradient
__global__ void k_stencil_hess(StencilArgs a);  // Hessian of systems still to be solved
__global__ void k_rows_rod(RowArgs a);       // residual and band rows
__global__ void k_rows_rod_res(RowArgs a);   // residual rows
__global__ void k_rows_rod_band(RowArgs a);  // band rows of systems still to be solved
__global__ void k_solve_rod(SolveArgs a);

struct StepArgs {
  int nd, ne, ns, nsys;
  double dt;
  double *q, *qn, *vn, *d1n, *tn, *beta_n;
  const double *ef, *beta_it;
  const uint8_t *fixed;
  int32_t *sys_active, *sys_iters, *sys_status;
  unsigned long long *sys_res;
  const double *vnew;  // NULL: qdot = (q - q_n)/dt; else the staged qdot_{n+1}
};
// Frame chain of a rollout adjoint (dm_adjoint_frame_chain).
struct FrameChainArgs {
  int ne, nlnode;
  double dt;                   // the backward-Euler step (dt/2 for implicit midpoint)
  int midpoint;                // the energy of a step is taken at (q + q_next)/2
  const int32_t *edge_lay;     // [Ne] layout index of each edge's start node x
  const int32_t *lnode_lay, *lnode_ein, *lnode_eout;  // per layout node
  const int32_t *layout2dof;
  const uint8_t *fixed;        // DOF order
  const double *q_prev, *q, *q_next, *gq, *gv, *gv0;
  double *phibar, *gq0;
  double *g;                   // [Ne][3] scratch
};
__global__ void k_frame_chain_edges(FrameChainArgs a);
__global__ void k_frame_chain_nodes(FrameChainArgs a);
__global__ void k_frames_out(int ne, const double *soa, double *aos);
__global__ void k_frames_in(int ne, const double *aos, double *soa);
__global__ void k_begin_step(StepArgs a);
__global__ void k_project_lengths(int nsys, const int32_t *sys_kind, const int32_t *sys_dof0,
                                  const int32_t *sys_ndof, const uint8_t *fixed,
                                  const double *qn, double *q, int midpoint);
__global__ void k_commit(StepArgs a);
__global__ void k_restore(StepArgs a);
__global__ void k_round_continue(int32_t *ctrl, int max_rounds, cudaGraphConditionalHandle h);
__global__ void k_round_count(int32_t *ctrl);
__global__ void k_reset_res(int lo, int hi, const int32_t *sys_active,
                            unsigned long long *sys_res);

__global__ void k_midpoint_finish(StepArgs a, double *vnew);
// Newton round of the long rods: bookkeeping, partitioned solve, q += dq.
cudaError_t long_rods_round(LongRods *L, const SolveArgs &v, cudaStream_t st);
__global__ void k_collect_failures(int nsys, const int32_t *sys_status, int32_t *ctrl);
__global__ void k_tangents(int ne, const int32_t *edge_a, const int32_t *edge_b,
                           const double *q, double *tn, int32_t *bad);

// Counts the active threads of a block into *units (all threads must call).
__device__ __forceinline__ void count_units(unsigned long long *units, bool act) {
  if (units == nullptr) return;
  const int n = __syncthreads_count(act ? 1 : 0);
  if (threadIdx.x == 0 && n) atomicAdd(units, (unsigned long long)n);
}

}  // namespace dm
