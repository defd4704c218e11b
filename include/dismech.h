/*
 * dismech.h -- C ABI of the GB300 implicit Discrete Elastic Rods step.
 *
 * The library advances batches of independent rod systems (single rods and
 * rods joined at elastic joints) by the fully implicit step of the DisMech
 * paper (arXiv 2311.18126), backward Euler or implicit midpoint:
 *
 *   Sec. III, Eq. 1    DOF vector q = [q_0, theta^0, q_1, ..., q_{N-1}] per rod
 *                      (node positions, edge twist angles), 4N-1 entries.
 *   Sec. III-A, Eq. 2-9  stretching, bending and twisting energies over edges
 *                      and node stencils, with time-parallel reference frames,
 *                      reference twist and material curvatures kappa1, kappa2.
 *   Sec. III-B, Eq. 10-13  IMC ground / edge-edge contact, smooth Coulomb
 *                      friction, gravity and viscous damping.
 *   Sec. III-C, Eq. 14-16  residual M/dt((q_{n+1}-q_n)/dt - qdot_n) - F = 0
 *                      solved by Newton's method with J = M/dt^2 - dF/dq,
 *                      then qdot_{n+1} = (q_{n+1}-q_n)/dt.
 *   Sec. III-D         elastic joints: bending and twisting for every pair of
 *                      edges meeting at a joint node.
 *   Sec. III-E         natural curvature kappabar as the control input.
 *
 * Everything on the step runs in hand-written sm_103a CUDA kernels in FP64.
 *
 * Conventions
 *  - Every call returns dm_status; no C++ exception crosses the ABI.  On an
 *    error, dm_last_error() returns a message for the calling thread.
 *  - A dm_system handle is not thread-safe: one host thread at a time.
 *  - The caller owns every buffer it passes; the library copies what it
 *    needs before returning (device-side copies are ordered on the system's
 *    stream).  The library owns all device memory behind the handle.
 *  - Units are SI.  Arrays are row-major, FP64 unless stated.
 *  - A "system" is a connected component of rods under the joints.  Systems
 *    are numbered in the order of their lowest rod index.
 */
#ifndef DISMECH_H
#define DISMECH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dm_system dm_system; /* opaque */

typedef enum dm_status {
  DM_OK = 0,
  DM_ERR_INVALID_ARG = 1,   /* bad descriptor, size or pointer               */
  DM_ERR_NOT_CONVERGED = 2, /* Newton hit max_iter; state kept at last step  */
  DM_ERR_NONFINITE = 3,     /* NaN/Inf in the residual or the update         */
  DM_ERR_DEGENERATE = 4,    /* zero-length edge, antiparallel edges at a
                               stencil (kappa b singular, Eq. 4), an edge
                               reversed within one step, or a pivot that is
                               zero or tiny against its row's diagonal (or,
                               in the rod and limb eliminations, outside
                               [2^-126, 2^126), the reciprocal's range)     */
  DM_ERR_PENETRATION = 5,   /* edge-edge distance D <= 0 (Eq. 10 undefined)  */
  DM_ERR_CUDA = 6,          /* a CUDA runtime call failed                    */
  DM_ERR_OOM = 7            /* device allocation failed                      */
} dm_status;

/* Rod geometry, materials and boundary conditions (Sec. III, III-D).
 * All arrays are host memory and are copied by dm_create_system. */
typedef struct dm_system_desc {
  int32_t n_rods;
  const int32_t *nodes_per_rod; /* [n_rods], N_r >= 2                          */
  const double *x0;             /* [sum N_r][3] rest = initial node positions   */
  const double *v0;             /* [sum N_r][3] initial velocities, or NULL (0) */
  const double *theta0;         /* [sum (N_r-1)] initial twist angles, or NULL  */
  const double *theta_dot0;     /* [sum (N_r-1)] or NULL                        */
  const double *E;              /* [n_rods] Young's modulus                     */
  const double *nu;             /* [n_rods] Poisson ratio (G = E/(2(1+nu)))     */
  const double *rho;            /* [n_rods] density                             */
  const double *radius;         /* [n_rods] rod radius h                        */
  /* Elastic joints: joint j merges the nodes joint_members[k] = (rod, node)
   * for k in [joint_offsets[j], joint_offsets[j+1]) into one shared node. */
  int32_t n_joints;
  const int32_t *joint_offsets; /* [n_joints+1] or NULL when n_joints == 0      */
  const int32_t *joint_members; /* [joint_offsets[n_joints]][2]                 */
  /* Fixed DOFs in the per-rod layout of Eq. 1 (nonzero = fixed), or NULL. */
  const uint8_t *fixed;         /* [sum (4 N_r - 1)]                            */
  /* Ground friction coefficient and contact stiffness per rod (a shared
   * joint node takes the values of its lowest-numbered rod), or NULL (0). */
  const double *ground_mu;      /* [n_rods]                                     */
  const double *ground_kc;      /* [n_rods] k_c multiplying Eq. 10, N/m         */
  /* Contact groups (edge-edge contact between rods, params.self_contact):
   * group g solves the rods contact_group_rods[k], k in
   * [contact_group_offsets[g], contact_group_offsets[g+1]), consecutive in
   * the descriptor and without joints, as one system, so that their edges
   * can touch each other (reading C26: contact acts within a system).  0 /
   * NULL: every rod is its own system. */
  int32_t n_contact_groups;
  const int32_t *contact_group_offsets; /* [n_contact_groups+1]                   */
  const int32_t *contact_group_rods;    /* [contact_group_offsets[n]]              */
} dm_system_desc;

/* Step parameters (Sec. III-B, III-C). */
typedef struct dm_params {
  double dt;            /* time step                                           */
  double newton_tol;    /* convergence: max_i |f_i| / (D_i l_i) <= newton_tol,
                           D_i = M_i/dt^2 + rest stretch (position DOFs) or
                           twist (angle DOFs) stiffness, l_i = total rest
                           length of the system (positions) or 1 (angles)     */
  int32_t max_iter;     /* Newton iterations per step before giving up         */
  double gravity[3];    /* m/s^2                                               */
  double damping;       /* viscous damping eta: F_i = -eta V_i (x_i - x_i^n)/dt */
  int32_t ground;       /* nonzero: ground plane z = ground_z with IMC contact  */
  double ground_z;
  double delta;         /* contact distance tolerance delta (K1 = 15/delta)    */
  double slip_nu;       /* slipping tolerance nu (K2 = 15/nu), m/s             */
  int32_t self_contact; /* nonzero: edge-edge IMC contact within each system   */
  double pair_kc;       /* k_c of edge-edge contact                            */
  double pair_mu;       /* edge-edge friction coefficient                      */
  int32_t line_search;  /* nonzero: backtracking after each Newton update: a
                           trial point whose 2-norm of the scaled residual
                           f_i / (D_i l_i) is not below (1 - 1e-4 alpha) times
                           that of the last accepted iterate is pulled halfway
                           back to it (alpha halves), at most 12 times, before
                           it is accepted (Sec. III-C notes a line search as an
                           optional safeguard)                                */
  void *stream;         /* cudaStream_t for all work, NULL = default stream    */
  int32_t integrator;   /* 0: backward Euler (Eq. 15); 1: implicit midpoint
                           (Sec. III-C offers both; the textbook rule:
                           q_{n+1} - q_n = dt (qdot_n + qdot_{n+1})/2,
                           M (qdot_{n+1} - qdot_n)/dt = F at (q_n + q_{n+1})/2,
                           velocity-dependent forces at (x_{n+1} - x_n)/dt).
                           Solved as backward Euler over dt/2 for the midpoint
                           configuration y, whose residual is the same
                           function, then q_{n+1} = 2y - q_n; newton_tol and
                           line_search then act on that residual (D_i with
                           M_i/(dt/2)^2).  Frames and reference twist are
                           committed at q_{n+1}.  The step adjoint rejects it. */
  int32_t long_rod_dofs; /* single rods with at least this many DOFs are solved
                           by the partitioned band solve (dm_solve_band_
                           partitioned, interiors of 502 rows) instead of the
                           twisted LDL^T chain; 0 = 2048 (512 nodes),
                           negative = never */
  int32_t predictor;    /* Newton's starting guess (the paper leaves it open;
                           Newton runs to the same tolerance from any guess):
                           0: q_n + dt qdot_n, fixed DOFs at q_n; 1: the same,
                           then for every system of a single rod each edge
                           rescaled to its committed length, node positions
                           rebuilt outward from the rod's first node along
                           the guess's edge directions (nodes with a fixed
                           position DOF keep theirs), also applied to a
                           learned guess.  Implicit midpoint: applied to
                           the step's end guess 2y - q_n, the midpoint guess
                           y rebuilt as its mean with q_n.                  */
} dm_params;

/* Optional per-call statistics (caller-owned arrays may be NULL). */
typedef struct dm_step_stats {
  int32_t capacity;          /* entries available in iterations[]/residual[]  */
  int32_t *iterations;       /* [n_systems] Newton iterations of the last step */
  double *residual;          /* [n_systems] final scaled residual              */
  int32_t first_failed;      /* out: -1, or the first failing system           */
  int32_t steps_done;        /* out: steps completed                           */
  int64_t sum_iterations;    /* out: sum over steps and systems of iterations  */
  int32_t max_iterations;    /* out: max over steps and systems                */
} dm_step_stats;

/* Builds the systems of `desc` on the current CUDA device (Sec. III, III-D):
 * merges joint nodes, numbers the DOFs, computes rest lengths, masses
 * (node: sum over incident edges of rho A l/2; twist: rho A h^2 l/2),
 * initial reference frames (z projected off the first tangent of each rod,
 * then space-parallel transport along the rod), initial reference twist,
 * natural strains (kappabar, taubar = initial values), and uploads it all.
 * `out` receives the handle; on error *out is NULL.  Bend-twist stencils
 * are numbered by node (nodes in order of their lowest (rod, node) entry),
 * then by the pair of incident edges (edges in descriptor order). */
dm_status dm_create_system(const dm_system_desc *desc, const dm_params *params,
                           dm_system **out);

/* Frees all device and host memory of the handle.  NULL-safe. */
void dm_destroy(dm_system *sys);

/* Natural curvature control (Sec. III-E, Eq. 6): kbar holds
 * (kappabar1, kappabar2) -- integrated curvature, dimensionless as in Eq. 5 --
 * for every interior node of rods [rod_begin, rod_end), rods in order,
 * nodes 1..N_r-2 in order: 2 * sum (N_r - 2) doubles.  Joint stencils keep
 * their initial natural curvature.  `kbar` is host memory, or device memory
 * when is_device != 0.  Takes effect at the next dm_step, in stream order. */
dm_status dm_set_natural_curvature(dm_system *sys, int32_t rod_begin,
                                   int32_t rod_end, const double *kbar,
                                   int32_t is_device);

/* Advances every system by `nsteps` implicit steps: backward Euler (Eq.
 * 15-16) or implicit midpoint, as dm_params.integrator selects, each solved
 * by Newton's method to newton_tol.  Each step is all-or-nothing: if any
 * system fails (status != DM_OK) the step is not committed, the state stays
 * at the last completed step and the call returns that status.  `stats` may
 * be NULL. */
dm_status dm_step(dm_system *sys, int32_t nsteps, dm_step_stats *stats);

/* Copies q and qdot out in the per-rod layout of Eq. 1, rods concatenated
 * (a shared joint node appears in every rod that contains it).  q and qdot
 * are host buffers (or device buffers when is_device != 0) of at least
 * dm_state_size() doubles each; qdot may be NULL.  Synchronises the stream
 * for host buffers. */
dm_status dm_get_state(dm_system *sys, double *q, double *qdot, size_t cap,
                       int32_t is_device);

/* Sets q and qdot (same layout as dm_get_state; joint-node copies must
 * agree, the lowest rod's copy wins).  Reference frames are kept; the
 * committed tangents are recomputed from the new q. */
dm_status dm_set_state(dm_system *sys, const double *q, const double *qdot,
                       size_t cap, int32_t is_device);

/* History a bitwise resume needs: reference director d1 per edge
 * ([sum (N_r-1)][3], descriptor edge order) and reference twist beta per
 * bend-twist stencil ([dm_num_stencils]).  Host buffers (the calls
 * synchronise the stream), or device buffers when is_device != 0 (ordered
 * on the system's stream, no synchronisation).  Either may be NULL. */
dm_status dm_get_frames(dm_system *sys, double *d1, double *beta, int32_t is_device);
dm_status dm_set_frames(dm_system *sys, const double *d1, const double *beta,
                        int32_t is_device);

/* Sizes. */
int64_t dm_state_size(const dm_system *sys);  /* sum (4 N_r - 1) */
int32_t dm_num_systems(const dm_system *sys);
int64_t dm_num_stencils(const dm_system *sys);
int64_t dm_num_edges(const dm_system *sys);

/* Solves J x = rhs for a batch of independent symmetric banded systems of
 * half bandwidth 10 -- the Jacobian layout of a single rod in the order of
 * Eq. 1 (Sec. III-C, Eq. 16 is solved with this kernel inside dm_step) --
 * with the library's twisted banded LDL^T kernel (no pivoting).
 *   nsys, sys_dof0[nsys], sys_ndof[nsys]: host arrays; system k occupies
 *     entries [sys_dof0[k], sys_dof0[k] + sys_ndof[k]) of the vectors; the
 *     systems may come in any order but may not share entries.
 *   ntot: length of the vectors.
 *   band: device, [11][ntot], band[d * ntot + i] = J[i][i - d] (the lower
 *     band; entries reaching outside a system are ignored).  Not modified.
 *   rhs: device [ntot]; x: device [ntot] output, overlapping neither band
 *     nor rhs.
 * Breaking these rules gives DM_ERR_INVALID_ARG before any device work.
 * Work is ordered on `stream` (NULL = default stream); the call allocates
 * device scratch and returns after the solve has finished.
 * J need not be positive definite: the rod Jacobian M/dt^2 - dF/dq is
 * indefinite for compressed or buckling rods and at large steps.  Without
 * pivoting, the factorisation of such a matrix is accurate as long as no
 * pivot D_i is small against its row; a pivot that is zero, not finite,
 * below 2^-43 |J_ii| (1.1e-13) or outside [2^-126, 2^126) returns
 * DM_ERR_DEGENERATE (the system is then numerically singular for this
 * solver) instead of an inaccurate x. */
dm_status dm_solve_band(int32_t nsys, const int32_t *sys_dof0, const int32_t *sys_ndof,
                        int64_t ntot, const double *band, const double *rhs, double *x,
                        void *stream);

/* The same solve for long systems (rods of thousands of nodes), without
 * the sequential chain over the whole system: each system is cut into
 * interiors of part_rows - 10 rows separated by 10-row separators (interiors
 * do not couple); a warp per interior factors it (band L D L^T) and forms
 * its Schur contributions to the neighbouring separators (forward solves
 * only, by symmetry), a warp per system solves the block-tridiagonal
 * separator system (10 x 10 blocks, Gauss-Jordan), and a warp per interior
 * back-substitutes.  Arguments and batch rules as dm_solve_band, plus
 * part_rows (0 = 512; otherwise 21..1024).  Nothing is pivoted: interiors
 * and separator blocks are eliminated in order, like the full band, and a
 * pivot that is zero, not finite or below 1e-13 times its row's (or its
 * Schur block's) starting diagonal entry returns DM_ERR_DEGENERATE.
 * Allocates device scratch (about 170 bytes per DOF); returns after the
 * solve has finished. */
dm_status dm_solve_band_partitioned(int32_t nsys, const int32_t *sys_dof0,
                                    const int32_t *sys_ndof, int64_t ntot, const double *band,
                                    const double *rhs, double *x, int32_t part_rows,
                                    void *stream);

/* dm_solve_band without any device allocation.
 *
 * Some callers cannot allocate device memory at the point where they need a
 * solve: a real-time control loop cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree imply, and a process whose device
 * memory is already reserved by another allocator (a framework's caching
 * pool, a fixed arena) may have none left to give.  This entry point takes
 * the same arguments and returns the same result as dm_solve_band, but keeps
 * all of its scratch in one fixed device array inside the library, sized for
 * DM_NOALLOC_MAX_SYSTEMS systems and DM_NOALLOC_MAX_DOFS DOFs in total
 * (about 3.3 MiB).  Larger batches are rejected with DM_ERR_INVALID_ARG and
 * a message naming the limit.  It calls no allocating CUDA routine itself.
 *  - The array belongs to the library's module: the CUDA driver reserves it
 *    on a device when it loads that module there, and keeps it until the
 *    process exits.  Under CUDA's default lazy module loading that happens
 *    inside the first call of this entry point on the device, which can
 *    then fail with DM_ERR_CUDA if the device has no 3.3 MiB left; make one
 *    call at set-up, while memory is still free and before any stream
 *    capture, to take that reservation early.
 *  - Each call looks the array's address up in the current context, with
 *    that device current (no address is cached across calls).
 *  - Every call reuses the same array and leaves its contents behind; each
 *    call re-initialises what it reads.  Calls whose work overlaps on the
 *    GPU (other streams, other host threads) race on the array: serialise
 *    them.
 *  - It returns after the solve has finished, like dm_solve_band.
 * The paper has no counterpart to this entry point. */
#define DM_NOALLOC_MAX_SYSTEMS 2048
#define DM_NOALLOC_MAX_DOFS 32768
dm_status dm_solve_band_noalloc(int32_t nsys, const int32_t *sys_dof0,
                                const int32_t *sys_ndof, int64_t ntot,
                                const double *band, const double *rhs, double *x,
                                void *stream);

/* BF16 tensor-core GEMM used by the learned warm start (no counterpart in
 * the paper): C = act(A B^T + bias) with A [M][K], B [N][K] bf16 row-major
 * device arrays, bias [N] fp32 device array or NULL, C [M][N] row-major bf16
 * (out_f32 = 0) or fp32 (out_f32 != 0), act = ReLU when relu != 0.
 * Accumulation is fp32 in tensor memory (tcgen05).  Requires M % 128 == 0,
 * K % 64 == 0, 16 <= N <= 256, N % 16 == 0 and 16-byte aligned A, B, C
 * (DM_ERR_INVALID_ARG otherwise).  Synchronises `stream`. */
dm_status dm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, const void *B,
                       const float *bias, void *C, int32_t relu, int32_t out_f32,
                       void *stream);

/* Warm-start network (no counterpart in the paper): a 4-layer MLP
 * in_dim (<= 64) -> 256 -> 256 -> 256 -> out_dim (<= 64), ReLU, BF16 operands
 * with FP32 accumulation on the tensor cores, FP32 master weights, Adam.
 * Inputs are [M][64] bf16 device arrays (columns >= in_dim zero), outputs
 * and targets fp32 device arrays, M a multiple of 128.  All work is ordered
 * on `stream`; the calls synchronise it.  Parameters travel as one fp32 host
 * array: per layer W [out][in] then b [out] on the padded shapes 256x64,
 * 256x256, 256x256, 64x256 (dm_mlp_num_params entries). */
typedef struct dm_mlp dm_mlp;
dm_status dm_mlp_create(int32_t in_dim, int32_t out_dim, uint64_t seed, void *stream,
                        dm_mlp **out);
void dm_mlp_destroy(dm_mlp *m);
int64_t dm_mlp_num_params(void);
dm_status dm_mlp_get_params(dm_mlp *m, float *host);
dm_status dm_mlp_set_params(dm_mlp *m, const float *host);
/* Y [M][64] = network(X) (fp32, columns >= out_dim are zero).  By default
 * one persistent kernel runs the four layers per 128-row tile on chip (TMA
 * loads with 128-byte swizzle, the hidden activations in shared memory);
 * dm_mlp_set_fused(m, 0) switches inference (and the warm start's) to one
 * GEMM launch per layer through global memory, with the same arithmetic.
 * dm_mlp_forward synchronises the network's stream and reports a
 * tensor-core barrier timeout (DM_ERR_CUDA); dm_mlp_forward_async only
 * enqueues the work (X and Y must stay valid until it has run), and
 * dm_mlp_check synchronises and reports (and clears) a timeout of any
 * earlier asynchronous call. */
dm_status dm_mlp_forward(dm_mlp *m, const void *X, float *Y, int32_t M);
dm_status dm_mlp_forward_async(dm_mlp *m, const void *X, float *Y, int32_t M);
dm_status dm_mlp_check(dm_mlp *m);
dm_status dm_mlp_set_fused(dm_mlp *m, int32_t enable);
/* One Adam step (learning rate lr; lr = 0 computes gradients only) on the
 * mean squared error against Y [M][out_dim]; grads (device, optional) gets
 * the gradient in the parameter layout, loss the loss before the update. */
dm_status dm_mlp_train_step(dm_mlp *m, const void *X, const float *Y, int32_t M, float lr,
                            float *grads, double *loss);

/* Learned warm start of the Newton iteration (no counterpart in the paper;
 * the paper starts each step from the previous state).  One segment per rod
 * node i >= 1: the network maps 64 features of the committed step, in the
 * local frame of edge i-1, to a correction (3 position components in units
 * of the edge rest length, 1 twist angle) of the guess q_n + dt qdot_n for
 * node i and edge i-1.  Newton then runs to the same tolerance from the
 * corrected guess, so only the iteration count changes.
 *
 * dm_ws_enable builds the segment tables (idempotent).  dm_ws_num_segments
 * returns their number S (0 before enabling).  dm_ws_capture_features writes
 * the raw fp32 features [S][64] of the committed state to device memory and
 * remembers the extrapolated guess; after dm_step, dm_ws_capture_targets
 * writes the fp32 targets [S][4] (converged q minus that guess, local frame)
 * to device memory.  Both are asynchronous on the system's stream.
 * dm_ws_set_model attaches a network (dm_mlp with out_dim 4; NULL detaches)
 * and its normalisation, 132 host floats: input mean [64], input std [64],
 * output scale [4]; the system does not own the network, which must outlive
 * its use.  While attached, every dm_step evaluates it on the tensor cores
 * before the first Newton iteration.
 * dm_ws_prepare_batch gathers rows idx[M] of device feature/target arrays
 * into a normalised bf16 input [M][64] and fp32 target [M][4] (all device
 * pointers, norm included).  dm_ws_column_stats writes the mean and standard
 * deviation of each column of a device fp32 [rows][cols] array to stats
 * [2][cols] (device).  Errors: DM_ERR_INVALID_ARG on NULL or unenabled. */
dm_status dm_ws_enable(dm_system *sys);
int64_t dm_ws_num_segments(const dm_system *sys);
dm_status dm_ws_capture_features(dm_system *sys, float *features);
dm_status dm_ws_capture_targets(dm_system *sys, float *targets);
dm_status dm_ws_set_model(dm_system *sys, dm_mlp *net, const float *norm);
dm_status dm_ws_prepare_batch(const float *features, const float *targets, const int64_t *idx,
                              int32_t M, const float *norm, void *X, float *Y, void *stream);
dm_status dm_ws_column_stats(const float *data, int64_t rows, int32_t cols, float *stats,
                             void *stream);

/* Adjoint of one implicit step (no counterpart in the paper, whose
 * calibration uses finite differences): gradients of a loss L(q_{n+1},
 * qdot_{n+1}) with respect to the step's natural curvatures and its initial
 * state, by J^T lambda = dL/dq_{n+1} + dL/dqdot_{n+1} / dt with the
 * Jacobian of Eq. 16 at q_{n+1} (single rods: banded LDL^T, J symmetric;
 * rod networks and rods on the ground: the condensation solve applied to
 * J^T, which friction makes nonsymmetric), then
 * dL/dkappabar = -lambda . df/dkappabar, dL/dq_n = -lambda . df/dq_n -
 * dL/dqdot_{n+1}/dt, dL/dqdot_n = -lambda . df/dqdot_n.  The committed
 * reference frames (d1, beta, tangents) of step n are held fixed.
 * Precondition: the system holds the state of step n (dm_set_state and
 * dm_set_frames to the values before the step) and q_next is the converged
 * q_{n+1} of that step.  q_next, gq, gv (inputs) and gq0, gv0 (outputs) are
 * in the dm_get_state layout; gkbar (output) holds 2 values per interior node
 * in the dm_set_natural_curvature layout (all rods).  A joint node appears
 * once per rod in the layout: its loss gradients are summed over the copies
 * and its output gradients are written to its first copy (zeros in the
 * others), so that outputs can be fed back as inputs.  is_device: the
 * pointers are device (1) or host (0) memory.  Rods with edge-edge contact
 * solve J^T lambda with the transposed dense-band LU of the contact path;
 * edge-edge friction (pair_mu != 0), and networks with a limb jointed at
 * both ends, are rejected (DM_ERR_INVALID_ARG); the ground friction
 * force's dependence on x_n enters
 * dL/dq_n; fixed DOFs pass dL/dq_{n+1} through and get no velocity
 * gradient.  Implicit midpoint (solved as backward Euler over h = dt/2 in
 * y = (q_n + q_{n+1})/2): the same adjoint over h at y with the loss
 * gradients doubled (q_{n+1} = 2y - q_n, qdot_{n+1} = 2 (y - q_n)/h -
 * qdot_n), then dL/dq_n -= dL/dq_{n+1} and, on free DOFs, dL/dqdot_n -=
 * dL/dqdot_{n+1}.  Synchronises the stream; the state of step n is left in
 * place. */
dm_status dm_step_adjoint(dm_system *sys, const double *q_next, const double *gq,
                          const double *gv, double *gkbar, double *gq0, double *gv0,
                          int32_t is_device);

/* Frame chain of the adjoint of a rollout (no counterpart in the paper,
 * whose calibration uses finite differences).  dm_step_adjoint holds the
 * committed reference frames of its step fixed; over a rollout they come
 * from the earlier tangents by time-parallel transport (Sec. III), which
 * this call adds, one step at a time, going backwards:
 *   sigma_e = -((gq + gv/dt) - gv0/dt) at edge e's twist angle (0 if fixed)
 *             -- the adjoint of a rotation of e's committed director;
 *   phibar_e <- phibar_e + sigma_e;
 *   gq0 += the node-position gradient of -phibar_e [w(t_e, t_e') + w(t_e'', t_e)]
 *          through t = e/|e|, with w(a, b) = (a x b)/(1 + a . b) the
 *          holonomy of the transport, t_e, t_e', t_e'' the tangents in q,
 *          q_next and q_prev.
 * q_prev (the state before q, or NULL at the start of the rollout), q and
 * q_next (the step's states), gq, gv (the loss gradients given to
 * dm_step_adjoint for this step) and gv0 (its dL/dqdot_n output) are in the
 * dm_get_state layout; phibar is [sum (N_r-1)] (descriptor edge order, in:
 * the value carried from the later steps, zeros at the end of the rollout;
 * out: the value to carry to the earlier ones); gq0 (dm_step_adjoint's
 * dL/dq_n output) is updated in place.  Implicit midpoint, whose step energy
 * sees step n's frames transported to the tangents t_y of y = (q + q_next)/2:
 * sigma_e = -(2 gq + (gv - gv0)/h) with h = dt/2, and the source term of the
 * transport out of t_e splits into phibar_e(in) w(t_e, t_e') +
 * sigma_e w(t_e, t_y).  All device pointers; ordered on the system's stream
 * without synchronisation. */
dm_status dm_adjoint_frame_chain(dm_system *sys, const double *q_prev, const double *q,
                                 const double *q_next, const double *gq, const double *gv,
                                 const double *gv0, double *phibar, double *gq0);

/* Edge-edge contact (Sec. III-B, Eq. 10-11; params.self_contact != 0):
 * number of edge pairs closer than C + delta at the last evaluated Newton
 * iterate, summed over the systems (0 without edge-edge contact, -1 on a
 * CUDA error).  Synchronises the stream.  Contact acts within single rods
 * and within contact groups of rods (dm_system_desc.contact_groups; no
 * joints), on the ground or not; friction at the closest points (Eq. 12-13)
 * when pair_mu > 0, with the slip tolerance slip_nu.  dm_create_system
 * rejects rods with joints under edge-edge contact (DM_ERR_INVALID_ARG). */
int64_t dm_contact_pairs(dm_system *sys);

/* Per-kernel profile of dm_step calls made while profiling is on: CUDA-event
 * time on the system's stream, launch count and work units processed
 * (edges, stencils, DOF rows, systems) per kernel id.  Kernel ids:
 * 0 edge frames + stretch, 1 bend-twist stencils, 2 residual/Jacobian rows,
 * 3 banded solve, 4 step begin, 5 step commit, 6 ground contact/friction,
 * 7 general residual rows, 8 general assembly, 9 limb/Schur solve,
 * 10 learned warm start (features + network + apply), 11 edge-edge contact
 * (broadphase, pairs, derivatives), 12 contact-system LU, 13 bend-twist
 * Hessians (the Jacobian pass of a round), 14 Jacobian band rows, 15
 * bend-twist gradients and Hessians in one pass (the first round of a step;
 * every round of batches with rod networks), 16 residual and band rows in
 * one pass.  Ids 1 and 2 are then the residual pass (reference twist and
 * gradients; residual rows).  launches[k] counts the launches of id k's
 * phase, which for ids 8, 9, 11 and 12 is a short sequence of kernels.
 * Profiling adds two event records per launch; it is off by default. */
#define DM_NUM_KERNELS 17
typedef struct dm_profile {
  int64_t launches[DM_NUM_KERNELS];
  int64_t units[DM_NUM_KERNELS];
  double ms[DM_NUM_KERNELS];
} dm_profile;
dm_status dm_set_profiling(dm_system *sys, int32_t enable); /* also resets */
/* Newton rounds as a CUDA graph (default on): dm_step launches, per step,
 * one graph whose while node runs a round (every phase's kernels) and then a
 * one-thread kernel that keeps the loop going while a system is active, at
 * most the host loop's round limit; the host reads the control words once
 * per step instead of once per round.  The results are the same kernels in
 * the same order, so they are identical.  Off (0): the host drives the
 * rounds.  With a learned guess tried against the extrapolation, the trial
 * round runs before the graph.  Steps with profiling on use the host loop
 * (per-launch events). */
dm_status dm_set_graphs(dm_system *sys, int32_t enable);

/* The first Newton round of a step (whose guess essentially never meets the
 * tolerance) runs the fused passes: one kernel for the bend-twist
 * gradients and Hessians, one for the residual and band rows (default, 1).
 * Off (0): it runs the split passes of the later rounds (residual pass,
 * then the Jacobian pass for the systems above the tolerance), the same
 * arithmetic per entry in a different kernel grouping: results equal to
 * rounding.  Batches with rod networks always run the fused passes. */
dm_status dm_set_fused_first(dm_system *sys, int32_t enable);

/* Launch shapes chosen by dm_autotune. */
typedef struct dm_tuning {
  int32_t edge_threads;        /* threads per block, edge frames + stretch        */
  int32_t stencil_threads;     /* threads per block, bend-twist stencils          */
  int32_t stencil_per_thread;  /* stencils per thread (stencils per warp / 32)    */
  int32_t rows_threads;        /* threads per block, residual/Jacobian rows       */
  int32_t solve_warps;         /* rod solver: warps per block (2 rods per warp)   */
  int32_t solve_blocks_per_sm; /* rod solver: resident blocks per SM              */
  int32_t limb_factor_warps;   /* condensation: limbs (warps) per factor block    */
  int32_t limb_back_warps;     /* condensation: limbs (warps) per back-subst block */
  double us_per_launch[8];     /* measured time per launch of the chosen shapes:
                                  edge, stencil, rows, rod solve, limb solve with
                                  the chosen factor shape, with both chosen (us) */
} dm_tuning;
/* Autotuner: from the current committed state, runs `steps` steps per
 * candidate launch shape with per-kernel CUDA events and keeps, kernel by
 * kernel, the fastest shape (the default unless another is faster by more
 * than 2 %): threads per block and stencils per thread of the stencil
 * kernel, threads per block of the edge and row kernels, warps per block
 * (systems per block = 2 x warps) and blocks per SM of the persistent rod
 * solver, limbs per block of the condensation kernels.  Every shape computes
 * the same arithmetic per system.  The committed state, the profiling
 * switch and the counters are restored before returning; `out` (optional,
 * caller-owned) receives the choice.  Rejects a system on which the
 * learned warm start is enabled (DM_ERR_INVALID_ARG: it keeps a history of
 * the state).  Synchronises the stream. */
dm_status dm_autotune(dm_system *sys, int32_t steps, dm_tuning *out);
/* Applies launch shapes found by an earlier dm_autotune (for instance on
 * another system of the same workload) without timing anything:
 * edge_threads in {128, 256, 512}, stencil_threads in {32, 64, 128} with
 * stencil_per_thread in {1, 2}, rows_threads in {64, 128, 256},
 * solve_warps in {1, 2, 4} with solve_blocks_per_sm >= 1 within the rod
 * solver's occupancy, limb_factor_warps and limb_back_warps in {1, 2, 4}
 * within the shared memory of a block; us_per_launch is ignored.  Any other
 * value: DM_ERR_INVALID_ARG, nothing changed.  The shapes of kernels the
 * system does not launch are accepted and kept. */
dm_status dm_set_tuning(dm_system *sys, const dm_tuning *t);
dm_status dm_get_profile(dm_system *sys, dm_profile *out);
const char *dm_kernel_name(int32_t id); /* "" for unused ids */

/* Diagnostics: copies an internal device buffer of the last Newton
 * iteration to host memory (`out`, capacity n doubles).  Names: "q" (iterate),
 * "f" (residual, DOF order), "sg"/"sh" (stencil gradients [11][Ns] and packed
 * Hessians [66][Ns]), "es" (stretch force/Hessian [9][Ne]), "ef" (edge frames
 * [13][Ne]), "nt" (node contact terms [12][Nn]), "gen" (general-path matrix
 * storage).  Synchronises the stream.  Not part of the solve. */
dm_status dm_debug_copy(dm_system *sys, const char *name, double *out, int64_t n);

/* Measures the FP64 FMA throughput of the current device (GFLOP/s, an FMA
 * counted as 2 flops) with a short register-resident DFMA kernel: the
 * denominator of the FP64 roofline.  Returns a negative value on error. */
double dm_fp64_peak_gflops(void);

/* Message of the last failing call on this thread ("" if none). */
const char *dm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DISMECH_H */
