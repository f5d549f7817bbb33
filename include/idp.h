/*
 * libidp: GPU (sm_103a) explicit stage of the invariant-domain preserving,
 * second-order Q1 finite-element scheme for the compressible Euler equations
 * with convex limiting, after Maier & Kronbichler, "Efficient parallel 3D
 * computation of the compressible Euler equations with an invariant-domain
 * preserving second-order finite-element scheme" (arXiv:2007.00094).
 *
 * One context owns one mesh, its precomputed matrices (Sec. 3.2) and all
 * device buffers of the stage; every call returns an idp_status and no C++
 * exception crosses this boundary.  Work is enqueued on the stream given to
 * idp_create (NULL = the legacy default stream); calls that hand data back to
 * the host synchronise that stream, the others do not.
 *
 * Conventions for every call:
 *  - Conserved states are struct-of-arrays of float64, U[f*n + i] for the
 *    fields f = 0..4 = (rho, m_x, m_y, m_z, E) (Sec. 2), in the caller's node
 *    order.  The library may renumber nodes internally and always translates.
 *  - "on_device = 0": pointers are host memory owned by the caller and only
 *    read/written during the call.  "on_device = 1": pointers are device
 *    memory of the context's GPU (e.g. torch tensors), borrowed for the call
 *    and accessed in stream order on the context's stream.
 *  - Sizes are element counts, not bytes.
 */
#ifndef IDP_H
#define IDP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idp_ctx idp_ctx;

typedef enum {
  IDP_OK = 0,
  IDP_ERR_ARG = 1,                  /* invalid argument or mesh */
  IDP_ERR_CUDA = 2,                 /* a CUDA runtime call failed (see idp_last_error) */
  IDP_ERR_OOM = 3,                  /* device or host allocation failed */
  IDP_ERR_STATE_NOT_ADMISSIBLE = 4, /* rho <= 0 or epsilon <= 0 somewhere (Sec. 3.3) */
  IDP_ERR_CFL = 5,                  /* tau of RK stage 1 exceeds min_i m_i/(-2 d_ii) of a later stage */
  IDP_ERR_NONFINITE = 6,            /* a NaN or Inf appeared in the state */
  IDP_ERR_BOUNDS = 7,               /* idp_check_bounds found a violated invariant */
  IDP_ERR_TIMEOUT = 8,              /* a bounded device wait gave up */
  IDP_ERR_STATE = 9                 /* call out of order (e.g. step before mesh and state) */
} idp_status;

enum { IDP_PRECISION_FP64 = 0, IDP_PRECISION_MIXED = 1 };

/* Solver parameters (Sec. 3, Alg. 1-3). */
typedef struct {
  double gamma;             /* ratio of specific heats; the kernels require 7/5 (Sec. 2) */
  double cfl;               /* c_cfl in (0, 1] of the time-step rule (Sec. 3.3) */
  int limiter_passes;       /* passes of eq. (iterative-limiter), >= 2 (Sec. 3.5) */
  int newton_max;           /* Newton steps of Alg. 2 */
  double newton_tol;        /* Alg. 2 stops when Psi(t_L) <= newton_tol * rho*eps(U) */
  double newton_eps;        /* eps of Alg. 3 */
  int precision;            /* IDP_PRECISION_FP64, or IDP_PRECISION_MIXED: per-entry flux, wavespeed,
                               antidiffusive-flux and limiter arithmetic in FP32; state, its
                               accumulation, mass division, tau and the final limiter check in FP64 */
  int schedule;             /* kernel schedule id; 0 = default */
  int64_t barrier_spin_limit; /* iteration limit of any device-side wait */
  int relax;                /* != 0: relax the local bounds, rho_min (1 - r_i), rho_max (1 + r_i),
                               phi_min (1 - r_i) with r_i = (m_i / |Omega|)^(1/2), |Omega| the volume of
                               the node's instance (Sec. 3.9 remark; the formula is project-defined);
                               0 (default): the bounds as Alg. 1 states them */
  int entry_table;          /* 1 (default): in the FP32-mixed stage, when the mesh has at most 4096 distinct
                               FP32 entries (c_ij, m_ij, |c_ij|, 1/|c_ij|) -- uniform tensor grids --
                               store each stored entry as a 16-bit index into a table of the distinct
                               values instead of six per-entry floats (the matrices of Sec. 3.1,
                               precomputed once as Sec. 3.2 asks), and, when the rows fall into at
                               most 4096 patterns, read column indices and transposed positions from
                               the patterns (idp_row_pattern_count; the FP64 stage reads its column
                               indices, transposed positions and flags from patterns too, on any mesh
                               whose rows fall into at most 4096); 0: per-entry arrays.  Results are
                               bitwise the same either way. */
  int adjoint_store_stages; /* 1 (default): idp_adjoint_record also reserves, when the device has the
                               memory (112 B per stored entry and 200 B per node, for each of the
                               3 x checkpoint_every stages of a segment, plus 4 GiB to spare), room
                               for the traces of one checkpoint segment, so that idp_adjoint_backward
                               evaluates each stage forward once instead of twice; 0: the traced
                               stages are recomputed.  Gradients are bitwise the same either way. */
  int renumber;             /* row order of the library, for the locality of the neighbour gathers on
                               meshes whose nodes come in an arbitrary order.  0 (default): the
                               caller's node order; 1: reverse Cuthill-McKee over the stencil graph,
                               every row sum in the caller's column order, so results are bitwise
                               those of 0; 2: Morton (Z-order) of the node coordinates, so that the 32
                               rows of a slice are a compact block of space, and every row's entries
                               ordered by their offset in the reference cell, so that a warp's gathers
                               at one slot are neighbours at one offset whatever order the caller's ids
                               come in: results equal those of 0 up to the rounding of the reordered
                               sums (mesh uploads only: with
                               idp_upload_sparsity, which has no coordinates, IDP_ERR_ARG).  States,
                               fields, gradients, matrices and instance offsets stay in the caller's
                               numbering at this interface. */
} idp_config;

/* Fills the defaults: gamma 1.4, cfl 0.5, 2 limiter passes, 2 Newton steps,
 * newton_tol 1e-10, newton_eps = DBL_EPSILON, FP64, schedule 0, no bound
 * relaxation, entry table on, adjoint stage traces stored. */
void idp_config_default(idp_config* cfg);

/* Creates a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t (may be NULL).  *out receives the context; the caller releases
 * it with idp_destroy.  Fails with IDP_ERR_ARG for a gamma other than 7/5,
 * cfl outside (0,1] or limiter_passes < 1. */
idp_status idp_create(const idp_config* cfg, void* cuda_stream, idp_ctx** out);
void idp_destroy(idp_ctx* ctx);
const char* idp_last_error(const idp_ctx* ctx);
const char* idp_status_string(idp_status s);

/* Uploads a hexahedral Q1 mesh and precomputes the matrices of Sec. 3.1
 * eq. (matrices): m_ij, m_i and c_ij, by exact Gauss quadrature on each
 * trilinear cell; n_ij and b_ij are formed on the fly (Sec. 3.2).
 *   n_nodes, n_cells : sizes
 *   cells            : host, 8*n_cells node ids, local vertex v = a + 2b + 4c
 *                      at reference corner (a, b, c) in {0,1}^3
 *   cell_xyz         : host, 24*n_cells vertex positions seen from each cell
 *                      (unwrapped across periodic seams); every cell must have
 *                      a positive Jacobian at its Gauss points (else IDP_ERR_ARG)
 *   node_bc          : host, n_nodes flags or NULL: bits 1, 2, 4 = slip wall
 *                      with an x-, y-, z-normal face; 8 = inflow (Dirichlet)
 *   inflow_state     : host, 5 conserved values used at inflow nodes, or NULL
 * Set-up work runs on the host and is not part of a stage. */
idp_status idp_upload_mesh_hex(idp_ctx* ctx, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                               const double* cell_xyz, const int32_t* node_bc, const double* inflow_state);
/* The same for a 2D mesh of Q1 quadrilaterals (Sec. 3.1 with d = 2, 9-point
 * stencil): cells holds 4 node ids per cell (local vertex v = a + 2b for the
 * reference corner (a, b)), cell_xy 2 coordinates per vertex (unwrapped on
 * periodic axes), node_bc as for hexahedra (IDP_BC_SLIP_Z unused).  The state
 * keeps 5 fields (rho, m_x, m_y, m_z, E): c_ij has no z component, so an
 * initial m_z = 0 stays exactly 0 and the update is the 2D one. */
idp_status idp_upload_mesh_quad(idp_ctx* ctx, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                                const double* cell_xy, const int32_t* node_bc, const double* inflow_state);

/* Uploads pre-assembled matrices instead of a mesh.  The scheme needs only
 * the matrices of Sec. 3.1 eq. (matrices), precomputed once (Sec. 3.2):
 * callers that assemble them themselves (other element types, their own
 * quadrature) pass them here in CSR form, in their own node numbering.
 *   n_nodes      : number of nodes (rows)
 *   rowptr       : host, n_nodes+1 offsets, rowptr[0] = 0, nnz = rowptr[n_nodes]
 *   col          : host, nnz column ids, strictly increasing within each row;
 *                  every row holds its diagonal and at least one neighbour, and
 *                  the pattern is structurally symmetric (entry (j,i) exists
 *                  for every entry (i,j)), else IDP_ERR_ARG
 *   mij          : host, nnz consistent masses m_ij
 *   cij          : host, 3*nnz, c_ij component-major (x row, y row, z row;
 *                  a zero z row for d = 2)
 *   mi           : host, n_nodes lumped masses m_i > 0, or NULL for the row
 *                  sums of m_ij (equal to int phi_i by partition of unity)
 *   node_bc, inflow_state : as for idp_upload_mesh_hex
 * Entries must be finite (else IDP_ERR_ARG).  Pairs with c_ji = -c_ij
 * bitwise share one wavespeed evaluation; all others evaluate both
 * orientations (Sec. 3.3).  The buffers are copied during the call. */
idp_status idp_upload_sparsity(idp_ctx* ctx, int64_t n_nodes, const int64_t* rowptr, const int64_t* col,
                               const double* mij, const double* cij, const double* mi, const int32_t* node_bc,
                               const double* inflow_state);

/* Number of nodes and of stored matrix entries (the stencil sizes I(i) of
 * Sec. 3.1 summed over i). */
idp_status idp_mesh_info(idp_ctx* ctx, int64_t* n_nodes, int64_t* nnz);

/* Number of distinct FP32 entries in the table of idp_config.entry_table
 * (*n_values = 0: the mixed stage reads per-entry arrays, because the context
 * is FP64, the table is off, or the mesh has more than 4096 distinct entries).
 * IDP_ERR_STATE before a mesh is uploaded. */
idp_status idp_entry_table_size(idp_ctx* ctx, int64_t* n_values);

/* Number of row patterns of the stage (meshes with grid connectivity, with
 * idp_config.entry_table = 1): rows whose entries have the same column
 * offsets j - i, the same transposed-entry positions, flags and (FP32-mixed)
 * table codes share one pattern, and the kernels read each entry's column and
 * transposed position from the pattern (a small table) instead of per-entry
 * index arrays.  In FP64 contexts the patterns carry no table code and also
 * serve jittered meshes, whose connectivity is still the grid's.
 * *n_patterns = 0: per-entry index arrays (table off, an FP32-mixed context
 * without an entry table, or more than 4096 patterns, as on renumbered or
 * unstructured meshes).  Results are bitwise the same either way.
 * IDP_ERR_STATE before a mesh is uploaded. */
idp_status idp_row_pattern_count(idp_ctx* ctx, int64_t* n_patterns);

/* Copies the assembled matrices back in the caller's numbering as CSR with
 * columns sorted by the caller's node id: rowptr (n+1), col (nnz), mij (nnz),
 * cij (3*nnz, component-major), mi (n).  Host pointers; any may be NULL. */
idp_status idp_get_matrices(idp_ctx* ctx, int64_t* rowptr, int64_t* col, double* mij, double* cij, double* mi);

/* Sets the current state U^n (5*n values).  Rejects states with rho <= 0 or
 * epsilon <= 0 (Sec. 3.3, admissible snapshots) with
 * IDP_ERR_STATE_NOT_ADMISSIBLE; synchronises the stream. */
idp_status idp_init_state(idp_ctx* ctx, const double* U, int on_device);

/* Copies the current state out (5*n values); synchronises the stream. */
idp_status idp_get_state(idp_ctx* ctx, double* U, int on_device);

/* Enqueues n_steps SSP-RK3 steps (Sec. 3.6 eq. ssprk3), each three
 * euler_steps (Alg. 1) with tau_n fixed by the first one.  Returns without
 * waiting for the GPU; device-side errors (CFL, non-finite) are latched and
 * returned by idp_synchronize.  A step that meets a CFL violation leaves the
 * state at its beginning and every later step of the same call is skipped. */
idp_status idp_step(idp_ctx* ctx, int n_steps);

/* One euler_step (Alg. 1 plus boundary post-processing) applied to the
 * current state in place, U <- E(U).  tau <= 0: tau_n is computed from the
 * CFL rule; tau > 0: tau is used and checked against min_i m_i/(-2 d_ii).
 * With trace != 0 the intermediate fields of this stage are kept for
 * idp_get_field.  Synchronises and returns the stage's status. */
idp_status idp_euler_step(idp_ctx* ctx, double tau, int trace, double* tau_out);

/* Waits for the context's stream and returns (then clears) the latched
 * device status. */
idp_status idp_synchronize(idp_ctx* ctx);

/* Simulated time accumulated by idp_step and the last tau_n; synchronises. */
idp_status idp_get_time(idp_ctx* ctx, double* t, double* last_tau);
idp_status idp_set_time(idp_ctx* ctx, double t);

/* Intermediate fields of the last traced euler_step, in caller order. */
enum {
  IDP_FIELD_D = 0,      /* d^L_ij, nnz CSR (diagonal = d_ii) */
  IDP_FIELD_ALPHA = 1,  /* alpha_i, n */
  IDP_FIELD_UL = 2,     /* low-order update, 5n */
  IDP_FIELD_R = 3,      /* R_i, 5n */
  IDP_FIELD_BOUNDS = 4, /* rho_min, rho_max, phi_min: 3n */
  IDP_FIELD_P = 5,      /* P_ij of Step 4, 5*nnz field-major */
  IDP_FIELD_L4 = 6,     /* limiter values of Step 4, nnz */
  IDP_FIELD_U5 = 7,     /* state after limiter pass 1, 5n */
  IDP_FIELD_L5 = 8,     /* limiter values recomputed in pass 1, nnz */
  IDP_FIELD_ULIM = 9,   /* state after the last pass, before boundary conditions, 5n */
  IDP_FIELD_TAU_MAX = 10 /* min_i m_i/(-2 d_ii): 1 value */
};
idp_status idp_get_field(idp_ctx* ctx, int which, double* out);

/* Invariant checks (Sec. 3.3: the admissible set; Sec. 3.9: the local
 * bounds that the limiter enforces).
 *
 * idp_check_bounds checks
 *  (a) the current state: counts of nodes with rho <= 0, epsilon <= 0 or a
 *      non-finite value, and the smallest rho and epsilon;
 *  (b) the output of the last euler_step the context ran on the current state
 *      (idp_step, idp_euler_step, or a forward evaluation inside the
 *      idp_adjoint_* calls), after its last limiter pass and before boundary
 *      values and the SSP-RK3 blend, against that stage's own bounds
 *      rho_min_i <= rho_i <= rho_max_i and phi(U_i) >= phi_min_i.  The
 *      entropy bound is tested as the limiter tests it (Alg. 2):
 *      Psi = rho eps - phi_min rho^(gamma+1) >= -slack_phi (|rho eps| +
 *      phi_min rho^(gamma+1)); the density bounds with a relative slack
 *      slack_rho.  Slacks: FP64 1e-13 (rho) and 2e-13 (Psi: the limiter
 *      accepts Psi down to -1e-13 of this scale, plus rounding of the row
 *      sum); FP32-mixed 1e-7 and 1e-6 (increments summed in FP32).  Before
 *      any stage has run on the state, n_bound_rows is 0 and (b) is skipped.
 * Synchronises.  Returns IDP_ERR_BOUNDS when any count is non-zero.
 *
 * idp_check_local_bounds runs the same two checks on a caller-given state U
 * (5 x n, caller order) against caller-given bounds (3 x n: rho_min,
 * rho_max, phi_min, caller order, the layout of IDP_FIELD_BOUNDS); host
 * pointers, or device pointers with on_device != 0.  It uses stage scratch
 * buffers of the context and leaves its state untouched. */
typedef struct {
  int64_t n_rho_nonpositive;  /* (a) */
  int64_t n_eps_nonpositive;
  int64_t n_nonfinite;
  double rho_min;
  double eps_min;
  int64_t n_bound_rows;       /* (b): rows checked, 0 when skipped */
  int64_t n_rho_below_min;    /* rho < rho_min - slack_rho |rho_min| (or NaN) */
  int64_t n_rho_above_max;    /* rho > rho_max + slack_rho |rho_max| (or NaN) */
  int64_t n_phi_below_min;    /* Psi below -slack_phi of its scale (or NaN) */
  double rho_min_violation;   /* max_i (rho_min_i - rho_i) / |rho_min_i|; <= 0: the bound holds everywhere */
  double rho_max_violation;   /* max_i (rho_i - rho_max_i) / |rho_max_i| */
  double phi_min_violation;   /* max_i -Psi_i / (|rho eps| + phi_min rho^(gamma+1))_i */
  double slack_rho;           /* the relative slacks the counts use */
  double slack_phi;
} idp_bounds_report;
idp_status idp_check_bounds(idp_ctx* ctx, idp_bounds_report* out);
idp_status idp_check_local_bounds(idp_ctx* ctx, const double* U, const double* bounds, int on_device,
                                  idp_bounds_report* out);

/* Number of kernel launches the last idp_step/idp_euler_step enqueued. */
int64_t idp_launch_count(const idp_ctx* ctx);

/* Per-kernel timing for benchmarks.  idp_profile(ctx, 1) synchronises the
 * stream, clears earlier records and from then on records a CUDA event pair
 * on the context's stream around every kernel launch (Alg. 1 steps 0-6);
 * idp_profile(ctx, 0) stops recording.  idp_profile_read synchronises and
 * writes, per kernel id, the summed event time in milliseconds and the
 * launch count since recording started (arrays of IDP_N_KERNELS); the
 * reverse-mode calls record their kernels too. */
enum {
  IDP_KERNEL_NODE = 0,        /* Step 0: per-node quantities */
  IDP_KERNEL_EDGE = 1,        /* Step 1: d_ij and alpha_i */
  IDP_KERNEL_DIAG = 2,        /* Step 2: d_ii and tau */
  IDP_KERNEL_LOW_ORDER = 3,   /* Step 3: low-order update, R_i, bounds */
  IDP_KERNEL_FLUX_LIMIT = 4,  /* Step 4: P_ij and l_ij */
  IDP_KERNEL_LIMITER_PASS = 5,/* Step 5: limiter pass with new l_ij */
  IDP_KERNEL_FINAL = 6,       /* Step 6: last pass, boundary values, RK blend */
  /* reverse mode (idp_adjoint_*): one id per reversed step */
  IDP_KERNEL_ADJ_FINAL = 7,   /* Step 6 reversed: boundary values, last pass */
  IDP_KERNEL_ADJ_PASS = 8,    /* Step 5 reversed */
  IDP_KERNEL_ADJ_FLUX = 9,    /* Step 4 reversed: P_ij, first limiter */
  IDP_KERNEL_ADJ_LOW = 10,    /* Step 3 reversed: U^L, R_i, bounds */
  IDP_KERNEL_ADJ_TAU = 11,    /* adjoint of tau_n: sum, CFL arg-min */
  IDP_KERNEL_ADJ_DIAG = 12,   /* Step 2 reversed */
  IDP_KERNEL_ADJ_EDGE = 13,   /* Step 1 reversed: alpha_i, fluxes, d_ij */
  IDP_KERNEL_ADJ_GATHER = 14, /* transposed-entry gather of the input adjoint */
  IDP_N_KERNELS = 15
};
idp_status idp_profile(idp_ctx* ctx, int enable);
idp_status idp_profile_read(idp_ctx* ctx, double* ms, int64_t* launches);

/* Many independent instances in one context (batches of small problems): the
 * uploaded mesh is the union of instance meshes whose nodes occupy the
 * contiguous ranges [node_offsets[k], node_offsets[k+1]) (n_instances + 1
 * host values, 0 first, n_nodes last) and share no matrix entry (else
 * IDP_ERR_ARG).  Every instance then takes its own tau_n = c_cfl min over its
 * nodes of m_i/(-2 d_ii) (Sec. 3.3) and keeps its own time; all instances
 * advance in the same kernel launches.  Call after idp_upload_mesh_hex;
 * synchronises. */
idp_status idp_set_instances(idp_ctx* ctx, int64_t n_instances, const int64_t* node_offsets);
/* Per-instance time and last tau_n (host arrays of n_instances, either may be
 * NULL); synchronises. */
idp_status idp_get_instance_times(idp_ctx* ctx, double* t, double* last_tau);

/* Launch schedule of the stage kernels: block_size 64, 128 or 256 threads
 * (one row per thread); use_graph != 0 captures one SSP-RK3 step in a CUDA
 * graph on first use and replays it in idp_step; persistent != 0 runs each
 * euler_step as ONE cooperative launch (all blocks co-resident, grid-stride
 * over the rows, a grid barrier where the paper's global synchronisations
 * are, Fig. 2).  A barrier wait is bounded by idp_config.barrier_spin_limit
 * polls; one that runs out ends the launch and latches IDP_ERR_TIMEOUT.
 * Traced and profiled stages always take the per-step kernels.  Results do
 * not depend on the schedule.  A new context uses block 64, per-step kernels
 * and no graph. */
idp_status idp_set_schedule(idp_ctx* ctx, int block_size, int use_graph, int persistent);
/* Self-test of the persistent schedule's grid barrier: a cooperative launch
 * of `blocks` blocks (64 threads) that pass `rounds` barriers, each wait
 * bounded by spin_limit polls; with skip_block0 != 0 block 0 never arrives,
 * so the others' waits run out.  *passes (may be NULL) receives the number
 * of block-passes (blocks x rounds when nothing is skipped).  Returns
 * IDP_ERR_TIMEOUT when a wait ran out (the context stays usable), IDP_ERR_CUDA
 * when the device cannot hold the blocks at once; synchronises. */
idp_status idp_barrier_selftest(idp_ctx* ctx, int blocks, int rounds, int skip_block0, long long spin_limit,
                                int* passes);
/* Times every schedule (block size x graph replay x persistent) for `steps`
 * SSP-RK3 steps on the current state, skips schedules the device cannot run,
 * keeps the fastest and restores the state and clocks; writes the choice and
 * its milliseconds per step (any output pointer may be NULL); synchronises. */
idp_status idp_autotune(idp_ctx* ctx, int steps, int* block_size, int* use_graph, int* persistent,
                        double* ms_per_step);

/* Reverse mode (discrete adjoint) of the FP64 scheme, for gradients of a
 * functional J(U^N) with respect to the state U^0 it evolved from.  The
 * adjoint differentiates the stage as computed (Alg. 1 with the limiter of
 * Alg. 2/3 and the bound of Sec. 3.7, Newton steps included); at
 * non-smooth points it takes the branch the forward pass took:
 * min(l_ij, l_ji) and every min/max bound go to the first extremal entry
 * (in the row's column order: the caller's, or the cell-offset order of
 * idp_config.renumber = 2),
 * tau_n = c_cfl min_i m_i/(-2 d_ii) (Sec. 3.3) to the first row attaining
 * the minimum.  Supported for precision IDP_PRECISION_FP64,
 * limiter_passes = 2 and a single instance, else IDP_ERR_ARG.  The
 * adjoint buffers (about 32 doubles per stencil entry) are allocated on
 * first use.  Arrays are (5, n_nodes) field-major doubles in caller order;
 * on_device != 0: device pointers, else host pointers.
 *
 * idp_adjoint_euler_step: the adjoint gU of the input U of one euler_step
 * (Alg. 1, boundary post-processing included) given the adjoint gE of its
 * output.  tau > 0: fixed tau_n, and *g_tau (host, may be NULL) receives
 * dJ/dtau_n; tau <= 0: tau_n is computed from U (first RK stage) and gU
 * includes its dependence on U (*g_tau then holds the partial derivative
 * at fixed tau_n).  Leaves the context's state untouched; synchronises. */
idp_status idp_adjoint_euler_step(idp_ctx* ctx, const double* U, double tau, const double* gE, double* gU,
                                  double* g_tau, int on_device);
/* idp_adjoint_record: advances the context's state by n_steps SSP-RK3 steps
 * (eq. ssprk3, as idp_step) and keeps what the backward sweep needs: a
 * checkpoint of the state every checkpoint_every steps (clamped to n_steps)
 * and tau_n of every step, replacing any earlier record.  Device memory:
 * ceil(n_steps/checkpoint_every) + 3 checkpoint_every states.  Synchronises.
 * idp_adjoint_backward: given the adjoint gU_final of the state after the
 * recorded steps, writes the adjoint gU_initial of the state before them.
 * Each checkpoint segment is recomputed forward once, then every stage is
 * re-evaluated with its trace and reversed (eq. ssprk3 blends included).
 * The context's state, time and record stay as they were; synchronises.
 * IDP_ERR_STATE without a record. */
idp_status idp_adjoint_record(idp_ctx* ctx, int n_steps, int checkpoint_every);
idp_status idp_adjoint_backward(idp_ctx* ctx, const double* gU_final, double* gU_initial, int on_device);

/* Domain decomposition (Sec. 4.1, Fig. 1): the rows split into contiguous
 * ranges, each shard owning one range and holding one ghost layer (the
 * neighbours of its rows that other shards own), and the values shards
 * exchange at the stage's synchronisation points (Fig. 2).
 *
 * idp_shard_plan_create builds the plan of a CSR pattern (the conventions of
 * idp_upload_sparsity: host rowptr n_nodes+1, col nnz, columns increasing in
 * each row, structurally symmetric) for n_shards ranges row_begin (host,
 * n_shards+1 values, 0 first, n_nodes last, strictly increasing; NULL: equal
 * ranges).  IDP_ERR_ARG for a bad pattern or partition.  The plan is host
 * memory only (no GPU needed); release it with idp_shard_plan_destroy.
 * Queries, all host arrays sized by idp_shard_plan_info:
 *  - info: local node count (own rows and ghosts), the local ids of the own
 *    rows [own_begin, own_end), local entry count; any pointer may be NULL;
 *  - nodes: the global id of every local node, increasing (local ids keep
 *    the global order, so each row keeps its column order);
 *  - csr: the local CSR (rowptr, local col) of the entries between local nodes
 *    (all entries of an own row, those inside the shard of a ghost row) and
 *    the global CSR entry of each (any pointer may be NULL);
 *  - list: the exchange list of kind IDP_SEND_NODES (own rows that are ghosts
 *    of peer), IDP_RECV_NODES (ghosts owned by peer), IDP_SEND_ENTRIES
 *    (entries (g, i) of own rows g with i owned by peer), IDP_RECV_ENTRIES
 *    (entries (g, i) of ghost rows g owned by peer with i an own row), as
 *    local node or local entry ids in the order of global ids: a shard's send
 *    list for a peer and the peer's receive list for it enumerate the same
 *    values.  *count receives the length; ids (may be NULL) the list. */
typedef struct idp_shard_plan idp_shard_plan;
enum { IDP_SEND_NODES = 0, IDP_RECV_NODES = 1, IDP_SEND_ENTRIES = 2, IDP_RECV_ENTRIES = 3 };
idp_status idp_shard_plan_create(int64_t n_nodes, const int64_t* rowptr, const int64_t* col, int n_shards,
                                 const int64_t* row_begin, idp_shard_plan** out);
void idp_shard_plan_destroy(idp_shard_plan* plan);
idp_status idp_shard_plan_info(const idp_shard_plan* plan, int shard, int64_t* n_local, int64_t* own_begin,
                               int64_t* own_end, int64_t* nnz_local);
idp_status idp_shard_plan_nodes(const idp_shard_plan* plan, int shard, int64_t* nodes);
idp_status idp_shard_plan_csr(const idp_shard_plan* plan, int shard, int64_t* rowptr, int64_t* col, int64_t* entry);
idp_status idp_shard_plan_list(const idp_shard_plan* plan, int shard, int peer, int kind, int64_t* count,
                               int64_t* ids);

/* The sharded stage on the current GPU: one context per shard of the plan
 * (its rows and ghosts, the matrices of idp_upload_sparsity restricted to
 * them), all on cuda_stream.  Each euler_step runs phase by phase over the
 * shards, and between phases the shards exchange, at the synchronisation
 * points of Fig. 2 (Sec. 4.1): alpha_j and a min-reduction of the CFL bound
 * after Step 2, R_j after Step 3, l_ji after Step 4 and after every limiter
 * pass, U_j after Step 6.  Ghost rows run Steps 0-1 only.  Every shard works
 * on a stream of its own (created by the group, ordered after cuda_stream at
 * the start of idp_shards_step and joined into it at the end), and the
 * exchanges order the shards by events: a gather kernel on the sender's
 * stream, one device-to-device cudaMemcpyAsync into the receiver's buffer, a
 * scatter kernel on the receiver's stream.  Every own row computes what an
 * unsharded context computes, in the same order: states, time and tau_n are
 * bitwise those of idp_step on the same matrices.
 *   cfg           : NULL for the defaults; FP64 or FP32-mixed precision (the
 *                   mixed stage exchanges its FP32 alpha, R and l), relax = 0,
 *                   renumber = 0 (else IDP_ERR_ARG)
 *   plan          : borrowed during the call (the group keeps a copy)
 *   mij, cij, mi, node_bc, inflow_state : the whole mesh's arrays, as for
 *                   idp_upload_sparsity with the plan's pattern; mi NULL: the
 *                   row sums of m_ij
 * idp_shards_init_state / idp_shards_get_state take the whole state (5 x
 * n_nodes host doubles, global numbering; init rejects non-admissible states)
 * and wait for all shards first;
 * idp_shards_step enqueues n_steps SSP-RK3 steps (eq. ssprk3) without waiting;
 * idp_shards_synchronize waits and returns the first latched error of any
 * shard (a shard with an error in the third stage keeps its state, the others
 * may not); idp_shards_get_time as idp_get_time.  idp_shards_context lends the
 * context of one shard (for idp_get_field and the like; local numbering, its
 * ghost rows hold exchanged or partial values); it stays owned by the group.
 * idp_shards_halo_size: values per exchange summed over all links (node
 * values per field, entry values) and the launches of the last
 * idp_shards_step; any pointer may be NULL. */
typedef struct idp_shards idp_shards;
idp_status idp_shards_create(const idp_config* cfg, void* cuda_stream, const idp_shard_plan* plan, const double* mij,
                             const double* cij, const double* mi, const int32_t* node_bc, const double* inflow_state,
                             idp_shards** out);
void idp_shards_destroy(idp_shards* sh);
const char* idp_shards_last_error(const idp_shards* sh);
idp_status idp_shards_init_state(idp_shards* sh, const double* U);
idp_status idp_shards_get_state(idp_shards* sh, double* U);
idp_status idp_shards_step(idp_shards* sh, int n_steps);
idp_status idp_shards_synchronize(idp_shards* sh);
idp_status idp_shards_get_time(idp_shards* sh, double* t, double* last_tau);
idp_status idp_shards_context(idp_shards* sh, int shard, idp_ctx** out);
idp_status idp_shards_halo_size(const idp_shards* sh, int64_t* node_values, int64_t* entry_values,
                                int64_t* launches);

/* FP64 fused multiply-add rate of the current GPU, for the roofline of the
 * FP64 stage (its heavy kernels are bound by the FP64 pipe; the paper has no
 * counterpart, it measures CPU peaks instead, Sec. 5, Table 1).  Runs one
 * launch of independent FMA chains on a full grid of the current device, on
 * cuda_stream (may be NULL), fma_per_thread (>= 16) FMAs per thread, and
 * writes the rate in TFLOP/s (2 flops per FMA) and, if ms is not NULL, the
 * launch's CUDA-event time.  Synchronises the stream; allocates nothing. */
idp_status idp_probe_fp64_peak(void* cuda_stream, int64_t fma_per_thread, double* tflops, double* ms);

/* Time-step bound without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory themselves, such as a host framework that hands out all
 * device memory from its own pool (an allocation behind its back escapes its
 * accounting and may fail under its memory cap), or a long-running service
 * that allocates everything at start-up and forbids allocation afterwards.
 * Those callers cannot create an idp_ctx, which allocates, so they pass their
 * own device arrays instead.
 *
 * Computes tau_max = min_i m_i / (-2 d_ii), the bound that idp_euler_step
 * scales by c_cfl and reports as IDP_FIELD_TAU_MAX, for the state U:
 *   n_nodes, nnz : sizes; 1 <= n_nodes <= IDP_NOALLOC_MAX_NODES, else IDP_ERR_ARG
 *   rowptr, col  : device, CSR pattern (n_nodes+1, nnz), columns sorted per row
 *   cij          : device, 3*nnz, c_ij component-major (as idp_get_matrices)
 *   mi           : device, n_nodes lumped masses
 *   U            : device, 5*n_nodes conserved state
 *   tau_max      : device, 1 double written by the kernel; NaN when some node
 *                  of U is not admissible (rho <= 0, epsilon <= 0 or NaN)
 *   cuda_stream  : cudaStream_t (may be NULL); the call does not synchronise.
 * It calls no cudaMalloc or cudaFree.  Its scratch is a fixed device array in
 * the library (one partial minimum per 128 nodes, 128 KiB), which every GPU
 * that loads the library keeps until the process exits.  Each call looks up
 * that array's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing); the first call on a device may also load the
 * library's device code, so make that first call before any stream capture.
 * All calls share the array, so calls that overlap on the GPU (e.g. on two
 * streams at once) race and give wrong results; the call clears what must
 * start at zero itself. */
#define IDP_NOALLOC_MAX_NODES 2097152
idp_status idp_tau_max_noalloc(int64_t n_nodes, int64_t nnz, const int64_t* rowptr, const int64_t* col,
                               const double* cij, const double* mi, const double* U, double* tau_max,
                               void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
