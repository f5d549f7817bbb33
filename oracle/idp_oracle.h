/*
 * FP64 CPU oracle for one explicit stage of the invariant-domain preserving
 * Q1 Euler scheme with convex limiting (Maier & Kronbichler, arXiv:2007.00094,
 * Sec. 3, Alg. 1-3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path includes, links or
 * calls this code: only tests/, the smoke check and the CPU-baseline leg of
 * bench.py do.  It shares no code, header or table with the CUDA library.
 *
 * Layout: conserved states are struct-of-arrays, U[f*n + i] for the fields
 * f = 0..4 = (rho, m_x, m_y, m_z, E).  Matrices are CSR with sorted columns
 * (the diagonal included); vector-valued c_ij is stored component-major,
 * c[d*nnz + k].
 */
#ifndef IDP_ORACLE_H
#define IDP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double gamma;       /* ratio of specific heats (Sec. 2), 7/5 */
  double cfl;         /* c_cfl in (0,1] (Sec. 3.3) */
  int limiter_passes; /* passes of eq. (iterative-limiter), >= 2 (Sec. 3.5) */
  int newton_max;     /* Newton steps of Alg. 2 */
  double newton_tol;  /* Alg. 2 stops once Psi(t_L) <= newton_tol * rho*eps(U) */
  double newton_eps;  /* eps of Alg. 3 */
  int n_threads;      /* OpenMP threads over rows (results do not depend on it) */
  int relax;          /* != 0: relax the local bounds (Sec. 3.9 remark; Reading A14) */
  double psi_margin;  /* Psi >= -psi_margin (|rho eps| + |phi_min rho^(gamma+1)|) counts as admissible in
                         Alg. 2 (Reading A27, the round-off safeguard of Alg. 3's caption); 0: strict */
} orc_params;

typedef struct {
  int64_t n;             /* number of nodes */
  const int64_t* rowptr; /* n+1 */
  const int64_t* col;    /* nnz, sorted within each row */
  const double* mij;     /* consistent mass m_ij, nnz */
  const double* cij;     /* c_ij, 3*nnz component-major */
  const double* mi;      /* lumped mass m_i, n */
  const int32_t* bc;     /* boundary flags per node (1,2,4 slip x,y,z; 8 inflow) */
  const double* inflow;  /* 5 conserved inflow values, or NULL */
} orc_mesh;

/* Optional intermediate outputs of one euler_step (any pointer may be NULL). */
typedef struct {
  double* d;       /* d^L_ij, nnz (diagonal = d_ii) */
  double* alpha;   /* alpha_i, n */
  double* tau_max; /* 1: min_i m_i / (-2 d_ii) */
  double* UL;      /* low-order update, 5n */
  double* R;       /* R_i, 5n */
  double* bounds;  /* rho_min, rho_max, phi_min, 3n (field-major) */
  double* P;       /* P_ij after Step 4, 5*nnz field-major */
  double* l4;      /* limiter values after Step 4, nnz */
  double* U5;      /* state after limiter pass 1, 5n */
  double* l5;      /* limiter values recomputed in pass 1, nnz */
  double* Ulim;    /* state after the last pass, before boundary conditions, 5n */
} orc_trace;

enum { ORC_OK = 0, ORC_ERR_CFL = 1, ORC_ERR_STATE = 2, ORC_ERR_ARG = 3 };

/* ---- mesh set-up (Sec. 3.1, eq. "matrices") ---- */
int64_t orc_sparsity(int64_t n_nodes, int64_t n_cells, const int64_t* cells, int64_t* rowptr, int64_t* col);
int orc_assemble(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xyz,
                 const int64_t* rowptr, const int64_t* col, double* mij, double* cij, double* mi);
/* d = 2: Q1 quadrilaterals, 4 vertices and 2 coordinates per vertex; c_ij z row zero */
int64_t orc_sparsity_nv(int64_t n_nodes, int64_t n_cells, int nv, const int64_t* cells, int64_t* rowptr,
                        int64_t* col);
int orc_assemble_quad(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xy,
                      const int64_t* rowptr, const int64_t* col, double* mij, double* cij, double* mi);

/* ---- pointwise building blocks ---- */
void orc_node_quantities(const double* U, double gamma, double* out /* p, c, phi, eta, eta'(5) */);
double orc_lambda_max(const double* n, const double* Ui, const double* Uj, double gamma);
double orc_limiter(const double* U, const double* P, double rho_min, double rho_max, double phi_min,
                   const orc_params* prm);
double orc_psi(const double* U, double phi_min, double gamma);
/* orc_limiter, also reporting the admissibility tests decided by the Psi
 * margin (count, and the largest |Psi| / scale among them); either may be NULL */
double orc_limiter_ex(const double* U, const double* P, double rho_min, double rho_max, double phi_min,
                      const orc_params* prm, int* margin_hits, double* margin_worst);
void orc_limiter_many(int64_t m, const double* U, const double* P, const double* bounds, const orc_params* prm,
                      double* t, int* hits, double* worst);

/* ---- one euler_step (Alg. 1) and one SSP-RK3 step (eq. "ssprk3") ---- */
int orc_euler_step(const orc_mesh* M, const orc_params* prm, const double* U, double* tau, int fixed_tau,
                   double* U_out, orc_trace* tr);
int orc_ssprk3_step(const orc_mesh* M, const orc_params* prm, double* U, double* tau_out);
/* eq. "ssprk3" with a given tau_n for all three stages */
int orc_ssprk3_step_fixed(const orc_mesh* M, const orc_params* prm, double* U, double tau);

#ifdef __cplusplus
}
#endif
#endif
