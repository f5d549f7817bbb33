/*
 * FP64 CPU oracle for one explicit stage of the invariant-domain preserving
 * Q1 Euler scheme with convex limiting (Maier & Kronbichler, arXiv:2007.00094).
 *
 * TEST INFRASTRUCTURE ONLY: called by tests/, the smoke check and the CPU
 * baseline leg of bench.py, never by the product path.  It shares no code with
 * the CUDA library.  Every loop follows the paper's statement in its own order:
 * rows i in index order, stencil entries j in increasing column order, one
 * floating-point operation at a time (build with -ffp-contract=off).
 *
 * Where the paper is silent, garbled or inconsistent the reading taken is
 * marked "Reading A<k>" and stated at the place it is used.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form Q1 matrices on uniform
 * grids (hexahedra and quadrilaterals; the quadrilateral matrices also against
 * the hexahedral ones of the mesh extruded over a periodic axis), linear
 * reproduction on jittered meshes, equal-state wavespeeds and a
 * brute-force check against an exact Riemann solver, alpha in [0,1], limiter
 * admissibility against bisection, conservation, positivity and local bounds,
 * free-stream preservation, exact Sod and vortex convergence, third-order
 * temporal convergence of eq. (ssprk3), and the Psi margin of Reading A27
 * (it changes only limiter calls in which some Psi lay within the margin,
 * and it keeps rounding-level input perturbations from flipping limiter
 * decisions).  The limiter's t at the default Newton settings: the exact
 * root of Psi where Psi is a quadratic in t (rho(P) = 0: Alg. 3's step is then
 * exact, checked against the quadratic formula), admissible and below the
 * bisection root otherwise, converging to it as the Newton steps grow.
 */
#include "idp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF 5 /* d + 2 conserved fields for d = 3 */

/* ------------------------------------------------------------------------ */
/* Q1 assembly, Sec. 3.1 eq. (matrices)                                      */
/* ------------------------------------------------------------------------ */

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Stencil I(i) = { j : supp(phi_i) and supp(phi_j) overlap } (Sec. 3.1): all
 * nodes of all cells that contain node i, for cells of nv vertices (8 for
 * hexahedra, 4 for quadrilaterals).  With col == NULL only the row pointer is
 * filled; returns nnz. */
int64_t orc_sparsity_nv(int64_t n_nodes, int64_t n_cells, int nv, const int64_t* cells, int64_t* rowptr,
                        int64_t* col) {
  int64_t* cnt = (int64_t*)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  for (int64_t c = 0; c < n_cells; ++c)
    for (int v = 0; v < nv; ++v) cnt[cells[nv * c + v] + 1]++;
  for (int64_t i = 0; i < n_nodes; ++i) cnt[i + 1] += cnt[i];
  int64_t* inc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[n_nodes] + 1));
  int64_t* fill = (int64_t*)calloc((size_t)n_nodes, sizeof(int64_t));
  for (int64_t c = 0; c < n_cells; ++c)
    for (int v = 0; v < nv; ++v) {
      int64_t i = cells[nv * c + v];
      inc[cnt[i] + fill[i]++] = c;
    }
  int64_t nnz = 0;
  int64_t buf[8 * 64];
  rowptr[0] = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    int64_t m = 0;
    for (int64_t q = cnt[i]; q < cnt[i + 1] && m + nv <= 8 * 64; ++q)
      for (int v = 0; v < nv; ++v) buf[m++] = cells[nv * inc[q] + v];
    qsort(buf, (size_t)m, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t q = 0; q < m; ++q)
      if (q == 0 || buf[q] != buf[q - 1]) {
        if (col) col[nnz + u] = buf[q];
        ++u;
      }
    nnz += u;
    rowptr[i + 1] = nnz;
  }
  free(cnt);
  free(inc);
  free(fill);
  return nnz;
}

int64_t orc_sparsity(int64_t n_nodes, int64_t n_cells, const int64_t* cells, int64_t* rowptr, int64_t* col) {
  return orc_sparsity_nv(n_nodes, n_cells, 8, cells, rowptr, col);
}

static int64_t find_col(const int64_t* rowptr, const int64_t* col, int64_t i, int64_t j) {
  int64_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] == j) return mid;
    if (col[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* m_ij = int phi_i phi_j, c_ij = int phi_i grad phi_j, m_i = int phi_i
 * (Sec. 3.1 eq. "matrices"), by 3-point Gauss quadrature per direction on the
 * trilinear map of each hexahedron, which integrates these polynomials exactly
 * (Reading A22).  Local vertex v = a + 2b + 4c at reference corner (a,b,c). */
int orc_assemble(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xyz,
                 const int64_t* rowptr, const int64_t* col, double* mij, double* cij, double* mi) {
  const int64_t nnz = rowptr[n_nodes];
  memset(mij, 0, sizeof(double) * (size_t)nnz);
  memset(cij, 0, sizeof(double) * 3 * (size_t)nnz);
  memset(mi, 0, sizeof(double) * (size_t)n_nodes);
  const double g[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int64_t c = 0; c < n_cells; ++c) {
    const double* X = cell_xyz + 24 * c;
    double Mloc[8][8], Cloc[8][8][3], mloc[8];
    memset(Mloc, 0, sizeof Mloc);
    memset(Cloc, 0, sizeof Cloc);
    memset(mloc, 0, sizeof mloc);
    for (int qx = 0; qx < 3; ++qx)
      for (int qy = 0; qy < 3; ++qy)
        for (int qz = 0; qz < 3; ++qz) {
          const double xi[3] = {g[qx], g[qy], g[qz]};
          const double wq = w[qx] * w[qy] * w[qz];
          double phi[8], dphi[8][3];
          for (int v = 0; v < 8; ++v) {
            double f[3], df[3];
            for (int d = 0; d < 3; ++d) {
              int bit = (v >> d) & 1;
              f[d] = bit ? xi[d] : 1.0 - xi[d];
              df[d] = bit ? 1.0 : -1.0;
            }
            phi[v] = f[0] * f[1] * f[2];
            dphi[v][0] = df[0] * f[1] * f[2];
            dphi[v][1] = f[0] * df[1] * f[2];
            dphi[v][2] = f[0] * f[1] * df[2];
          }
          /* J[r][s] = d x_r / d xi_s */
          double J[3][3] = {{0}};
          for (int v = 0; v < 8; ++v)
            for (int r = 0; r < 3; ++r)
              for (int s = 0; s < 3; ++s) J[r][s] += X[3 * v + r] * dphi[v][s];
          double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
          if (!(det > 0.0)) return ORC_ERR_ARG;
          /* inverse of J: Jinv[s][r] = d xi_s / d x_r */
          double Jinv[3][3];
          Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
          Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
          Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
          Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
          Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
          Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
          Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
          Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
          Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
          double grad[8][3];
          for (int v = 0; v < 8; ++v)
            for (int r = 0; r < 3; ++r)
              grad[v][r] = dphi[v][0] * Jinv[0][r] + dphi[v][1] * Jinv[1][r] + dphi[v][2] * Jinv[2][r];
          const double dx = wq * det;
          for (int a = 0; a < 8; ++a) {
            mloc[a] += phi[a] * dx;
            for (int b = 0; b < 8; ++b) {
              Mloc[a][b] += phi[a] * phi[b] * dx;
              for (int r = 0; r < 3; ++r) Cloc[a][b][r] += phi[a] * grad[b][r] * dx;
            }
          }
        }
    for (int a = 0; a < 8; ++a) {
      int64_t i = cells[8 * c + a];
      mi[i] += mloc[a];
      for (int b = 0; b < 8; ++b) {
        int64_t k = find_col(rowptr, col, i, cells[8 * c + b]);
        if (k < 0) return ORC_ERR_ARG;
        mij[k] += Mloc[a][b];
        for (int r = 0; r < 3; ++r) cij[r * nnz + k] += Cloc[a][b][r];
      }
    }
  }
  return ORC_OK;
}

/* The same matrices for d = 2 (Sec. 3.1 with Q1 quadrilaterals): 3x3 Gauss
 * points on the bilinear map of each quadrilateral, local vertex v = a + 2b at
 * reference corner (a,b), two coordinates per vertex in cell_xy.  c_ij keeps
 * three rows with the z row zero, so the stage is the 3D one with m_z = 0. */
int orc_assemble_quad(int64_t n_nodes, int64_t n_cells, const int64_t* cells, const double* cell_xy,
                      const int64_t* rowptr, const int64_t* col, double* mij, double* cij, double* mi) {
  const int64_t nnz = rowptr[n_nodes];
  memset(mij, 0, sizeof(double) * (size_t)nnz);
  memset(cij, 0, sizeof(double) * 3 * (size_t)nnz);
  memset(mi, 0, sizeof(double) * (size_t)n_nodes);
  const double g[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int64_t c = 0; c < n_cells; ++c) {
    const double* X = cell_xy + 8 * c;
    double Mloc[4][4], Cloc[4][4][2], mloc[4];
    memset(Mloc, 0, sizeof Mloc);
    memset(Cloc, 0, sizeof Cloc);
    memset(mloc, 0, sizeof mloc);
    for (int qx = 0; qx < 3; ++qx)
      for (int qy = 0; qy < 3; ++qy) {
        const double xi[2] = {g[qx], g[qy]};
        const double wq = w[qx] * w[qy];
        double phi[4], dphi[4][2];
        for (int v = 0; v < 4; ++v) {
          const double fx = (v & 1) ? xi[0] : 1.0 - xi[0];
          const double fy = (v & 2) ? xi[1] : 1.0 - xi[1];
          const double dfx = (v & 1) ? 1.0 : -1.0;
          const double dfy = (v & 2) ? 1.0 : -1.0;
          phi[v] = fx * fy;
          dphi[v][0] = dfx * fy;
          dphi[v][1] = fx * dfy;
        }
        /* J[r][s] = d x_r / d xi_s */
        double J[2][2] = {{0}};
        for (int v = 0; v < 4; ++v)
          for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) J[r][s] += X[2 * v + r] * dphi[v][s];
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(det > 0.0)) return ORC_ERR_ARG;
        /* Jinv[s][r] = d xi_s / d x_r */
        const double Jinv[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
        double grad[4][2];
        for (int v = 0; v < 4; ++v)
          for (int r = 0; r < 2; ++r) grad[v][r] = dphi[v][0] * Jinv[0][r] + dphi[v][1] * Jinv[1][r];
        const double dx = wq * det;
        for (int a = 0; a < 4; ++a) {
          mloc[a] += phi[a] * dx;
          for (int b = 0; b < 4; ++b) {
            Mloc[a][b] += phi[a] * phi[b] * dx;
            for (int r = 0; r < 2; ++r) Cloc[a][b][r] += phi[a] * grad[b][r] * dx;
          }
        }
      }
    for (int a = 0; a < 4; ++a) {
      int64_t i = cells[4 * c + a];
      mi[i] += mloc[a];
      for (int b = 0; b < 4; ++b) {
        int64_t k = find_col(rowptr, col, i, cells[4 * c + b]);
        if (k < 0) return ORC_ERR_ARG;
        mij[k] += Mloc[a][b];
        for (int r = 0; r < 2; ++r) cij[r * nnz + k] += Cloc[a][b][r];
      }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Euler flux and derived quantities, Sec. 2                                 */
/* ------------------------------------------------------------------------ */

/* epsilon = E - |m|^2/(2 rho) (internal energy), p = (gamma-1) epsilon. */
static double internal_energy(const double* U) {
  const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  return U[4] - m2 / (2.0 * U[0]);
}
static double pressure(const double* U, double gamma) { return (gamma - 1.0) * internal_energy(U); }

/* phi(U) = epsilon rho^(-gamma), eq. (specific_entropy). */
static double specific_entropy(const double* U, double gamma) {
  return internal_energy(U) * pow(U[0], -gamma);
}

/* eta(U) = (rho epsilon)^(1/(gamma+1)) (Harten entropy, Sec. 2). */
static double harten_entropy(const double* U, double gamma) {
  return pow(U[0] * internal_energy(U), 1.0 / (gamma + 1.0));
}

/* eta'(U) = (rho epsilon)^(-gamma/(gamma+1)) / (gamma+1) * (E, -m, rho),
 * derivative with respect to (rho, m, E) (Sec. 3.8; Reading A7). */
static void harten_entropy_derivative(const double* U, double gamma, double* out) {
  const double s = pow(U[0] * internal_energy(U), -gamma / (gamma + 1.0)) / (gamma + 1.0);
  out[0] = s * U[4];
  out[1] = -s * U[1];
  out[2] = -s * U[2];
  out[3] = -s * U[3];
  out[4] = s * U[0];
}

/* f(U) in R^{5x3}, eq. (flux): rows m ; v (x) m + p I ; v (E + p). */
static void flux(const double* U, double gamma, double F[NF][3]) {
  const double rho = U[0], E = U[4];
  const double v[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
  const double p = pressure(U, gamma);
  for (int d = 0; d < 3; ++d) {
    F[0][d] = U[1 + d];
    for (int r = 0; r < 3; ++r) F[1 + r][d] = v[r] * U[1 + d] + (r == d ? p : 0.0);
    F[4][d] = v[d] * (E + p);
  }
}

/* (F . c)_f = sum_d F[f][d] c_d */
static void contract(double F[NF][3], const double* c, double* out) {
  for (int f = 0; f < NF; ++f) out[f] = F[f][0] * c[0] + F[f][1] * c[1] + F[f][2] * c[2];
}

void orc_node_quantities(const double* U, double gamma, double* out) {
  out[0] = pressure(U, gamma);
  out[1] = sqrt(gamma * out[0] / U[0]);
  out[2] = specific_entropy(U, gamma);
  out[3] = harten_entropy(U, gamma);
  harten_entropy_derivative(U, gamma, out + 4);
}

/* ------------------------------------------------------------------------ */
/* Two-rarefaction maximum wavespeed bound, Sec. 3.7                         */
/* ------------------------------------------------------------------------ */

static double positive_part(double x) { return 0.5 * (fabs(x) + x); }
/* [x]_neg = (|x| - x)/2: the paper uses the negative part without defining
 * its sign convention (Reading A3) */
static double negative_part(double x) { return 0.5 * (fabs(x) - x); }

typedef struct { double rho, u, p, c; } state1d;

/* Projected 1D state: rho~ = rho, m~ = n.m, E~ = E - |m - m~ n|^2/(2 rho);
 * u~ = m~/rho, p~ from the 1D state, c~ = sqrt(gamma p~/rho). */
static state1d project(const double* n, const double* U, double gamma) {
  state1d s;
  const double rho = U[0];
  const double mt = n[0] * U[1] + n[1] * U[2] + n[2] * U[3];
  const double q0 = U[1] - mt * n[0], q1 = U[2] - mt * n[1], q2 = U[3] - mt * n[2];
  const double Et = U[4] - (q0 * q0 + q1 * q1 + q2 * q2) / (2.0 * rho);
  s.rho = rho;
  s.u = mt / rho;
  s.p = (gamma - 1.0) * (Et - mt * mt / (2.0 * rho));
  s.c = sqrt(gamma * s.p / rho);
  return s;
}

/* f(U, p) of the pressure function psi (Sec. 3.7). */
static double riemann_f(const state1d* s, double p, double gamma) {
  if (p >= s->p) return sqrt(2.0) * (p - s->p) / sqrt(s->rho * ((gamma + 1.0) * p + (gamma - 1.0) * s->p));
  return (pow(p / s->p, (gamma - 1.0) / (2.0 * gamma)) - 1.0) * 2.0 * s->c / (gamma - 1.0);
}

/* lambda~_max(n, U_i, U_j) of Sec. 3.7 with U_i as the left and U_j as the
 * right state. */
double orc_lambda_max(const double* n, const double* Ui, const double* Uj, double gamma) {
  const state1d L = project(n, Ui, gamma), R = project(n, Uj, gamma);
  const double e = (gamma - 1.0) / (2.0 * gamma);
  /* two-rarefaction pressure; a non-positive numerator gives p~* = 0 (Reading A4) */
  double num = L.c + R.c - 0.5 * (gamma - 1.0) * (R.u - L.u);
  if (num < 0.0) num = 0.0;
  const double den = L.c * pow(L.p / R.p, -e) + R.c;
  const double p_tr = R.p * pow(num / den, 1.0 / e);
  const double p_max = L.p > R.p ? L.p : R.p;
  const double psi = riemann_f(&L, p_max, gamma) + riemann_f(&R, p_max, gamma) + R.u - L.u;
  double p_star = p_tr;
  if (!(psi < 0.0)) p_star = p_max < p_tr ? p_max : p_tr;
  const double k = (gamma + 1.0) / (2.0 * gamma);
  const double lam1 = L.u - L.c * sqrt(1.0 + k * positive_part((p_star - L.p) / L.p));
  const double lam3 = R.u + R.c * sqrt(1.0 + k * positive_part((p_star - R.p) / R.p));
  const double a = negative_part(lam1), b = positive_part(lam3);
  return a > b ? a : b;
}

/* ------------------------------------------------------------------------ */
/* Convex limiter, Sec. 3.9, Alg. 2 and Alg. 3                               */
/* ------------------------------------------------------------------------ */

/* Psi(U) = rho^(gamma+1) (phi(U) - phi_min).  Since rho^(gamma+1) phi(U) =
 * rho epsilon by eq. (specific_entropy), this is rho epsilon - phi_min
 * rho^(gamma+1) with rho epsilon = rho E - |m|^2/2. */
double orc_psi(const double* U, double phi_min, double gamma) {
  const double rho_eps = U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
  return rho_eps - phi_min * pow(U[0], gamma + 1.0);
}

/* d/dt Psi(U + t P) */
static double dpsi_dt(const double* V, const double* P, double phi_min, double gamma) {
  const double drho_eps = P[0] * V[4] + V[0] * P[4] - (V[1] * P[1] + V[2] * P[2] + V[3] * P[3]);
  return drho_eps - phi_min * (gamma + 1.0) * pow(V[0], gamma) * P[0];
}

/* Admissibility test Psi(V) >= 0 of Alg. 2, taken with a relative margin
 * (Reading A27): Psi(V) >= -margin (|rho eps| + |phi_min rho^(gamma+1)|).
 * The caption of Alg. 3 states that an implementation must add safeguards
 * against round-off; this is one of them.  Where phi is close to phi_min
 * (isentropic flow) the two terms of Psi nearly cancel and the sign of a Psi
 * that small depends on the rounding of its inputs, which differ between any
 * two implementations of the stage at the 1e-13 level.  margin = 0 gives the
 * strict test.  When the outcome was decided by the margin (-slack <= Psi <
 * 0), *hits is incremented and *worst raised to |Psi| / scale. */
static int psi_admissible(const double* V, double phi_min, double gamma, double margin, int* hits,
                          double* worst) {
  const double rho_eps = V[0] * V[4] - 0.5 * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]);
  const double scale = fabs(rho_eps) + fabs(phi_min * pow(V[0], gamma + 1.0));
  const double psi = orc_psi(V, phi_min, gamma);
  const int ok = psi >= -margin * scale;
  if (ok && psi < 0.0) {
    ++*hits;
    if (-psi / scale > *worst) *worst = -psi / scale;
  }
  return ok;
}

static void axpy_state(const double* U, double t, const double* P, double* out) {
  for (int f = 0; f < NF; ++f) out[f] = U[f] + t * P[f];
}

static double clamp(double x, double lo, double hi) {
  if (!(x >= lo)) x = lo;
  if (!(x <= hi)) x = hi;
  return x;
}

/* Alg. 3, quadratic Newton step with divided differences, sign = -1
 * (Reading A10), with the safeguards the caption asks for: a negative
 * discriminant is set to 0 (Reading A10). */
static void quadratic_newton_step(double* tL, double* tR, double PsiL, double PsiR, double dPsiL, double dPsiR,
                                  double sign, double eps) {
  const double scaling = 1.0 / (*tR - *tL + eps);
  const double d11 = dPsiL;
  const double d12 = (PsiR - PsiL) * scaling;
  const double d22 = dPsiR;
  const double d112 = (d12 - d11) * scaling;
  const double d122 = (d22 - d12) * scaling;
  double LamL = dPsiL * dPsiL - 4.0 * PsiL * d112;
  double LamR = dPsiR * dPsiR - 4.0 * PsiR * d122;
  if (LamL < 0.0) LamL = 0.0;
  if (LamR < 0.0) LamR = 0.0;
  *tL = *tL - 2.0 * PsiL / (dPsiL + sign * sqrt(LamL));
  *tR = *tR - 2.0 * PsiR / (dPsiR + sign * sqrt(LamR));
}

/* limiter.compute(U, P, bounds) of Alg. 2: the largest t in [0,1] found by
 * the density interval and the quadratic Newton iteration such that U + t P
 * keeps rho in [rho_min, rho_max] and Psi >= 0.  Readings A9-A12, A26, A27.
 * margin_hits / margin_worst (may be NULL) receive the number of
 * admissibility tests whose outcome the Psi margin decided and the largest
 * |Psi| / scale among them. */
double orc_limiter_ex(const double* U, const double* P, double rho_min, double rho_max, double phi_min,
                      const orc_params* prm, int* margin_hits, double* margin_worst) {
  const double gamma = prm->gamma;
  const double margin = prm->psi_margin;
  int hits = 0;
  double worst = 0.0;
  double tL = 0.0, tR = 1.0;
  const double rhoU = U[0], rhoP = P[0];
  /* density interval (Reading A12) */
  if (rhoU + tR * rhoP > rho_max && rhoP != 0.0) tR = fabs(rho_max - rhoU) / fabs(rhoP);
  if (rhoU + tR * rhoP < rho_min && rhoP != 0.0) tR = fabs(rho_min - rhoU) / fabs(rhoP);
  tR = clamp(tR, 0.0, 1.0);
  const double tol = prm->newton_tol * (U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]));
  double V[NF];
  for (int step = 0; step < prm->newton_max; ++step) {
    axpy_state(U, tR, P, V);
    const double PsiR = orc_psi(V, phi_min, gamma);
    if (psi_admissible(V, phi_min, gamma, margin, &hits, &worst)) { /* t_R admissible: close the interval */
      tL = tR;
      break;
    }
    axpy_state(U, tL, P, V);
    const double PsiL = orc_psi(V, phi_min, gamma);
    if (PsiL <= tol) break; /* t_L is a root within the tolerance (Reading A11) */
    const double dPsiL = dpsi_dt(V, P, phi_min, gamma); /* at t_L (Reading A9) */
    axpy_state(U, tR, P, V);
    const double dPsiR = dpsi_dt(V, P, phi_min, gamma); /* at t_R */
    double nL = tL, nR = tR;
    quadratic_newton_step(&nL, &nR, PsiL, PsiR, dPsiL, dPsiR, -1.0, prm->newton_eps);
    /* keep t_L admissible and the bracket ordered (Reading A10): the new
     * left end is checked before it bounds the new right end (a step that
     * lands on the root within rounding must not fall back to the old t_L) */
    nL = clamp(nL, tL, tR);
    axpy_state(U, nL, P, V);
    if (!psi_admissible(V, phi_min, gamma, margin, &hits, &worst)) nL = tL;
    nR = clamp(nR, nL, tR);
    tL = nL;
    tR = nR;
  }
  if (margin_hits) *margin_hits = hits;
  if (margin_worst) *margin_worst = worst;
  return tL;
}

double orc_limiter(const double* U, const double* P, double rho_min, double rho_max, double phi_min,
                   const orc_params* prm) {
  return orc_limiter_ex(U, P, rho_min, rho_max, phi_min, prm, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* euler_step, Alg. 1                                                        */
/* ------------------------------------------------------------------------ */

static void load(const double* U, int64_t n, int64_t i, double* u) {
  for (int f = 0; f < NF; ++f) u[f] = U[f * n + i];
}
static void store(double* U, int64_t n, int64_t i, const double* u) {
  for (int f = 0; f < NF; ++f) U[f * n + i] = u[f];
}

static void cvec(const orc_mesh* M, int64_t k, double* c) {
  const int64_t nnz = M->rowptr[M->n];
  c[0] = M->cij[k];
  c[1] = M->cij[nnz + k];
  c[2] = M->cij[2 * nnz + k];
}

/* Boundary post-processing after each euler_step (Reading A20): slip nodes
 * drop the momentum components normal to their axis-aligned wall faces,
 * inflow nodes take the inflow state. */
static void apply_boundary(const orc_mesh* M, double* U) {
  const int64_t n = M->n;
  if (!M->bc) return;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t b = M->bc[i];
    if (b & 8) {
      if (M->inflow)
        for (int f = 0; f < NF; ++f) U[f * n + i] = M->inflow[f];
      continue;
    }
    for (int d = 0; d < 3; ++d)
      if (b & (1 << d)) U[(1 + d) * n + i] = 0.0;
  }
}

int orc_euler_step(const orc_mesh* M, const orc_params* prm, const double* U, double* tau, int fixed_tau,
                   double* U_out, orc_trace* tr) {
  const int64_t n = M->n, nnz = M->rowptr[n];
  const int64_t* rp = M->rowptr;
  const int64_t* col = M->col;
  const double gamma = prm->gamma;
  const int nt = prm->n_threads > 0 ? prm->n_threads : 1;
  (void)nt;

  for (int64_t i = 0; i < n; ++i) {
    double u[NF];
    load(U, n, i, u);
    if (!(u[0] > 0.0) || !(internal_energy(u) > 0.0)) return ORC_ERR_STATE;
  }

  /* transpose position: entry (j,i) for every entry (i,j) */
  int64_t* kT = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) kT[k] = find_col(rp, col, col[k], i);

  double* d = (double*)calloc((size_t)nnz, sizeof(double));
  double* alpha = (double*)calloc((size_t)n, sizeof(double));
  double* UL = (double*)malloc(sizeof(double) * NF * (size_t)n);
  double* R = (double*)malloc(sizeof(double) * NF * (size_t)n);
  double* bnd = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* P = (double*)calloc(NF * (size_t)nnz, sizeof(double));
  double* l = (double*)calloc((size_t)nnz, sizeof(double));
  double* lnew = (double*)calloc((size_t)nnz, sizeof(double));
  double* Ucur = (double*)malloc(sizeof(double) * NF * (size_t)n);
  double* Unext = (double*)malloc(sizeof(double) * NF * (size_t)n);

  /* Step 1: off-diagonal d_ij for j > i (Sec. 3.3) and the indicator alpha_i
   * (Sec. 3.8); the indicator runs over all j in I(i) (Reading A2). */
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ui[NF], uj[NF], Fi[NF][3], Fj[NF][3], c[3], cT[3], fi[NF], fj[NF], etap[NF];
    load(U, n, i, ui);
    flux(ui, gamma, Fi);
    const double s_i = harten_entropy(ui, gamma) / ui[0];
    harten_entropy_derivative(ui, gamma, etap);
    double a = 0.0, b[NF] = {0, 0, 0, 0, 0};
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      load(U, n, j, uj);
      cvec(M, k, c);
      if (j > i) {
        cvec(M, kT[k], cT);
        const double nc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double ncT = sqrt(cT[0] * cT[0] + cT[1] * cT[1] + cT[2] * cT[2]);
        double lij = 0.0, lji = 0.0;
        if (nc > 0.0) {
          const double nij[3] = {c[0] / nc, c[1] / nc, c[2] / nc};
          lij = orc_lambda_max(nij, ui, uj, gamma) * nc;
        }
        if (ncT > 0.0) {
          const double nji[3] = {cT[0] / ncT, cT[1] / ncT, cT[2] / ncT};
          lji = orc_lambda_max(nji, uj, ui, gamma) * ncT;
        }
        d[k] = lij > lji ? lij : lji;
      }
      const double s_j = harten_entropy(uj, gamma) / uj[0];
      a += (s_j - s_i) * (uj[1] * c[0] + uj[2] * c[1] + uj[3] * c[2]);
      flux(uj, gamma, Fj);
      contract(Fj, c, fj);
      contract(Fi, c, fi);
      for (int f = 0; f < NF; ++f) b[f] += fj[f] - fi[f];
    }
    double num = a - (etap[0] * b[0] + etap[1] * b[1] + etap[2] * b[2] + etap[3] * b[3] + etap[4] * b[4]) +
                 s_i * b[0];
    double N_i = fabs(num);
    double D_i = fabs(a);
    /* the denominator sums all five components (the printed range stops one
     * short), which keeps alpha_i in [0, 1] (Reading A6) */
    for (int f = 0; f < NF; ++f) D_i += fabs(etap[f] - (f == 0 ? s_i : 0.0)) * fabs(b[f]);
    alpha[i] = D_i > 0.0 ? N_i / D_i : 0.0;
  }

  /* Step 2: lower part d_ij = d_ji, d_ii = -sum_{j != i} d_ij and
   * tau_n = c_cfl min_i m_i / (-2 d_ii) (Sec. 3.3). */
  double tau_max = INFINITY;
#pragma omp parallel for num_threads(nt) schedule(static) reduction(min : tau_max)
  for (int64_t i = 0; i < n; ++i) {
    int64_t kd = -1;
    double sum = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      if (j < i) d[k] = d[kT[k]];
      if (j == i) kd = k;
    }
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] != i) sum += d[k];
    d[kd] = -sum;
    const double t = M->mi[i] / (-2.0 * d[kd]);
    if (t < tau_max) tau_max = t;
  }
  if (tr && tr->tau_max) *tr->tau_max = tau_max;
  int status = ORC_OK;
  if (!fixed_tau) {
    *tau = prm->cfl * tau_max;
  } else if (*tau > tau_max) {
    status = ORC_ERR_CFL; /* a given tau above this stage's bound is reported (Reading A17) */
  }
  const double dt = *tau;

  /* Bound relaxation (Reading A14, project-defined; the paper leaves the
   * formula to the literature): r_i = (m_i / |Omega|)^(1/2), |Omega| = sum_i m_i. */
  double volume = 0.0;
  if (prm->relax)
    for (int64_t i = 0; i < n; ++i) volume += M->mi[i];

  /* Step 3: low-order update via bar states (Sec. 3.3 eq. def-ubar, Reading
   * A1), R_i (eq. high-order-final) and the local bounds (Sec. 3.9). */
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ui[NF], uj[NF], Fi[NF][3], Fj[NF][3], c[3], fi[NF], fj[NF], r[NF], ul[NF];
    load(U, n, i, ui);
    flux(ui, gamma, Fi);
    for (int f = 0; f < NF; ++f) {
      r[f] = 0.0;
      ul[f] = ui[f];
    }
    double rho_min = INFINITY, rho_max = -INFINITY, phi_min = INFINITY;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      load(U, n, j, uj);
      cvec(M, k, c);
      flux(uj, gamma, Fj);
      contract(Fj, c, fj);
      contract(Fi, c, fi);
      const double dH = d[k] * (alpha[i] + alpha[j]) / 2.0;
      for (int f = 0; f < NF; ++f) r[f] += -fj[f] + dH * (uj[f] - ui[f]);
      if (d[k] != 0.0) { /* an entry with d_ij = 0 has no bar state and is skipped (Reading A19) */
        double ubar[NF];
        for (int f = 0; f < NF; ++f) ubar[f] = 0.5 * (ui[f] + uj[f]) - (fj[f] - fi[f]) / (2.0 * d[k]);
        const double coef = 2.0 * dt / M->mi[i] * d[k];
        for (int f = 0; f < NF; ++f) ul[f] += coef * ubar[f];
        if (ubar[0] < rho_min) rho_min = ubar[0];
        if (ubar[0] > rho_max) rho_max = ubar[0];
      }
      const double phj = specific_entropy(uj, gamma); /* j ranges over I(i), i included (Reading A13) */
      if (phj < phi_min) phi_min = phj;
    }
    if (prm->relax) {
      const double ri = sqrt(M->mi[i] / volume);
      rho_min *= 1.0 - ri;
      rho_max *= 1.0 + ri;
      phi_min *= 1.0 - ri;
    }
    store(UL, n, i, ul);
    store(R, n, i, r);
    bnd[i] = rho_min;
    bnd[n + i] = rho_max;
    bnd[2 * n + i] = phi_min;
  }

  /* Step 4: P_ij (eq. def-p) with b_ij = delta_ij - m_ij/m_j and
   * lambda_i = 1/(card I(i) - 1) (Reading A18); first limiter values. */
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ui[NF], uj[NF], ri[NF], rj[NF], ul[NF], pij[NF];
    load(U, n, i, ui);
    load(R, n, i, ri);
    load(UL, n, i, ul);
    const double lam = 1.0 / (double)(rp[i + 1] - rp[i] - 1);
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      if (j == i) {
        for (int f = 0; f < NF; ++f) P[f * nnz + k] = 0.0;
        l[k] = 0.0;
        continue;
      }
      load(U, n, j, uj);
      load(R, n, j, rj);
      const double b_ij = -M->mij[k] / M->mi[j];
      const double b_ji = -M->mij[kT[k]] / M->mi[i];
      const double dH = d[k] * (alpha[i] + alpha[j]) / 2.0;
      for (int f = 0; f < NF; ++f) {
        pij[f] = dt / (M->mi[i] * lam) * (b_ij * rj[f] - b_ji * ri[f] + (dH - d[k]) * (uj[f] - ui[f]));
        P[f * nnz + k] = pij[f];
      }
      l[k] = orc_limiter(ul, pij, bnd[i], bnd[n + i], bnd[2 * n + i], prm);
    }
  }
  if (tr && tr->P) memcpy(tr->P, P, sizeof(double) * NF * (size_t)nnz);
  if (tr && tr->l4) memcpy(tr->l4, l, sizeof(double) * (size_t)nnz);

  /* Steps 5, 6, ...: eq. (iterative-limiter) with l_ij -> min(l_ij, l_ji)
   * (Reading A15); the last pass only updates U (Reading A16). */
  memcpy(Ucur, UL, sizeof(double) * NF * (size_t)n);
  for (int pass = 1; pass <= prm->limiter_passes; ++pass) {
    const int last = pass == prm->limiter_passes;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double u[NF];
      load(Ucur, n, i, u);
      const double lam = 1.0 / (double)(rp[i + 1] - rp[i] - 1);
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (col[k] == i) continue;
        const double lk = l[k] < l[kT[k]] ? l[k] : l[kT[k]];
        for (int f = 0; f < NF; ++f) u[f] += lam * lk * P[f * nnz + k];
      }
      store(Unext, n, i, u);
      if (!last) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
          if (col[k] == i) {
            lnew[k] = 0.0;
            continue;
          }
          const double lk = l[k] < l[kT[k]] ? l[k] : l[kT[k]];
          double pij[NF];
          for (int f = 0; f < NF; ++f) {
            P[f * nnz + k] = (1.0 - lk) * P[f * nnz + k];
            pij[f] = P[f * nnz + k];
          }
          lnew[k] = orc_limiter(u, pij, bnd[i], bnd[n + i], bnd[2 * n + i], prm);
        }
      }
    }
    double* tmp = Ucur;
    Ucur = Unext;
    Unext = tmp;
    if (!last) {
      double* t2 = l;
      l = lnew;
      lnew = t2;
    }
    if (pass == 1 && tr && tr->U5) memcpy(tr->U5, Ucur, sizeof(double) * NF * (size_t)n);
    if (pass == 1 && !last && tr && tr->l5) memcpy(tr->l5, l, sizeof(double) * (size_t)nnz);
  }
  if (tr && tr->Ulim) memcpy(tr->Ulim, Ucur, sizeof(double) * NF * (size_t)n);
  apply_boundary(M, Ucur);
  memcpy(U_out, Ucur, sizeof(double) * NF * (size_t)n);

  if (tr && tr->d) memcpy(tr->d, d, sizeof(double) * (size_t)nnz);
  if (tr && tr->alpha) memcpy(tr->alpha, alpha, sizeof(double) * (size_t)n);
  if (tr && tr->UL) memcpy(tr->UL, UL, sizeof(double) * NF * (size_t)n);
  if (tr && tr->R) memcpy(tr->R, R, sizeof(double) * NF * (size_t)n);
  if (tr && tr->bounds) memcpy(tr->bounds, bnd, sizeof(double) * 3 * (size_t)n);

  free(kT);
  free(d);
  free(alpha);
  free(UL);
  free(R);
  free(bnd);
  free(P);
  free(l);
  free(lnew);
  free(Ucur);
  free(Unext);
  return status;
}

/* ------------------------------------------------------------------------ */
/* SSP-RK3, Sec. 3.6 eq. (ssprk3): tau fixed by the first stage               */
/* ------------------------------------------------------------------------ */
/* One step of eq. (ssprk3).  fixed_tau = 0: tau_n comes from the CFL rule of
 * the first stage and is written to *tau; fixed_tau != 0: *tau is used by all
 * three stages (each checks it against its own bound, Reading A17). */
static int ssprk3(const orc_mesh* M, const orc_params* prm, double* U, double* tau, int fixed_tau) {
  const int64_t n = M->n;
  const size_t sz = sizeof(double) * NF * (size_t)n;
  double* U1 = (double*)malloc(sz);
  double* U2 = (double*)malloc(sz);
  double* E = (double*)malloc(sz);
  int st = orc_euler_step(M, prm, U, tau, fixed_tau, U1, NULL);
  if (st == ORC_OK) st = orc_euler_step(M, prm, U1, tau, 1, E, NULL);
  if (st == ORC_OK) {
    for (int64_t q = 0; q < NF * n; ++q) U2[q] = 0.75 * U[q] + 0.25 * E[q];
    st = orc_euler_step(M, prm, U2, tau, 1, E, NULL);
  }
  if (st == ORC_OK)
    for (int64_t q = 0; q < NF * n; ++q) U[q] = 1.0 / 3.0 * U[q] + 2.0 / 3.0 * E[q];
  free(U1);
  free(U2);
  free(E);
  return st;
}

int orc_ssprk3_step_fixed(const orc_mesh* M, const orc_params* prm, double* U, double tau) {
  return ssprk3(M, prm, U, &tau, 1);
}

int orc_ssprk3_step(const orc_mesh* M, const orc_params* prm, double* U, double* tau_out) {
  double tau = 0.0;
  const int st = ssprk3(M, prm, U, &tau, 0);
  if (tau_out) *tau_out = tau;
  return st;
}

/* limiter.compute of Alg. 2 for m independent calls: U, P (5 x m), bounds
 * (3 x m: rho_min, rho_max, phi_min), all field-major; t, hits and worst as
 * in orc_limiter_ex (hits and worst may be NULL). */
void orc_limiter_many(int64_t m, const double* U, const double* P, const double* bounds, const orc_params* prm,
                      double* t, int* hits, double* worst) {
  for (int64_t q = 0; q < m; ++q) {
    double u[NF], p[NF];
    for (int f = 0; f < NF; ++f) {
      u[f] = U[f * m + q];
      p[f] = P[f * m + q];
    }
    int h = 0;
    double w = 0.0;
    t[q] = orc_limiter_ex(u, p, bounds[q], bounds[m + q], bounds[2 * m + q], prm, &h, &w);
    if (hits) hits[q] = h;
    if (worst) worst[q] = w;
  }
}
