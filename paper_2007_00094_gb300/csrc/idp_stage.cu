// FP64 kernels of one euler_step (Alg. 1), thread per row over the
// sliced-ELL graph.  Kernel boundaries are the global dependencies of the
// algorithm (Fig. 2): alpha_j and d_ji after Step 1, tau after Step 2, R_j
// after Step 3, l_ji after Steps 4 and 5.
#include <algorithm>
#include <cfloat>

#include "idp_internal.h"
#include "idp_stage.cuh"

namespace idp {

namespace {

constexpr int kBlock = 128;  // state-check kernels

__device__ __forceinline__ int64_t slot_base(const DeviceGraph& G, int64_t r) {
  return (int64_t)G.slice_ptr[r >> 5] + (r & 31);
}

__device__ __forceinline__ void load5(const double* U, int64_t n, int64_t i, double* u) {
#pragma unroll
  for (int f = 0; f < kFields; ++f) u[f] = U[f * n + i];
}

__device__ __forceinline__ Side load_side(const double* U, const double* Q, int64_t n, int64_t i) {
  Side s;
  s.rho = U[i];
  s.mx = U[n + i];
  s.my = U[2 * n + i];
  s.mz = U[3 * n + i];
  s.inv_rho = Q[kQInvRho * n + i];
  s.p = Q[kQP * n + i];
  s.c = Q[kQC * n + i];
  s.pm = Q[kQPm * n + i];
  s.inv_p = Q[kQInvP * n + i];
  return s;
}

// Step 0: per-node quantities (Sec. 2): 1/rho, p, c, p^(-1/7), 1/p,
// eta/rho with eta = (rho eps)^(5/12), (E + p)/rho and phi = eps rho^(-7/5).
__device__ __forceinline__ void row_node(int64_t n, const double* U, double* Q,
                                         DeviceScalars* scal, int64_t i) {
  double u[kFields];
  load5(U, n, i, u);
  const double rho = u[0];
  const double inv_rho = 1.0 / rho;
  const double eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * inv_rho;
  if (!(rho > 0.0) || !(eps > 0.0)) atomicOr(&scal->status, kStatusNotAdmissible);
  const double p = 0.4 * eps;
  const double rho_eps = rho * eps;
  const double w12 = inv_root<12>(rho_eps);  // (rho eps)^(-1/12)
  double w7 = w12 * w12 * w12;
  w7 = w7 * w7 * w12;  // (rho eps)^(-7/12)
  const double eta = rho_eps * w7;
  const double w5 = inv_root<5>(rho);
  double r7 = w5 * w5 * w5;
  r7 = r7 * r7 * w5;  // rho^(-7/5)
  Q[kQInvRho * n + i] = inv_rho;
  Q[kQP * n + i] = p;
  Q[kQC * n + i] = sqrt(1.4 * p * inv_rho);
  Q[kQPm * n + i] = inv_root<7>(p);
  Q[kQInvP * n + i] = 1.0 / p;
  Q[kQS * n + i] = eta * inv_rho;
  Q[kQH * n + i] = (u[4] + p) * inv_rho;
  Q[kQPhi * n + i] = eps * r7;
  Q[kQVx * n + i] = __dmul_rn(u[1], inv_rho);
  Q[kQVy * n + i] = __dmul_rn(u[2], inv_rho);
  Q[kQVz * n + i] = __dmul_rn(u[3], inv_rho);
}

__global__ void __launch_bounds__(kMaxBlock) k_node(int64_t n, const double* __restrict__ U, double* __restrict__ Q,
                                                 DeviceScalars* scal) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) row_node(n, U, Q, scal, i);
}

// Step 1: for every unordered pair {i, j} that this row owns (kEntryUpper),
// d^L_ij with 1/(2 d_ij), and the flux differences (f_j - f_i).c_ij with
// m_j.c_ij, stored at both of the pair's slots.  For a bitwise skew pair
// (c_ji = -c_ij) the transposed slot's values are bitwise those its own row
// would compute, (f_i - f_j).c_ji = (f_j - f_i).c_ij and m_i.c_ji = -m_i.c_ij,
// because every product and difference is rounded alike on both sides;
// boundary pairs evaluate the transposed orientation separately.  The
// indicator alpha_i (Sec. 3.8), which sums these over all j in I(i), is
// formed in Step 2, and Step 3 reuses the differences for the bar states and
// R_i.
__device__ __forceinline__ void flux_diff(const Side& si, const Side& sj, double vxi, double vyi, double vzi,
                                          double vxj, double vyj, double vzj, double hi, double hj, double cx,
                                          double cy, double cz, double* df, double* mcj_out, double* mci_out) {
  // (f_j - f_i).c_ij formed from m.c of both sides and the pressure
  // difference: every term is rounded alike on both sides, so equal states
  // still give exact zeros, with fewer FP64 operations than two fluxes
  const double mcj = m_dot_c(sj.mx, sj.my, sj.mz, cx, cy, cz);
  const double mci = m_dot_c(si.mx, si.my, si.mz, cx, cy, cz);
  const double dp = sj.p - si.p;
  df[0] = mcj - mci;
  df[1] = fma(dp, cx, __dmul_rn(vxj, mcj) - __dmul_rn(vxi, mci));
  df[2] = fma(dp, cy, __dmul_rn(vyj, mcj) - __dmul_rn(vyi, mci));
  df[3] = fma(dp, cz, __dmul_rn(vzj, mcj) - __dmul_rn(vzi, mci));
  df[4] = __dmul_rn(hj, mcj) - __dmul_rn(hi, mci);
  *mcj_out = mcj;
  *mci_out = mci;
}

__device__ __forceinline__ void row_edge(const DeviceGraph& G, const double* U,
                                         const double* Q, double* d,
                                         double* dinv, double* dF, double* mc, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const Side si = load_side(U, Q, n, r);
  const double h_i = Q[kQH * n + r];
  const double vxi = Q[kQVx * n + r], vyi = Q[kQVy * n + r], vzi = Q[kQVz * n + r];
  const uint2* pat = row_pattern64(G, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const Slot64 sl = slot64(G, pat, r, k, p);
    const unsigned int fl = sl.fl;
    if (fl & kEntryDiag) {  // (f_i - f_i).c_ii = 0; the diagonal's m_i.c_ii is not used
#pragma unroll
      for (int f = 0; f < kFields; ++f) dF[f * ns + p] = 0.0;
      mc[p] = 0.0;
      continue;
    }
    if (!(fl & kEntryUpper)) continue;  // written by the pair's owner
    const int64_t j = sl.j;
    const int64_t pt = sl.pt;
    const double cx = G.cx[p], cy = G.cy[p], cz = G.cz[p];
    const Side sj = load_side(U, Q, n, j);
    const double h_j = Q[kQH * n + j];
    const double vxj = Q[kQVx * n + j], vyj = Q[kQVy * n + j], vzj = Q[kQVz * n + j];
    double df[kFields], mcj, mci;
    flux_diff(si, sj, vxi, vyi, vzi, vxj, vyj, vzj, h_i, h_j, cx, cy, cz, df, &mcj, &mci);
#pragma unroll
    for (int f = 0; f < kFields; ++f) dF[f * ns + p] = df[f];
    mc[p] = mcj;
    const double nc = G.cn[p];
    double dij = 0.0;
    if (positive_k(nc)) {
      const double inv = G.inv_cn[p];
      dij = lambda_max_u(normal_speed(mci, si.inv_rho, inv), normal_speed(mcj, sj.inv_rho, inv), si, sj) * nc;
    }
    if (fl & kEntrySkew) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) dF[f * ns + pt] = df[f];
      mc[pt] = -mci;
    } else {  // boundary pair: the transposed orientation separately
      const double tx = G.cx[pt], ty = G.cy[pt], tz = G.cz[pt];
      double dft[kFields], mcjt, mcit;
      flux_diff(sj, si, vxj, vyj, vzj, vxi, vyi, vzi, h_j, h_i, tx, ty, tz, dft, &mcjt, &mcit);
#pragma unroll
      for (int f = 0; f < kFields; ++f) dF[f * ns + pt] = dft[f];
      mc[pt] = mcjt;
      const double nt = G.cn[pt];
      if (positive_k(nt)) {
        const double inv = G.inv_cn[pt];
        dij = fmax(dij, lambda_max(tx * inv, ty * inv, tz * inv, sj, si) * nt);
      }
    }
    d[p] = dij;
    dinv[p] = !dzero(dij) ? div_pos(0.5, dij) : 0.0;
  }
}

__global__ void __launch_bounds__(kMaxBlock) k_edge(DeviceGraph G, const double* __restrict__ U,
                                                 const double* __restrict__ Q, double* __restrict__ d,
                                                 double* __restrict__ dinv, double* __restrict__ dF,
                                                 double* __restrict__ mc, DeviceScalars* scal) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < G.n_inst) G.tau_min[r] = 0x7ff0000000000000ull;  // +inf, read by the next kernel
  if (r < G.n) row_edge(G, U, Q, d, dinv, dF, mc, r);
}

// Step 2: d_ij = d_ji below the diagonal, d_ii = -sum_{j != i} d_ij and the
// CFL bound min_i m_i / (-2 d_ii) (a deterministic min over all rows); and the
// indicator alpha_i = N_i / D_i of Sec. 3.8 from the flux differences and
// m_j.c_ij of Step 1, summed over all j in I(i) in slot order.
__device__ __forceinline__ double row_diag(const DeviceGraph& G, const double* U, const double* Q, double* d,
                                           double* dinv, const double* dF, const double* mc, double* alpha,
                                           double* ab, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double s_i = Q[kQS * n + r];
  double sum = 0.0;
  double a = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0, b4 = 0.0;
  int64_t pd = base;
  const uint2* pat = row_pattern64(G, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const Slot64 sl = slot64(G, pat, r, k, p);
    const int64_t j = sl.j;
    a = fma(Q[kQS * n + j] - s_i, mc[p], a);
    b0 += dF[p];
    b1 += dF[ns + p];
    b2 += dF[2 * ns + p];
    b3 += dF[3 * ns + p];
    b4 += dF[4 * ns + p];
    if (j == r) {
      pd = p;
      continue;
    }
    double v;
    if (!(sl.fl & kEntryUpper)) {  // lower entry: copy from the owning row
      const int64_t pt = sl.pt;
      v = d[pt];
      d[p] = v;
      dinv[p] = dinv[pt];
    } else {
      v = d[p];
    }
    sum += v;
  }
  d[pd] = -sum;
  // eta'(U_i) = (rho eps)^(-7/12)/(gamma+1) (E, -m, rho) = (eta/rho) / (6 p) (E, -m, rho)
  const double rho = U[r], mx = U[n + r], my = U[2 * n + r], mz = U[3 * n + r], Ei = U[4 * n + r];
  const double sc = s_i * Q[kQInvP * n + r] * (1.0 / 6.0);
  const double e0 = sc * Ei, e1 = -sc * mx, e2 = -sc * my, e3 = -sc * mz, e4 = sc * rho;
  const double num = a - (e0 * b0 + e1 * b1 + e2 * b2 + e3 * b3 + e4 * b4) + s_i * b0;
  const double D = fabs(a) + fabs(e0 - s_i) * fabs(b0) + fabs(e1) * fabs(b1) + fabs(e2) * fabs(b2) +
                   fabs(e3) * fabs(b3) + fabs(e4) * fabs(b4);
  alpha[r] = positive_k(D) ? fabs(num) / D : 0.0;
  if (ab) {  // traced for the adjoint
    ab[r] = a;
    ab[n + r] = b0;
    ab[2 * n + r] = b1;
    ab[3 * n + r] = b2;
    ab[4 * n + r] = b3;
    ab[5 * n + r] = b4;
  }
  return G.mi[r] / (2.0 * sum);
}

__global__ void __launch_bounds__(kMaxBlock) k_diag(DeviceGraph G, const double* __restrict__ U,
                                                 const double* __restrict__ Q, double* __restrict__ d,
                                                 double* __restrict__ dinv, const double* __restrict__ dF,
                                                 const double* __restrict__ mc, double* __restrict__ alpha,
                                                 double* __restrict__ ab, DeviceScalars* scal) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  reduce_tau_candidate(G, r, computes_row(G, r) ? row_diag(G, U, Q, d, dinv, dF, mc, alpha, ab, r) : INFINITY);
}

// Step 3: low-order update through the bar states (eq. def-ubar), R_i
// (eq. high-order-final) and the local bounds rho_min, rho_max over
// rho(Ubar_ij) and phi_min over phi(U_j), j in I(i) (Sec. 3.9).  With the
// flux differences df_ij = (f_j - f_i).c_ij of Step 1,
// Ubar_ij = (U_i + U_j)/2 - df_ij/(2 d_ij) and, since sum_j c_ij = s_i,
// sum_j -f_j.c_ij = -sum_j df_ij - f_i.s_i (s_i is zero up to rounding).
__device__ __forceinline__ void row_low_order(const DeviceGraph& G, const StageConfig& C, const double* U,
                                              const double* Q, const double* d,
                                              const double* dinv, const double* dF,
                                              const double* alpha, double* UL,
                                              double* R, double* bnd, int tau_mode,
                                              int64_t r) {
  const double tau = stage_tau(G, instance_of(G, r), tau_mode, C.cfl);
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double ui[kFields];
  load5(U, n, r, ui);
  const double a_i = alpha[r];
  const double tau_m = tau * G.inv_mi[r];
  double ul[kFields], rr[kFields];
  {
    double fs[kFields];  // f_i . s_i
    flux_dot(ui[1], ui[2], ui[3], Q[kQInvRho * n + r], Q[kQP * n + r], Q[kQH * n + r], G.csx[r], G.csy[r],
             G.csz[r], fs);
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      ul[f] = ui[f];
      rr[f] = -fs[f];
    }
  }
  // The bar states are formed doubled, 2 Ubar_ij = U_i + U_j - (f_j - f_i).c_ij / d_ij,
  // against half the coefficient, tau d_ij / m_i: the same products (scaling by
  // 2 is exact) without the multiplications by 1/2; the bounds are halved once.
  double rho_min2 = INFINITY, rho_max2 = -INFINITY, phi_min = INFINITY;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    const double dij = d[p];
    double uj[kFields], df[kFields];
    load5(U, n, j, uj);
#pragma unroll
    for (int f = 0; f < kFields; ++f) df[f] = dF[f * ns + p];
    const double dH = dij * (a_i + alpha[j]) * 0.5;
#pragma unroll
    for (int f = 0; f < kFields; ++f) rr[f] += -df[f] + dH * (uj[f] - ui[f]);
    if (!dzero(dij)) {
      const double inv_d = 2.0 * dinv[p];  // 1/d_ij
      const double coef_h = tau_m * dij;   // (2 tau d_ij / m_i) / 2
      double ub2[kFields];
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        ub2[f] = fma(-df[f], inv_d, ui[f] + uj[f]);
        ul[f] = fma(coef_h, ub2[f], ul[f]);
      }
      rho_min2 = min_k(rho_min2, ub2[0]);
      rho_max2 = max_k(rho_max2, ub2[0]);
    }
    phi_min = min_k(phi_min, Q[kQPhi * n + j]);
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    UL[f * n + r] = ul[f];
    R[f * n + r] = rr[f];
  }
  double rho_min = 0.5 * rho_min2, rho_max = 0.5 * rho_max2;
  if (G.relax) {  // bound relaxation (off unless configured)
    const double q = G.relax[r];
    rho_min *= 1.0 - q;
    rho_max *= 1.0 + q;
    phi_min *= 1.0 - q;
  }
  bnd[r] = rho_min;
  bnd[n + r] = rho_max;
  bnd[2 * n + r] = phi_min;
}

__global__ void __launch_bounds__(kMaxBlock) k_low_order(DeviceGraph G, StageConfig C, const double* __restrict__ U,
                                                      const double* __restrict__ Q, const double* __restrict__ d,
                                                      const double* __restrict__ dinv, const double* __restrict__ dF,
                                                      const double* __restrict__ alpha, double* __restrict__ UL,
                                                      double* __restrict__ R, double* __restrict__ bnd,
                                                      DeviceScalars* scal, int tau_mode, int accumulate_time) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  instance_books(G, t, tau_mode, C.cfl, accumulate_time, scal);
  const int64_t r = row_start(G) + t;
  if (computes_row(G, r)) row_low_order(G, C, U, Q, d, dinv, dF, alpha, UL, R, bnd, tau_mode, r);
}

// Step 4: antidiffusive fluxes P_ij (eq. def-p) with b_ij = -m_ij/m_j,
// b_ji = -m_ij/m_i (j != i) and the first limiter values l_ij.
__device__ __forceinline__ void row_flux_limit(const DeviceGraph& G, const StageConfig& C,
                                               const double* U, const double* d,
                                               const double* alpha, const double* UL,
                                               const double* R, const double* bnd,
                                               double* P, double* l, int tau_mode,
                                               int64_t r) {
  const double tau = stage_tau(G, instance_of(G, r), tau_mode, C.cfl);
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double ui[kFields], ri[kFields], ul[kFields];
  load5(U, n, r, ui);
  load5(R, n, r, ri);
  load5(UL, n, r, ul);
  const double rmin = bnd[r], rmax = bnd[n + r], pmin = bnd[2 * n + r];
  const PsiCheck32 pre = make_psi_check(ul, pmin);
  const double a_i = alpha[r];
  const double inv_mi = G.inv_mi[r];
  const double scale = tau * inv_mi * (double)(len - 1);  // tau / (m_i lambda_i)
  const double scale_i = scale * inv_mi;
  const uint2* pat = row_pattern64(G, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = slot64(G, pat, r, k, p).j;
    if (j == r) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) P[f * ns + p] = 0.0;
      l[p] = 0.0;
      continue;
    }
    double uj[kFields], rj[kFields], pij[kFields];
    load5(U, n, j, uj);
    load5(R, n, j, rj);
    // the coefficients scaled once per entry instead of each field:
    // scale b_ij = -scale m_ij / m_j, scale b_ji = -m_ij scale / m_i,
    // scale (d^H_ij - d^L_ij)
    const double m = G.mij[p];
    const double sb_ij = -(scale * m) * G.inv_mi[j];
    const double sb_ji = -m * scale_i;
    const double dij = d[p];
    const double sdd = scale * (dij * (a_i + alpha[j]) * 0.5 - dij);
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      pij[f] = fma(sb_ij, rj[f], fma(-sb_ji, ri[f], sdd * (uj[f] - ui[f])));
      P[f * ns + p] = pij[f];
    }
    l[p] = limiter(ul, pij, rmin, rmax, pmin, C.lim, &pre);
  }
}

__global__ void __launch_bounds__(kMaxBlock) k_flux_limit(DeviceGraph G, StageConfig C, const double* __restrict__ U,
                                                       const double* __restrict__ d, const double* __restrict__ alpha,
                                                       const double* __restrict__ UL, const double* __restrict__ R,
                                                       const double* __restrict__ bnd, double* __restrict__ P,
                                                       double* __restrict__ l, const DeviceScalars* scal,
                                                       int tau_mode) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_flux_limit(G, C, U, d, alpha, UL, R, bnd, P, l, tau_mode, r);
}

// Steps 5, 6, ...: U_i += sum_j lambda_i min(l_ij, l_ji) P_ij, then (not in
// the last pass) P_ij <- (1 - min(l_ij, l_ji)) P_ij and new l_ij.
__device__ __forceinline__ void row_limiter_pass(const DeviceGraph& G, const StageConfig& C,
                                                 const double* Ucur, double* Unext,
                                                 double* P, const double* lold,
                                                 double* lnew, const double* bnd, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double lam = G.lam[r];
  double u[kFields];
  load5(Ucur, n, r, u);
  const uint2* pat = row_pattern64(G, r);
  {
    // loads of entry k + 1 issued before entry k's accumulation
    bool dg_n = false;
    double la_n = 0.0, lb_n = 0.0, p_n[kFields];
    auto fetch1 = [&](int k) {
      const int64_t q = base + 32 * (int64_t)k;
      const Slot64 sl = slot64(G, pat, r, k, q);
      dg_n = sl.j == r;
      la_n = lold[q];
      lb_n = lold[sl.pt];
#pragma unroll
      for (int f = 0; f < kFields; ++f) p_n[f] = P[f * ns + q];
    };
    if (len > 0) fetch1(0);
    for (int k = 0; k < len; ++k) {
      const bool dg = dg_n;
      const double la = la_n, lb = lb_n;
      double pk[kFields];
#pragma unroll
      for (int f = 0; f < kFields; ++f) pk[f] = p_n[f];
      if (k + 1 < len) fetch1(k + 1);
      if (dg) continue;
      // min of two limiter values in [0, 1] on their bit patterns (integer pipe)
      const double w = lam * min_k(la, lb);
#pragma unroll
      for (int f = 0; f < kFields; ++f) u[f] += w * pk[f];
    }
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) Unext[f * n + r] = u[f];
  const double rmin = bnd[r], rmax = bnd[n + r], pmin = bnd[2 * n + r];
  const PsiCheck32 pre = make_psi_check(u, pmin);
  // Software pipeline: entry k + 1's loads are issued before entry k's limiter.
  bool diag_n = false;
  double lk_n = 0.0, p_n[kFields];
  auto fetch = [&](int k) {
    const int64_t q = base + 32 * (int64_t)k;
    const Slot64 sl = slot64(G, pat, r, k, q);
    diag_n = sl.j == r;
    lk_n = min_k(lold[q], lold[sl.pt]);
#pragma unroll
    for (int f = 0; f < kFields; ++f) p_n[f] = P[f * ns + q];
  };
  if (len > 0) fetch(0);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const bool diag = diag_n;
    const double lk = lk_n;
    double pold[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) pold[f] = p_n[f];
    if (k + 1 < len) fetch(k + 1);
    if (diag) {
      lnew[p] = 0.0;
      continue;
    }
    double pij[kFields];
    bool zero = true;
    if (is_one(lk)) {
      // l = 1: (1 - l) P_ij is a zero with the sign of P_ij
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        pij[f] = __hiloint2double(__double2hiint(pold[f]) & (int)0x80000000, 0);
        P[f * ns + p] = pij[f];
      }
    } else {
      const bool keep = is_pos_zero(lk);
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        // l = 0 leaves P_ij as it is
        pij[f] = keep ? pold[f] : (1.0 - lk) * pold[f];
        if (!keep) P[f * ns + p] = pij[f];
        zero &= ((((unsigned int)__double2hiint(pij[f])) << 1) | (unsigned int)__double2loint(pij[f])) == 0u;
      }
    }
    // A zero P_ij (the previous pass accepted it in full, so P_ji is zero
    // too) is moved by no value of l_ij: skip the limiter.
    lnew[p] = zero ? 1.0 : limiter(u, pij, rmin, rmax, pmin, C.lim, &pre);
  }
}

__global__ void __launch_bounds__(kMaxBlock) k_limiter_pass(DeviceGraph G, StageConfig C, const double* __restrict__ Ucur,
                                                         double* __restrict__ Unext, double* __restrict__ P,
                                                         const double* __restrict__ lold, double* __restrict__ lnew,
                                                         const double* __restrict__ bnd) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_limiter_pass(G, C, Ucur, Unext, P, lold, lnew, bnd, r);
}

// Last limiter pass, boundary post-processing (slip walls drop the flagged
// normal momentum components, inflow nodes take the inflow state) and the
// SSP-RK3 blend (Sec. 3.6): stage 2 3/4 U^n + 1/4 E, stage 3 1/3 U^n + 2/3 E.
__device__ __forceinline__ void row_final(const DeviceGraph& G, const StageConfig& C, const double* Ucur,
                                          const double* P, const double* l,
                                          const double* Un, double* Uout,
                                          double* Ulim, DeviceScalars* scal, int blend,
                                          int skip_write_on_error, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double lam = G.lam[r];
  double u[kFields];
  load5(Ucur, n, r, u);
  const uint2* pat = row_pattern64(G, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const Slot64 sl = slot64(G, pat, r, k, p);
    if (sl.j == r) continue;
    const double lk = min_k(l[p], l[sl.pt]);
    const double w = lam * lk;
#pragma unroll
    for (int f = 0; f < kFields; ++f) u[f] += w * P[f * ns + p];
  }
  if (Ulim) {
#pragma unroll
    for (int f = 0; f < kFields; ++f) Ulim[f * n + r] = u[f];
  }
  const int bc = G.bc[r];
  if (bc & 8) {
#pragma unroll
    for (int f = 0; f < kFields; ++f) u[f] = C.inflow[f];
  } else {
    if (bc & 1) u[1] = 0.0;
    if (bc & 2) u[2] = 0.0;
    if (bc & 4) u[3] = 0.0;
  }
  double out[kFields];
  bool finite = true;
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    double v = u[f];
    if (blend == kBlendStage2) v = 0.75 * Un[f * n + r] + 0.25 * u[f];
    if (blend == kBlendStage3) v = (1.0 / 3.0) * Un[f * n + r] + (2.0 / 3.0) * u[f];
    out[f] = v;
    finite &= (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;  // not inf/nan
  }
  if (!finite) atomicOr(&scal->status, kStatusNonFinite);
  if (skip_write_on_error && *(volatile int*)&scal->status != 0) return;
#pragma unroll
  for (int f = 0; f < kFields; ++f) Uout[f * n + r] = out[f];
}

__global__ void __launch_bounds__(kMaxBlock) k_final(DeviceGraph G, StageConfig C, const double* __restrict__ Ucur,
                                                  const double* __restrict__ P, const double* __restrict__ l,
                                                  const double* __restrict__ Un, double* __restrict__ Uout,
                                                  double* __restrict__ Ulim, DeviceScalars* scal, int blend,
                                                  int skip_write_on_error) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_final(G, C, Ucur, P, l, Un, Uout, Ulim, scal, blend, skip_write_on_error, r);
}

// One euler_step in a single cooperative launch: the phases of the kernels
// above run over all rows (tiles of 32 rows handed out dynamically) with a
// grid barrier between them, where the kernel boundaries were.  Data a phase
// reads was written before the barrier that precedes it (or before the
// launch), never earlier in the launch by another block, so no block can
// hold a stale copy of it.
__global__ void __launch_bounds__(kMaxBlock, 2) k_stage_persistent(PersistentStage a) {
  const DeviceGraph& G = a.G;
  const StageConfig& C = a.C;
  const StageBuffers& B = a.B;
  const int64_t n = G.n;
  unsigned int* tile = a.bar->tile;
  for_each_row_tile(&tile[0], n, [&](int64_t i) {
    if (i < n) row_node(n, a.Uin, B.node, B.scal, i);
    if (i < G.n_inst) G.tau_min[i] = 0x7ff0000000000000ull;
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[1], n, [&](int64_t r) {
    if (r < n) row_edge(G, a.Uin, B.node, B.d, B.dinv, B.P, B.l[1], r);
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[2], n, [&](int64_t r) {
    reduce_tau_candidate(G, r, r < n ? row_diag(G, a.Uin, B.node, B.d, B.dinv, B.P, B.l[1], B.alpha, nullptr, r) : INFINITY);
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[3], n, [&](int64_t r) {
    instance_books(G, r, a.tau_mode, C.cfl, a.accumulate_time, B.scal);
    if (r < n) row_low_order(G, C, a.Uin, B.node, B.d, B.dinv, B.P, B.alpha, B.UL, B.R, B.bnd, a.tau_mode, r);
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[4], n, [&](int64_t r) {
    if (r < n) row_flux_limit(G, C, a.Uin, B.d, B.alpha, B.UL, B.R, B.bnd, B.P, B.l[0], a.tau_mode, r);
  });
  const double* cur = B.UL;
  int lbuf = 0, wbuf = 0;
  for (int pass = 1; pass < C.limiter_passes; ++pass) {
    if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
    double* next = B.Uw[wbuf];
    const int ph = 4 + pass < 11 ? 4 + pass : 11;
    for_each_row_tile(&tile[ph], n, [&](int64_t r) {
      if (r < n) row_limiter_pass(G, C, cur, next, B.P, B.l[lbuf], B.l[lbuf ^ 1], B.bnd, r);
    });
    cur = next;
    wbuf ^= 1;
    lbuf ^= 1;
  }
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[11], n, [&](int64_t r) {
    if (r < n) row_final(G, C, cur, B.P, B.l[lbuf], a.Un, a.Uout, B.Ulast, B.scal, a.blend, a.skip_write_on_error, r);
  });
}

// Self-test of the grid barrier: every block passes `rounds` barriers and
// counts its passes; with skip_block0 block 0 never arrives, so the other
// blocks' waits run out after spin_limit polls.
__global__ void k_barrier_selftest(GridBarrier* bar, long long spin_limit, int rounds, int skip_block0,
                                   unsigned int* passes, DeviceScalars* scal) {
  if (skip_block0 && blockIdx.x == 0) return;
  for (int k = 0; k < rounds; ++k) {
    if (!grid_barrier(bar, spin_limit, scal)) return;
    if (threadIdx.x == 0) atomicAdd(passes, 1u);
  }
}

// Order-preserving map of doubles to unsigned 64-bit keys (negative values
// reverse their bit order), so that atomicMin on keys is a min on values.
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double from_order_key(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Invariant check of a state: counts of rho <= 0, eps <= 0 and non-finite
// nodes, and the minima of rho and eps, accumulated with atomics into
// acc = {count_rho, count_eps, count_nonfinite, key(rho_min), key(eps_min)}.
__global__ void __launch_bounds__(kBlock) k_check_state(const double* __restrict__ U, int64_t n,
                                                        unsigned long long* acc) {
  double rmin = INFINITY, emin = INFINITY;
  unsigned long long c0 = 0, c1 = 0, c2 = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double u[kFields];
    load5(U, n, i, u);
    bool fin = true;
#pragma unroll
    for (int f = 0; f < kFields; ++f) fin &= isfinite(u[f]);
    const double eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
    c0 += !(u[0] > 0.0);
    c1 += !(eps > 0.0);
    c2 += !fin;
    rmin = fmin(rmin, u[0]);
    emin = fmin(emin, eps);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(&acc[0], c0);
    if (c1) atomicAdd(&acc[1], c1);
    if (c2) atomicAdd(&acc[2], c2);
    atomicMin(&acc[3], order_key(rmin));
    atomicMin(&acc[4], order_key(emin));
  }
}

__global__ void k_check_finish(const unsigned long long* acc, double* out) {
  out[0] = (double)acc[0];
  out[1] = (double)acc[1];
  out[2] = (double)acc[2];
  out[3] = from_order_key(acc[3]);
  out[4] = from_order_key(acc[4]);
}

// Local bounds of Sec. 3.9 on a stage output: rho in [rho_min, rho_max] and
// phi >= phi_min, the latter in the form the limiter tests (Alg. 2), Psi =
// rho eps - phi_min rho^(gamma+1) >= -slack (|rho eps| + phi_min
// rho^(gamma+1)).  acc = {n_rho_below, n_rho_above, n_phi_below, key(worst
// (rho_min - rho)/|rho_min|), key(worst (rho - rho_max)/|rho_max|),
// key(worst -Psi/scale), rows}.  A NaN counts as a violation.  Off the
// stage's path: runs only when a caller asks for the check.
__global__ void __launch_bounds__(kBlock) k_check_local(const double* __restrict__ U, const double* __restrict__ bnd,
                                                        int64_t n, double slack_rho, double slack_phi,
                                                        unsigned long long* acc) {
  double w0 = -INFINITY, w1 = -INFINITY, w2 = -INFINITY;
  unsigned long long c0 = 0, c1 = 0, c2 = 0, rows = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double u[kFields];
    load5(U, n, i, u);
    const double rmin = bnd[i], rmax = bnd[n + i], pmin = bnd[2 * n + i];
    const double v0 = (rmin - u[0]) / fabs(rmin);
    const double v1 = (u[0] - rmax) / fabs(rmax);
    const double re = u[0] * u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
    const double pw = pmin * pow(u[0], 2.4);
    const double v2 = -(re - pw) / (fabs(re) + fabs(pw));
    c0 += !(v0 <= slack_rho);
    c1 += !(v1 <= slack_rho);
    c2 += !(v2 <= slack_phi);
    w0 = fmax(w0, v0);
    w1 = fmax(w1, v1);
    w2 = fmax(w2, v2);
    ++rows;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    w0 = fmax(w0, __shfl_xor_sync(0xffffffffu, w0, o));
    w1 = fmax(w1, __shfl_xor_sync(0xffffffffu, w1, o));
    w2 = fmax(w2, __shfl_xor_sync(0xffffffffu, w2, o));
    c0 += __shfl_xor_sync(0xffffffffu, c0, o);
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    rows += __shfl_xor_sync(0xffffffffu, rows, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(&acc[0], c0);
    if (c1) atomicAdd(&acc[1], c1);
    if (c2) atomicAdd(&acc[2], c2);
    atomicMax(&acc[3], order_key(w0));
    atomicMax(&acc[4], order_key(w1));
    atomicMax(&acc[5], order_key(w2));
    if (rows) atomicAdd(&acc[6], rows);
  }
}

__global__ void k_check_local_finish(const unsigned long long* acc, double* out) {
  out[0] = (double)acc[6];
  out[1] = (double)acc[0];
  out[2] = (double)acc[1];
  out[3] = (double)acc[2];
  out[4] = from_order_key(acc[3]);
  out[5] = from_order_key(acc[4]);
  out[6] = from_order_key(acc[5]);
}

}  // namespace

void Profiler::begin(int id, cudaStream_t s) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  ev.push_back(a);
  ev.push_back(b);
  kernel.push_back(id);
  cudaEventRecord(a, s);
}

void Profiler::end(cudaStream_t s) { cudaEventRecord(ev.back(), s); }

void Profiler::clear() {
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  ev.clear();
  kernel.clear();
}

int launch_euler_step(const DeviceGraph& G, const StageBuffers& B, const StageConfig& C, const double* Uin,
                      double* Uout, const double* Un, int blend, int tau_mode, bool accumulate_time,
                      bool skip_write_on_error, bool trace, cudaStream_t s, Profiler* prof, int block,
                      GridBarrier* bar) {
  const int kBlock = block;  // block size of this schedule (<= kMaxBlock)
  const unsigned grid = (unsigned)((G.n + kBlock - 1) / kBlock);
  const bool p = prof && prof->enabled;
  if (bar && !trace && !p) {
    PersistentStage a{G, C, B, Uin, Uout, Un, bar, blend, tau_mode, accumulate_time ? 1 : 0,
                      skip_write_on_error ? 1 : 0};
    const int limit = persistent_grid_limit(kBlock, false);
    const unsigned pgrid = (unsigned)(limit < (int)grid ? limit : grid);
    cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    void* args[] = {&a};
    cudaLaunchCooperativeKernel((const void*)k_stage_persistent, dim3(pgrid), dim3(kBlock), args, 0, s);
    return 1;
  }
  int launches = 0;
  auto run = [&](int id, auto&& launch) {
    if (p) prof->begin(id, s);
    launch();
    if (p) prof->end(s);
    ++launches;
  };
  run(kKNode, [&] { k_node<<<grid, kBlock, 0, s>>>(G.n, Uin, B.node, B.scal); });
  // m_j.c_ij of Step 1 lives in l[1] until Step 2 (l[1] is next written by the first limiter pass);
  // the flux differences live in P until Step 3, or in the trace when tracing
  double* dF = trace ? B.tdF : B.P;
  run(kKEdge, [&] { k_edge<<<grid, kBlock, 0, s>>>(G, Uin, B.node, B.d, B.dinv, dF, B.l[1], B.scal); });
  run(kKDiag, [&] {
    k_diag<<<grid, kBlock, 0, s>>>(G, Uin, B.node, B.d, B.dinv, dF, B.l[1], B.alpha, trace ? B.tab : nullptr,
                                   B.scal);
  });
  run(kKLowOrder, [&] {
    k_low_order<<<grid, kBlock, 0, s>>>(G, C, Uin, B.node, B.d, B.dinv, dF, B.alpha, B.UL, B.R, B.bnd, B.scal,
                                        tau_mode, accumulate_time ? 1 : 0);
  });
  run(kKFluxLimit, [&] {
    k_flux_limit<<<grid, kBlock, 0, s>>>(G, C, Uin, B.d, B.alpha, B.UL, B.R, B.bnd, B.P, B.l[0], B.scal, tau_mode);
  });
  if (trace) {
    cudaMemcpyAsync(B.tP, B.P, sizeof(double) * kFields * G.n_slots, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(B.tl4, B.l[0], sizeof(double) * G.n_slots, cudaMemcpyDeviceToDevice, s);
  }
  const double* cur = B.UL;
  int lbuf = 0, wbuf = 0;
  for (int pass = 1; pass < C.limiter_passes; ++pass) {
    double* next = B.Uw[wbuf];
    run(kKLimiterPass,
        [&] { k_limiter_pass<<<grid, kBlock, 0, s>>>(G, C, cur, next, B.P, B.l[lbuf], B.l[lbuf ^ 1], B.bnd); });
    if (trace && pass == 1) {
      cudaMemcpyAsync(B.tU5, next, sizeof(double) * kFields * G.n, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(B.tl5, B.l[lbuf ^ 1], sizeof(double) * G.n_slots, cudaMemcpyDeviceToDevice, s);
    }
    cur = next;
    wbuf ^= 1;
    lbuf ^= 1;
  }
  // the stage output before boundary values and blend: kept in B.Ulast for
  // the local-bound check, and copied to the trace when tracing
  double* ulim = B.Ulast ? B.Ulast : (trace ? B.tUlim : nullptr);
  run(kKFinal, [&] {
    k_final<<<grid, kBlock, 0, s>>>(G, C, cur, B.P, B.l[lbuf], Un, Uout, ulim, B.scal, blend,
                                    skip_write_on_error ? 1 : 0);
  });
  if (trace && B.Ulast)
    cudaMemcpyAsync(B.tUlim, B.Ulast, sizeof(double) * kFields * G.n, cudaMemcpyDeviceToDevice, s);
  return launches;
}

int euler_phase_count(const StageConfig& C) { return 3 + C.limiter_passes; }

double* phase_l_buffer(const StageBuffers& B, int phase) { return B.l[(phase - 2) & 1]; }

int launch_euler_phase(const DeviceGraph& G, const StageBuffers& B, const StageConfig& C, const double* Uin,
                       double* Uout, const double* Un, int blend, int tau_mode, bool accumulate_time,
                       bool skip_write_on_error, int phase, cudaStream_t s, int block) {
  const unsigned grid = (unsigned)((G.n + block - 1) / block);
  const unsigned grid_own = own_row_grid(G, block);  // Steps 2-6
  const int passes = C.limiter_passes;
  if (phase == 0) {
    k_node<<<grid, block, 0, s>>>(G.n, Uin, B.node, B.scal);
    k_edge<<<grid, block, 0, s>>>(G, Uin, B.node, B.d, B.dinv, B.P, B.l[1], B.scal);
    k_diag<<<grid_own, block, 0, s>>>(G, Uin, B.node, B.d, B.dinv, B.P, B.l[1], B.alpha, nullptr, B.scal);
    return 3;
  }
  if (phase == 1) {
    k_low_order<<<grid_own, block, 0, s>>>(G, C, Uin, B.node, B.d, B.dinv, B.P, B.alpha, B.UL, B.R, B.bnd, B.scal,
                                       tau_mode, accumulate_time ? 1 : 0);
    return 1;
  }
  if (phase == 2) {
    k_flux_limit<<<grid_own, block, 0, s>>>(G, C, Uin, B.d, B.alpha, B.UL, B.R, B.bnd, B.P, B.l[0], B.scal, tau_mode);
    return 1;
  }
  // pass p reads the state of pass p - 1 (U^L for p = 1) and l of pass p - 1;
  // the buffers alternate as in launch_euler_step
  auto state_after = [&](int p) -> double* { return p == 0 ? B.UL : B.Uw[(p - 1) & 1]; };
  const int p = phase - 2;
  if (p >= 1 && p < passes) {
    k_limiter_pass<<<grid_own, block, 0, s>>>(G, C, state_after(p - 1), B.Uw[(p - 1) & 1], B.P, B.l[(p - 1) & 1],
                                          B.l[p & 1], B.bnd);
    return 1;
  }
  if (p == passes) {
    k_final<<<grid_own, block, 0, s>>>(G, C, state_after(passes - 1), B.P, B.l[(passes - 1) & 1], Un, Uout, B.Ulast,
                                   B.scal, blend, skip_write_on_error ? 1 : 0);
    return 1;
  }
  return 0;
}

cudaError_t launch_barrier_selftest(GridBarrier* bar, long long spin_limit, int blocks, int rounds, int skip_block0,
                                    unsigned int* passes, DeviceScalars* scal, cudaStream_t s) {
  cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  cudaMemsetAsync(passes, 0, sizeof(unsigned int), s);
  void* args[] = {&bar, &spin_limit, &rounds, &skip_block0, &passes, &scal};
  return cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(blocks), dim3(64), args, 0, s);
}

int persistent_grid_limit(int block, bool mixed) {
  // occupancy is a property of the kernel and the block size: cache it
  static int cache[2][3] = {{0, 0, 0}, {0, 0, 0}};
  const int slot = block == 64 ? 0 : (block == 128 ? 1 : 2);
  int& v = cache[mixed ? 1 : 0][slot];
  if (v == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mixed ? persistent_kernel_mixed() : (const void*)k_stage_persistent,
                                                  block, 0);
    v = sms * (per_sm > 0 ? per_sm : 1);
  }
  return v;
}

void launch_check_local(const double* U, const double* bnd, int64_t n, double slack_rho, double slack_phi,
                        double* out, unsigned long long* acc, cudaStream_t s) {
  // counts start at 0, maximum keys at the smallest key
  cudaMemsetAsync(acc, 0, 7 * sizeof(unsigned long long), s);
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  const unsigned grid = (unsigned)(blocks < 152 * 8 ? blocks : 152 * 8);
  k_check_local<<<grid, kBlock, 0, s>>>(U, bnd, n, slack_rho, slack_phi, acc);
  k_check_local_finish<<<1, 1, 0, s>>>(acc, out);
}

void launch_check_state(const double* U, int64_t n, double* out, unsigned long long* acc, cudaStream_t s) {
  // counts start at 0, minimum keys at the largest key
  cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), s);
  cudaMemsetAsync(acc + 3, 0xff, 2 * sizeof(unsigned long long), s);
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  const unsigned grid = (unsigned)(blocks < 152 * 8 ? blocks : 152 * 8);
  k_check_state<<<grid, kBlock, 0, s>>>(U, n, acc);
  k_check_finish<<<1, 1, 0, s>>>(acc, out);
}

}  // namespace idp
