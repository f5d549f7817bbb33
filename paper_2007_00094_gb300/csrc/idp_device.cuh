// Device building blocks of the stage for gamma = 7/5 (Sec. 2): powers with
// fixed rational exponents, the two-rarefaction wavespeed bound (Sec. 3.7)
// and the convex limiter (Sec. 3.9, Alg. 2 and Alg. 3), in FP64.
#pragma once
#include <cstdint>

namespace idp {

// w^K by repeated squaring (K = 5, 7, 12 in this file).
template <int K>
__device__ __forceinline__ double ipow(double w) {
  if constexpr (K == 1) {
    return w;
  } else if constexpr (K % 2 == 0) {
    const double h = ipow<K / 2>(w);
    return h * h;
  } else {
    return ipow<K - 1>(w) * w;
  }
}

// x^(-1/K) for x > 0.  A single-precision seed w0 = powf(x, -1/K) (relative
// error below 3e-7) is corrected with the second-order series of
// (1 - delta)^(-1/K) = 1 + delta/K + (K+1) delta^2/(2K^2) + O(delta^3), where
// delta = 1 - x w0^K; the neglected term is ~delta^3 < 1e-17 for K <= 12.
template <int K>
__device__ __forceinline__ double inv_root(double x) {
  const double w0 = (double)powf((float)x, -1.0f / (float)K);
  const double delta = 1.0 - x * ipow<K>(w0);
  const double c1 = 1.0 / (double)K, c2 = (double)(K + 1) / (2.0 * (double)K * (double)K);
  return fma(w0, fma(c2, delta, c1) * delta, w0);
}

// rho^(gamma+1) = rho^(12/5) = rho^3 * (rho^(-1/5))^3
__device__ __forceinline__ double pow_12_5(double rho) {
  const double w = inv_root<5>(rho);
  return rho * rho * rho * (w * w * w);
}

// Per-node quantities of the stage (Step 0, "precompute entropies").
enum NodeQ : int {
  kQInvRho = 0,  // 1/rho
  kQP = 1,       // p = (gamma-1) epsilon
  kQC = 2,       // c = sqrt(gamma p / rho)
  kQPm = 3,      // p^(-(gamma-1)/(2 gamma)) = p^(-1/7), two-rarefaction pressure
  kQInvP = 4,    // 1/p
  kQS = 5,       // eta/rho, eta = (rho epsilon)^(1/(gamma+1)) (Harten entropy)
  kQH = 6,       // (E + p)/rho, energy flux factor
  kQPhi = 7,     // phi = epsilon rho^(-gamma) (specific entropy)
  kNodeQ = 8
};

struct Side {
  double rho, inv_rho, mx, my, mz, p, c, pm, inv_p;
};

// f(U) . c of eq. (flux): (m.c, v (m.c) + p c, (E+p)/rho (m.c)), with an
// operation sequence pinned by rounding intrinsics so that equal states give
// bitwise equal fluxes (differences f_j - f_i then vanish exactly, as in the
// oracle).
__device__ __forceinline__ void flux_dot(double m1, double m2, double m3, double inv_rho, double p, double h,
                                         double cx, double cy, double cz, double* f) {
  const double mc = __fma_rn(m3, cz, __fma_rn(m2, cy, __dmul_rn(m1, cx)));
  f[0] = mc;
  f[1] = __fma_rn(p, cx, __dmul_rn(__dmul_rn(m1, inv_rho), mc));
  f[2] = __fma_rn(p, cy, __dmul_rn(__dmul_rn(m2, inv_rho), mc));
  f[3] = __fma_rn(p, cz, __dmul_rn(__dmul_rn(m3, inv_rho), mc));
  f[4] = __dmul_rn(h, mc);
}


// lambda~_max(n, U_L, U_R) of Sec. 3.7.  For gamma = 7/5 the two-rarefaction
// pressure is p~* = ((c_L + c_R - (u_R - u_L)/5) / (c_L p_L^(-1/7) +
// c_R p_R^(-1/7)))^7 (the printed form divided through by p_R^(1/7)); the
// projection leaves the pressure unchanged (E~ - m~^2/(2 rho) = epsilon).
// psi is needed at p_max, where only the side with the smaller pressure
// contributes (its shock branch); the other side's f vanishes.
__device__ __forceinline__ double lambda_max(double nx, double ny, double nz, const Side& L, const Side& R) {
  const double uL = (L.mx * nx + L.my * ny + L.mz * nz) * L.inv_rho;
  const double uR = (R.mx * nx + R.my * ny + R.mz * nz) * R.inv_rho;
  double num = L.c + R.c - 0.2 * (uR - uL);
  num = num > 0.0 ? num : 0.0;  // vacuum: p~* = 0
  const double x = num / (L.c * L.pm + R.c * R.pm);
  const double x2 = x * x, x3 = x2 * x, x6 = x3 * x3;
  const double p_tr = x6 * x;
  const bool left_high = L.p >= R.p;
  const double p_max = left_high ? L.p : R.p;
  const double p_low = left_high ? R.p : L.p;
  const double rho_low = left_high ? R.rho : L.rho;
  // psi(p_max) = A/B + du with A = sqrt(2)(p_max - p_low) >= 0 and
  // B = sqrt(rho_low (2.4 p_max + 0.4 p_low)) > 0, so psi < 0 exactly when
  // du < 0 and A^2 < du^2 B^2: the same decision without a square root or a
  // division
  const double du = uR - uL;
  const double dp = p_max - p_low;
  const bool psi_negative = du < 0.0 && 2.0 * dp * dp < du * du * (rho_low * (2.4 * p_max + 0.4 * p_low));
  const double p_star = psi_negative ? p_tr : fmin(p_max, p_tr);
  const double k = 6.0 / 7.0;  // (gamma+1)/(2 gamma)
  const double lam1 = uL - L.c * sqrt(1.0 + k * fmax((p_star - L.p) * L.inv_p, 0.0));
  const double lam3 = uR + R.c * sqrt(1.0 + k * fmax((p_star - R.p) * R.inv_p, 0.0));
  return fmax(fmax(-lam1, 0.0), fmax(lam3, 0.0));
}

struct LimiterParams {
  int newton_max;
  double newton_tol;
  double newton_eps;
};

// rho epsilon = rho E - |m|^2 / 2 of U + t P
__device__ __forceinline__ double rho_eps_at(const double* U, const double* P, double t, double* rho_out) {
  const double r = U[0] + t * P[0];
  const double m1 = U[1] + t * P[1], m2 = U[2] + t * P[2], m3 = U[3] + t * P[3];
  const double E = U[4] + t * P[4];
  *rho_out = r;
  return r * E - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3);
}

// d/dt of rho epsilon along U + t P
__device__ __forceinline__ double drho_eps_at(const double* U, const double* P, double t) {
  const double r = U[0] + t * P[0];
  const double m1 = U[1] + t * P[1], m2 = U[2] + t * P[2], m3 = U[3] + t * P[3];
  const double E = U[4] + t * P[4];
  return P[0] * E + r * P[4] - (m1 * P[1] + m2 * P[2] + m3 * P[3]);
}

// Admissibility margin of Psi = rho eps - phi_min rho^(gamma+1): its two
// terms nearly cancel where phi ~ phi_min (isentropic flow), so the sign of
// a Psi within rounding of zero is arbitrary; Psi >= -1e-13 (|rho eps| +
// |phi_min rho^(gamma+1)|) counts as admissible, a margin far above rounding
// and far below the tolerance of the invariant checks.
__device__ __forceinline__ double psi_slack(double rho_eps, double phi_term) {
  return 1e-13 * (fabs(rho_eps) + fabs(phi_term));
}

// limiter.compute(U, P, bounds) of Alg. 2: density interval, then the
// quadratic Newton iteration of Alg. 3 (sign -1) on
// Psi(t) = rho eps(U + tP) - phi_min rho(U + tP)^(gamma+1), with the
// safeguards: non-negative discriminants, t_L kept admissible, bracket
// ordered; Psi >= -psi_slack counts as admissible (for t_R and the new
// t_L alike).  Returns t_L.
__device__ __forceinline__ double limiter(const double* U, const double* P, double rho_min, double rho_max,
                                          double phi_min, const LimiterParams& prm) {
  double tL = 0.0, tR = 1.0;
  const double rhoU = U[0], rhoP = P[0];
  if (rhoU + tR * rhoP > rho_max && rhoP != 0.0) tR = fabs(rho_max - rhoU) / fabs(rhoP);
  if (rhoU + tR * rhoP < rho_min && rhoP != 0.0) tR = fabs(rho_min - rhoU) / fabs(rhoP);
  tR = fmin(fmax(tR, 0.0), 1.0);
  // Psi and rho^(gamma+1) at the current t_L (t_L = 0 at the start)
  double psiL = 0.0, powL = 0.0;
  bool haveL = false;
  for (int step = 0; step < prm.newton_max; ++step) {
    double rR;
    const double reR = rho_eps_at(U, P, tR, &rR);
    const double powR = pow_12_5(rR);
    const double psiR = reR - phi_min * powR;
    if (psiR >= -psi_slack(reR, phi_min * powR)) {
      tL = tR;
      break;
    }
    if (!haveL) {
      double rL;
      const double reL = rho_eps_at(U, P, tL, &rL);
      powL = pow_12_5(rL);
      psiL = reL - phi_min * powL;
      haveL = true;
    }
    // tolerance relative to rho eps(U) (Reading A11), only needed on this path
    const double tol = prm.newton_tol * (U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]));
    if (psiL <= tol) break;
    const double rhoL = U[0] + tL * P[0];
    const double dpsiL = drho_eps_at(U, P, tL) - phi_min * 2.4 * (powL / rhoL) * P[0];
    const double dpsiR = drho_eps_at(U, P, tR) - phi_min * 2.4 * (powR / rR) * P[0];
    // Alg. 3 with divided differences
    const double scaling = 1.0 / (tR - tL + prm.newton_eps);
    const double d12 = (psiR - psiL) * scaling;
    const double d112 = (d12 - dpsiL) * scaling;
    const double d122 = (dpsiR - d12) * scaling;
    const double lamL = fmax(dpsiL * dpsiL - 4.0 * psiL * d112, 0.0);
    const double lamR = fmax(dpsiR * dpsiR - 4.0 * psiR * d122, 0.0);
    double nL = tL - 2.0 * psiL / (dpsiL - sqrt(lamL));
    double nR = tR - 2.0 * psiR / (dpsiR - sqrt(lamR));
    if (!(nL >= tL)) nL = tL;
    if (!(nL <= tR)) nL = tR;
    double rN;
    const double reN = rho_eps_at(U, P, nL, &rN);
    const double powN = pow_12_5(rN);
    const double psiN = reN - phi_min * powN;
    if (psiN < -psi_slack(reN, phi_min * powN)) {
      nL = tL;  // keep the admissible end; psiL, powL stay valid
    } else {
      psiL = psiN;
      powL = powN;
    }
    if (!(nR >= nL)) nR = nL;
    if (!(nR <= tR)) nR = tR;
    tL = nL;
    tR = nR;
  }
  return tL;
}

}  // namespace idp
