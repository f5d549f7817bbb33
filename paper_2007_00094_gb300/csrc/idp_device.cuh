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
// error below 3e-7; x enters and w0 leaves FP32 by exponent and mantissa bit
// arithmetic on the integer pipe, the FP64 pipe being the bottleneck) is
// corrected with the second-order series of
// (1 - delta)^(-1/K) = 1 + delta/K + (K+1) delta^2/(2K^2) + O(delta^3), where
// delta = 1 - x w0^K; the neglected term is ~delta^3 < 1e-17 for K <= 12.
// Seed for x outside the normal float range (out of line, so that its
// conversions are not executed speculatively on the common path).
template <int K>
__device__ __noinline__ double inv_root_seed_wide(double x) {
  return (double)powf((float)x, -1.0f / (float)K);
}

template <int K>
__device__ __forceinline__ double inv_root(double x) {
  double w0;
  {
    const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
    const int e = (int)(hi >> 20) - 1023 + 127;
    if (e > 0 && e < 255) {
      const float xf = __uint_as_float(((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
      const unsigned int wb = __float_as_uint(powf(xf, -1.0f / (float)K));
      const unsigned int we = ((wb >> 23) & 0xffu) - 127u + 1023u;
      w0 = __hiloint2double((int)((we << 20) | ((wb & 0x7fffffu) >> 3)), (int)((wb & 7u) << 29));
    } else {
      w0 = inv_root_seed_wide<K>(x);
    }
  }
  const double delta = 1.0 - x * ipow<K>(w0);
  const double c1 = 1.0 / (double)K, c2 = (double)(K + 1) / (2.0 * (double)K * (double)K);
  return fma(w0, fma(c2, delta, c1) * delta, w0);
}

// num / den for den > 0: an FP32 reciprocal seed of den (den enters FP32 and
// the seed leaves it by exponent and mantissa bit arithmetic on the integer
// pipe, as in inv_root), one Newton step w <- w + w (1 - den w) in FP64
// (relative error below 2^-44 from the seed's 2^-22), and one correction of
// the quotient q0 = num w by its residual, q = q0 + (num - den q0) w, which
// leaves q within about half an ulp of num / den: 5 FP64 operations, about
// half of what the IEEE division issues on the FP64 pipe.  den whose
// reciprocal is not a normal float takes the IEEE division (out of line).
static __device__ __noinline__ double div_pos_wide(double num, double den) { return num / den; }

__device__ __forceinline__ double div_pos(double num, double den) {
  const unsigned int hi = (unsigned int)__double2hiint(den), lo = (unsigned int)__double2loint(den);
  const int e = (int)(hi >> 20) - 1023 + 127;
  if (!(e > 0 && e < 253)) return div_pos_wide(num, den);
  const float xf = __uint_as_float(((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  const unsigned int wb = __float_as_uint(rf);
  const unsigned int we = ((wb >> 23) & 0xffu) - 127u + 1023u;
  double w = __hiloint2double((int)((we << 20) | ((wb & 0x7fffffu) >> 3)), (int)((wb & 7u) << 29));
  w = fma(w, fma(-den, w, 1.0), w);
  const double q0 = num * w;
  return fma(fma(-den, q0, num), w, q0);
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
  kQVx = 8,      // velocity m/rho (FP64 stage only)
  kQVy = 9,
  kQVz = 10,
  kNodeQ = 11
};

struct Side {
  double rho, inv_rho, mx, my, mz, p, c, pm, inv_p;
};

// Comparisons of doubles on the integer pipe, from the two 32-bit words of
// each value (the FP64 pipe, which executes FP64 compares and min/max and is
// slow for 64-bit integer operations too, is the bottleneck of the FP64
// stage).  dle(a, b) is a <= b in IEEE order without NaNs: the words of a
// negative value are reflected so that the (signed high, unsigned low) pair
// orders like the value; ties keep the first operand in min_k / max_k.
__device__ __forceinline__ bool dzero(double x) {
  return ((((unsigned int)__double2hiint(x)) << 1) | (unsigned int)__double2loint(x)) == 0u;
}
__device__ __forceinline__ bool dle(double a, double b) {
  int ha = __double2hiint(a), hb = __double2hiint(b);
  unsigned int la = (unsigned int)__double2loint(a), lb = (unsigned int)__double2loint(b);
  const int ma = ha >> 31, mb = hb >> 31;
  ha ^= ma & 0x7fffffff;
  la ^= (unsigned int)ma;
  hb ^= mb & 0x7fffffff;
  lb ^= (unsigned int)mb;
  return ha < hb || (ha == hb && la <= lb);
}
__device__ __forceinline__ double min_k(double a, double b) { return dle(a, b) ? a : b; }
__device__ __forceinline__ double max_k(double a, double b) { return dle(b, a) ? a : b; }
// x > 0 and x < 0 (+0 and -0 are neither)
__device__ __forceinline__ bool positive_k(double x) { return __double2hiint(x) >= 0 && !dzero(x); }
__device__ __forceinline__ bool negative_k(double x) { return __double2hiint(x) < 0 && !dzero(x); }
// exactly 1.0 and exactly +0
__device__ __forceinline__ bool is_one(double x) { return __double2hiint(x) == 0x3ff00000 && __double2loint(x) == 0; }
__device__ __forceinline__ bool is_pos_zero(double x) { return __double2hiint(x) == 0 && __double2loint(x) == 0; }

// f(U) . c of eq. (flux): (m.c, v (m.c) + p c, (E+p)/rho (m.c)), with an
// operation sequence pinned by rounding intrinsics so that equal states give
// bitwise equal fluxes (differences f_j - f_i then vanish exactly, as in the
// oracle).
// m . c with a pinned operation sequence (the f[0] of flux_dot)
__device__ __forceinline__ double m_dot_c(double m1, double m2, double m3, double cx, double cy, double cz) {
  return __fma_rn(m3, cz, __fma_rn(m2, cy, __dmul_rn(m1, cx)));
}

__device__ __forceinline__ void flux_dot(double m1, double m2, double m3, double inv_rho, double p, double h,
                                         double cx, double cy, double cz, double* f) {
  const double mc = m_dot_c(m1, m2, m3, cx, cy, cz);
  f[0] = mc;
  f[1] = __fma_rn(p, cx, __dmul_rn(__dmul_rn(m1, inv_rho), mc));
  f[2] = __fma_rn(p, cy, __dmul_rn(__dmul_rn(m2, inv_rho), mc));
  f[3] = __fma_rn(p, cz, __dmul_rn(__dmul_rn(m3, inv_rho), mc));
  f[4] = __dmul_rn(h, mc);
}


// flux_dot with the velocity v = m/rho given (rounded as __dmul_rn(m, 1/rho),
// so that the result is bitwise that of flux_dot)
__device__ __forceinline__ void flux_dot_v(double m1, double m2, double m3, double v1, double v2, double v3, double p,
                                           double h, double cx, double cy, double cz, double* f) {
  const double mc = m_dot_c(m1, m2, m3, cx, cy, cz);
  f[0] = mc;
  f[1] = __fma_rn(p, cx, __dmul_rn(v1, mc));
  f[2] = __fma_rn(p, cy, __dmul_rn(v2, mc));
  f[3] = __fma_rn(p, cz, __dmul_rn(v3, mc));
  f[4] = __dmul_rn(h, mc);
}

// lambda~_max(n, U_L, U_R) of Sec. 3.7.  For gamma = 7/5 the two-rarefaction
// pressure is p~* = ((c_L + c_R - (u_R - u_L)/5) / (c_L p_L^(-1/7) +
// c_R p_R^(-1/7)))^7 (the printed form divided through by p_R^(1/7)); the
// projection leaves the pressure unchanged (E~ - m~^2/(2 rho) = epsilon).
// psi is needed at p_max, where only the side with the smaller pressure
// contributes (its shock branch); the other side's f vanishes.
// lambda_max_u takes the normal velocities u_L = m_L.n / rho_L, u_R directly.
__device__ __forceinline__ double lambda_max_u(double uL, double uR, const Side& L, const Side& R) {
  double num = L.c + R.c - 0.2 * (uR - uL);
  num = positive_k(num) ? num : 0.0;  // vacuum: p~* = 0
  const double x = div_pos(num, L.c * L.pm + R.c * R.pm);
  const double x2 = x * x, x3 = x2 * x, x6 = x3 * x3;
  const double p_tr = x6 * x;
  const bool left_high = dle(R.p, L.p);
  const double p_max = left_high ? L.p : R.p;
  const double p_low = left_high ? R.p : L.p;
  const double rho_low = left_high ? R.rho : L.rho;
  // psi(p_max) = A/B + du with A = sqrt(2)(p_max - p_low) >= 0 and
  // B = sqrt(rho_low (2.4 p_max + 0.4 p_low)) > 0, so psi < 0 exactly when
  // du < 0 and A^2 < du^2 B^2: the same decision without a square root or a
  // division
  const double du = uR - uL;
  const double dp = p_max - p_low;
  const bool psi_negative = negative_k(du) && 2.0 * dp * dp < du * du * (rho_low * (2.4 * p_max + 0.4 * p_low));
  const double p_star = psi_negative ? p_tr : min_k(p_max, p_tr);
  const double k = 6.0 / 7.0;  // (gamma+1)/(2 gamma)
  // sqrt(1 + k [z]_+) is exactly 1 where z <= 0 (no shock on that side)
  const double zL = (p_star - L.p) * L.inv_p, zR = (p_star - R.p) * R.inv_p;
  const double lam1 = uL - L.c * (positive_k(zL) ? sqrt(1.0 + k * zL) : 1.0);
  const double lam3 = uR + R.c * (positive_k(zR) ? sqrt(1.0 + k * zR) : 1.0);
  const double a = negative_k(-lam1) ? 0.0 : -lam1, b = negative_k(lam3) ? 0.0 : lam3;
  return max_k(a, b);
}

__device__ __forceinline__ double lambda_max(double nx, double ny, double nz, const Side& L, const Side& R) {
  const double uL = (L.mx * nx + L.my * ny + L.mz * nz) * L.inv_rho;
  const double uR = (R.mx * nx + R.my * ny + R.mz * nz) * R.inv_rho;
  return lambda_max_u(uL, uR, L, R);
}

// u = m.n / rho with n = c/|c| from m.c (as m_dot_c gives it), 1/rho and
// 1/|c|: the normal velocities of lambda_max_u for the orientation c_ij,
// reusing the m.c of the flux contractions
__device__ __forceinline__ double normal_speed(double mc, double inv_rho, double inv_cn) {
  return __dmul_rn(__dmul_rn(mc, inv_rho), inv_cn);
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
// (|x| by clearing the sign bit, on the integer pipe)
__device__ __forceinline__ double dabs_k(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ double psi_slack(double rho_eps, double phi_term) {
  return 1e-13 * (dabs_k(rho_eps) + dabs_k(phi_term));
}

// Double to float rounded toward zero by bit arithmetic (integer pipe): the
// sign, the exponent rebiased and the top 23 mantissa bits; relative error
// below 2^-23.  Zero maps to zero.  A double outside the normal float range
// maps to NaN, which fails every test of the FP32 pre-check below, so such
// inputs take the FP64 path (no conversion instruction, whose FP64-pipe cost
// the compiler would otherwise pay speculatively on every call).
__device__ __forceinline__ float to_float_rz(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e > 0 && e < 255)
    return __uint_as_float((hi & 0x80000000u) | ((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  return ((hi << 1) | lo) == 0u ? 0.0f : __uint_as_float(0x7fc00000u);
}

// FP32 pre-check of the FP64 limiter's acceptance test.  Per row, Psi(0) =
// rho eps(U) - phi_min rho^(gamma+1) and phi_min rho^(gamma+1) come from FP64;
// per entry Psi(t) = Psi(0) + t (g + t h) - phi_min rho^(gamma+1) q along
// U + tP (g, h the coefficients of rho eps(U + tP), q = (1 + t P_rho/rho)^2.4
// - 1) is evaluated in FP32 with a bound on its error: the roundings of the
// FP32 copies of U, P, t and of the anchor (u = 2^-24, 2^-23 for the copies
// rounded toward zero), of g, h and s (a few per term), of log1p/expm1 (an
// ulp each, amplified by 2.4 (1 + q)) and of the combining operations, plus
// 1e-15 (|rho E| + |m|^2/2 + phi_min rho^(gamma+1)) at t and at 0 for the
// FP64 evaluations.  The FP64 test accepts when its Psi(t) >= -1e-13 (|rho
// eps| + phi_min rho^(gamma+1)); the pre-check answers "accepts" only when
// that holds for every value within the bounds (0.9 of the slack), so a
// limiter that takes its answer returns exactly what the FP64 test returns.
struct PsiCheck32 {
  float u[5];    // U in FP32
  float psi0;    // Psi(0), rounded from FP64
  float pp;      // phi_min rho^(gamma+1), rounded from FP64
  float inv_rho; // 1/rho in FP32
  float k0;      // |rho E| + |m|^2/2 + pp in FP32
};

__device__ __forceinline__ PsiCheck32 make_psi_check(const double* U, double phi_min) {
  PsiCheck32 a;
#pragma unroll
  for (int f = 0; f < 5; ++f) a.u[f] = to_float_rz(U[f]);
  const double re = U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
  const double pp = U[0] > 0.0 ? phi_min * pow_12_5(U[0]) : 0.0;
  a.psi0 = to_float_rz(re - pp);
  a.pp = to_float_rz(pp);
  a.inv_rho = 1.0f / a.u[0];
  a.k0 = fabsf(a.u[0] * a.u[4]) + 0.5f * (a.u[1] * a.u[1] + a.u[2] * a.u[2] + a.u[3] * a.u[3]) + a.pp;
  return a;
}

__device__ __forceinline__ bool psi_accepts_fp32(const PsiCheck32& a, const double* P, double t) {
  float p[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) p[f] = to_float_rz(P[f]);
  const float tf = to_float_rz(t);
  const float s = tf * p[0] * a.inv_rho;
  if (!(s > -0.5f) || !(a.u[0] > 0.0f)) return false;  // leave strong expansions to FP64
  const float g = p[0] * a.u[4] + a.u[0] * p[4] - (a.u[1] * p[1] + a.u[2] * p[2] + a.u[3] * p[3]);
  const float gabs = fabsf(p[0] * a.u[4]) + fabsf(a.u[0] * p[4]) + fabsf(a.u[1] * p[1]) + fabsf(a.u[2] * p[2]) +
                     fabsf(a.u[3] * p[3]);
  const float h = p[0] * p[4] - 0.5f * (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const float habs = fabsf(p[0] * p[4]) + 0.5f * (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const float lg = log1pf(s);
  const float q = expm1f(2.4f * lg);
  const float qa = fabsf(q);
  const float qe = (1.0f + q) * (7.2f * fabsf(lg) + 24.0f * fabsf(s) / (1.0f + s)) + 3.0f * qa;
  const float tg = tf * gabs, th = tf * tf * habs;
  const float psi = a.psi0 + tf * (g + tf * h) - a.pp * q;
  const float err = 5.9604645e-8f * (8.0f * fabsf(a.psi0) + 18.0f * (tg + th) + a.pp * (8.0f * qa + qe));
  const float re_t = a.psi0 + a.pp + tf * (g + tf * h);
  const float r = a.u[0] + tf * p[0], E = a.u[4] + tf * p[4];
  const float m1 = a.u[1] + tf * p[1], m2 = a.u[2] + tf * p[2], m3 = a.u[3] + tf * p[3];
  const float ppt = a.pp * (1.0f + q);
  const float kt = fabsf(r * E) + 0.5f * (m1 * m1 + m2 * m2 + m3 * m3) + ppt;
  return psi - err >= 1e-15f * (kt + a.k0) - 0.9e-13f * (fabsf(re_t) + ppt);
}

// limiter.compute(U, P, bounds) of Alg. 2: density interval, then the
// quadratic Newton iteration of Alg. 3 (sign -1) on
// Psi(t) = rho eps(U + tP) - phi_min rho(U + tP)^(gamma+1), with the
// safeguards: non-negative discriminants, t_L kept admissible, bracket
// ordered; Psi >= -psi_slack counts as admissible (for t_R and the new
// t_L alike).  Returns t_L.
// With pre (the row's PsiCheck32), an FP32 evaluation settles the first
// acceptance test where it can (see psi_accepts_fp32); the result is the
// same.
__device__ __forceinline__ double limiter(const double* U, const double* P, double rho_min, double rho_max,
                                          double phi_min, const LimiterParams& prm,
                                          const PsiCheck32* pre = nullptr) {
  double tL = 0.0, tR = 1.0;
  const double rhoU = U[0], rhoP = P[0];
  if (!dzero(rhoP)) {  // rho(P) != 0
    bool cut = false;
    if (!dle(rhoU + tR * rhoP, rho_max)) {
      tR = fabs(rho_max - rhoU) / fabs(rhoP);
      cut = true;
    }
    if (!dle(rho_min, rhoU + tR * rhoP)) {
      tR = fabs(rho_min - rhoU) / fabs(rhoP);
      cut = true;
    }
    if (cut) tR = fmin(fmax(tR, 0.0), 1.0);  // t_R = 1 needs no clamp
  }
  if (pre && prm.newton_max > 0 && psi_accepts_fp32(*pre, P, tR)) return tR;
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
