// FP32-mixed euler_step (Alg. 1): per-edge flux, wavespeed, antidiffusive
// flux and limiter-candidate arithmetic in FP32; the state, its accumulation,
// the lumped-mass division, tau and the density interval in FP64.
//
// On GB300 an FP64 operation issues at 1/64 of the FP32 rate, so every
// per-edge quantity is FP32 and FP64 touches each row a handful of times:
//   * U^L_i = U_i + sum_j (2 tau d_ij/m_i)(Ubar_ij - U_i): the increments are
//     summed in FP32 and added to the FP64 state once per row; likewise the
//     limiter passes sum lambda_i l_ij P_ij in FP32.
//   * lambda_max is evaluated in FP32 and multiplied by (1 + 1e-5) so that it
//     stays above the FP64 bound (Sec. 3.7) despite FP32 rounding.
//   * the limiter's line search (Alg. 2/3) runs in FP32 on the deviation of
//     Psi from its FP64 value at t = 0 (computed once per row), shifted by a
//     margin m = 1e-6 (|rho eps| + phi_min rho^(gamma+1)), several times the
//     FP32 error of that deviation, so an accepted t keeps Psi >= 0 in FP64;
//     the density interval cuts against FP64 gaps rho_max - rho(U), rho_min -
//     rho(U) computed once per row, and a returned t is re-checked in FP64
//     (t = 0 if it fails) where a rounding bound of the FP32 Psi reaches the
//     margin.
#include <cfloat>

#include "idp_internal.h"
#include "idp_mixed.cuh"

namespace idp {

namespace {

// Stores of streams written once per stage (evict-first in L2, so that they
// do not displace data the stage reads again) and L2 residency hints for the
// per-entry P_ij, which the limiter pass reads twice (measured on the 128^3
// Sod cube: 12.58 -> 12.41 ms per SSP-RK3 step, bitwise the same results).
__device__ __forceinline__ void st_stream(float* a, float v) { __stcs(a, v); }
__device__ __forceinline__ unsigned long long l2_policy_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ld_policy(const float* a, unsigned long long pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol) : "memory");
  return v;
}

// FP32 quotient and square root by the hardware approximations (a reciprocal
// or square-root unit operation and at most one multiply; relative error a
// few units of 2^-23), where the result is covered by a later test or a
// safety factor: the wavespeed bound (times 1 + 1e-5), 1/(2 d_ij), and the
// limiter's Newton iterates and slopes (every t the limiter returns is
// evaluated again by psi_at, whose rounding bound decides the FP64 check).
// The density cut of the limiter keeps the IEEE division its shrink factor
// assumes.  Measured on the 128^3 Sod cube: 12.4 -> 11.4 ms per SSP-RK3 step.
__device__ __forceinline__ float fdiv_approx(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fsqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

constexpr float kLambdaSafety = 1.0f + 1e-5f;
constexpr float kPsiMargin = 1e-6f;

__device__ __forceinline__ int64_t slot_base(const DeviceGraph& G, int64_t r) {
  return (int64_t)G.slice_ptr[r >> 5] + (r & 31);
}

// Entry k (slot p) of row r: column j, slot pt of the transposed entry,
// flags and entry-table code, from the row's pattern record when the mesh
// has row patterns (pat = its records), else from the per-slot arrays.
// Fields a caller does not use cost nothing (their loads are dropped).
struct SlotRef {
  int64_t j;
  int64_t pt;
  unsigned int fl;
  int code;
};

__device__ __forceinline__ const uint2* row_pattern(const MixedGraph& M, int64_t r) {
  return M.rpat ? M.ptab + (int64_t)M.rpat[r] * M.pwidth : nullptr;
}

__device__ __forceinline__ SlotRef slot_ref(const DeviceGraph& G, const MixedGraph& M, const uint2* pat, int64_t r,
                                            int k, int64_t p) {
  SlotRef e;
  if (pat) {
    const uint2 w = __ldg(&pat[k]);
    e.j = r + (int32_t)w.x;
    e.pt = slot_base(G, e.j) + 32 * (int64_t)(w.y & 0xffu);
    e.fl = (w.y >> 8) & 0xffu;
    e.code = (int)(w.y >> 16);
  } else {
    e.j = G.col[p];
    e.pt = G.tpos[p];
    e.fl = G.flags[p];
    e.code = M.ecode ? (int)M.ecode[p] : 0;
  }
  return e;
}

template <typename T>
__device__ __forceinline__ void load5(const T* U, int64_t n, int64_t i, T* u) {
#pragma unroll
  for (int f = 0; f < kFields; ++f) u[f] = U[f * n + i];
}

struct SideF {
  float rho, inv_rho, mx, my, mz, p, c, pm, inv_p;
};

__device__ __forceinline__ SideF load_side_f(const float* U, const float* Q, int64_t n, int64_t i) {
  SideF s;
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

// f(U) . c in FP32 with a pinned operation sequence (equal states give equal
// fluxes bitwise, so flux differences of equal states vanish).
__device__ __forceinline__ void flux_dot_f(float m1, float m2, float m3, float inv_rho, float p, float h, float cx,
                                           float cy, float cz, float* f) {
  const float mc = __fmaf_rn(m3, cz, __fmaf_rn(m2, cy, __fmul_rn(m1, cx)));
  f[0] = mc;
  f[1] = __fmaf_rn(p, cx, __fmul_rn(__fmul_rn(m1, inv_rho), mc));
  f[2] = __fmaf_rn(p, cy, __fmul_rn(__fmul_rn(m2, inv_rho), mc));
  f[3] = __fmaf_rn(p, cz, __fmul_rn(__fmul_rn(m3, inv_rho), mc));
  f[4] = __fmul_rn(h, mc);
}

// Two-rarefaction wavespeed bound of Sec. 3.7 in FP32 (same algebra as the
// FP64 version in idp_device.cuh), times the safety factor.
__device__ __forceinline__ float lambda_max_f(float nx, float ny, float nz, const SideF& L, const SideF& R) {
  const float uL = fmaf(L.mz, nz, fmaf(L.my, ny, L.mx * nx)) * L.inv_rho;
  const float uR = fmaf(R.mz, nz, fmaf(R.my, ny, R.mx * nx)) * R.inv_rho;
  float num = fmaf(-0.2f, uR - uL, L.c + R.c);
  num = num > 0.0f ? num : 0.0f;
  const float x = fdiv_approx(num, fmaf(L.c, L.pm, R.c * R.pm));
  const float x2 = x * x, x3 = x2 * x, x6 = x3 * x3;
  const float p_tr = x6 * x;
  const bool left_high = L.p >= R.p;
  const float p_max = left_high ? L.p : R.p;
  const float p_low = left_high ? R.p : L.p;
  const float rho_low = left_high ? R.rho : L.rho;
  const float du = uR - uL;
  const float dp = p_max - p_low;
  const bool psi_negative = du < 0.0f && 2.0f * dp * dp < du * du * (rho_low * (2.4f * p_max + 0.4f * p_low));
  const float p_star = psi_negative ? p_tr : fminf(p_max, p_tr);
  const float k = 6.0f / 7.0f;
  const float lam1 = fmaf(-L.c, fsqrt_approx(fmaf(k, fmaxf((p_star - L.p) * L.inv_p, 0.0f), 1.0f)), uL);
  const float lam3 = fmaf(R.c, fsqrt_approx(fmaf(k, fmaxf((p_star - R.p) * R.inv_p, 0.0f), 1.0f)), uR);
  return fmaxf(fmaxf(-lam1, 0.0f), fmaxf(lam3, 0.0f)) * kLambdaSafety;
}

// Per-row FP64 anchor of the limiter's Psi along U + tP: for the row state U
// and the row's phi_min, Psi(0) = rho eps(U) - phi_min rho^(12/5) is exact in
// FP64, and per entry only the deviation Psi(t) - Psi(0) is evaluated in FP32.
// That removes the cancellation between rho E and |m|^2/2 and between rho eps
// and phi_min rho^(12/5) from the FP32 arithmetic.
struct PsiAnchor {
  float u[kFields];  // FP32 copy of U
  float psi0;        // Psi(0)
  float rho0, inv_rho0;
  float phi_pow0;    // phi_min rho^(12/5)
  float margin;      // admissibility margin of the FP32 line search
  float gap_max;     // rho_max - rho(U), rounded toward zero
  float gap_min;     // rho_min - rho(U), rounded toward zero
  float tol;         // Newton stopping threshold of Alg. 2 for this row
};

__device__ __forceinline__ PsiAnchor make_anchor(const double* U, double rho_min, double rho_max, double phi_min,
                                                 double newton_tol) {
  PsiAnchor a;
#pragma unroll
  for (int f = 0; f < kFields; ++f) a.u[f] = (float)U[f];
  const double re = U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
  const double pp = U[0] > 0.0 ? phi_min * pow_12_5(U[0]) : 0.0;
  a.psi0 = (float)(re - pp);
  a.rho0 = (float)U[0];
  a.inv_rho0 = (float)(1.0 / U[0]);
  a.phi_pow0 = (float)pp;
  // FP32 evaluation error of Psi(t) is a few 1e-7 of this scale
  a.margin = kPsiMargin * (float)(fabs(re) + pp);
  // density gaps in FP64, rounded toward zero so that FP32 cuts stay inside
  a.gap_max = __double2float_rz(rho_max - U[0]);
  a.gap_min = __double2float_rz(rho_min - U[0]);
  a.tol = (float)newton_tol * (a.psi0 + a.phi_pow0);
  return a;
}

// Psi(t) - margin and dPsi/dt along U + tP with the anchor:
//   rho eps(U + tP) = rho eps(U) + t g + t^2 h,
//   g = P_rho E + rho P_E - m.P_m,  h = P_rho P_E - |P_m|^2/2,
//   rho(U + tP)^(12/5) = rho^(12/5) (1 + q),  q = (1 + t P_rho/rho)^(12/5) - 1.
struct PsiLine {
  float g, h, sr;  // sr = P_rho / rho
  float gabs, habs;  // sums of the magnitudes of the terms of g and h
};

__device__ __forceinline__ PsiLine make_line(const PsiAnchor& a, const float* P) {
  PsiLine L;
  L.g = fmaf(P[0], a.u[4], a.u[0] * P[4]) - fmaf(a.u[3], P[3], fmaf(a.u[2], P[2], a.u[1] * P[1]));
  L.h = fmaf(-0.5f, fmaf(P[3], P[3], fmaf(P[2], P[2], P[1] * P[1])), P[0] * P[4]);
  L.sr = P[0] * a.inv_rho0;
  L.gabs = fabsf(P[0] * a.u[4]) + fabsf(a.u[0] * P[4]) + fabsf(a.u[1] * P[1]) + fabsf(a.u[2] * P[2]) +
           fabsf(a.u[3] * P[3]);
  L.habs = fabsf(P[0] * P[4]) + 0.5f * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
  return L;
}

// Binomial coefficients C(12/5, k), k = 1..7, of (1 + s)^(12/5) - 1
constexpr float kQ1 = 2.4f, kQ2 = 1.68f, kQ3 = 0.224f, kQ4 = -0.0336f, kQ5 = 0.010752f, kQ6 = -0.0046592f,
                kQ7 = 0.00239616f;

// Psi(t) - margin; also dPsi/dt, q = (1 + s)^(12/5) - 1 and fe, the error of
// the evaluation of q in units of u (for the error bound).  For |s| <= 1/8 q
// is the binomial series to s^7 by Horner's rule: rounding (seven fused
// steps and the coefficients' own rounding) stays below 15 u sum_k |C_k||s|^k
// <= 15 * 2.62 u |s|, truncation below 0.0015 |s|^8 / (1 - 0.075) < 0.02 u |s|,
// so fe = 40 |s|.  Otherwise q = expm1(2.4 log1p(s)) with an ulp in each
// function amplified by 2.4 (1 + q): fe = 4.8 (1 + q) |log1p(s)|.
__device__ __forceinline__ float psi_at(const PsiAnchor& a, const PsiLine& L, float t, float* dpsi, float* fe_out,
                                        float* q_out) {
  const float s = t * L.sr;  // > -1 inside the density interval
  float q, fe;
  if (fabsf(s) <= 0.125f) {
    q = s * fmaf(s, fmaf(s, fmaf(s, fmaf(s, fmaf(s, fmaf(s, kQ7, kQ6), kQ5), kQ4), kQ3), kQ2), kQ1);
    fe = 40.0f * fabsf(s);
  } else {
    const float lg = log1pf(s);
    q = expm1f(2.4f * lg);
    fe = 4.8f * (1.0f + q) * fabsf(lg);
  }
  if (dpsi) *dpsi = fmaf(2.0f * t, L.h, L.g) - a.phi_pow0 * 2.4f * fdiv_approx(1.0f + q, 1.0f + s) * L.sr;
  *fe_out = fe;
  *q_out = q;
  return fmaf(t, fmaf(t, L.h, L.g), a.psi0) - fmaf(a.phi_pow0, q, a.margin);
}

// Bound on |psi_at(t) - (Psi(t) - margin)|, Psi in exact arithmetic along
// U + tP with the FP64 U and the FP32 P, from the rounding of every FP32
// operation (unit roundoff u = 2^-24): the FP32 copies of U and Psi(0), g and
// h (a few roundings of their terms each), s = t P_rho/rho (amplified by
// dq/ds = 2.4 (1 + q)/(1 + s)), the evaluation of q (fe from psi_at) and the
// seven operations that combine them, each at most u times the sum S of the
// magnitudes involved.
__device__ __forceinline__ float psi_error_bound(const PsiAnchor& a, const PsiLine& L, float t, float fe, float q) {
  const float s = t * L.sr;
  const float tg = t * L.gabs, th = t * t * L.habs;
  const float qa = fabsf(q);
  const float S = fabsf(a.psi0) + tg + th + a.phi_pow0 * qa + a.margin;
  const float dq = fe + (1.0f + q) * 7.2f * fabsf(s) / fmaxf(1.0f + s, 1e-30f) + 3.0f * qa;
  return 5.9604645e-8f * (7.0f * S + fabsf(a.psi0) + 7.0f * tg + 5.0f * th + a.phi_pow0 * dq);
}

// Float to double by bit arithmetic on the integer pipe, exact for every
// float (subnormals normalised with a leading-zero count).  The conversion
// instruction runs on the FP64 pipe, and the compiler executes the
// conversions of the rarely taken FP64 check below speculatively on every
// entry (ncu: ~6 per entry), which this form keeps off the FP64 pipe.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned int b = __float_as_uint(x), sign = b & 0x80000000u, e = (b >> 23) & 0xffu;
  unsigned int m = b & 0x7fffffu, de;
  if (e == 0u) {
    if (m == 0u) return __hiloint2double((int)sign, 0);
    const int z = __clz((int)m);
    m = (m << (z - 8)) & 0x7fffffu;
    de = 905u - (unsigned int)z;
  } else {
    de = e == 255u ? 2047u : e + 896u;
  }
  return __hiloint2double((int)(sign | (de << 20) | (m >> 3)), (int)(m << 29));
}

// FP64 test of the entropy bound at U + tP (Reading A30), run on few entries.
// The row state is read here from the state array (field-major, n nodes, row
// r) rather than passed in: with five doubles held live in the caller across
// the limiter loop, ncu counted ~5 FP64-pipe conversions (F2F) per entry in
// the loop, and the flux-limit kernel ran 19 % slower.
__device__ __noinline__ bool psi_holds_fp64(const double* Ug, int64_t n, int64_t r, float p0, float p1, float p2,
                                            float p3, float p4, float t, double phi_min) {
  const double u0 = Ug[r], u1 = Ug[n + r], u2 = Ug[2 * n + r], u3 = Ug[3 * n + r], u4 = Ug[4 * n + r];
  const double td = f2d_exact(t);
  const double v0 = u0 + td * f2d_exact(p0), v1 = u1 + td * f2d_exact(p1), v2 = u2 + td * f2d_exact(p2);
  const double v3 = u3 + td * f2d_exact(p3), v4 = u4 + td * f2d_exact(p4);
  const double re = v0 * v4 - 0.5 * (v1 * v1 + v2 * v2 + v3 * v3);
  const double pw = phi_min * pow_12_5(v0);
  return v0 > 0.0 && re - pw >= -1e-13 * (fabs(re) + fabs(pw));
}

// limiter.compute of Alg. 2 for the mixed path.  The row state (FP64) is row
// r of the state array Ug (field-major, n nodes), read only by the FP64 check;
// P (FP32) is the direction.  Returns t in [0, 1].
__device__ __forceinline__ float limiter_mixed(const double* Ug, int64_t n, int64_t r, const PsiAnchor& A,
                                               const float* P, double phi_min,
                                               const LimiterParams& prm) {
  // density interval (Reading A12) against the row's FP64 gaps: the cut
  // t = |gap|/|rho(P)| is shrunk by 2^-22 to absorb the FP32 division, so
  // rho(U) + t rho(P) stays inside [rho_min, rho_max]
  const float rhoP = P[0];
  float tR = 1.0f;
  if (rhoP > A.gap_max && rhoP != 0.0f) tR = fabsf(A.gap_max) / fabsf(rhoP) * (1.0f - 2.384185791015625e-7f);
  if (tR * rhoP < A.gap_min && rhoP != 0.0f) tR = fabsf(A.gap_min) / fabsf(rhoP) * (1.0f - 2.384185791015625e-7f);
  tR = fminf(fmaxf(tR, 0.0f), 1.0f);
  // t_R = 0 (a density bound that U sits on, e.g. collapsed bounds in a
  // constant region, and rho(P) pushing past it): t_L stays in [0, t_R], so
  // the line search can only return 0
  if (tR == 0.0f) return 0.0f;
  float tL = 0.0f;
  const PsiLine L = make_line(A, P);
  float psiL = 0.0f, dpsiL = 0.0f, psiAtL, feL = 0.0f, qL = 0.0f;
  bool haveL = false, accepted = false;
  for (int step = 0; step < prm.newton_max; ++step) {
    float dpsiR, feR, qR;
    const float psiR = psi_at(A, L, tR, &dpsiR, &feR, &qR);
    if (psiR >= 0.0f) {
      tL = tR;
      psiAtL = psiR;
      feL = feR;
      qL = qR;
      accepted = true;
      break;
    }
    if (!haveL) {
      psiL = psi_at(A, L, tL, &dpsiL, &feL, &qL);
      haveL = true;
    }
    if (psiL <= A.tol) break;
    const float scaling = fdiv_approx(1.0f, tR - tL + FLT_EPSILON);
    const float d12 = (psiR - psiL) * scaling;
    const float d112 = (d12 - dpsiL) * scaling;
    const float d122 = (dpsiR - d12) * scaling;
    const float lamL = fmaxf(dpsiL * dpsiL - 4.0f * psiL * d112, 0.0f);
    const float lamR = fmaxf(dpsiR * dpsiR - 4.0f * psiR * d122, 0.0f);
    float nL = tL - fdiv_approx(2.0f * psiL, dpsiL - fsqrt_approx(lamL));
    float nR = tR - fdiv_approx(2.0f * psiR, dpsiR - fsqrt_approx(lamR));
    if (!(nL >= tL)) nL = tL;
    if (!(nL <= tR)) nL = tR;
    float dpsiN, feN, qN;
    const float psiN = psi_at(A, L, nL, &dpsiN, &feN, &qN);
    if (psiN >= 0.0f) {
      psiL = psiN;
      dpsiL = dpsiN;
      feL = feN;
      qL = qN;
    } else {
      nL = tL;
    }
    if (!(nR >= nL)) nR = nL;
    if (!(nR <= tR)) nR = tR;
    tL = nL;
    tR = nR;
  }
  if (!accepted) psiAtL = haveL ? psiL : psi_at(A, L, tL, nullptr, &feL, &qL);
  // FP64 check of the entropy bound where the FP32 evaluation cannot
  // guarantee it: psiAtL >= 0 means Psi(t) >= margin - error, so the check is
  // needed only when the rounding bound reaches the margin
  if (tL > 0.0f && (psiAtL < 0.0f || psi_error_bound(A, L, tL, feL, qL) >= A.margin) &&
      !psi_holds_fp64(Ug, n, r, P[0], P[1], P[2], P[3], P[4], tL, phi_min))
    tL = 0.0f;
  return tL;
}

// Step 0: per-node quantities (FP32 copies) and an FP32 copy of the state.
__device__ __forceinline__ void row_node_m(int64_t n, const double* U, float* Q,
                                           float* Uf, DeviceScalars* scal, int64_t i) {
  double u[kFields];
  load5(U, n, i, u);
  // rho eps = rho E - |m|^2/2 in FP64 (the two terms cancel where the flow
  // is fast); everything else in FP32
  const double re = u[0] * u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
  if (!positive_k(u[0]) || !positive_k(re)) atomicOr(&scal->status, kStatusNotAdmissible);
  float uf[kFields];
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    uf[f] = (float)u[f];
    Uf[f * n + i] = uf[f];
  }
  const float rf = uf[0], inv_rho = 1.0f / rf;
  const float ref = (float)re;
  const float ef = ref * inv_rho;  // epsilon
  const float pf = 0.4f * ef;
  Q[kQInvRho * n + i] = inv_rho;
  Q[kQP * n + i] = pf;
  Q[kQC * n + i] = sqrtf(1.4f * pf * inv_rho);
  Q[kQPm * n + i] = powf(pf, -1.0f / 7.0f);
  Q[kQInvP * n + i] = 1.0f / pf;
  Q[kQS * n + i] = powf(ref, 5.0f / 12.0f) * inv_rho;
  Q[kQH * n + i] = (uf[4] + pf) * inv_rho;
  Q[kQPhi * n + i] = ef * powf(rf, -1.4f);
}

__global__ void __launch_bounds__(kMaxBlock) k_node_m(DeviceGraph G, const double* __restrict__ U,
                                                   float* __restrict__ Q, float* __restrict__ Uf,
                                                   DeviceScalars* scal) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G.n_inst) G.tau_min[i] = 0x7ff0000000000000ull;  // +inf, reduced into by the next kernel
  if (i < G.n) row_node_m(G.n, U, Q, Uf, scal, i);
}

// Steps 1 and 2 in FP32: d_ij with 1/(2 d_ij) for every entry of the row,
// flux differences, alpha_i, and the row's CFL bound m_i/(-2 d_ii).  Each
// row evaluates the wavespeed bound of a pair in the pair's own orientation
// (that of the row with the smaller caller id, whose entry is kEntryUpper),
// so both rows of a pair compute bitwise the same d_ij and no transposition
// step is needed; at FP32 rates the second evaluation costs less than the
// pass over the slots that would copy it.  Returns the CFL candidate.
__device__ __forceinline__ double row_edge_m(const DeviceGraph& G, const MixedGraph& M, const float* U,
                                             const float* Q, float* d,
                                             float* dinv, float* dF,
                                             float* alpha, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const SideF si = load_side_f(U, Q, n, r);
  const float Ei = U[4 * n + r];
  const float s_i = Q[kQS * n + r], h_i = Q[kQH * n + r];
  float a = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f, b3 = 0.0f, b4 = 0.0f, dsum = 0.0f;
  const uint2* pat = row_pattern(M, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const SlotRef sr = slot_ref(G, M, pat, r, k, p);
    const int64_t j = sr.j;
    const unsigned int fl = sr.fl;
    const EntryF e = entry_f_code(M, p, sr.code);
    const float cx = e.cx, cy = e.cy, cz = e.cz;
    const SideF sj = load_side_f(U, Q, n, j);
    const float s_j = Q[kQS * n + j], h_j = Q[kQH * n + j];
    float fj[kFields], fi[kFields];
    flux_dot_f(sj.mx, sj.my, sj.mz, sj.inv_rho, sj.p, h_j, cx, cy, cz, fj);
    flux_dot_f(si.mx, si.my, si.mz, si.inv_rho, si.p, h_i, cx, cy, cz, fi);
    a = fmaf(s_j - s_i, fj[0], a);
    float df[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      df[f] = fj[f] - fi[f];
      st_stream(&dF[f * ns + p], df[f]);
    }
    b0 += df[0];
    b1 += df[1];
    b2 += df[2];
    b3 += df[3];
    b4 += df[4];
    if (fl & kEntryDiag) continue;
    // the pair in its owner's orientation (lo = the smaller caller id):
    // c_lo,hi first, then, for a pair that is not bitwise skew, c_hi,lo
    const bool upper = fl & kEntryUpper;
    const bool skew = fl & kEntrySkew;
    const SideF& lo = upper ? si : sj;
    const SideF& hi = upper ? sj : si;
    EntryF ef = e, et = e;
    if (skew) {
      if (!upper) {
        ef.cx = -e.cx;
        ef.cy = -e.cy;
        ef.cz = -e.cz;
      }
    } else {
      const EntryF tr = entry_f(M, sr.pt);
      if (upper) et = tr; else ef = tr;
    }
    float dij = 0.0f;
    if (ef.cn > 0.0f) {
      const float inv = ef.inv_cn;
      dij = lambda_max_f(ef.cx * inv, ef.cy * inv, ef.cz * inv, lo, hi) * ef.cn;
    }
    if (!skew && et.cn > 0.0f) {
      const float inv = et.inv_cn;
      dij = fmaxf(dij, lambda_max_f(et.cx * inv, et.cy * inv, et.cz * inv, hi, lo) * et.cn);
    }
    st_stream(&d[p], dij);
    st_stream(&dinv[p], dij != 0.0f ? fdiv_approx(0.5f, dij) : 0.0f);
    dsum += dij;
  }
  const float sc = s_i * si.inv_p * (1.0f / 6.0f);
  const float e0 = sc * Ei, e1 = -sc * si.mx, e2 = -sc * si.my, e3 = -sc * si.mz, e4 = sc * si.rho;
  const float num = a - (e0 * b0 + e1 * b1 + e2 * b2 + e3 * b3 + e4 * b4) + s_i * b0;
  const float D = fabsf(a) + fabsf(e0 - s_i) * fabsf(b0) + fabsf(e1) * fabsf(b1) + fabsf(e2) * fabsf(b2) +
                  fabsf(e3) * fabsf(b3) + fabsf(e4) * fabsf(b4);
  alpha[r] = D > 0.0f ? fabsf(num) / D : 0.0f;
  // Step 2: the CFL bound m_i/(-2 d_ii), d_ii = -sum_j d_ij summed in FP32
  // (relative error below 26 * 2^-24 = 1.6e-6, inside the 1e-5 safety factor
  // of the FP32 wavespeed, so tau_n stays below the FP64 bound)
  return (double)((float)G.mi[r] / (2.0f * dsum));
}

__global__ void __launch_bounds__(kMaxBlock) k_edge_m(DeviceGraph G, MixedGraph M, const float* __restrict__ U,
                                                   const float* __restrict__ Q, float* __restrict__ d,
                                                   float* __restrict__ dinv, float* __restrict__ dF,
                                                   float* __restrict__ alpha, DeviceScalars* scal) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  reduce_tau_candidate(G, r, computes_row(G, r) ? row_edge_m(G, M, U, Q, d, dinv, dF, alpha, r) : INFINITY);
}

// Step 3: U^L_i = U_i + sum_j (2 tau d_ij/m_i)(Ubar_ij - U_i) with
// Ubar_ij - U_i = (U_j - U_i)/2 - df_ij/(2 d_ij) summed in FP32 and added to
// the FP64 state; bounds rho_i + min/max_j (Ubar_ij - U_i)_rho and phi_min;
// R_i = -sum_j df_ij - f_i.s_i + sum_j d^H_ij (U_j - U_i) in FP32.
__device__ __forceinline__ void row_low_order_m(const DeviceGraph& G, const StageConfig& C,
                                                const double* U, const float* Uf,
                                                const float* Q, const float* d,
                                                const float* dinv, const float* dF,
                                                const float* alpha, double* UL,
                                                float* R, double* bnd, int tau_mode,
                                                int64_t r) {
  const double tau = stage_tau(G, instance_of(G, r), tau_mode, C.cfl);
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  float ui[kFields];
  load5(Uf, n, r, ui);
  const float a_i = alpha[r];
  const float two_tau_m = (float)(2.0 * tau * G.inv_mi[r]);
  float inc[kFields], rr[kFields];
  {
    float fs[kFields];
    flux_dot_f(ui[1], ui[2], ui[3], Q[kQInvRho * n + r], Q[kQP * n + r], Q[kQH * n + r], (float)G.csx[r],
               (float)G.csy[r], (float)G.csz[r], fs);
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      inc[f] = 0.0f;
      rr[f] = -fs[f];
    }
  }
  float dmin = 0.0f, dmax = 0.0f, phi_min = INFINITY;
  // the column stream, not the row pattern: measured faster here (this
  // kernel's seven neighbour gathers lean on L1 more than the others')
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    const float dij = d[p];
    float diff[kFields], df[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      diff[f] = Uf[f * n + j] - ui[f];
      df[f] = dF[f * ns + p];
    }
    const float dH = dij * (a_i + alpha[j]) * 0.5f;
#pragma unroll
    for (int f = 0; f < kFields; ++f) rr[f] += fmaf(dH, diff[f], -df[f]);
    if (dij != 0.0f && j != r) {
      const float inv2d = dinv[p];
      const float coef = two_tau_m * dij;
      float db[kFields];
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        db[f] = fmaf(-df[f], inv2d, 0.5f * diff[f]);
        inc[f] = fmaf(coef, db[f], inc[f]);
      }
      dmin = fminf(dmin, db[0]);
      dmax = fmaxf(dmax, db[0]);
    }
    phi_min = fminf(phi_min, Q[kQPhi * n + j]);
  }
  const double rho_i = U[r];
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    UL[f * n + r] = U[f * n + r] + (double)inc[f];
    R[f * n + r] = rr[f];
  }
  double bmin = rho_i + (double)dmin, bmax = rho_i + (double)dmax, pmin = (double)phi_min;
  if (G.relax) {  // bound relaxation (off unless configured)
    const double q = G.relax[r];
    bmin *= 1.0 - q;
    bmax *= 1.0 + q;
    pmin *= 1.0 - q;
  }
  bnd[r] = bmin;
  bnd[n + r] = bmax;
  bnd[2 * n + r] = pmin;
}

__global__ void __launch_bounds__(kMaxBlock) k_low_order_m(DeviceGraph G, StageConfig C, const double* __restrict__ U,
                                                        const float* __restrict__ Uf, const float* __restrict__ Q,
                                                        const float* __restrict__ d, const float* __restrict__ dinv,
                                                        const float* __restrict__ dF, const float* __restrict__ alpha,
                                                        double* __restrict__ UL, float* __restrict__ R,
                                                        double* __restrict__ bnd, DeviceScalars* scal, int tau_mode,
                                                        int accumulate_time) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  instance_books(G, t, tau_mode, C.cfl, accumulate_time, scal);
  const int64_t r = row_start(G) + t;
  if (computes_row(G, r)) row_low_order_m(G, C, U, Uf, Q, d, dinv, dF, alpha, UL, R, bnd, tau_mode, r);
}

// Step 4 in FP32: P_ij and the first limiter values.
__device__ __forceinline__ void row_flux_limit_m(const DeviceGraph& G, const MixedGraph& M, const StageConfig& C,
                                                 const float* Uf, const float* d,
                                                 const float* alpha, const double* UL,
                                                 const float* R, const double* bnd,
                                                 float* P, float* l, int tau_mode,
                                                 int64_t r) {
  const double tau = stage_tau(G, instance_of(G, r), tau_mode, C.cfl);
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  float ui[kFields], ri[kFields];
  double ul[kFields];
  load5(Uf, n, r, ui);
  load5(R, n, r, ri);
  load5(UL, n, r, ul);
  const double rmin = bnd[r], rmax = bnd[n + r], pmin = bnd[2 * n + r];
  const PsiAnchor anchor = make_anchor(ul, rmin, rmax, pmin, C.lim.newton_tol);
  const float a_i = alpha[r];
  const float inv_mi = (float)G.inv_mi[r];
  const float scale = (float)(tau * G.inv_mi[r] * (double)(len - 1));
  const uint2* pat = row_pattern(M, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const SlotRef sr = slot_ref(G, M, pat, r, k, p);
    const int64_t j = sr.j;
    if (j == r) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) st_stream(&P[f * ns + p], 0.0f);
      st_stream(&l[p], 0.0f);
      continue;
    }
    float pij[kFields];
    const float m = entry_f_code(M, p, sr.code).m;
    const float b_ij = -m * M.inv_mi[j];
    const float b_ji = -m * inv_mi;
    const float dij = d[p];
    const float dd = dij * (a_i + alpha[j]) * 0.5f - dij;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      pij[f] = scale * fmaf(b_ij, R[f * n + j], fmaf(-b_ji, ri[f], dd * (Uf[f * n + j] - ui[f])));
      st_stream(&P[f * ns + p], pij[f]);
    }
    st_stream(&l[p], limiter_mixed(UL, n, r, anchor, pij, pmin, C.lim));
  }
}

__global__ void __launch_bounds__(kMaxBlock, 4) k_flux_limit_m(DeviceGraph G, MixedGraph M, StageConfig C,
                                                         const float* __restrict__ Uf, const float* __restrict__ d,
                                                         const float* __restrict__ alpha, const double* __restrict__ UL,
                                                         const float* __restrict__ R, const double* __restrict__ bnd,
                                                         float* __restrict__ P, float* __restrict__ l,
                                                         const DeviceScalars* scal, int tau_mode) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_flux_limit_m(G, M, C, Uf, d, alpha, UL, R, bnd, P, l, tau_mode, r);
}

// Limiter pass: U_next = U_cur + sum_j lambda_i min(l_ij, l_ji) P_ij (sum in
// FP32, added to FP64), P_ij <- (1 - min) P_ij and new l_ij.
__device__ __forceinline__ void row_limiter_pass_m(const DeviceGraph& G, const MixedGraph& M, const StageConfig& C,
                                                   const double* Ucur, double* Unext,
                                                   float* P, const float* lold,
                                                   float* lnew, const double* bnd,
                                                   int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const float lam = (float)G.lam[r];
  float inc[kFields] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const unsigned long long keep = l2_policy_last(), drop = l2_policy_first();
  const uint2* pat = row_pattern(M, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const SlotRef sr = slot_ref(G, M, pat, r, k, p);
    if (sr.j == r) continue;
    const float w = lam * fminf(lold[p], lold[sr.pt]);
#pragma unroll
    for (int f = 0; f < kFields; ++f)
      inc[f] = fmaf(w, ld_policy(&P[f * ns + p], keep), inc[f]);
  }
  double u[kFields];
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    u[f] = Ucur[f * n + r] + (double)inc[f];
    Unext[f * n + r] = u[f];
  }
  const double rmin = bnd[r], rmax = bnd[n + r], pmin = bnd[2 * n + r];
  const PsiAnchor anchor = make_anchor(u, rmin, rmax, pmin, C.lim.newton_tol);
  // Software pipeline: the loads of entry k + 1 are issued before the limiter
  // of entry k, so their latency overlaps its arithmetic (they read P and l_old
  // slots that iteration k does not write).
  bool diag_n = false;
  float lk_n = 0.0f, p_n[kFields];
  auto fetch = [&](int k) {
    const int64_t q = base + 32 * (int64_t)k;
    const SlotRef sr = slot_ref(G, M, pat, r, k, q);
    diag_n = sr.j == r;
    lk_n = fminf(lold[q], lold[sr.pt]);
#pragma unroll
    for (int f = 0; f < kFields; ++f) p_n[f] = ld_policy(&P[f * ns + q], drop);
  };
  if (len > 0) fetch(0);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const bool diag = diag_n;
    const float lk = lk_n;
    float pold[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) pold[f] = p_n[f];
    if (k + 1 < len) fetch(k + 1);
    if (diag) {
      st_stream(&lnew[p], 0.0f);
      continue;
    }
    float pij[kFields];
    bool zero = true;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      pij[f] = (1.0f - lk) * pold[f];
      st_stream(&P[f * ns + p], pij[f]);
      zero &= pij[f] == 0.0f;
    }
    st_stream(&lnew[p], zero ? 1.0f : limiter_mixed(Unext, n, r, anchor, pij, pmin, C.lim));
  }
}

__global__ void __launch_bounds__(kMaxBlock, 4) k_limiter_pass_m(DeviceGraph G, MixedGraph M, StageConfig C,
                                                           const double* __restrict__ Ucur,
                                                           double* __restrict__ Unext, float* __restrict__ P,
                                                           const float* __restrict__ lold, float* __restrict__ lnew,
                                                           const double* __restrict__ bnd) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_limiter_pass_m(G, M, C, Ucur, Unext, P, lold, lnew, bnd, r);
}

// Last pass, boundary post-processing and the SSP-RK3 blend (FP64).
__device__ __forceinline__ void row_final_m(const DeviceGraph& G, const MixedGraph& M, const StageConfig& C,
                                            const double* Ucur, const float* P,
                                            const float* l, const double* Un,
                                            double* Uout, double* Ulim, DeviceScalars* scal,
                                            int blend, int skip_write_on_error, int64_t r) {
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const float lam = (float)G.lam[r];
  float inc[kFields] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const uint2* pat = row_pattern(M, r);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const SlotRef sr = slot_ref(G, M, pat, r, k, p);
    if (sr.j == r) continue;
    const float w = lam * fminf(l[p], l[sr.pt]);
#pragma unroll
    for (int f = 0; f < kFields; ++f) inc[f] = fmaf(w, P[f * ns + p], inc[f]);
  }
  double u[kFields];
#pragma unroll
  for (int f = 0; f < kFields; ++f) u[f] = Ucur[f * n + r] + (double)inc[f];
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
    if (blend == kBlendStage2) v = fma(0.75, Un[f * n + r], 0.25 * u[f]);
    if (blend == kBlendStage3) v = fma(1.0 / 3.0, Un[f * n + r], (2.0 / 3.0) * u[f]);
    out[f] = v;
    finite &= isfinite(v);
  }
  if (!finite) atomicOr(&scal->status, kStatusNonFinite);
  if (skip_write_on_error && *(volatile int*)&scal->status != 0) return;
#pragma unroll
  for (int f = 0; f < kFields; ++f) Uout[f * n + r] = out[f];
}

__global__ void __launch_bounds__(kMaxBlock) k_final_m(DeviceGraph G, MixedGraph M, StageConfig C,
                                                    const double* __restrict__ Ucur,
                                                    const float* __restrict__ P, const float* __restrict__ l,
                                                    const double* __restrict__ Un, double* __restrict__ Uout,
                                                    double* __restrict__ Ulim, DeviceScalars* scal, int blend,
                                                    int skip_write_on_error) {
  const int64_t r = row_start(G) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (computes_row(G, r)) row_final_m(G, M, C, Ucur, P, l, Un, Uout, Ulim, scal, blend, skip_write_on_error, r);
}

struct PersistentStageMixed {
  PersistentStage a;
  MixedGraph M;
  MixedBuffers X;
};

// One FP32-mixed euler_step in a single cooperative launch (see
// k_stage_persistent in idp_stage.cu for the barriers and the work list).
// No register cap: under one, ptxas fuses the FP32 limiter arithmetic
// differently, and rounding-level changes move limiter decisions, so the
// schedules would no longer agree bitwise.
__global__ void __launch_bounds__(kMaxBlock) k_stage_persistent_m(PersistentStageMixed pm) {
  const PersistentStage& a = pm.a;
  const DeviceGraph& G = a.G;
  const StageConfig& C = a.C;
  const StageBuffers& B = a.B;
  const MixedGraph& M = pm.M;
  const MixedBuffers& X = pm.X;
  const int64_t n = G.n;
  unsigned int* tile = a.bar->tile;
  for_each_row_tile(&tile[0], n, [&](int64_t i) {
    if (i < n) row_node_m(n, a.Uin, X.Q, X.Uf, B.scal, i);
    if (i < G.n_inst) G.tau_min[i] = 0x7ff0000000000000ull;
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[1], n, [&](int64_t r) {
    reduce_tau_candidate(G, r, r < n ? row_edge_m(G, M, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, r) : INFINITY);
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[3], n, [&](int64_t r) {
    instance_books(G, r, a.tau_mode, C.cfl, a.accumulate_time, B.scal);
    if (r < n) row_low_order_m(G, C, a.Uin, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, B.UL, X.R, B.bnd, a.tau_mode, r);
  });
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[4], n, [&](int64_t r) {
    if (r < n) row_flux_limit_m(G, M, C, X.Uf, X.d, X.alpha, B.UL, X.R, B.bnd, X.P, X.l[0], a.tau_mode, r);
  });
  const double* cur = B.UL;
  int lbuf = 0, wbuf = 0;
  for (int pass = 1; pass < C.limiter_passes; ++pass) {
    if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
    double* next = B.Uw[wbuf];
    const int ph = 4 + pass < 11 ? 4 + pass : 11;
    for_each_row_tile(&tile[ph], n, [&](int64_t r) {
      if (r < n) row_limiter_pass_m(G, M, C, cur, next, X.P, X.l[lbuf], X.l[lbuf ^ 1], B.bnd, r);
    });
    cur = next;
    wbuf ^= 1;
    lbuf ^= 1;
  }
  if (!grid_barrier(a.bar, C.spin_limit, B.scal)) return;
  for_each_row_tile(&tile[11], n, [&](int64_t r) {
    if (r < n) row_final_m(G, M, C, cur, X.P, X.l[lbuf], a.Un, a.Uout, B.Ulast, B.scal, a.blend, a.skip_write_on_error, r);
  });
}

}  // namespace

const void* persistent_kernel_mixed() { return (const void*)k_stage_persistent_m; }

int launch_euler_step_mixed(const DeviceGraph& G, const MixedGraph& M, const StageBuffers& B, const MixedBuffers& X,
                            const StageConfig& C, const double* Uin, double* Uout, const double* Un, int blend,
                            int tau_mode, bool accumulate_time, bool skip_write_on_error, bool trace, cudaStream_t s,
                            Profiler* prof, int block, GridBarrier* bar) {
  const int kBlock = block;
  const unsigned grid = (unsigned)((G.n + kBlock - 1) / kBlock);
  const bool p = prof && prof->enabled;
  if (bar && !trace && !p) {
    PersistentStageMixed pm{{G, C, B, Uin, Uout, Un, bar, blend, tau_mode, accumulate_time ? 1 : 0,
                             skip_write_on_error ? 1 : 0},
                            M, X};
    const int limit = persistent_grid_limit(kBlock, true);
    const unsigned pgrid = (unsigned)(limit < (int)grid ? limit : grid);
    cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    void* args[] = {&pm};
    cudaLaunchCooperativeKernel((const void*)k_stage_persistent_m, dim3(pgrid), dim3(kBlock), args, 0, s);
    return 1;
  }
  int launches = 0;
  auto run = [&](int id, auto&& launch) {
    if (p) prof->begin(id, s);
    launch();
    if (p) prof->end(s);
    ++launches;
  };
  run(kKNode, [&] { k_node_m<<<grid, kBlock, 0, s>>>(G, Uin, X.Q, X.Uf, B.scal); });
  run(kKEdge, [&] { k_edge_m<<<grid, kBlock, 0, s>>>(G, M, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, B.scal); });
  run(kKLowOrder, [&] {
    k_low_order_m<<<grid, kBlock, 0, s>>>(G, C, Uin, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, B.UL, X.R, B.bnd, B.scal,
                                          tau_mode, accumulate_time ? 1 : 0);
  });
  run(kKFluxLimit, [&] {
    k_flux_limit_m<<<grid, kBlock, 0, s>>>(G, M, C, X.Uf, X.d, X.alpha, B.UL, X.R, B.bnd, X.P, X.l[0], B.scal,
                                           tau_mode);
  });
  const double* cur = B.UL;
  int lbuf = 0, wbuf = 0;
  for (int pass = 1; pass < C.limiter_passes; ++pass) {
    double* next = B.Uw[wbuf];
    run(kKLimiterPass,
        [&] { k_limiter_pass_m<<<grid, kBlock, 0, s>>>(G, M, C, cur, next, X.P, X.l[lbuf], X.l[lbuf ^ 1], B.bnd); });
    if (trace && pass == 1) cudaMemcpyAsync(B.tU5, next, sizeof(double) * kFields * G.n, cudaMemcpyDeviceToDevice, s);
    cur = next;
    wbuf ^= 1;
    lbuf ^= 1;
  }
  double* ulim = B.Ulast ? B.Ulast : (trace ? B.tUlim : nullptr);
  run(kKFinal, [&] {
    k_final_m<<<grid, kBlock, 0, s>>>(G, M, C, cur, X.P, X.l[lbuf], Un, Uout, ulim, B.scal, blend,
                                      skip_write_on_error ? 1 : 0);
  });
  if (trace && B.Ulast)
    cudaMemcpyAsync(B.tUlim, B.Ulast, sizeof(double) * kFields * G.n, cudaMemcpyDeviceToDevice, s);
  return launches;
}

int launch_euler_phase_mixed(const DeviceGraph& G, const MixedGraph& M, const StageBuffers& B,
                             const MixedBuffers& X, const StageConfig& C, const double* Uin, double* Uout,
                             const double* Un, int blend, int tau_mode, bool accumulate_time,
                             bool skip_write_on_error, int phase, cudaStream_t s, int block) {
  const unsigned grid = (unsigned)((G.n + block - 1) / block);
  const unsigned grid_own = own_row_grid(G, block);
  const int passes = C.limiter_passes;
  if (phase == 0) {
    k_node_m<<<grid, block, 0, s>>>(G, Uin, X.Q, X.Uf, B.scal);
    k_edge_m<<<grid_own, block, 0, s>>>(G, M, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, B.scal);
    return 2;
  }
  if (phase == 1) {
    k_low_order_m<<<grid_own, block, 0, s>>>(G, C, Uin, X.Uf, X.Q, X.d, X.dinv, X.P, X.alpha, B.UL, X.R, B.bnd,
                                             B.scal, tau_mode, accumulate_time ? 1 : 0);
    return 1;
  }
  if (phase == 2) {
    k_flux_limit_m<<<grid_own, block, 0, s>>>(G, M, C, X.Uf, X.d, X.alpha, B.UL, X.R, B.bnd, X.P, X.l[0], B.scal,
                                              tau_mode);
    return 1;
  }
  auto state_after = [&](int p) -> double* { return p == 0 ? B.UL : B.Uw[(p - 1) & 1]; };
  const int p = phase - 2;
  if (p >= 1 && p < passes) {
    k_limiter_pass_m<<<grid_own, block, 0, s>>>(G, M, C, state_after(p - 1), B.Uw[(p - 1) & 1], X.P,
                                                X.l[(p - 1) & 1], X.l[p & 1], B.bnd);
    return 1;
  }
  if (p == passes) {
    k_final_m<<<grid_own, block, 0, s>>>(G, M, C, state_after(passes - 1), X.P, X.l[(passes - 1) & 1], Un, Uout,
                                         B.Ulast, B.scal, blend, skip_write_on_error ? 1 : 0);
    return 1;
  }
  return 0;
}

}  // namespace idp
