// Forward-mode dual numbers for the local derivatives of the adjoint: the
// per-node quantities of Step 0 and the limiter (Alg. 2 / Alg. 3).
//
// Dual<N> carries a value and N directional derivatives.  The functions
// below mirror their FP64 counterparts in idp_device.cuh / idp_stage.cu
// operation by operation; branches (clamps, the limiter's exits) are decided
// on values, so the derivatives are those of the branch the forward pass
// takes.
#pragma once
#include "idp_device.cuh"

namespace idp {

template <int N>
struct Dual {
  double v;
  double d[N];
};

__device__ __forceinline__ double val(double x) { return x; }
template <int N>
__device__ __forceinline__ double val(const Dual<N>& x) {
  return x.v;
}

template <int N>
__device__ __forceinline__ Dual<N> dconst(double x) {
  Dual<N> r;
  r.v = x;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = 0.0;
  return r;
}

// x seeded with direction k (derivative 1 in slot k)
template <int N>
__device__ __forceinline__ Dual<N> dseed(double x, int k) {
  Dual<N> r = dconst<N>(x);
  if (k >= 0 && k < N) r.d[k] = 1.0;
  return r;
}

#define IDP_DUAL_BIN(op, vexpr, dexpr)                                                         \
  template <int N>                                                                             \
  __device__ __forceinline__ Dual<N> operator op(const Dual<N>& a, const Dual<N>& b) {         \
    Dual<N> r;                                                                                 \
    r.v = vexpr;                                                                               \
    _Pragma("unroll") for (int q = 0; q < N; ++q) r.d[q] = dexpr;                              \
    return r;                                                                                  \
  }
IDP_DUAL_BIN(+, a.v + b.v, a.d[q] + b.d[q])
IDP_DUAL_BIN(-, a.v - b.v, a.d[q] - b.d[q])
IDP_DUAL_BIN(*, a.v * b.v, a.d[q] * b.v + a.v * b.d[q])
#undef IDP_DUAL_BIN

template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = (a.d[q] - r.v * b.d[q]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = -a.d[q];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v = a.v + b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(double b, const Dual<N>& a) {
  return a + b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v = a.v - b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(double b, const Dual<N>& a) {
  Dual<N> r;
  r.v = b - a.v;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = -a.d[q];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = a.d[q] * b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double b, const Dual<N>& a) {
  return a * b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) {
  return a * (1.0 / b);
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) {
  return dconst<N>(a) / b;
}

// chain rule for a scalar function with value fv and derivative fd at x
template <int N>
__device__ __forceinline__ Dual<N> dchain(const Dual<N>& x, double fv, double fd) {
  Dual<N> r;
  r.v = fv;
#pragma unroll
  for (int q = 0; q < N; ++q) r.d[q] = fd * x.d[q];
  return r;
}

// the double overloads stay visible next to the Dual ones below
using ::fabs;
using ::fmax;
using ::fmin;
using ::sqrt;

template <int N>
__device__ __forceinline__ Dual<N> sqrt(const Dual<N>& x) {
  const double s = ::sqrt(x.v);
  return dchain(x, s, s > 0.0 ? 0.5 / s : 0.0);
}
template <int N>
__device__ __forceinline__ Dual<N> fabs(const Dual<N>& x) {
  return x.v < 0.0 ? -x : x;
}
template <int N>
__device__ __forceinline__ Dual<N> fmax(const Dual<N>& a, const Dual<N>& b) {
  return a.v >= b.v ? a : b;
}
template <int N>
__device__ __forceinline__ Dual<N> fmin(const Dual<N>& a, const Dual<N>& b) {
  return a.v <= b.v ? a : b;
}
template <int N>
__device__ __forceinline__ Dual<N> fmax(const Dual<N>& a, double b) {
  return a.v >= b ? a : dconst<N>(b);
}
template <int N>
__device__ __forceinline__ Dual<N> fmin(const Dual<N>& a, double b) {
  return a.v <= b ? a : dconst<N>(b);
}

// x^(-1/K) and rho^(12/5) with the forward's values and exact derivatives
template <int K>
__device__ __forceinline__ double inv_root_t(double x) {
  return inv_root<K>(x);
}
template <int K, int N>
__device__ __forceinline__ Dual<N> inv_root_t(const Dual<N>& x) {
  const double w = inv_root<K>(x.v);
  return dchain(x, w, -w / ((double)K * x.v));
}
__device__ __forceinline__ double pow_12_5_t(double x) { return pow_12_5(x); }
template <int N>
__device__ __forceinline__ Dual<N> pow_12_5_t(const Dual<N>& x) {
  const double v = pow_12_5(x.v);
  return dchain(x, v, 2.4 * v / x.v);
}

// ---------------------------------------------------------------------------
// Stage functions for a generic scalar (double or Dual<N>)
// ---------------------------------------------------------------------------

template <typename T>
struct SideT {
  T rho, inv_rho, mx, my, mz, p, c, pm, inv_p;
};

// per-node quantities of Step 0 as functions of the conserved state
template <typename T>
__device__ __forceinline__ SideT<T> side_of_state(const T* u) {
  SideT<T> s;
  s.rho = u[0];
  s.mx = u[1];
  s.my = u[2];
  s.mz = u[3];
  s.inv_rho = 1.0 / u[0];
  const T eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * s.inv_rho;
  s.p = 0.4 * eps;
  s.c = sqrt(1.4 * s.p * s.inv_rho);
  s.pm = inv_root_t<7>(s.p);
  s.inv_p = 1.0 / s.p;
  return s;
}

// eta/rho with eta = (rho eps)^(5/12), and phi = eps rho^(-7/5)
template <typename T>
__device__ __forceinline__ T entropy_s(const T* u) {
  const T inv_rho = 1.0 / u[0];
  const T eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * inv_rho;
  const T rho_eps = u[0] * eps;
  const T w12 = inv_root_t<12>(rho_eps);
  T w7 = w12 * w12 * w12;
  w7 = w7 * w7 * w12;
  return rho_eps * w7 * inv_rho;
}
template <typename T>
__device__ __forceinline__ T entropy_phi(const T* u) {
  const T inv_rho = 1.0 / u[0];
  const T eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * inv_rho;
  const T w5 = inv_root_t<5>(u[0]);
  T r7 = w5 * w5 * w5;
  r7 = r7 * r7 * w5;
  return eps * r7;
}

// ---------------------------------------------------------------------------
// The limiter as a function of its line scalars
// ---------------------------------------------------------------------------

// limiter(U, P, bounds) depends on U and P only through rho(t) = U0 + t P0
// and the quadratic rho eps(t) = a0 + a1 t + a2 t^2 along U + t P, with
// a0 = rho eps(U), a1 = U0 P4 + P0 U4 - m_U.m_P, a2 = P0 P4 - |m_P|^2/2.
// LimiterLine carries these five scalars as duals (plus U and P in FP64):
// values, and with them every branch, are evaluated exactly as in the FP64
// limiter, derivatives through the line scalars.
template <int N>
struct LimiterLine {
  const double* U;
  const double* P;
  Dual<N> U0, P0, a0, a1, a2;
};

template <int N>
__device__ __forceinline__ Dual<N> line_rho_eps(const LimiterLine<N>& L, const Dual<N>& t, Dual<N>* rho) {
  double r;
  Dual<N> out;
  out.v = rho_eps_at(L.U, L.P, t.v, &r);
  rho->v = r;
  const double slope = L.a1.v + 2.0 * L.a2.v * t.v;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    rho->d[q] = L.U0.d[q] + t.v * L.P0.d[q] + L.P0.v * t.d[q];
    out.d[q] = L.a0.d[q] + t.v * (L.a1.d[q] + t.v * L.a2.d[q]) + slope * t.d[q];
  }
  return out;
}

template <int N>
__device__ __forceinline__ Dual<N> line_drho_eps(const LimiterLine<N>& L, const Dual<N>& t) {
  Dual<N> out;
  out.v = drho_eps_at(L.U, L.P, t.v);
#pragma unroll
  for (int q = 0; q < N; ++q) out.d[q] = L.a1.d[q] + 2.0 * (t.v * L.a2.d[q] + L.a2.v * t.d[q]);
  return out;
}

// Mirror of limiter() in idp_device.cuh (Alg. 2 / Alg. 3 with the same
// safeguards, margins and exits), returning t_L as a dual.
template <int N>
__device__ __forceinline__ Dual<N> limiter_line(const LimiterLine<N>& L, const Dual<N>& rho_min,
                                                const Dual<N>& rho_max, const Dual<N>& phi_min,
                                                const LimiterParams& prm) {
  Dual<N> tL = dconst<N>(0.0), tR = dconst<N>(1.0);
  const Dual<N>&rhoU = L.U0, &rhoP = L.P0;
  if (rhoU.v + tR.v * rhoP.v > rho_max.v && rhoP.v != 0.0) tR = fabs(rho_max - rhoU) / fabs(rhoP);
  if (rhoU.v + tR.v * rhoP.v < rho_min.v && rhoP.v != 0.0) tR = fabs(rho_min - rhoU) / fabs(rhoP);
  if (tR.v < 0.0) tR = dconst<N>(0.0);
  if (tR.v > 1.0) tR = dconst<N>(1.0);
  Dual<N> psiL = tL, powL = tL;
  bool haveL = false;
  for (int step = 0; step < prm.newton_max; ++step) {
    Dual<N> rR;
    const Dual<N> reR = line_rho_eps(L, tR, &rR);
    const Dual<N> powR = pow_12_5_t(rR);
    const Dual<N> psiR = reR - phi_min * powR;
    if (psiR.v >= -psi_slack(reR.v, phi_min.v * powR.v)) {
      tL = tR;
      break;
    }
    if (!haveL) {
      Dual<N> rL;
      const Dual<N> reL = line_rho_eps(L, tL, &rL);
      powL = pow_12_5_t(rL);
      psiL = reL - phi_min * powL;
      haveL = true;
    }
    const double tol =
        prm.newton_tol * (L.U[0] * L.U[4] - 0.5 * (L.U[1] * L.U[1] + L.U[2] * L.U[2] + L.U[3] * L.U[3]));
    if (psiL.v <= tol) break;
    const Dual<N> rhoL = rhoU + tL * rhoP;
    const Dual<N> dpsiL = line_drho_eps(L, tL) - phi_min * 2.4 * (powL / rhoL) * rhoP;
    const Dual<N> dpsiR = line_drho_eps(L, tR) - phi_min * 2.4 * (powR / rR) * rhoP;
    const Dual<N> scaling = 1.0 / (tR - tL + prm.newton_eps);
    const Dual<N> d12 = (psiR - psiL) * scaling;
    const Dual<N> d112 = (d12 - dpsiL) * scaling;
    const Dual<N> d122 = (dpsiR - d12) * scaling;
    Dual<N> lamL = dpsiL * dpsiL - 4.0 * psiL * d112;
    Dual<N> lamR = dpsiR * dpsiR - 4.0 * psiR * d122;
    if (lamL.v < 0.0) lamL = dconst<N>(0.0);
    if (lamR.v < 0.0) lamR = dconst<N>(0.0);
    Dual<N> nL = tL - 2.0 * psiL / (dpsiL - sqrt(lamL));
    Dual<N> nR = tR - 2.0 * psiR / (dpsiR - sqrt(lamR));
    if (!(nL.v >= tL.v)) nL = tL;
    if (!(nL.v <= tR.v)) nL = tR;
    Dual<N> rN;
    const Dual<N> reN = line_rho_eps(L, nL, &rN);
    const Dual<N> powN = pow_12_5_t(rN);
    const Dual<N> psiN = reN - phi_min * powN;
    if (psiN.v < -psi_slack(reN.v, phi_min.v * powN.v)) {
      nL = tL;
    } else {
      psiL = psiN;
      powL = powN;
    }
    if (!(nR.v >= nL.v)) nR = nL;
    if (!(nR.v <= tR.v)) nR = tR;
    tL = nL;
    tR = nR;
  }
  return tL;
}

}  // namespace idp
