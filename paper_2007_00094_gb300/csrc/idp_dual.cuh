// Forward-mode dual numbers and the stage's per-entry functions written for
// a generic scalar type, for the local Jacobians of the adjoint.
//
// Dual<N> carries a value and N directional derivatives.  Every function
// below mirrors its FP64 counterpart in idp_device.cuh / idp_stage.cu
// operation by operation; branches (min, max, clamps, the limiter's exits)
// are decided on values, so the derivatives are those of the branch the
// forward pass takes.
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

// f(U) . c of eq. (flux)
template <typename T>
__device__ __forceinline__ void flux_dot_t(const T* u, double cx, double cy, double cz, T* f) {
  const T inv_rho = 1.0 / u[0];
  const T eps = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * inv_rho;
  const T p = 0.4 * eps;
  const T h = (u[4] + p) * inv_rho;
  const T mc = u[1] * cx + u[2] * cy + u[3] * cz;
  f[0] = mc;
  f[1] = u[1] * inv_rho * mc + p * cx;
  f[2] = u[2] * inv_rho * mc + p * cy;
  f[3] = u[3] * inv_rho * mc + p * cz;
  f[4] = h * mc;
}

// two-rarefaction bound of Sec. 3.7 (mirror of lambda_max)
template <typename T>
__device__ __forceinline__ T lambda_max_t(double nx, double ny, double nz, const SideT<T>& L, const SideT<T>& R) {
  const T uL = (L.mx * nx + L.my * ny + L.mz * nz) * L.inv_rho;
  const T uR = (R.mx * nx + R.my * ny + R.mz * nz) * R.inv_rho;
  T num = L.c + R.c - 0.2 * (uR - uL);
  if (val(num) < 0.0) num = num * 0.0;
  const T x = num / (L.c * L.pm + R.c * R.pm);
  const T x2 = x * x, x3 = x2 * x, x6 = x3 * x3;
  const T p_tr = x6 * x;
  const bool left_high = val(L.p) >= val(R.p);
  const T p_max = left_high ? L.p : R.p;
  const T p_low = left_high ? R.p : L.p;
  const T rho_low = left_high ? R.rho : L.rho;
  const double du = val(uR) - val(uL);
  const double dp = val(p_max) - val(p_low);
  const bool psi_negative =
      du < 0.0 && 2.0 * dp * dp < du * du * (val(rho_low) * (2.4 * val(p_max) + 0.4 * val(p_low)));
  const T p_star = psi_negative ? p_tr : fmin(p_max, p_tr);
  const double k = 6.0 / 7.0;
  const T lam1 = uL - L.c * sqrt(1.0 + k * fmax((p_star - L.p) * L.inv_p, 0.0));
  const T lam3 = uR + R.c * sqrt(1.0 + k * fmax((p_star - R.p) * R.inv_p, 0.0));
  return fmax(fmax(-lam1, 0.0), fmax(lam3, 0.0));
}

template <typename T>
__device__ __forceinline__ T rho_eps_at_t(const T* U, const T* P, const T& t, T* rho_out) {
  const T r = U[0] + t * P[0];
  const T m1 = U[1] + t * P[1], m2 = U[2] + t * P[2], m3 = U[3] + t * P[3];
  const T E = U[4] + t * P[4];
  *rho_out = r;
  return r * E - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3);
}

template <typename T>
__device__ __forceinline__ T drho_eps_at_t(const T* U, const T* P, const T& t) {
  const T r = U[0] + t * P[0];
  const T m1 = U[1] + t * P[1], m2 = U[2] + t * P[2], m3 = U[3] + t * P[3];
  const T E = U[4] + t * P[4];
  return P[0] * E + r * P[4] - (m1 * P[1] + m2 * P[2] + m3 * P[3]);
}

template <typename T>
__device__ __forceinline__ double psi_slack_t(const T& rho_eps, const T& phi_term) {
  return 1e-13 * (::fabs(val(rho_eps)) + ::fabs(val(phi_term)));
}

// limiter.compute of Alg. 2 / Alg. 3 (mirror of limiter in idp_device.cuh)
template <typename T>
__device__ __forceinline__ T limiter_t(const T* U, const T* P, const T& rho_min, const T& rho_max, const T& phi_min,
                                       const LimiterParams& prm) {
  T tL = U[0] * 0.0, tR = tL + 1.0;
  const T rhoU = U[0], rhoP = P[0];
  if (val(rhoU) + val(tR) * val(rhoP) > val(rho_max) && val(rhoP) != 0.0) tR = fabs(rho_max - rhoU) / fabs(rhoP);
  if (val(rhoU) + val(tR) * val(rhoP) < val(rho_min) && val(rhoP) != 0.0) tR = fabs(rho_min - rhoU) / fabs(rhoP);
  if (val(tR) < 0.0) tR = tR * 0.0;
  if (val(tR) > 1.0) tR = tR * 0.0 + 1.0;
  T psiL = tL, powL = tL;
  bool haveL = false;
  for (int step = 0; step < prm.newton_max; ++step) {
    T rR;
    const T reR = rho_eps_at_t(U, P, tR, &rR);
    const T powR = pow_12_5_t(rR);
    const T psiR = reR - phi_min * powR;
    if (val(psiR) >= -psi_slack_t(reR, phi_min * powR)) {
      tL = tR;
      break;
    }
    if (!haveL) {
      T rL;
      const T reL = rho_eps_at_t(U, P, tL, &rL);
      powL = pow_12_5_t(rL);
      psiL = reL - phi_min * powL;
      haveL = true;
    }
    const double tol =
        prm.newton_tol * (val(U[0]) * val(U[4]) - 0.5 * (val(U[1]) * val(U[1]) + val(U[2]) * val(U[2]) + val(U[3]) * val(U[3])));
    if (val(psiL) <= tol) break;
    const T rhoL = U[0] + tL * P[0];
    const T dpsiL = drho_eps_at_t(U, P, tL) - phi_min * 2.4 * (powL / rhoL) * P[0];
    const T dpsiR = drho_eps_at_t(U, P, tR) - phi_min * 2.4 * (powR / rR) * P[0];
    const T scaling = 1.0 / (tR - tL + prm.newton_eps);
    const T d12 = (psiR - psiL) * scaling;
    const T d112 = (d12 - dpsiL) * scaling;
    const T d122 = (dpsiR - d12) * scaling;
    T lamL = dpsiL * dpsiL - 4.0 * psiL * d112;
    T lamR = dpsiR * dpsiR - 4.0 * psiR * d122;
    if (val(lamL) < 0.0) lamL = lamL * 0.0;
    if (val(lamR) < 0.0) lamR = lamR * 0.0;
    T nL = tL - 2.0 * psiL / (dpsiL - sqrt(lamL));
    T nR = tR - 2.0 * psiR / (dpsiR - sqrt(lamR));
    if (!(val(nL) >= val(tL))) nL = tL;
    if (!(val(nL) <= val(tR))) nL = tR;
    T rN;
    const T reN = rho_eps_at_t(U, P, nL, &rN);
    const T powN = pow_12_5_t(rN);
    const T psiN = reN - phi_min * powN;
    if (val(psiN) < -psi_slack_t(reN, phi_min * powN)) {
      nL = tL;
    } else {
      psiL = psiN;
      powL = powN;
    }
    if (!(val(nR) >= val(nL))) nR = nL;
    if (!(val(nR) <= val(tR))) nR = tR;
    tL = nL;
    tR = nR;
  }
  return tL;
}

}  // namespace idp
