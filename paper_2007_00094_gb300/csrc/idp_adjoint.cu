// Discrete adjoint (reverse mode) of one FP64 euler_step (Alg. 1): given the
// adjoint of the stage output, the adjoint of the stage input.
//
// The reverse kernels run the forward sweeps backwards (Step 6 -> Step 0)
// over the intermediates of a traced forward evaluation of the stage.
// Non-smooth points take the branch the forward pass took: min(l_ij, l_ji)
// routes to the smaller value (own entry on ties), each bound to the first
// entry attaining it, tau_n to the first row attaining the CFL minimum, the
// limiter and the wavespeed bound to their evaluated branches, |x| has the
// derivative sign(x) with sign(0) = 0.  Per-entry local derivatives (fluxes,
// entropies, the wavespeed bound and the limiter with its Newton steps) come
// from forward-mode dual numbers.  A row never writes another row's adjoint:
// a contribution to neighbour j of entry (i, j) is stored at that entry and
// row j gathers it through the transposed entry, so results do not depend
// on thread scheduling.
#include <cfloat>

#include "idp_adjoint.cuh"
#include "idp_dual.cuh"
#include "idp_internal.h"

namespace idp {

namespace {

constexpr int kB = 128;

__device__ __forceinline__ int64_t slot_base(const DeviceGraph& G, int64_t r) {
  return (int64_t)G.slice_ptr[r >> 5] + (r & 31);
}

__device__ __forceinline__ void load5(const double* U, int64_t n, int64_t i, double* u) {
#pragma unroll
  for (int f = 0; f < kFields; ++f) u[f] = U[f * n + i];
}

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// gl times the derivative of limiter(U, P, rho_min, rho_max, phi_min),
// added to gU, gP and gb = (g rho_min, g rho_max, g phi_min): one dual pass
// over the eight scalars the limiter depends on (U0, P0, the coefficients
// a0, a1, a2 of rho eps(t) and the three bounds), then the chain rule
// through a0 = U0 U4 - |m_U|^2/2, a1 = U0 P4 + P0 U4 - m_U.m_P and
// a2 = P0 P4 - |m_P|^2/2.
__device__ void limiter_vjp(const double* U, const double* P, double rmin, double rmax, double pmin, double gl,
                            const LimiterParams& prm, double* gU, double* gP, double* gb) {
  LimiterLine<8> L;
  L.U = U;
  L.P = P;
  L.U0 = dseed<8>(U[0], 0);
  L.P0 = dseed<8>(P[0], 1);
  L.a0 = dseed<8>(U[0] * U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]), 2);
  L.a1 = dseed<8>(U[0] * P[4] + P[0] * U[4] - (U[1] * P[1] + U[2] * P[2] + U[3] * P[3]), 3);
  L.a2 = dseed<8>(P[0] * P[4] - 0.5 * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]), 4);
  const Dual<8> t = limiter_line(L, dseed<8>(rmin, 5), dseed<8>(rmax, 6), dseed<8>(pmin, 7), prm);
  const double g0 = gl * t.d[2], g1 = gl * t.d[3], g2 = gl * t.d[4];
  gU[0] += gl * t.d[0] + g0 * U[4] + g1 * P[4];
  gP[0] += gl * t.d[1] + g1 * U[4] + g2 * P[4];
#pragma unroll
  for (int f = 1; f < 4; ++f) {
    gU[f] -= g0 * U[f] + g1 * P[f];
    gP[f] -= g1 * U[f] + g2 * P[f];
  }
  gU[4] += g0 * U[0] + g1 * P[0];
  gP[4] += g1 * U[0] + g2 * P[0];
  gb[0] += gl * t.d[5];
  gb[1] += gl * t.d[6];
  gb[2] += gl * t.d[7];
}

// out += sign * J^T g, J the Jacobian of U -> f(U).c (eq. flux) at the state
// u with 1/rho and H = (E + p)/rho.  With v = m/rho, A = g_m.m, B = g_m.c
// and T = B + g_E v.c:
//   d/drho = -(A/rho) v.c + 0.2|v|^2 T - g_E H v.c
//   d/dm   = c (g_rho + A/rho + g_E H) + g_m v.c - 0.4 v T
//   d/dE   = 0.4 T + g_E v.c
__device__ __forceinline__ void flux_vjp(const double* u, double inv_rho, double H, double cx, double cy, double cz,
                                         const double* g, double sign, double* out) {
  const double vx = u[1] * inv_rho, vy = u[2] * inv_rho, vz = u[3] * inv_rho;
  const double vc = vx * cx + vy * cy + vz * cz;
  const double Ai = (g[1] * u[1] + g[2] * u[2] + g[3] * u[3]) * inv_rho;
  const double T = g[1] * cx + g[2] * cy + g[3] * cz + g[4] * vc;
  const double cc = g[0] + Ai + g[4] * H;
  out[0] += sign * (0.2 * (vx * vx + vy * vy + vz * vz) * T - (Ai + g[4] * H) * vc);
  out[1] += sign * (cx * cc + g[1] * vc - 0.4 * vx * T);
  out[2] += sign * (cy * cc + g[2] * vc - 0.4 * vy * T);
  out[3] += sign * (cz * cc + g[3] * vc - 0.4 * vz * T);
  out[4] += sign * (0.4 * T + g[4] * vc);
}

// out += g * grad s(U), s = eta/rho: grad s = (s/(6 p rho)) (E, -m, rho) - (s/rho) e_rho
__device__ __forceinline__ void entropy_s_vjp(const double* u, double s, double inv_rho, double inv_p, double g,
                                              double* out) {
  const double sc = g * s * inv_p * inv_rho * (1.0 / 6.0);
  out[0] += sc * u[4] - g * s * inv_rho;
  out[1] -= sc * u[1];
  out[2] -= sc * u[2];
  out[3] -= sc * u[3];
  out[4] += sc * u[0];
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

// Adjoints of one side's primitives (normal velocity u, sound speed c,
// pressure p, p^(-1/7)) to its conserved state, added to out.
__device__ __forceinline__ void side_vjp(double nx, double ny, double nz, const Side& S, double gu, double gc,
                                         double gp, double gpm, double* out) {
  const double vx = S.mx * S.inv_rho, vy = S.my * S.inv_rho, vz = S.mz * S.inv_rho;
  const double u = vx * nx + vy * ny + vz * nz;
  // c = sqrt(1.4 p / rho), pm = p^(-1/7), u = m.n/rho, p = 0.4 (E - |m|^2/(2 rho))
  const double gpt = gp + (0.5 * gc * S.c - gpm * S.pm * (1.0 / 7.0)) * S.inv_p;
  out[0] += (-0.5 * gc * S.c - gu * u) * S.inv_rho + 0.2 * (vx * vx + vy * vy + vz * vz) * gpt;
  out[1] += gu * nx * S.inv_rho - 0.4 * vx * gpt;
  out[2] += gu * ny * S.inv_rho - 0.4 * vy * gpt;
  out[3] += gu * nz * S.inv_rho - 0.4 * vz * gpt;
  out[4] += 0.4 * gpt;
}

// Reverse of lambda_max (idp_device.cuh): adds g d lambda/dU_L to gL and
// g d lambda/dU_R to gR, on the branches the forward evaluation takes.  The
// values that decide the branches are formed as the forward sweep forms
// them, bitwise: the normal speeds u_fwd (m.c (1/rho)(1/|c|), as the forward
// sweep takes them from its flux contractions) where given, else m.n/rho as
// lambda_max forms them, and the quotient of the two-rarefaction pressure by
// div_pos.
__device__ void lambda_max_vjp(double nx, double ny, double nz, const Side& L, const Side& R, double g, double* gL,
                               double* gR, const double* u_fwd = nullptr) {
  const double uL = u_fwd ? u_fwd[0] : (L.mx * nx + L.my * ny + L.mz * nz) * L.inv_rho;
  const double uR = u_fwd ? u_fwd[1] : (R.mx * nx + R.my * ny + R.mz * nz) * R.inv_rho;
  const double num0 = L.c + R.c - 0.2 * (uR - uL);
  const double num = num0 > 0.0 ? num0 : 0.0;
  const double den = L.c * L.pm + R.c * R.pm;
  const double x = div_pos(num, den);
  const double x2 = x * x, x3 = x2 * x, x6 = x3 * x3;
  const double p_tr = x6 * x;
  const bool left_high = L.p >= R.p;
  const double p_max = left_high ? L.p : R.p;
  const double p_low = left_high ? R.p : L.p;
  const double rho_low = left_high ? R.rho : L.rho;
  const double du = uR - uL;
  const double dp = p_max - p_low;
  const bool psi_negative = du < 0.0 && 2.0 * dp * dp < du * du * (rho_low * (2.4 * p_max + 0.4 * p_low));
  const bool star_is_max = !psi_negative && p_max <= p_tr;
  const double p_star = star_is_max ? p_max : p_tr;
  const double k = 6.0 / 7.0;
  const double zL = (p_star - L.p) * L.inv_p, zR = (p_star - R.p) * R.inv_p;
  const double SL = sqrt(1.0 + k * fmax(zL, 0.0)), SR = sqrt(1.0 + k * fmax(zR, 0.0));
  const double lam1 = uL - L.c * SL, lam3 = uR + R.c * SR;
  const double a = fmax(-lam1, 0.0), b = fmax(lam3, 0.0);
  double g1 = 0.0, g3 = 0.0;  // adjoints of lam1, lam3
  if (a >= b) {
    if (-lam1 >= 0.0) g1 = -g;
  } else if (lam3 >= 0.0) {
    g3 = g;
  }
  if (g1 == 0.0 && g3 == 0.0) return;
  double guL = g1, guR = g3, gcL = -g1 * SL, gcR = g3 * SR, gpL = 0.0, gpR = 0.0, gstar = 0.0;
  if (g1 != 0.0 && zL >= 0.0) {
    const double gz = -g1 * L.c * k / (2.0 * SL);
    gstar += gz * L.inv_p;
    gpL -= gz * p_star * L.inv_p * L.inv_p;
  }
  if (g3 != 0.0 && zR >= 0.0) {
    const double gz = g3 * R.c * k / (2.0 * SR);
    gstar += gz * R.inv_p;
    gpR -= gz * p_star * R.inv_p * R.inv_p;
  }
  double gpmL = 0.0, gpmR = 0.0;
  if (star_is_max) {
    if (left_high) gpL += gstar; else gpR += gstar;
  } else if (gstar != 0.0) {
    const double gx = 7.0 * x6 * gstar;
    const double gnum = gx / den, gden = -x / den * gx;
    gcL += L.pm * gden;
    gcR += R.pm * gden;
    gpmL = L.c * gden;
    gpmR = R.c * gden;
    if (num0 >= 0.0) {
      gcL += gnum;
      gcR += gnum;
      guL += 0.2 * gnum;
      guR -= 0.2 * gnum;
    }
  }
  side_vjp(nx, ny, nz, L, guL, gcL, gpL, gpmL, gL);
  side_vjp(nx, ny, nz, R, guR, gcR, gpR, gpmR, gR);
}

// Step 6 reverse: boundary post-processing and the last limiter pass
// U6 = U5 + sum_j lambda_i min(l_ij, l_ji) P'_ij.
__global__ void __launch_bounds__(kB) ka_final(DeviceGraph G, const double* __restrict__ gE, const double* __restrict__ Pp,
                                               const double* __restrict__ l5, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  double g[kFields];
  load5(gE, n, r, g);
  const int bc = G.bc[r];
  if (bc & 8) {
#pragma unroll
    for (int f = 0; f < kFields; ++f) g[f] = 0.0;
  } else {
    if (bc & 1) g[1] = 0.0;
    if (bc & 2) g[2] = 0.0;
    if (bc & 4) g[3] = 0.0;
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) A.gU5[f * n + r] = g[f];
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double lam = G.lam[r];
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (G.col[p] == r) continue;
    const double lij = l5[p], lji = l5[G.tpos[p]];
    const double m = fmin(lij, lji);
    double gm = 0.0;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      A.gPp[f * ns + p] = lam * m * g[f];
      gm += lam * Pp[f * ns + p] * g[f];
    }
    A.gl5_own[p] = lij <= lji ? gm : 0.0;
    A.gl5_tr[p] = lij <= lji ? 0.0 : gm;
  }
}

// The limiter's derivative (a Dual<8> pass, ~255 registers) is needed only
// at the entries whose limiter value lies strictly inside (0, 1) and whose
// l_ij has a non-zero adjoint (a few per cent of the entries, spread over
// most warps' rows): ka_lim_select lists them, ka_lim_eval runs the dual pass
// with one thread per listed entry, and ka_lim_gather adds each row's
// contributions in slot order, so that the sums do not depend on the order
// of the list.  The rest of each reversed step runs at a higher occupancy.
// Used for Step 5 (l5 = limiter(U5, P', bounds)) and Step 4 (l4 =
// limiter(U^L, P, bounds)).
__global__ void __launch_bounds__(kB) ka_lim_select(DeviceGraph G, const double* __restrict__ l,
                                                    const double* __restrict__ gl_own,
                                                    const double* __restrict__ gl_tr, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int64_t base = 0;
  int len = 0;
  unsigned int cnt = 0;
  if (r < G.n) {
    base = slot_base(G, r);
    len = G.row_len[r];
    for (int k = 0; k < len; ++k) {
      const int64_t p = base + 32 * (int64_t)k;
      uint8_t fl = 0;
      if (G.col[p] != r) {
        const double gl = gl_own[p] + gl_tr[G.tpos[p]];
        const double lv = l[p];
        // l = 0 and l = 1 are clamped (or skipped) values: locally constant
        if (gl != 0.0 && lv > 0.0 && lv < 1.0) {
          fl = 1;
          A.lim_gl[p] = gl;
          ++cnt;
        }
      }
      A.lim_flag[p] = fl;
    }
  }
  // warp-aggregated append: inclusive scan of the rows' counts
  unsigned int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned int start = 0;
  if (lane == 31 && total) start = atomicAdd(A.lim_count, total);
  start = __shfl_sync(0xffffffffu, start, 31);
  if (!cnt) return;
  unsigned int pos = start + incl - cnt;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (A.lim_flag[p]) {
      A.lim_slot[pos] = (int32_t)p;
      A.lim_row[pos] = (int32_t)r;
      ++pos;
    }
  }
}

// One thread per listed entry: gl times the derivative of the limiter at
// (U_r, P_p, bounds_r); the P part is added to gP at the entry, the row-state
// and bound parts are kept at the entry for ka_lim_gather.
__global__ void __launch_bounds__(kB) ka_lim_eval(DeviceGraph G, StageConfig C, const double* __restrict__ Ur,
                                                  const double* __restrict__ P, const double* __restrict__ bnd,
                                                  double* __restrict__ gP, AdjointBuffers A) {
  const int64_t n = G.n, ns = G.n_slots;
  const unsigned int count = *A.lim_count;
  for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    const int64_t p = A.lim_slot[q];
    const int64_t r = A.lim_row[q];
    double u[kFields], pij[kFields], gU[kFields], gPl[kFields], gb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      u[f] = Ur[f * n + r];
      pij[f] = P[f * ns + p];
      gU[f] = 0.0;
      gPl[f] = 0.0;
    }
    limiter_vjp(u, pij, bnd[r], bnd[n + r], bnd[2 * n + r], A.lim_gl[p], C.lim, gU, gPl, gb);
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      gP[f * ns + p] += gPl[f];
      A.lim_gU[f * ns + p] = gU[f];
    }
    A.lim_gb[p] = gb[0];
    A.lim_gb[ns + p] = gb[1];
    A.lim_gb[2 * ns + p] = gb[2];
  }
}

// Row r adds its listed entries' contributions in slot order to gUr (the
// adjoint of the state the limiter was evaluated at) and to the adjoint of
// its bounds: assigned (the first writer, Step 5) or added (Step 4, only
// where the row has listed entries).
__global__ void __launch_bounds__(kB) ka_lim_gather(DeviceGraph G, double* __restrict__ gUr, int assign_bounds,
                                                    AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double g[kFields], gb[3] = {0.0, 0.0, 0.0};
  bool touched = false;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (!A.lim_flag[p]) continue;
    if (!touched) {
      load5(gUr, n, r, g);
      touched = true;
    }
#pragma unroll
    for (int f = 0; f < kFields; ++f) g[f] += A.lim_gU[f * ns + p];
    gb[0] += A.lim_gb[p];
    gb[1] += A.lim_gb[ns + p];
    gb[2] += A.lim_gb[2 * ns + p];
  }
  if (touched) {
#pragma unroll
    for (int f = 0; f < kFields; ++f) gUr[f * n + r] = g[f];
  }
  if (assign_bounds) {
    A.gbnd[r] = gb[0];
    A.gbnd[n + r] = gb[1];
    A.gbnd[2 * n + r] = gb[2];
  } else if (touched) {
    A.gbnd[r] += gb[0];
    A.gbnd[n + r] += gb[1];
    A.gbnd[2 * n + r] += gb[2];
  }
}

// Step 5 reverse, the rest: P'_ij = (1 - m_ij) P_ij and
// U5 = U^L + sum_j lambda_i m_ij P_ij with m_ij = min(l4_ij, l4_ji).
__global__ void __launch_bounds__(kB) ka_pass(DeviceGraph G, const double* __restrict__ P,
                                              const double* __restrict__ l4, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double lam = G.lam[r];
  double gU5[kFields];
  load5(A.gU5, n, r, gU5);
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (G.col[p] == r) continue;
    const double lij = l4[p], lji = l4[G.tpos[p]];
    const double m = fmin(lij, lji);
    double gm = 0.0;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      const double gpp = A.gPp[f * ns + p];
      const double pf = P[f * ns + p];
      A.gP[f * ns + p] = (1.0 - m) * gpp + lam * m * gU5[f];
      gm += (lam * gU5[f] - gpp) * pf;
    }
    A.gl4_own[p] = lij <= lji ? gm : 0.0;
    A.gl4_tr[p] = lij <= lji ? 0.0 : gm;
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) A.gUL[f * n + r] = gU5[f];
}

// Step 4 reverse, the rest:
// P_ij = tau/(m_i lambda_i) (b_ij R_j - b_ji R_i + (d^H_ij - d_ij)(U_j - U_i)).
__global__ void __launch_bounds__(kB) ka_flux(DeviceGraph G, const double* __restrict__ U,
                                              const double* __restrict__ P, const double* __restrict__ d,
                                              const double* __restrict__ alpha, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double tau = G.tau[instance_of(G, r)];
  double ui[kFields];
  double gRi[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0}, gUi[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0};
  load5(U, n, r, ui);
  const double a_i = alpha[r];
  const double inv_mi = G.inv_mi[r];
  const double scale = tau * inv_mi * (double)(len - 1);
  double galpha_i = 0.0, tp_sum = 0.0;
  // the first writer of the entry adjoints gU_tr, gd and ga_tr and of gU_own
  // in the reversed stage: assigns them (zero on the diagonal)
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    if (j == r) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        A.gR_tr[f * ns + p] = 0.0;
        A.gU_tr[f * ns + p] = 0.0;
      }
      A.gd[p] = 0.0;
      A.ga_tr[p] = 0.0;
      continue;
    }
    double pij[kFields], gP[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      pij[f] = P[f * ns + p];
      gP[f] = A.gP[f * ns + p];
    }
    double uj[kFields];
    load5(U, n, j, uj);
    const double m = G.mij[p];
    const double b_ij = -m * G.inv_mi[j];
    const double b_ji = -m * inv_mi;
    const double dij = d[p];
    const double Aij = (a_i + alpha[j]) * 0.5;
    const double dd = dij * Aij - dij;
    double gdd = 0.0, tp = 0.0;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      gRi[f] -= scale * b_ji * gP[f];
      A.gR_tr[f * ns + p] = scale * b_ij * gP[f];
      gdd += scale * (uj[f] - ui[f]) * gP[f];
      A.gU_tr[f * ns + p] = scale * dd * gP[f];
      gUi[f] -= scale * dd * gP[f];
      tp += pij[f] * gP[f];
    }
    A.gd[p] = (Aij - 1.0) * gdd;
    galpha_i += 0.5 * dij * gdd;
    A.ga_tr[p] = 0.5 * dij * gdd;
    tp_sum += tp;
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    A.gR_own[f * n + r] = gRi[f];
    A.gU_own[f * n + r] = gUi[f];
  }
  A.ga_own[r] = galpha_i;
  A.gtau_part[r] = tau > 0.0 ? tp_sum / tau : 0.0;  // P_ij is linear in tau
}

// Step 3 reverse: U^L_i = U_i + sum_j (2 tau/m_i) d_ij Ubar_ij, the bounds
// over rho(Ubar_ij) and phi(U_j), and
// R_i = -f_i.s_i - sum_j (f_j - f_i).c_ij + sum_j d^H_ij (U_j - U_i).
__global__ void __launch_bounds__(kB) ka_low(DeviceGraph G, const double* __restrict__ U, const double* __restrict__ Q,
                                             const double* __restrict__ d, const double* __restrict__ dinv,
                                             const double* __restrict__ dF, const double* __restrict__ alpha,
                                             AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  const double tau = G.tau[instance_of(G, r)];
  double ui[kFields], gUL[kFields], gR[kFields], gUi[kFields];
  load5(U, n, r, ui);
  load5(A.gUL, n, r, gUL);
  load5(A.gR_own, n, r, gR);
  const double inv_rho_i = Q[kQInvRho * n + r], h_i = Q[kQH * n + r];
  // gather R's adjoint; locate the first entries attaining the bounds (the
  // doubled bar-state densities formed as Step 3 forms them, from its flux
  // differences)
  int kmin = -1, kmax = -1, kphi = -1;
  double vmin = INFINITY, vmax = -INFINITY, vphi = INFINITY;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    const int64_t pt = G.tpos[p];
#pragma unroll
    for (int f = 0; f < kFields; ++f) gR[f] += A.gR_tr[f * ns + pt];
    const double dij = d[p];
    if (dij != 0.0) {
      const double ub0 = j != r ? fma(-dF[p], 2.0 * dinv[p], ui[0] + U[j]) : ui[0] + ui[0];
      if (ub0 < vmin) {
        vmin = ub0;
        kmin = k;
      }
      if (ub0 > vmax) {
        vmax = ub0;
        kmax = k;
      }
    }
    const double phj = Q[kQPhi * n + j];
    if (phj < vphi) {
      vphi = phj;
      kphi = k;
    }
  }
  const double g_rmin = A.gbnd[r], g_rmax = A.gbnd[n + r], g_pmin = A.gbnd[2 * n + r];
#pragma unroll
  for (int f = 0; f < kFields; ++f) gUi[f] = gUL[f];
  // -f_i . s_i
  flux_vjp(ui, inv_rho_i, h_i, G.csx[r], G.csy[r], G.csz[r], gR, -1.0, gUi);
  const double a_i = alpha[r];
  const double two_tau_m = 2.0 * tau * G.inv_mi[r];
  double ga_i = 0.0, gtau = 0.0;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    const double dij = d[p];
    A.gphi_tr[p] = k == kphi ? g_pmin : 0.0;  // the only writer
    if (j == r) {
      // Ubar_ii = U_i
      if (dij != 0.0) {
        double ud = 0.0;
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          gUi[f] += two_tau_m * dij * gUL[f];
          ud += ui[f] * gUL[f];
        }
        A.gd[p] += two_tau_m * ud;
        gtau += 2.0 * G.inv_mi[r] * dij * ud;
        if (k == kmin) gUi[0] += g_rmin;
        if (k == kmax) gUi[0] += g_rmax;
      }
      continue;
    }
    double uj[kFields];
    load5(U, n, j, uj);
    double df[kFields], gdf[kFields];
    const double Aij = (a_i + alpha[j]) * 0.5;
    const double dH = dij * Aij;
    double gdH = 0.0;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      df[f] = dF[f * ns + p];
      gdf[f] = -gR[f];
      A.gU_tr[f * ns + p] += dH * gR[f];
      gUi[f] -= dH * gR[f];
      gdH += (uj[f] - ui[f]) * gR[f];
    }
    A.gd[p] += Aij * gdH;
    ga_i += 0.5 * dij * gdH;
    A.ga_tr[p] += 0.5 * dij * gdH;
    if (dij != 0.0) {
      // Ubar_ij = (U_i + U_j)/2 - df_ij inv2d with inv2d = 1/(2 d_ij)
      const double inv2d = dinv[p];
      const double coef = two_tau_m * dij;
      double gub[kFields], ud = 0.0;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        const double ub = 0.5 * (ui[f] + uj[f]) - df[f] * inv2d;
        gub[f] = coef * gUL[f];
        ud += ub * gUL[f];
      }
      if (k == kmin) gub[0] += g_rmin;
      if (k == kmax) gub[0] += g_rmax;
      A.gd[p] += two_tau_m * ud;
      gtau += 2.0 * G.inv_mi[r] * dij * ud;
      double gi2d = 0.0;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        gUi[f] += 0.5 * gub[f];
        A.gU_tr[f * ns + p] += 0.5 * gub[f];
        gdf[f] -= inv2d * gub[f];
        gi2d -= df[f] * gub[f];
      }
      A.gd[p] -= 2.0 * inv2d * inv2d * gi2d;
    }
#pragma unroll
    for (int f = 0; f < kFields; ++f) A.gdF[f * ns + p] = gdf[f];
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) A.gU_own[f * n + r] += gUi[f];
  A.ga_own[r] += ga_i;
  A.gtau_part[r] += gtau;
}

// Sum of the per-row adjoints of tau_n in a fixed order, in two levels:
// block b sums a contiguous range of caller nodes (a strided pass, then a
// tree in shared memory), then one block sums the block partials the same
// way.  gtau[1] = this stage's sum plus the carried sum when tau was
// computed here; gtau[0] accumulates over the stages.
constexpr int kTauThreads = 256;

__device__ __forceinline__ double block_tree_sum(double* part, double s) {
  part[threadIdx.x] = s;
  __syncthreads();
#pragma unroll
  for (int w = kTauThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  return part[0];
}

__global__ void __launch_bounds__(kTauThreads) ka_tau_part(DeviceGraph G, AdjointBuffers A) {
  __shared__ double part[kTauThreads];
  const int64_t chunk = (G.n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < G.n ? lo + chunk : G.n;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kTauThreads) s += A.gtau_part[G.row_of_node ? G.row_of_node[i] : i];
  const double t = block_tree_sum(part, s);
  if (threadIdx.x == 0) A.gtau_blk[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kTauThreads) ka_tau(AdjointBuffers A, int blocks, int add_carry) {
  __shared__ double part[kTauThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < blocks; i += kTauThreads) s += A.gtau_blk[i];
  const double t = block_tree_sum(part, s);
  if (threadIdx.x == 0) {
    A.gtau[1] = t + (add_carry ? A.gtau[0] : 0.0);
    A.gtau[0] += t;
  }
}

// CFL candidates m_i / (-2 d_ii) recomputed from the traced d_ii: their
// minimum (positive doubles order as their bits), then the first row with it.
__device__ __forceinline__ double cfl_candidate(const DeviceGraph& G, const double* d, int64_t r) {
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (G.col[p] == r) return G.mi[r] / (-2.0 * d[p]);
  }
  return INFINITY;
}

__global__ void __launch_bounds__(kB) ka_cfl_min(DeviceGraph G, const double* __restrict__ d, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double c = r < G.n ? cfl_candidate(G, d, r) : INFINITY;
  // the warp's minimum first (as bits: +inf and the positive candidates order like their values), one atomic per warp
  unsigned long long key = c > 0.0 && c < INFINITY ? (unsigned long long)__double_as_longlong(c) : ~0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, key, o);
    key = v < key ? v : key;
  }
  if ((threadIdx.x & 31) == 0 && key != ~0ull) atomicMin(&A.argmin[0], key);
}

__global__ void __launch_bounds__(kB) ka_cfl_arg(DeviceGraph G, const double* __restrict__ d, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const double c = cfl_candidate(G, d, r);
  // the first row in the caller's node order attaining the minimum
  const int64_t key = G.node_of_row ? G.node_of_row[r] : r;
  if ((unsigned long long)__double_as_longlong(c) == A.argmin[0]) atomicMin(&A.argmin[1], (unsigned long long)key);
}

// Step 2 reverse: d_ii = -sum_{j != i} d_ij; in the first RK stage also
// tau_n = c_cfl m_k / (-2 d_kk) of the arg-min row k.
__global__ void __launch_bounds__(kB) ka_diag(DeviceGraph G, StageConfig C, const double* __restrict__ d,
                                              AdjointBuffers A, int tau_computed) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double gdii = 0.0;
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (G.col[p] != r) continue;
    gdii = A.gd[p];
    if (tau_computed && (unsigned long long)(G.node_of_row ? G.node_of_row[r] : r) == A.argmin[1]) {
      const double dii = d[p];
      gdii += A.gtau[1] * C.cfl * G.mi[r] / (2.0 * dii * dii);
    }
  }
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    if (G.col[p] != r) A.gd[p] -= gdii;
  }
}

// Step 1 reverse: alpha_i (Sec. 3.8), the flux differences, the wavespeed
// bound d_ij of the edges this row owns, and phi(U_i) of the bounds.
// three blocks per SM: 168 registers (32 bytes spilled) instead of 180 at two
// blocks; 50 % more warps to hide its gathers (2.96 -> 2.83 ms at 64^3)
__global__ void __launch_bounds__(kB, 3) ka_edge(DeviceGraph G, const double* __restrict__ U, const double* __restrict__ Q,
                                              const double* __restrict__ ab, AdjointBuffers A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double ui[kFields], gUi[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0};
  load5(U, n, r, ui);
  double galpha = A.ga_own[r], gphi = 0.0;
  for (int k = 0; k < len; ++k) {
    const int64_t pt = G.tpos[base + 32 * (int64_t)k];
    galpha += A.ga_tr[pt];
    gphi += A.gphi_tr[pt];
  }
  const double inv_rho_i = Q[kQInvRho * n + r], h_i = Q[kQH * n + r];
  const double s_i = Q[kQS * n + r];
  // a_i and b_i of the indicator as the forward sweep formed them
  const double a = ab[r];
  const double b[kFields] = {ab[n + r], ab[2 * n + r], ab[3 * n + r], ab[4 * n + r], ab[5 * n + r]};
  // alpha = |num| / D with num = a - e.b + s_i b_0,
  // D = |a| + |e_0 - s_i||b_0| + sum_{f>0} |e_f||b_f|, e = eta'(U_i)
  double ga = 0.0, gb[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0}, ge[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0}, gs = 0.0;
  {
    const double sc = s_i * Q[kQInvP * n + r] * (1.0 / 6.0);
    const double e[kFields] = {sc * ui[4], -sc * ui[1], -sc * ui[2], -sc * ui[3], sc * ui[0]};
    const double num = a - (e[0] * b[0] + e[1] * b[1] + e[2] * b[2] + e[3] * b[3] + e[4] * b[4]) + s_i * b[0];
    double D = fabs(a);
#pragma unroll
    for (int f = 0; f < kFields; ++f) D += fabs(e[f] - (f == 0 ? s_i : 0.0)) * fabs(b[f]);
    if (D > 0.0 && galpha != 0.0) {
      const double al = fabs(num) / D;
      const double gD = -al / D * galpha;
      const double gnum = sgn(num) * galpha / D;
      ga = gnum + sgn(a) * gD;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        const double ef = e[f] - (f == 0 ? s_i : 0.0);
        gb[f] = -e[f] * gnum + fabs(ef) * sgn(b[f]) * gD;
        ge[f] = -b[f] * gnum + sgn(ef) * fabs(b[f]) * gD;
      }
      gb[0] += s_i * gnum;
      gs = b[0] * gnum - sgn(e[0] - s_i) * fabs(b[0]) * gD;
    }
  }
  // e(U_i), s(U_i) and phi(U_i)
  {
    Dual<5> ud[kFields];
#pragma unroll
    for (int f = 0; f < kFields; ++f) ud[f] = dseed<5>(ui[f], f);
    const Dual<5> sd = entropy_s(ud);
    const SideT<Dual<5>> side = side_of_state(ud);
    const Dual<5> sc = sd * side.inv_p * (1.0 / 6.0);
    const Dual<5> e0 = sc * ud[4], e1 = -(sc * ud[1]), e2 = -(sc * ud[2]), e3 = -(sc * ud[3]), e4 = sc * ud[0];
    const Dual<5> phid = entropy_phi(ud);
#pragma unroll
    for (int q = 0; q < kFields; ++q)
      gUi[q] += ge[0] * e0.d[q] + ge[1] * e1.d[q] + ge[2] * e2.d[q] + ge[3] * e3.d[q] + ge[4] * e4.d[q] +
                gs * sd.d[q] + gphi * phid.d[q];
  }
  // per-entry terms; U_i's flux adjoint is collected per direction,
  // sum_j J(U_i; c_ij)^T g_ij = sum_d J(U_i; e_d)^T (sum_j c_ij,d g_ij)
  const Side si = load_side(U, Q, n, r);
  const double inv_p_i = Q[kQInvP * n + r];
  double Gx[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0}, Gy[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0},
         Gz[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double gsi = 0.0;  // adjoint of s_i through a_i
  for (int k = 0; k < len; ++k) {
    const int64_t p = base + 32 * (int64_t)k;
    const int64_t j = G.col[p];
    if (j == r) continue;  // the diagonal terms of a_i and b_i vanish identically
    const double cx = G.cx[p], cy = G.cy[p], cz = G.cz[p];
    double uj[kFields], gj[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0}, gdf[kFields];
    load5(U, n, j, uj);
    const double inv_rho_j = Q[kQInvRho * n + j];
    // (f_j - f_i).c_ij: adjoint from Step 3 and from b_i
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
      gdf[f] = A.gdF[f * ns + p] + gb[f];
      Gx[f] += cx * gdf[f];
      Gy[f] += cy * gdf[f];
      Gz[f] += cz * gdf[f];
    }
    flux_vjp(uj, inv_rho_j, Q[kQH * n + j], cx, cy, cz, gdf, 1.0, gj);
    // a_i term (s_j - s_i)(m_j . c_ij)
    if (ga != 0.0) {
      const double mc = uj[1] * cx + uj[2] * cy + uj[3] * cz;
      const double sj = Q[kQS * n + j];
      const double ds = sj - s_i;
      entropy_s_vjp(uj, sj, inv_rho_j, Q[kQInvP * n + j], mc * ga, gj);
      gj[1] += ds * cx * ga;
      gj[2] += ds * cy * ga;
      gj[3] += ds * cz * ga;
      gsi -= mc * ga;
    }
    // d_ij of an edge this row owns: adjoint of both rows' uses
    if (G.flags[p] & kEntryUpper) {
      const int64_t pt = G.tpos[p];
      const double gdedge = A.gd[p] + A.gd[pt];
      if (gdedge != 0.0) {
        const Side sj = load_side(U, Q, n, j);
        const double nc = G.cn[p];
        bool transposed = false;
        if (!(G.flags[p] & kEntrySkew) && G.cn[pt] > 0.0) {
          // d1 as the forward sweep forms it (normal speeds from m.c)
          const double ic = G.inv_cn[p];
          const double d1 = nc > 0.0 ? lambda_max_u(normal_speed(m_dot_c(si.mx, si.my, si.mz, cx, cy, cz), si.inv_rho, ic),
                                                    normal_speed(m_dot_c(sj.mx, sj.my, sj.mz, cx, cy, cz), sj.inv_rho, ic),
                                                    si, sj) * nc
                                     : 0.0;
          const double it = G.inv_cn[pt];
          const double d2 = lambda_max(G.cx[pt] * it, G.cy[pt] * it, G.cz[pt] * it, sj, si) * G.cn[pt];
          transposed = !(d1 >= d2);
        }
        if (transposed) {
          const double it = G.inv_cn[pt];
          lambda_max_vjp(G.cx[pt] * it, G.cy[pt] * it, G.cz[pt] * it, sj, si, gdedge * G.cn[pt], gj, gUi);
        } else if (nc > 0.0) {
          const double inv = G.inv_cn[p];
          const double u_fwd[2] = {normal_speed(m_dot_c(si.mx, si.my, si.mz, cx, cy, cz), si.inv_rho, inv),
                                   normal_speed(m_dot_c(sj.mx, sj.my, sj.mz, cx, cy, cz), sj.inv_rho, inv)};
          lambda_max_vjp(cx * inv, cy * inv, cz * inv, si, sj, gdedge * nc, gUi, gj, u_fwd);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < kFields; ++f) A.gU_tr[f * ns + p] += gj[f];
  }
  flux_vjp(ui, inv_rho_i, h_i, 1.0, 0.0, 0.0, Gx, -1.0, gUi);
  flux_vjp(ui, inv_rho_i, h_i, 0.0, 1.0, 0.0, Gy, -1.0, gUi);
  flux_vjp(ui, inv_rho_i, h_i, 0.0, 0.0, 1.0, Gz, -1.0, gUi);
  if (gsi != 0.0) entropy_s_vjp(ui, s_i, inv_rho_i, inv_p_i, gsi, gUi);
#pragma unroll
  for (int f = 0; f < kFields; ++f) A.gU_own[f * n + r] += gUi[f];
}

// adjoint of U_i: own part plus the neighbours' contributions stored at the
// transposed entries
__global__ void __launch_bounds__(kB) ka_gather(DeviceGraph G, AdjointBuffers A, double* __restrict__ gIn) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G.n) return;
  const int64_t n = G.n, ns = G.n_slots;
  const int64_t base = slot_base(G, r);
  const int len = G.row_len[r];
  double g[kFields];
  load5(A.gU_own, n, r, g);
  for (int k = 0; k < len; ++k) {
    const int64_t pt = G.tpos[base + 32 * (int64_t)k];
#pragma unroll
    for (int f = 0; f < kFields; ++f) g[f] += A.gU_tr[f * ns + pt];
  }
#pragma unroll
  for (int f = 0; f < kFields; ++f) gIn[f * n + r] = g[f];
}

__global__ void k_axpby(double* __restrict__ out, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y ? a * x[i] + b * y[i] : a * x[i];
}

}  // namespace

// Grid of ka_lim_eval: the blocks that fit on the device at once (a
// grid-stride loop over the list, whose length stays on the device).
static unsigned lim_eval_grid() {
  static unsigned cached = 0;
  if (!cached) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)ka_lim_eval, kB, 0);
    cached = (unsigned)(sms > 0 ? sms : 1) * (unsigned)(per_sm > 0 ? per_sm : 1);
  }
  return cached;
}

int launch_adjoint_stage(const DeviceGraph& G, const StageBuffers& B, const AdjointBuffers& A, const StageConfig& C,
                         const double* Uin, const double* gE, double* gIn, bool tau_computed, cudaStream_t s,
                         Profiler* prof) {
  const unsigned grid = (unsigned)((G.n + kB - 1) / kB);
  const bool timed = prof && prof->enabled;
  int launches = 0;
  auto run = [&](int id, auto&& launch) {
    if (timed) prof->begin(id, s);
    launch();
    if (timed) prof->end(s);
  };
  // gU_own, gU_tr, gd and ga_tr are first written (assigned) by ka_flux,
  // gphi_tr only by ka_low
  // traced intermediates: P and l of Step 4 (tP, tl4), the state and l
  // after the first pass (tU5, tl5), P' of the first pass (left in B.P)
  run(kKAdjFinal, [&] { ka_final<<<grid, kB, 0, s>>>(G, gE, B.P, B.tl5, A); });
  const unsigned egrid = lim_eval_grid();
  // the limiter's derivative at the listed entries (see ka_lim_select)
  auto limiter_reverse = [&](const double* Ur, const double* P, const double* l, const double* gl_own,
                             const double* gl_tr, double* gUr, double* gP, int assign_bounds) {
    cudaMemsetAsync(A.lim_count, 0, sizeof(unsigned int), s);
    ka_lim_select<<<grid, kB, 0, s>>>(G, l, gl_own, gl_tr, A);
    ka_lim_eval<<<egrid, kB, 0, s>>>(G, C, Ur, P, B.bnd, gP, A);
    ka_lim_gather<<<grid, kB, 0, s>>>(G, gUr, assign_bounds, A);
  };
  run(kKAdjPass, [&] {
    limiter_reverse(B.tU5, B.P, B.tl5, A.gl5_own, A.gl5_tr, A.gU5, A.gPp, 1);
    ka_pass<<<grid, kB, 0, s>>>(G, B.tP, B.tl4, A);
  });
  run(kKAdjFlux, [&] {
    limiter_reverse(B.UL, B.tP, B.tl4, A.gl4_own, A.gl4_tr, A.gUL, A.gP, 0);
    ka_flux<<<grid, kB, 0, s>>>(G, Uin, B.tP, B.d, B.alpha, A);
  });
  run(kKAdjLow, [&] { ka_low<<<grid, kB, 0, s>>>(G, Uin, B.node, B.d, B.dinv, B.tdF, B.alpha, A); });
  launches += 10;
  run(kKAdjTau, [&] {
    const int64_t want = (G.n + 2047) / 2048;
    const int tblocks = (int)(want < kTauBlocks ? (want > 0 ? want : 1) : kTauBlocks);
    ka_tau_part<<<tblocks, kTauThreads, 0, s>>>(G, A);
    ka_tau<<<1, kTauThreads, 0, s>>>(A, tblocks, tau_computed ? 1 : 0);
    if (tau_computed) {
      cudaMemsetAsync(A.argmin, 0xff, 2 * sizeof(unsigned long long), s);
      ka_cfl_min<<<grid, kB, 0, s>>>(G, B.d, A);
      ka_cfl_arg<<<grid, kB, 0, s>>>(G, B.d, A);
    }
  });
  launches += tau_computed ? 4 : 2;
  run(kKAdjDiag, [&] { ka_diag<<<grid, kB, 0, s>>>(G, C, B.d, A, tau_computed ? 1 : 0); });
  run(kKAdjEdge, [&] { ka_edge<<<grid, kB, 0, s>>>(G, Uin, B.node, B.tab, A); });
  run(kKAdjGather, [&] { ka_gather<<<grid, kB, 0, s>>>(G, A, gIn); });
  return launches + 3;
}

void launch_axpby(double* out, double a, const double* x, double b, const double* y, int64_t count, cudaStream_t s) {
  const int64_t blocks = (count + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
  k_axpby<<<grid, 256, 0, s>>>(out, a, x, b, y, count);
}

}  // namespace idp
