// C ABI of libidp (include/idp.h): context, uploads, stepping, read-back.
#include <cuda_runtime.h>

#include <array>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "idp.h"
#include "idp_adjoint.cuh"
#include "idp_internal.h"
#include "idp_mixed.cuh"
#include "idp_stage.cuh"
#include "idp_context.cuh"

namespace {

idp_status fail(idp_ctx* ctx, idp_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define IDP_CUDA(ctx, expr)                                                                     \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return fail(ctx, IDP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
idp_status dalloc(idp_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, IDP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return IDP_OK;
}

template <typename T>
idp_status upload(idp_ctx* ctx, T** p, const std::vector<T>& v) {
  idp_status st = dalloc(ctx, p, v.size());
  if (st != IDP_OK) return st;
  IDP_CUDA(ctx, cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return IDP_OK;
}

void drop_graph(idp_ctx* ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
}

void free_instances(idp_ctx* ctx) {
  for (void* p : ctx->inst_allocs) cudaFree(p);
  ctx->inst_allocs.clear();
}

void free_record(idp_ctx* ctx) {
  for (void* p : ctx->rec_allocs) cudaFree(p);
  ctx->rec_allocs.clear();
  ctx->rec_steps = ctx->rec_every = 0;
  ctx->rec_ckpt = ctx->rec_tau = ctx->rec_seg = ctx->rec_snap = nullptr;
}

void free_all(idp_ctx* ctx) {
  drop_graph(ctx);
  free_instances(ctx);
  free_record(ctx);
  ctx->has_adjoint = false;
  for (void* p : ctx->allocations) cudaFree(p);
  ctx->allocations.clear();
}

// Per-instance tau, time, bound and reduction word for n_inst instances;
// inst (host, per library row) may be empty for a single instance.
idp_status alloc_instances(idp_ctx* ctx, int64_t n_inst, const std::vector<int32_t>& inst) {
  drop_graph(ctx);
  free_instances(ctx);
  auto get = [&](void** p, size_t bytes) -> idp_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, IDP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->inst_allocs.push_back(*p);
    return IDP_OK;
  };
  void *tau, *time, *tmax, *tmin, *ins = nullptr;
  idp_status st;
  if ((st = get(&tau, sizeof(double) * n_inst)) || (st = get(&time, sizeof(double) * n_inst)) ||
      (st = get(&tmax, sizeof(double) * n_inst)) || (st = get(&tmin, sizeof(unsigned long long) * n_inst)))
    return st;
  if (!inst.empty()) {
    if ((st = get(&ins, sizeof(int32_t) * inst.size()))) return st;
    IDP_CUDA(ctx, cudaMemcpy(ins, inst.data(), sizeof(int32_t) * inst.size(), cudaMemcpyHostToDevice));
  }
  IDP_CUDA(ctx, cudaMemset(tau, 0, sizeof(double) * n_inst));
  IDP_CUDA(ctx, cudaMemset(time, 0, sizeof(double) * n_inst));
  IDP_CUDA(ctx, cudaMemset(tmax, 0, sizeof(double) * n_inst));
  IDP_CUDA(ctx, cudaMemset(tmin, 0, sizeof(unsigned long long) * n_inst));
  idp::DeviceGraph& G = ctx->G;
  G.n_inst = n_inst;
  G.inst = static_cast<const int32_t*>(ins);
  G.tau = static_cast<double*>(tau);
  G.time = static_cast<double*>(time);
  G.tau_max = static_cast<double*>(tmax);
  G.tau_min = static_cast<unsigned long long*>(tmin);
  return IDP_OK;
}

idp_status device_status(idp_ctx* ctx, bool clear) {
  int st = 0;
  IDP_CUDA(ctx, cudaMemcpyAsync(&st, &ctx->B.scal->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (clear && st) IDP_CUDA(ctx, cudaMemsetAsync(&ctx->B.scal->status, 0, sizeof(int), ctx->stream));
  if (st & idp::kStatusNotAdmissible) return fail(ctx, IDP_ERR_STATE_NOT_ADMISSIBLE, "state not admissible");
  if (st & idp::kStatusCfl) return fail(ctx, IDP_ERR_CFL, "tau of the first RK stage violates the CFL bound of a later stage");
  if (st & idp::kStatusNonFinite) return fail(ctx, IDP_ERR_NONFINITE, "non-finite value in the state");
  if (st & idp::kStatusTimeout) return fail(ctx, IDP_ERR_TIMEOUT, "device wait timed out");
  return IDP_OK;
}

// Per-row bound relaxation r_i = (m_i / |Omega_k|)^(1/2), |Omega_k| the sum of
// m_i over the row's instance k (inst: instance per row, empty for one).
idp_status upload_relax(idp_ctx* ctx, const std::vector<int32_t>& inst) {
  const idp::SellLayout& L = ctx->L;
  const int64_t n = L.n;
  int64_t n_inst = 1;
  for (int32_t k : inst) n_inst = k + 1 > n_inst ? k + 1 : n_inst;
  std::vector<double> vol((size_t)n_inst, 0.0), r((size_t)n);
  for (int64_t c = 0; c < n; ++c) {  // summed in the caller's node order
    const int64_t i = L.perm[c];
    vol[inst.empty() ? 0 : inst[i]] += L.mi[i];
  }
  for (int64_t i = 0; i < n; ++i) r[i] = std::sqrt(L.mi[i] / vol[inst.empty() ? 0 : inst[i]]);
  if (!ctx->G.relax) {
    double* p = nullptr;
    idp_status st = dalloc(ctx, &p, (size_t)n);
    if (st != IDP_OK) return st;
    ctx->G.relax = p;
  }
  IDP_CUDA(ctx, cudaMemcpy(const_cast<double*>(ctx->G.relax), r.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  return IDP_OK;
}

// Trace copies of the stage intermediates (allocated on first traced stage).
idp_status ensure_trace(idp_ctx* ctx) {
  if (ctx->has_trace) return IDP_OK;
  idp::StageBuffers& B = ctx->B;
  const size_t n = (size_t)ctx->G.n, ns = (size_t)ctx->G.n_slots;
  idp_status st;
  if ((st = dalloc(ctx, &B.tP, 5 * ns)) || (st = dalloc(ctx, &B.tl4, ns)) || (st = dalloc(ctx, &B.tU5, 5 * n)) ||
      (st = dalloc(ctx, &B.tl5, ns)) || (st = dalloc(ctx, &B.tUlim, 5 * n)) || (st = dalloc(ctx, &B.tab, 6 * n)) ||
      (st = dalloc(ctx, &B.tdF, 5 * ns)))
    return st;
  ctx->has_trace = true;
  return IDP_OK;
}

// The reverse mode covers the FP64 stage with two limiter passes on one instance.
idp_status adjoint_supported(idp_ctx* ctx) {
  if (!ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (ctx->mixed) return fail(ctx, IDP_ERR_ARG, "the adjoint needs the FP64 precision mode");
  if (ctx->C.limiter_passes != 2) return fail(ctx, IDP_ERR_ARG, "the adjoint needs limiter_passes = 2");
  if (ctx->G.n_inst != 1) return fail(ctx, IDP_ERR_ARG, "the adjoint needs a single instance");
  if (ctx->cfg.relax) return fail(ctx, IDP_ERR_ARG, "the adjoint does not cover the bound relaxation");
  return IDP_OK;
}

idp_status ensure_adjoint(idp_ctx* ctx) {
  idp_status st = ensure_trace(ctx);
  if (st != IDP_OK || ctx->has_adjoint) return st;
  idp::AdjointBuffers& A = ctx->A;
  const size_t n = (size_t)ctx->G.n, ns = (size_t)ctx->G.n_slots;
  if ((st = dalloc(ctx, &A.gU5, 5 * n)) || (st = dalloc(ctx, &A.gUL, 5 * n)) || (st = dalloc(ctx, &A.gR_own, 5 * n)) ||
      (st = dalloc(ctx, &A.gU_own, 5 * n)) || (st = dalloc(ctx, &A.gbnd, 3 * n)) || (st = dalloc(ctx, &A.ga_own, n)) ||
      (st = dalloc(ctx, &A.gtau_part, n)) || (st = dalloc(ctx, &A.gPp, 5 * ns)) || (st = dalloc(ctx, &A.gP, 5 * ns)) ||
      (st = dalloc(ctx, &A.gR_tr, 5 * ns)) || (st = dalloc(ctx, &A.gU_tr, 5 * ns)) || (st = dalloc(ctx, &A.gdF, 5 * ns)) ||
      (st = dalloc(ctx, &A.gl5_own, ns)) || (st = dalloc(ctx, &A.gl5_tr, ns)) || (st = dalloc(ctx, &A.gl4_own, ns)) ||
      (st = dalloc(ctx, &A.gl4_tr, ns)) || (st = dalloc(ctx, &A.gd, ns)) || (st = dalloc(ctx, &A.ga_tr, ns)) ||
      (st = dalloc(ctx, &A.gphi_tr, ns)) || (st = dalloc(ctx, &A.gtau, 2)) || (st = dalloc(ctx, &A.argmin, 2)) ||
      (st = dalloc(ctx, &A.gtau_blk, idp::kTauBlocks)) || (st = dalloc(ctx, &A.lim_slot, ns)) ||
      (st = dalloc(ctx, &A.lim_row, ns)) || (st = dalloc(ctx, &A.lim_count, 1)) || (st = dalloc(ctx, &A.lim_flag, ns)) ||
      (st = dalloc(ctx, &A.lim_gl, ns)) || (st = dalloc(ctx, &A.lim_gU, 5 * ns)) || (st = dalloc(ctx, &A.lim_gb, 3 * ns)) ||
      (st = dalloc(ctx, &ctx->a_in, 5 * n)) || (st = dalloc(ctx, &ctx->a_out, 5 * n)) ||
      (st = dalloc(ctx, &ctx->a_g, 5 * n)) || (st = dalloc(ctx, &ctx->a_acc, 5 * n)) ||
      (st = dalloc(ctx, &ctx->a_e, 5 * n)) || (st = dalloc(ctx, &ctx->a_tmp, 5 * n)))
    return st;
  // entries no kernel writes (padding slots) are read by none either; start clean
  IDP_CUDA(ctx, cudaMemset(A.gl5_own, 0, sizeof(double) * ns));
  IDP_CUDA(ctx, cudaMemset(A.gl5_tr, 0, sizeof(double) * ns));
  IDP_CUDA(ctx, cudaMemset(A.gl4_own, 0, sizeof(double) * ns));
  IDP_CUDA(ctx, cudaMemset(A.gl4_tr, 0, sizeof(double) * ns));
  ctx->has_adjoint = true;
  return IDP_OK;
}

// One euler_step in the context's precision.
int launch(idp_ctx* ctx, const double* Uin, double* Uout, const double* Un, int blend, int tau_mode, bool acc_time,
           bool skip_write_on_error, bool trace, cudaStream_t s, idp::Profiler* prof) {
  idp::GridBarrier* bar = ctx->persistent ? ctx->bar : nullptr;
  ctx->stage_ran = true;
  if (ctx->mixed)
    return idp::launch_euler_step_mixed(ctx->G, ctx->MG, ctx->B, ctx->MB, ctx->C, Uin, Uout, Un, blend, tau_mode,
                                        acc_time, skip_write_on_error, trace, s, prof, ctx->block, bar);
  return idp::launch_euler_step(ctx->G, ctx->B, ctx->C, Uin, Uout, Un, blend, tau_mode, acc_time, skip_write_on_error,
                                trace, s, prof, ctx->block, bar);
}

// dst[c n + r] = src[c n + map[r]] for the 5 fields: states between the
// caller's node order and the library's row order (idp_config.renumber).
__global__ void k_gather_rows(int64_t n, const int64_t* __restrict__ map, const double* __restrict__ src,
                              double* __restrict__ dst, int comps) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t i = map[r];
  for (int c = 0; c < comps; ++c) dst[c * n + r] = src[c * n + i];
}

// A caller-order array of `comps` fields (host or device) into library row order.
idp_status copy_in(idp_ctx* ctx, double* dst_lib, const double* src, bool on_device, int comps = 5) {
  const int64_t n = ctx->G.n;
  const size_t bytes = sizeof(double) * comps * (size_t)n;
  if (!ctx->renumbered) {
    IDP_CUDA(ctx, cudaMemcpyAsync(dst_lib, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  ctx->stream));
    return IDP_OK;
  }
  const double* from = src;
  if (!on_device) {
    IDP_CUDA(ctx, cudaMemcpyAsync(ctx->perm_buf, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    from = ctx->perm_buf;
  }
  k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, ctx->d_iperm, from, dst_lib, comps);
  IDP_CUDA(ctx, cudaGetLastError());
  return IDP_OK;
}

// A library-order 5-field array back into the caller's order (host or device).
idp_status copy_out(idp_ctx* ctx, double* dst, const double* src_lib, bool on_device) {
  const int64_t n = ctx->G.n;
  const size_t bytes = sizeof(double) * 5 * (size_t)n;
  if (!ctx->renumbered) {
    IDP_CUDA(ctx, cudaMemcpyAsync(dst, src_lib, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  ctx->stream));
    return IDP_OK;
  }
  double* to = on_device ? dst : ctx->perm_buf;
  k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, ctx->d_perm, src_lib, to, 5);
  IDP_CUDA(ctx, cudaGetLastError());
  if (!on_device) IDP_CUDA(ctx, cudaMemcpyAsync(dst, ctx->perm_buf, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return IDP_OK;
}

// Doubles of one stage's stored trace: per node the node quantities, alpha,
// U^L, the bounds, U after the first pass and the indicator sums a_i, b_i;
// per slot d, 1/(2d), P' (after the first pass), P of Step 4, the flux
// differences of Step 1, l of Step 4 and l of the first pass.
size_t snapshot_doubles(const idp_ctx* ctx) {
  const size_t n = (size_t)ctx->G.n, ns = (size_t)ctx->G.n_slots;
  return (size_t)(idp::kNodeQ + 1 + 5 + 3 + 5 + 6) * n + (size_t)(1 + 1 + 5 + 5 + 5 + 1 + 1) * ns;
}

// The stage buffers of stored trace k: the stage's own node, d, 1/(2d),
// alpha, U^L, bounds, P, flux differences and trace arrays inside rec_snap, the rest (state
// scratch, R, limiter values, status) shared with ctx->B.
idp::StageBuffers snapshot_set(const idp_ctx* ctx, int k) {
  idp::StageBuffers B = ctx->B;
  const size_t n = (size_t)ctx->G.n, ns = (size_t)ctx->G.n_slots;
  double* p = ctx->rec_snap + (size_t)k * snapshot_doubles(ctx);
  auto take = [&](double** f, size_t count) {
    *f = p;
    p += count;
  };
  take(&B.node, (size_t)idp::kNodeQ * n);
  take(&B.alpha, n);
  take(&B.UL, 5 * n);
  take(&B.bnd, 3 * n);
  take(&B.tU5, 5 * n);
  take(&B.tab, 6 * n);
  take(&B.d, ns);
  take(&B.dinv, ns);
  take(&B.P, 5 * ns);
  take(&B.tP, 5 * ns);
  take(&B.tdF, 5 * ns);
  take(&B.tl4, ns);
  take(&B.tl5, ns);
  B.Ulast = nullptr;  // the stored traces leave the last stage's output and bounds alone
  return B;
}

// One traced FP64 euler_step on explicit stage buffers (the adjoint's stored
// traces).
int launch_traced(idp_ctx* ctx, const idp::StageBuffers& B, const double* Uin, double* Uout, const double* Un,
                  int blend, int tau_mode, cudaStream_t s, idp::Profiler* prof) {
  return idp::launch_euler_step(ctx->G, B, ctx->C, Uin, Uout, Un, blend, tau_mode, false, false, true, s, prof,
                                ctx->block, nullptr);
}

// The three euler_steps of one SSP-RK3 step (eq. ssprk3) on stream s.
int64_t launch_rk3(idp_ctx* ctx, cudaStream_t s, idp::Profiler* prof) {
  idp::StageBuffers& B = ctx->B;
  int64_t n = 0;
  n += launch(ctx, B.U, B.Us, B.U, idp::kBlendNone, 0, true, false, false, s, prof);
  n += launch(ctx, B.Us, B.Us, B.U, idp::kBlendStage2, 1, false, false, false, s, prof);
  n += launch(ctx, B.Us, B.U, B.U, idp::kBlendStage3, 1, false, true, false, s, prof);
  return n;
}

// Captures one SSP-RK3 step into a CUDA graph (on a private stream; the
// legacy default stream cannot be captured) and instantiates it.
idp_status build_graph(idp_ctx* ctx) {
  drop_graph(ctx);
  if (!ctx->cap_stream) IDP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  IDP_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  ctx->graph_launches = launch_rk3(ctx, ctx->cap_stream, nullptr);
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, IDP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->graph_exec = nullptr;
    return fail(ctx, IDP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return IDP_OK;
}

// The state check of Sec. 3.3 (rho > 0, epsilon > 0, finite) of a 5n
// library-order array: fills the first five fields of *out.
idp_status check_state(idp_ctx* ctx, const double* U, idp_bounds_report* out) {
  std::memset(out, 0, sizeof(*out));
  idp::launch_check_state(U, ctx->G.n, ctx->check, ctx->check_acc, ctx->stream);
  IDP_CUDA(ctx, cudaGetLastError());
  double h[5];
  IDP_CUDA(ctx, cudaMemcpyAsync(h, ctx->check, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out->n_rho_nonpositive = (int64_t)h[0];
  out->n_eps_nonpositive = (int64_t)h[1];
  out->n_nonfinite = (int64_t)h[2];
  out->rho_min = h[3];
  out->eps_min = h[4];
  return (out->n_rho_nonpositive || out->n_eps_nonpositive || out->n_nonfinite) ? IDP_ERR_BOUNDS : IDP_OK;
}

// The local bounds of Sec. 3.9 of a library-order state against library-
// order bounds (rho_min, rho_max, phi_min): fills the local-bound fields of
// *out.  Relative slacks: FP64 1e-13 on rho and 2e-13 on Psi (the limiter
// accepts Psi down to -1e-13 of its scale, Reading A27, and the row sum of
// the accepted increments adds rounding); FP32-mixed 1e-7 and 1e-6 (the
// increments are summed in FP32 before they reach the FP64 state).
idp_status check_local(idp_ctx* ctx, const double* U, const double* bnd, idp_bounds_report* out) {
  out->slack_rho = ctx->mixed ? 1e-7 : 1e-13;
  out->slack_phi = ctx->mixed ? 1e-6 : 2e-13;
  idp::launch_check_local(U, bnd, ctx->G.n, out->slack_rho, out->slack_phi, ctx->check + 5, ctx->check_acc + 5,
                          ctx->stream);
  IDP_CUDA(ctx, cudaGetLastError());
  double h[7];
  IDP_CUDA(ctx, cudaMemcpyAsync(h, ctx->check + 5, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out->n_bound_rows = (int64_t)h[0];
  out->n_rho_below_min = (int64_t)h[1];
  out->n_rho_above_max = (int64_t)h[2];
  out->n_phi_below_min = (int64_t)h[3];
  out->rho_min_violation = h[4];
  out->rho_max_violation = h[5];
  out->phi_min_violation = h[6];
  return (out->n_rho_below_min || out->n_rho_above_max || out->n_phi_below_min) ? IDP_ERR_BOUNDS : IDP_OK;
}

}  // namespace

extern "C" {

void idp_config_default(idp_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->gamma = 1.4;
  cfg->cfl = 0.5;
  cfg->limiter_passes = 2;
  cfg->newton_max = 2;
  cfg->newton_tol = 1e-10;
  cfg->newton_eps = DBL_EPSILON;
  cfg->precision = IDP_PRECISION_FP64;
  cfg->schedule = 0;
  cfg->barrier_spin_limit = 1 << 26;
  cfg->entry_table = 1;
  cfg->adjoint_store_stages = 1;
}

const char* idp_status_string(idp_status s) {
  switch (s) {
    case IDP_OK: return "ok";
    case IDP_ERR_ARG: return "invalid argument";
    case IDP_ERR_CUDA: return "CUDA error";
    case IDP_ERR_OOM: return "out of memory";
    case IDP_ERR_STATE_NOT_ADMISSIBLE: return "state not admissible";
    case IDP_ERR_CFL: return "CFL violation";
    case IDP_ERR_NONFINITE: return "non-finite state";
    case IDP_ERR_BOUNDS: return "invariant violated";
    case IDP_ERR_TIMEOUT: return "device wait timed out";
    case IDP_ERR_STATE: return "call out of order";
  }
  return "unknown";
}

idp_status idp_create(const idp_config* cfg, void* cuda_stream, idp_ctx** out) {
  if (!out) return IDP_ERR_ARG;
  *out = nullptr;
  idp_config c;
  if (cfg) c = *cfg; else idp_config_default(&c);
  if (c.gamma != 1.4) return IDP_ERR_ARG;
  if (!(c.cfl > 0.0 && c.cfl <= 1.0) || c.limiter_passes < 1 || c.newton_max < 0) return IDP_ERR_ARG;
  if (c.precision != IDP_PRECISION_FP64 && c.precision != IDP_PRECISION_MIXED) return IDP_ERR_ARG;
  idp_ctx* ctx = new (std::nothrow) idp_ctx;
  if (!ctx) return IDP_ERR_OOM;
  ctx->cfg = c;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return IDP_ERR_CUDA;
  }
  ctx->mixed = c.precision == IDP_PRECISION_MIXED;
  ctx->C.cfl = c.cfl;
  ctx->C.limiter_passes = c.limiter_passes;
  ctx->C.lim.newton_max = c.newton_max;
  ctx->C.lim.newton_tol = c.newton_tol;
  ctx->C.lim.newton_eps = c.newton_eps;
  ctx->C.spin_limit = c.barrier_spin_limit > 0 ? (long long)c.barrier_spin_limit : (1LL << 26);
  *out = ctx;
  return IDP_OK;
}

void idp_destroy(idp_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->prof.clear();
  free_all(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

const char* idp_last_error(const idp_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

namespace {
idp_status upload_mesh(idp_ctx* ctx, int dim, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                       const double* cell_x, const int32_t* node_bc, const double* inflow_state);
idp_status upload_matrices(idp_ctx* ctx, const double* inflow_state);
}

extern "C" idp_status idp_upload_mesh_hex(idp_ctx* ctx, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                                          const double* cell_xyz, const int32_t* node_bc,
                                          const double* inflow_state) {
  return upload_mesh(ctx, 3, n_nodes, n_cells, cells, cell_xyz, node_bc, inflow_state);
}

extern "C" idp_status idp_upload_mesh_quad(idp_ctx* ctx, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                                           const double* cell_xy, const int32_t* node_bc,
                                           const double* inflow_state) {
  return upload_mesh(ctx, 2, n_nodes, n_cells, cells, cell_xy, node_bc, inflow_state);
}

extern "C" idp_status idp_upload_sparsity(idp_ctx* ctx, int64_t n_nodes, const int64_t* rowptr, const int64_t* col,
                                          const double* mij, const double* cij, const double* mi,
                                          const int32_t* node_bc, const double* inflow_state) {
  if (!ctx) return IDP_ERR_ARG;
  if (n_nodes <= 0 || !rowptr || !col || !mij || !cij) return fail(ctx, IDP_ERR_ARG, "bad sparsity arguments");
  if (rowptr[0] != 0) return fail(ctx, IDP_ERR_ARG, "rowptr[0] must be 0");
  for (int64_t i = 0; i < n_nodes; ++i) {
    if (rowptr[i + 1] < rowptr[i] + 2) return fail(ctx, IDP_ERR_ARG, "every row needs its diagonal and a neighbour");
    bool diag = false;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n_nodes) return fail(ctx, IDP_ERR_ARG, "column index out of range");
      if (k > rowptr[i] && col[k] <= col[k - 1]) return fail(ctx, IDP_ERR_ARG, "columns must increase within a row");
      diag |= col[k] == i;
    }
    if (!diag) return fail(ctx, IDP_ERR_ARG, "a row lacks its diagonal entry");
  }
  const int64_t nnz = rowptr[n_nodes];
  for (int64_t k = 0; k < nnz; ++k)
    if (!std::isfinite(mij[k]) || !std::isfinite(cij[k]) || !std::isfinite(cij[nnz + k]) ||
        !std::isfinite(cij[2 * nnz + k]))
      return fail(ctx, IDP_ERR_ARG, "non-finite matrix entry");
  if (mi)
    for (int64_t i = 0; i < n_nodes; ++i)
      if (!(mi[i] > 0.0) || !std::isfinite(mi[i])) return fail(ctx, IDP_ERR_ARG, "lumped masses must be positive");
  if (ctx->has_mesh) {
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    ctx->has_mesh = ctx->has_state = ctx->has_trace = false;
  }
  idp::HostMatrices& M = ctx->M;
  M = idp::HostMatrices{};
  M.n = n_nodes;
  M.rowptr.assign(rowptr, rowptr + n_nodes + 1);
  M.col.assign(col, col + nnz);
  M.mij.assign(mij, mij + nnz);
  for (int d = 0; d < 3; ++d) M.cij[d].assign(cij + d * nnz, cij + (d + 1) * nnz);
  if (mi) {
    M.mi.assign(mi, mi + n_nodes);
    M.lumped_given = true;
  }
  M.bc.assign(n_nodes, 0);
  if (node_bc) M.bc.assign(node_bc, node_bc + n_nodes);
  return upload_matrices(ctx, inflow_state);
}

namespace {
// Entry table of the mixed stage (idp_config.entry_table): the distinct FP32
// tuples (c_x, c_y, c_z, m_ij, |c_ij|, 1/|c_ij|) of all slots, padding
// included, compared bitwise.  Left off when there are more than
// kEntryTableMax of them.
idp_status upload_entry_table(idp_ctx* ctx, const idp::HostEntriesF& E, std::vector<uint16_t>& code) {
  const size_t ns = E.cx.size();
  std::map<std::array<uint32_t, 6>, uint16_t> index;
  code.assign(ns, 0);
  std::vector<float4> tab;
  auto bits = [](float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
  };
  for (size_t p = 0; p < ns; ++p) {
    const std::array<uint32_t, 6> key = {bits(E.cx[p]), bits(E.cy[p]), bits(E.cz[p]),
                                         bits(E.m[p]),  bits(E.cn[p]), bits(E.inv_cn[p])};
    auto it = index.find(key);
    if (it == index.end()) {
      if ((int)index.size() == idp::kEntryTableMax) {  // not a table mesh: per-entry arrays
        code.clear();
        return IDP_OK;
      }
      it = index.emplace(key, (uint16_t)index.size()).first;
      tab.push_back(make_float4(E.cx[p], E.cy[p], E.cz[p], E.m[p]));
      tab.push_back(make_float4(E.cn[p], E.inv_cn[p], 0.0f, 0.0f));
    }
    code[p] = it->second;
  }
  uint16_t* dcode;
  float4* dtab;
  idp_status st;
  if ((st = upload(ctx, &dcode, code)) || (st = upload(ctx, &dtab, tab))) return st;
  ctx->MG.ecode = dcode;
  ctx->MG.etab = dtab;
  ctx->n_entry_values = (int64_t)index.size();
  return IDP_OK;
}

// Row patterns of the mixed stage (with idp_config.entry_table): each row's
// entries as (column offset j - r, index k' of the transposed entry in row
// j, flags, entry-table code); rows with equal sequences share a pattern.
// Left off (per-slot arrays) when there are more than kRowPatternMax
// patterns or an offset or index does not fit its field.  The records are
// derived from the SELL arrays themselves, so the kernels read the same
// columns, slots, flags and codes either way.
idp_status upload_row_patterns(idp_ctx* ctx, const std::vector<uint16_t>& code) {
  const idp::SellLayout& L = ctx->L;
  const int64_t n = L.n;
  int width = 0;
  for (int64_t r = 0; r < n; ++r) width = L.row_len[r] > width ? L.row_len[r] : width;
  if (n == 0 || width == 0 || width > 255) return IDP_OK;
  struct Hash {
    size_t operator()(const std::vector<uint64_t>& v) const {
      uint64_t h = 1469598103934665603ull;  // FNV-1a over the words
      for (uint64_t w : v) h = (h ^ w) * 1099511628211ull;
      return (size_t)h;
    }
  };
  std::unordered_map<std::vector<uint64_t>, uint16_t, Hash> index;
  std::vector<uint16_t> rpat((size_t)n);
  std::vector<uint2> tab;
  std::vector<uint64_t> sig;
  for (int64_t r = 0; r < n; ++r) {
    const int len = L.row_len[r];
    const int64_t base = (int64_t)L.slice_ptr[r >> 5] + (r & 31);
    sig.assign((size_t)len, 0);
    for (int k = 0; k < len; ++k) {
      const int64_t p = base + 32 * (int64_t)k;
      const int64_t j = L.col[p];
      const int64_t rel = L.tpos[p] - ((int64_t)L.slice_ptr[j >> 5] + (j & 31));
      const int64_t dj = j - r;
      if (rel < 0 || rel % 32 != 0 || rel / 32 >= L.row_len[j] || dj < -2147483647LL || dj > 2147483647LL) return IDP_OK;
      const uint32_t y = (uint32_t)(rel / 32) | ((uint32_t)L.flags[p] << 8) | ((uint32_t)(code.empty() ? 0 : code[p]) << 16);
      sig[k] = (uint64_t)(uint32_t)(int32_t)dj | ((uint64_t)y << 32);
    }
    auto it = index.find(sig);
    if (it == index.end()) {
      if ((int)index.size() == idp::kRowPatternMax) return IDP_OK;
      it = index.emplace(sig, (uint16_t)index.size()).first;
      for (int k = 0; k < width; ++k)
        tab.push_back(k < len ? make_uint2((uint32_t)sig[k], (uint32_t)(sig[k] >> 32)) : make_uint2(0u, 0u));
    }
    rpat[(size_t)r] = it->second;
  }
  uint16_t* drp;
  uint2* dtab;
  idp_status st;
  if ((st = upload(ctx, &drp, rpat)) || (st = upload(ctx, &dtab, tab))) return st;
  if (ctx->mixed) {
    ctx->MG.rpat = drp;
    ctx->MG.ptab = dtab;
    ctx->MG.pwidth = width;
  } else {
    ctx->G.rpat = drp;
    ctx->G.ptab = dtab;
    ctx->G.pwidth = width;
  }
  ctx->n_row_patterns = (int64_t)index.size();
  return IDP_OK;
}

idp_status upload_mesh(idp_ctx* ctx, int dim, int64_t n_nodes, int64_t n_cells, const int64_t* cells,
                       const double* cell_x, const int32_t* node_bc, const double* inflow_state) {
  if (!ctx || !cells || !cell_x || n_nodes <= 0 || n_cells <= 0) return fail(ctx, IDP_ERR_ARG, "bad mesh arguments");
  if (ctx->has_mesh) {
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    ctx->has_mesh = ctx->has_state = ctx->has_trace = false;
  }
  std::string msg = dim == 3 ? idp::assemble_q1(n_nodes, n_cells, cells, cell_x, ctx->M)
                             : idp::assemble_q1_2d(n_nodes, n_cells, cells, cell_x, ctx->M);
  if (!msg.empty()) return fail(ctx, IDP_ERR_ARG, msg);
  ctx->M.lumped_given = false;
  ctx->M.bc.assign(node_bc ? node_bc : nullptr, node_bc ? node_bc + n_nodes : nullptr);
  if (!node_bc) ctx->M.bc.assign(n_nodes, 0);
  return upload_matrices(ctx, inflow_state);
}

// Sliced-ELL layout of ctx->M, device copies and stage buffers (the part of
// a mesh upload that follows the matrices).
idp_status upload_matrices(idp_ctx* ctx, const double* inflow_state) {
  idp_status st;
  std::string msg = idp::build_sell(ctx->M, ctx->L, ctx->cfg.renumber);
  if (!msg.empty()) return fail(ctx, IDP_ERR_ARG, msg);
  for (int f = 0; f < 5; ++f) ctx->C.inflow[f] = inflow_state ? inflow_state[f] : 0.0;

  const idp::SellLayout& L = ctx->L;
  idp::DeviceGraph& G = ctx->G;
  G.n = L.n;
  G.n_slots = L.n_slots;
  G.row0 = 0;
  G.row1 = L.n;
  int32_t *slice_ptr, *row_len, *col, *tpos, *bc;
  uint8_t* flags;
  double *cx, *cy, *cz, *mij, *mi, *inv_mi, *lam, *cn, *inv_cn, *csx, *csy, *csz;
  if ((st = upload(ctx, &slice_ptr, L.slice_ptr)) || (st = upload(ctx, &row_len, L.row_len)) ||
      (st = upload(ctx, &col, L.col)) || (st = upload(ctx, &tpos, L.tpos)) || (st = upload(ctx, &flags, L.flags)) ||
      (st = upload(ctx, &cx, L.cx)) || (st = upload(ctx, &cy, L.cy)) || (st = upload(ctx, &cz, L.cz)) ||
      (st = upload(ctx, &mij, L.mij)) || (st = upload(ctx, &mi, L.mi)) || (st = upload(ctx, &inv_mi, L.inv_mi)) ||
      (st = upload(ctx, &lam, L.lam)) || (st = upload(ctx, &bc, L.bc)) || (st = upload(ctx, &cn, L.cn)) ||
      (st = upload(ctx, &inv_cn, L.inv_cn)) || (st = upload(ctx, &csx, L.csx)) || (st = upload(ctx, &csy, L.csy)) ||
      (st = upload(ctx, &csz, L.csz)))
    return st;
  G.slice_ptr = slice_ptr;
  G.row_len = row_len;
  G.col = col;
  G.tpos = tpos;
  G.flags = flags;
  G.cx = cx;
  G.cy = cy;
  G.cz = cz;
  G.mij = mij;
  G.cn = cn;
  G.inv_cn = inv_cn;
  G.csx = csx;
  G.csy = csy;
  G.csz = csz;
  G.mi = mi;
  G.inv_mi = inv_mi;
  G.lam = lam;
  G.bc = bc;
  G.relax = nullptr;
  G.rpat = nullptr;
  G.ptab = nullptr;
  G.pwidth = 0;
  if (ctx->cfg.relax && (st = upload_relax(ctx, std::vector<int32_t>()))) return st;

  ctx->renumbered = ctx->cfg.renumber != 0;
  G.node_of_row = G.row_of_node = nullptr;
  if (ctx->renumbered) {
    if ((st = upload(ctx, &ctx->d_perm, L.perm)) || (st = upload(ctx, &ctx->d_iperm, L.iperm)) ||
        (st = dalloc(ctx, &ctx->perm_buf, (size_t)5 * L.n)))
      return st;
    G.node_of_row = ctx->d_iperm;
    G.row_of_node = ctx->d_perm;
  }
  idp::StageBuffers& B = ctx->B;
  const size_t n = (size_t)L.n, ns = (size_t)L.n_slots;
  B = idp::StageBuffers{};
  if ((st = dalloc(ctx, &B.U, 5 * n)) || (st = dalloc(ctx, &B.Us, 5 * n)) || (st = dalloc(ctx, &B.UL, 5 * n)) ||
      (st = dalloc(ctx, &B.bnd, 3 * n)) || (st = dalloc(ctx, &B.Uw[0], 5 * n)) || (st = dalloc(ctx, &B.Uw[1], 5 * n)) ||
      (st = dalloc(ctx, &B.scal, 1)) || (st = dalloc(ctx, &ctx->check, 12)) || (st = dalloc(ctx, &ctx->check_acc, 12)) ||
      (st = dalloc(ctx, &ctx->bar, 1)) || (st = dalloc(ctx, &B.Ulast, 5 * n)))
    return st;
  if (!ctx->mixed) {
    if ((st = dalloc(ctx, &B.node, idp::kNodeQ * n)) || (st = dalloc(ctx, &B.d, ns)) || (st = dalloc(ctx, &B.dinv, ns)) ||
        (st = dalloc(ctx, &B.alpha, n)) || (st = dalloc(ctx, &B.R, 5 * n)) || (st = dalloc(ctx, &B.P, 5 * ns)) ||
        (st = dalloc(ctx, &B.l[0], ns)) || (st = dalloc(ctx, &B.l[1], ns)))
      return st;
    // d_ij of padding slots and 1/(2 d_ii) of the diagonal are never written
    // by the kernels: the diagonal bar state U_i reads a zero there
    IDP_CUDA(ctx, cudaMemset(B.d, 0, sizeof(double) * ns));
    IDP_CUDA(ctx, cudaMemset(B.dinv, 0, sizeof(double) * ns));
    // column, transpose and flags from row patterns where the rows fall into
    // few of them (the same indices, so bitwise the same results)
    ctx->n_row_patterns = 0;
    if (ctx->cfg.entry_table && (st = upload_row_patterns(ctx, std::vector<uint16_t>()))) return st;
  } else {
    // FP32 copies of the entries.  A component of c_ij below 2^-24 of the
    // largest |c| is assembly rounding of a zero (e.g. c_x between nodes of
    // equal x on a uniform grid) and beneath FP32 resolution on the matrix's
    // scale: it becomes an exact zero.
    double cscale = 0.0;
    for (size_t p = 0; p < ns; ++p) cscale = std::fmax(cscale, L.cn[p]);
    if (ctx->c_scale > 0.0) cscale = ctx->c_scale;
    auto to_float = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    auto c_float = [&](const std::vector<double>& v) {
      std::vector<float> f(v.size());
      for (size_t p = 0; p < v.size(); ++p) f[p] = std::fabs(v[p]) < cscale * 0x1p-24 ? 0.0f : (float)v[p];
      return f;
    };
    const idp::HostEntriesF E{c_float(L.cx), c_float(L.cy), c_float(L.cz), to_float(L.mij), to_float(L.cn),
                              to_float(L.inv_cn)};
    float* fimi;
    if ((st = upload(ctx, &fimi, to_float(L.inv_mi))) != IDP_OK) return st;
    ctx->MG = idp::MixedGraph{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, fimi,
                              nullptr, nullptr, nullptr, nullptr, 0};
    ctx->n_entry_values = 0;
    ctx->n_row_patterns = 0;
    if (ctx->cfg.entry_table) {
      std::vector<uint16_t> code;
      if ((st = upload_entry_table(ctx, E, code)) || (st = upload_row_patterns(ctx, code))) return st;
    }
    if (!ctx->MG.ecode) {
      float *fcx, *fcy, *fcz, *fm, *fcn, *finv;
      if ((st = upload(ctx, &fcx, E.cx)) || (st = upload(ctx, &fcy, E.cy)) || (st = upload(ctx, &fcz, E.cz)) ||
          (st = upload(ctx, &fm, E.m)) || (st = upload(ctx, &fcn, E.cn)) || (st = upload(ctx, &finv, E.inv_cn)))
        return st;
      ctx->MG.cx = fcx;
      ctx->MG.cy = fcy;
      ctx->MG.cz = fcz;
      ctx->MG.mij = fm;
      ctx->MG.cn = fcn;
      ctx->MG.inv_cn = finv;
    }
    idp::MixedBuffers& X = ctx->MB;
    if ((st = dalloc(ctx, &X.Uf, 5 * n)) || (st = dalloc(ctx, &X.Q, idp::kNodeQ * n)) || (st = dalloc(ctx, &X.d, ns)) ||
        (st = dalloc(ctx, &X.dinv, ns)) || (st = dalloc(ctx, &X.P, 5 * ns)) || (st = dalloc(ctx, &X.l[0], ns)) ||
        (st = dalloc(ctx, &X.l[1], ns)) || (st = dalloc(ctx, &X.alpha, n)) || (st = dalloc(ctx, &X.R, 5 * n)))
      return st;
    IDP_CUDA(ctx, cudaMemset(X.d, 0, sizeof(float) * ns));
    IDP_CUDA(ctx, cudaMemset(X.dinv, 0, sizeof(float) * ns));
  }
  B.tP = B.tl4 = B.tU5 = B.tl5 = B.tUlim = B.tab = B.tdF = nullptr;
  IDP_CUDA(ctx, cudaMemset(B.scal, 0, sizeof(idp::DeviceScalars)));
  if ((st = alloc_instances(ctx, 1, std::vector<int32_t>())) != IDP_OK) return st;
  ctx->has_mesh = true;
  return IDP_OK;
}
}  // namespace

idp_status idp_mesh_info(idp_ctx* ctx, int64_t* n_nodes, int64_t* nnz) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (n_nodes) *n_nodes = ctx->M.n;
  if (nnz) *nnz = ctx->M.rowptr[ctx->M.n];
  return IDP_OK;
}

idp_status idp_entry_table_size(idp_ctx* ctx, int64_t* n_values) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (n_values) *n_values = ctx->n_entry_values;
  return IDP_OK;
}

idp_status idp_row_pattern_count(idp_ctx* ctx, int64_t* n_patterns) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (n_patterns) *n_patterns = ctx->n_row_patterns;
  return IDP_OK;
}

idp_status idp_get_matrices(idp_ctx* ctx, int64_t* rowptr, int64_t* col, double* mij, double* cij, double* mi) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  const idp::HostMatrices& M = ctx->M;
  const int64_t nnz = M.rowptr[M.n];
  if (rowptr) std::memcpy(rowptr, M.rowptr.data(), sizeof(int64_t) * (M.n + 1));
  if (col) std::memcpy(col, M.col.data(), sizeof(int64_t) * nnz);
  if (mij) std::memcpy(mij, M.mij.data(), sizeof(double) * nnz);
  if (cij)
    for (int d = 0; d < 3; ++d) std::memcpy(cij + d * nnz, M.cij[d].data(), sizeof(double) * nnz);
  if (mi)
    for (int64_t i = 0; i < M.n; ++i) mi[i] = ctx->L.mi[ctx->L.perm[i]];
  return IDP_OK;
}

idp_status idp_init_state(idp_ctx* ctx, const double* U, int on_device) {
  if (!ctx || !U) return fail(ctx, IDP_ERR_ARG, "null state");
  if (!ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  idp_status cst = copy_in(ctx, ctx->B.U, U, on_device != 0);
  if (cst != IDP_OK) return cst;
  idp_bounds_report rep;
  ctx->has_state = true;
  ctx->stage_ran = false;
  idp_status st = check_state(ctx, ctx->B.U, &rep);
  if (st == IDP_ERR_BOUNDS) {
    ctx->has_state = false;
    return fail(ctx, IDP_ERR_STATE_NOT_ADMISSIBLE, "initial state has rho <= 0, epsilon <= 0 or non-finite values");
  }
  if (st != IDP_OK) ctx->has_state = false;
  return st;
}

idp_status idp_get_state(idp_ctx* ctx, double* U, int on_device) {
  if (!ctx || !U) return fail(ctx, IDP_ERR_ARG, "null state");
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  idp_status st = copy_out(ctx, U, ctx->B.U, on_device != 0);
  if (st != IDP_OK) return st;
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return IDP_OK;
}

idp_status idp_profile(idp_ctx* ctx, int enable) {
  if (!ctx) return IDP_ERR_ARG;
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->prof.clear();
  ctx->prof.enabled = enable != 0;
  return IDP_OK;
}

idp_status idp_profile_read(idp_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return IDP_ERR_ARG;
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < IDP_N_KERNELS; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  const idp::Profiler& P = ctx->prof;
  for (size_t q = 0; q < P.kernel.size(); ++q) {
    float t = 0.0f;
    IDP_CUDA(ctx, cudaEventElapsedTime(&t, P.ev[2 * q], P.ev[2 * q + 1]));
    ms[P.kernel[q]] += t;
    launches[P.kernel[q]] += 1;
  }
  return IDP_OK;
}

idp_status idp_step(idp_ctx* ctx, int n_steps) {
  if (!ctx) return IDP_ERR_ARG;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  if (n_steps < 0) return fail(ctx, IDP_ERR_ARG, "negative step count");
  int64_t launches = 0;
  if (ctx->use_graph && !ctx->prof.enabled) {
    if (!ctx->graph_exec) {
      idp_status st = build_graph(ctx);
      if (st != IDP_OK) return st;
    }
    for (int s = 0; s < n_steps; ++s) IDP_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    launches = ctx->graph_launches * n_steps;
  } else {
    for (int s = 0; s < n_steps; ++s) launches += launch_rk3(ctx, ctx->stream, &ctx->prof);
  }
  ctx->launches = launches;
  IDP_CUDA(ctx, cudaGetLastError());
  return IDP_OK;
}

idp_status idp_euler_step(idp_ctx* ctx, double tau, int trace, double* tau_out) {
  if (!ctx) return IDP_ERR_ARG;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  idp::StageBuffers& B = ctx->B;
  if (trace) {
    idp_status st = ensure_trace(ctx);
    if (st != IDP_OK) return st;
  }
  if (tau > 0.0) {
    std::vector<double> t(ctx->G.n_inst, tau);
    IDP_CUDA(ctx, cudaMemcpy(ctx->G.tau, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice));
  }
  ctx->launches = launch(ctx, B.U, B.U, B.U, idp::kBlendNone, tau > 0.0 ? 1 : 0, false, false, trace != 0,
                         ctx->stream, &ctx->prof);
  IDP_CUDA(ctx, cudaGetLastError());
  if (tau_out) {
    IDP_CUDA(ctx, cudaMemcpyAsync(tau_out, ctx->G.tau, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  return device_status(ctx, true);
}

idp_status idp_synchronize(idp_ctx* ctx) {
  if (!ctx) return IDP_ERR_ARG;
  if (!ctx->has_mesh) {
    IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return IDP_OK;
  }
  return device_status(ctx, true);
}

idp_status idp_get_time(idp_ctx* ctx, double* t, double* last_tau) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (t) IDP_CUDA(ctx, cudaMemcpyAsync(t, ctx->G.time, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (last_tau) IDP_CUDA(ctx, cudaMemcpyAsync(last_tau, ctx->G.tau, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return IDP_OK;
}

idp_status idp_set_time(idp_ctx* ctx, double t) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<double> v(ctx->G.n_inst, t);
  IDP_CUDA(ctx, cudaMemcpy(ctx->G.time, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
  return IDP_OK;
}

idp_status idp_set_instances(idp_ctx* ctx, int64_t n_instances, const int64_t* node_offsets) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (n_instances < 1 || !node_offsets) return fail(ctx, IDP_ERR_ARG, "bad instance list");
  const int64_t n = ctx->M.n;
  if (node_offsets[0] != 0 || node_offsets[n_instances] != n)
    return fail(ctx, IDP_ERR_ARG, "instance offsets must start at 0 and end at n_nodes");
  std::vector<int32_t> of_node(n);
  for (int64_t k = 0; k < n_instances; ++k) {
    if (node_offsets[k + 1] <= node_offsets[k]) return fail(ctx, IDP_ERR_ARG, "empty or decreasing instance range");
    for (int64_t i = node_offsets[k]; i < node_offsets[k + 1]; ++i) of_node[i] = (int32_t)k;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = ctx->M.rowptr[i]; e < ctx->M.rowptr[i + 1]; ++e)
      if (of_node[ctx->M.col[e]] != of_node[i]) return fail(ctx, IDP_ERR_ARG, "a matrix entry couples two instances");
  std::vector<int32_t> of_row(n);
  for (int64_t i = 0; i < n; ++i) of_row[ctx->L.perm[i]] = of_node[i];
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->cfg.relax) {
    idp_status st = upload_relax(ctx, of_row);
    if (st != IDP_OK) return st;
  }
  return alloc_instances(ctx, n_instances, of_row);
}

idp_status idp_get_instance_times(idp_ctx* ctx, double* t, double* last_tau) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  const size_t bytes = sizeof(double) * ctx->G.n_inst;
  if (t) IDP_CUDA(ctx, cudaMemcpyAsync(t, ctx->G.time, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (last_tau) IDP_CUDA(ctx, cudaMemcpyAsync(last_tau, ctx->G.tau, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return IDP_OK;
}

idp_status idp_set_schedule(idp_ctx* ctx, int block_size, int use_graph, int persistent) {
  if (!ctx) return IDP_ERR_ARG;
  if (block_size != 64 && block_size != 128 && block_size != 256) return fail(ctx, IDP_ERR_ARG, "block size");
  if (block_size != ctx->block || (persistent != 0) != ctx->persistent) drop_graph(ctx);
  ctx->block = block_size;
  ctx->use_graph = use_graph != 0;
  ctx->persistent = persistent != 0;
  return IDP_OK;
}

idp_status idp_autotune(idp_ctx* ctx, int steps, int* block_size, int* use_graph, int* persistent,
                        double* ms_per_step) {
  if (!ctx) return IDP_ERR_ARG;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  if (steps < 1) return fail(ctx, IDP_ERR_ARG, "steps");
  const size_t n = (size_t)ctx->G.n, ni = (size_t)ctx->G.n_inst;
  // the trial steps advance the state: keep U and the instance clocks
  std::vector<double> U0(5 * n), t0(ni), tau0(ni);
  IDP_CUDA(ctx, cudaMemcpyAsync(U0.data(), ctx->B.U, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, ctx->stream));
  idp_status st = idp_get_instance_times(ctx, t0.data(), tau0.data());
  if (st != IDP_OK) return st;
  const int blocks[3] = {64, 128, 256};
  double best = 1e300;
  int best_b = ctx->block, best_g = ctx->use_graph ? 1 : 0, best_p = ctx->persistent ? 1 : 0;
  cudaEvent_t a, b;
  IDP_CUDA(ctx, cudaEventCreate(&a));
  IDP_CUDA(ctx, cudaEventCreate(&b));
  for (int pers = 0; pers < 2 && st == IDP_OK; ++pers)
    for (int g = 0; g < 2 && st == IDP_OK; ++g)
      for (int q = 0; q < 3 && st == IDP_OK; ++q) {
        if ((st = idp_set_schedule(ctx, blocks[q], g, pers))) break;
        // a schedule this device or driver cannot run (e.g. a cooperative
        // launch in a captured graph) is skipped, not fatal
        idp_status trial = idp_step(ctx, 1);  // warm-up (and graph capture)
        float ms = -1.0f;
        if (trial == IDP_OK) {
          IDP_CUDA(ctx, cudaEventRecord(a, ctx->stream));
          trial = idp_step(ctx, steps);
          IDP_CUDA(ctx, cudaEventRecord(b, ctx->stream));
          if (trial == IDP_OK) {
            IDP_CUDA(ctx, cudaEventSynchronize(b));
            IDP_CUDA(ctx, cudaEventElapsedTime(&ms, a, b));
          }
        }
        if (trial == IDP_ERR_CUDA) {
          cudaGetLastError();
          drop_graph(ctx);
        } else if (trial != IDP_OK) {
          st = trial;
          break;
        }
        if (ms >= 0.0f && ms / steps < best) {
          best = ms / steps;
          best_b = blocks[q];
          best_g = g;
          best_p = pers;
        }
        IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        IDP_CUDA(ctx, cudaMemcpyAsync(ctx->B.U, U0.data(), sizeof(double) * 5 * n, cudaMemcpyHostToDevice, ctx->stream));
        IDP_CUDA(ctx, cudaMemcpyAsync(ctx->G.time, t0.data(), sizeof(double) * ni, cudaMemcpyHostToDevice, ctx->stream));
        IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != IDP_OK) return st;
  if (best >= 1e300) return fail(ctx, IDP_ERR_CUDA, "no schedule ran");
  if ((st = idp_set_schedule(ctx, best_b, best_g, best_p))) return st;
  if (block_size) *block_size = best_b;
  if (use_graph) *use_graph = best_g;
  if (persistent) *persistent = best_p;
  if (ms_per_step) *ms_per_step = best;
  return device_status(ctx, true);
}

idp_status idp_get_field(idp_ctx* ctx, int which, double* out) {
  if (!ctx || !out) return IDP_ERR_ARG;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  const idp::SellLayout& L = ctx->L;
  const idp::StageBuffers& B = ctx->B;
  const int64_t n = L.n, ns = L.n_slots, nnz = (int64_t)L.slot_of_entry.size();
  auto node_field = [&](const double* src, int comps) -> idp_status {
    std::vector<double> h((size_t)comps * n);
    IDP_CUDA(ctx, cudaMemcpyAsync(h.data(), src, sizeof(double) * comps * n, cudaMemcpyDeviceToHost, ctx->stream));
    IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < comps; ++c)
      for (int64_t i = 0; i < n; ++i) out[c * n + i] = h[c * n + L.perm[i]];
    return IDP_OK;
  };
  auto slot_field = [&](const double* src, int comps) -> idp_status {
    std::vector<double> h((size_t)comps * ns);
    IDP_CUDA(ctx, cudaMemcpyAsync(h.data(), src, sizeof(double) * comps * ns, cudaMemcpyDeviceToHost, ctx->stream));
    IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < comps; ++c)
      for (int64_t e = 0; e < nnz; ++e) out[c * nnz + e] = h[c * ns + L.slot_of_entry[e]];
    return IDP_OK;
  };
  auto node_field_f = [&](const float* src, int comps) -> idp_status {
    std::vector<float> h((size_t)comps * n);
    IDP_CUDA(ctx, cudaMemcpyAsync(h.data(), src, sizeof(float) * comps * n, cudaMemcpyDeviceToHost, ctx->stream));
    IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < comps; ++c)
      for (int64_t i = 0; i < n; ++i) out[c * n + i] = h[c * n + L.perm[i]];
    return IDP_OK;
  };
  auto slot_field_f = [&](const float* src, int comps) -> idp_status {
    std::vector<float> h((size_t)comps * ns);
    IDP_CUDA(ctx, cudaMemcpyAsync(h.data(), src, sizeof(float) * comps * ns, cudaMemcpyDeviceToHost, ctx->stream));
    IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < comps; ++c)
      for (int64_t e = 0; e < nnz; ++e) out[c * nnz + e] = h[c * ns + L.slot_of_entry[e]];
    return IDP_OK;
  };
  const bool traced = ctx->has_trace;
  if (ctx->mixed) {
    switch (which) {
      case IDP_FIELD_D: return slot_field_f(ctx->MB.d, 1);
      case IDP_FIELD_ALPHA: return node_field_f(ctx->MB.alpha, 1);
      case IDP_FIELD_R: return node_field_f(ctx->MB.R, 5);
      case IDP_FIELD_P:
      case IDP_FIELD_L4:
      case IDP_FIELD_L5: return fail(ctx, IDP_ERR_STATE, "field not kept in the mixed precision mode");
      default: break;
    }
  }
  switch (which) {
    case IDP_FIELD_D: return slot_field(B.d, 1);
    case IDP_FIELD_ALPHA: return node_field(B.alpha, 1);
    case IDP_FIELD_UL: return node_field(B.UL, 5);
    case IDP_FIELD_R: return node_field(B.R, 5);
    case IDP_FIELD_BOUNDS: return node_field(B.bnd, 3);
    case IDP_FIELD_P: return traced ? slot_field(B.tP, 5) : fail(ctx, IDP_ERR_STATE, "no traced stage");
    case IDP_FIELD_L4: return traced ? slot_field(B.tl4, 1) : fail(ctx, IDP_ERR_STATE, "no traced stage");
    case IDP_FIELD_U5: return traced ? node_field(B.tU5, 5) : fail(ctx, IDP_ERR_STATE, "no traced stage");
    case IDP_FIELD_L5: return traced ? slot_field(B.tl5, 1) : fail(ctx, IDP_ERR_STATE, "no traced stage");
    case IDP_FIELD_ULIM: return traced ? node_field(B.tUlim, 5) : fail(ctx, IDP_ERR_STATE, "no traced stage");
    case IDP_FIELD_TAU_MAX: {
      IDP_CUDA(ctx, cudaMemcpyAsync(out, ctx->G.tau_max, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      return IDP_OK;
    }
  }
  return fail(ctx, IDP_ERR_ARG, "unknown field");
}

idp_status idp_check_bounds(idp_ctx* ctx, idp_bounds_report* out) {
  if (!ctx || !out) return IDP_ERR_ARG;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  idp_status st = check_state(ctx, ctx->B.U, out);
  if (st != IDP_OK && st != IDP_ERR_BOUNDS) return st;
  const idp_status sl = ctx->stage_ran ? check_local(ctx, ctx->B.Ulast, ctx->B.bnd, out) : IDP_OK;
  if (sl != IDP_OK && sl != IDP_ERR_BOUNDS) return sl;
  if (st == IDP_ERR_BOUNDS || sl == IDP_ERR_BOUNDS)
    return fail(ctx, IDP_ERR_BOUNDS, st == IDP_ERR_BOUNDS ? "state violates rho > 0, epsilon > 0 or finiteness"
                                                          : "the last stage's output violates its local bounds");
  return IDP_OK;
}

idp_status idp_check_local_bounds(idp_ctx* ctx, const double* U, const double* bounds, int on_device,
                                  idp_bounds_report* out) {
  if (!ctx || !U || !bounds || !out) return fail(ctx, IDP_ERR_ARG, "null argument");
  if (!ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  // scratch: the limiter passes' state buffers, rewritten by every stage
  double* Uc = ctx->B.Uw[0];
  double* bc = ctx->B.Uw[1];
  idp_status st;
  if ((st = copy_in(ctx, Uc, U, on_device != 0)) != IDP_OK || (st = copy_in(ctx, bc, bounds, on_device != 0, 3)) != IDP_OK)
    return st;
  st = check_state(ctx, Uc, out);
  if (st != IDP_OK && st != IDP_ERR_BOUNDS) return st;
  const idp_status sl = check_local(ctx, Uc, bc, out);
  if (sl != IDP_OK && sl != IDP_ERR_BOUNDS) return sl;
  if (st == IDP_ERR_BOUNDS || sl == IDP_ERR_BOUNDS) return fail(ctx, IDP_ERR_BOUNDS, "bounds violated");
  return IDP_OK;
}

int64_t idp_launch_count(const idp_ctx* ctx) { return ctx ? ctx->launches : 0; }

idp_status idp_barrier_selftest(idp_ctx* ctx, int blocks, int rounds, int skip_block0, long long spin_limit,
                                int* passes) {
  if (!ctx || !ctx->has_mesh) return fail(ctx, IDP_ERR_STATE, "no mesh");
  if (blocks < 1 || rounds < 0 || spin_limit < 0) return fail(ctx, IDP_ERR_ARG, "bad self-test arguments");
  unsigned int* d_passes = reinterpret_cast<unsigned int*>(ctx->check_acc);  // scratch word
  IDP_CUDA(ctx, idp::launch_barrier_selftest(ctx->bar, spin_limit, blocks, rounds, skip_block0 ? 1 : 0, d_passes,
                                             ctx->B.scal, ctx->stream));
  unsigned int h = 0;
  IDP_CUDA(ctx, cudaMemcpyAsync(&h, d_passes, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  idp_status st = device_status(ctx, true);
  if (passes) *passes = (int)h;
  return st;
}

idp_status idp_adjoint_euler_step(idp_ctx* ctx, const double* U, double tau, const double* gE, double* gU,
                                  double* g_tau, int on_device) {
  if (!ctx || !U || !gE || !gU) return fail(ctx, IDP_ERR_ARG, "null argument");
  idp_status st = adjoint_supported(ctx);
  if (st != IDP_OK || (st = ensure_adjoint(ctx)) != IDP_OK) return st;
  cudaStream_t s = ctx->stream;
  if ((st = copy_in(ctx, ctx->a_in, U, on_device != 0)) != IDP_OK || (st = copy_in(ctx, ctx->a_e, gE, on_device != 0)) != IDP_OK)
    return st;
  if (tau > 0.0) IDP_CUDA(ctx, cudaMemcpyAsync(ctx->G.tau, &tau, sizeof(double), cudaMemcpyHostToDevice, s));
  IDP_CUDA(ctx, cudaMemsetAsync(ctx->A.gtau, 0, 2 * sizeof(double), s));
  int64_t launches = launch(ctx, ctx->a_in, ctx->a_out, ctx->a_in, idp::kBlendNone, tau > 0.0 ? 1 : 0, false, false,
                            true, s, &ctx->prof);
  launches += idp::launch_adjoint_stage(ctx->G, ctx->B, ctx->A, ctx->C, ctx->a_in, ctx->a_e, ctx->a_tmp, !(tau > 0.0), s,
                                        &ctx->prof);
  ctx->launches = launches;
  IDP_CUDA(ctx, cudaGetLastError());
  if ((st = copy_out(ctx, gU, ctx->a_tmp, on_device != 0)) != IDP_OK) return st;
  double gt = 0.0;
  IDP_CUDA(ctx, cudaMemcpyAsync(&gt, ctx->A.gtau, sizeof(double), cudaMemcpyDeviceToHost, s));
  st = device_status(ctx, true);  // synchronises the stream
  if (g_tau) *g_tau = gt;
  return st;
}

idp_status idp_adjoint_record(idp_ctx* ctx, int n_steps, int checkpoint_every) {
  if (!ctx) return IDP_ERR_ARG;
  idp_status st = adjoint_supported(ctx);
  if (st != IDP_OK) return st;
  if (!ctx->has_state) return fail(ctx, IDP_ERR_STATE, "no state");
  if (n_steps < 1 || checkpoint_every < 1) return fail(ctx, IDP_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
  if (checkpoint_every > n_steps) checkpoint_every = n_steps;
  IDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  free_record(ctx);
  const size_t n5 = (size_t)5 * ctx->G.n;
  const size_t n_ckpt = (size_t)((n_steps + checkpoint_every - 1) / checkpoint_every);
  auto get = [&](double** p, size_t count) -> idp_status {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(double) * count);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, IDP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->rec_allocs.push_back(q);
    *p = static_cast<double*>(q);
    return IDP_OK;
  };
  if ((st = get(&ctx->rec_ckpt, n_ckpt * n5)) || (st = get(&ctx->rec_tau, (size_t)n_steps)) ||
      (st = get(&ctx->rec_seg, (size_t)3 * checkpoint_every * n5))) {
    free_record(ctx);
    return st;
  }
  if (ctx->cfg.adjoint_store_stages) {
    // traces of the segment's 3 x checkpoint_every stages, if they fit with 4 GiB to spare
    const size_t want = sizeof(double) * snapshot_doubles(ctx) * (size_t)(3 * checkpoint_every);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b > want + ((size_t)4 << 30)) {
      void* q = nullptr;
      if (cudaMalloc(&q, want) == cudaSuccess) {
        ctx->rec_allocs.push_back(q);
        ctx->rec_snap = static_cast<double*>(q);
        // d and 1/(2d) of padding slots and of the diagonal are never written
        IDP_CUDA(ctx, cudaMemsetAsync(q, 0, want, ctx->stream));
      } else {
        cudaGetLastError();
      }
    }
  }
  cudaStream_t s = ctx->stream;
  int64_t launches = 0;
  for (int q = 0; q < n_steps; ++q) {
    if (q % checkpoint_every == 0)
      IDP_CUDA(ctx, cudaMemcpyAsync(ctx->rec_ckpt + (size_t)(q / checkpoint_every) * n5, ctx->B.U,
                                    sizeof(double) * n5, cudaMemcpyDeviceToDevice, s));
    launches += launch_rk3(ctx, s, &ctx->prof);
    IDP_CUDA(ctx, cudaMemcpyAsync(ctx->rec_tau + q, ctx->G.tau, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  ctx->launches = launches;
  IDP_CUDA(ctx, cudaGetLastError());
  ctx->rec_steps = n_steps;
  ctx->rec_every = checkpoint_every;
  return device_status(ctx, true);
}

idp_status idp_adjoint_backward(idp_ctx* ctx, const double* gU_final, double* gU_initial, int on_device) {
  if (!ctx || !gU_final || !gU_initial) return fail(ctx, IDP_ERR_ARG, "null argument");
  idp_status st = adjoint_supported(ctx);
  if (st != IDP_OK) return st;
  if (ctx->rec_steps < 1) return fail(ctx, IDP_ERR_STATE, "no recorded forward run");
  if ((st = ensure_adjoint(ctx)) != IDP_OK) return st;
  cudaStream_t s = ctx->stream;
  const idp::DeviceGraph& G = ctx->G;
  const idp::StageBuffers& B = ctx->B;
  const size_t n5 = (size_t)5 * G.n, bytes = sizeof(double) * n5;
  const int n_steps = ctx->rec_steps, every = ctx->rec_every;
  const int n_ckpt = (n_steps + every - 1) / every;
  double* g = ctx->a_g;     // adjoint of the current step's output
  double* acc = ctx->a_acc; // adjoint of U^n through the RK blends
  double* gE = ctx->a_e;
  double* tmp = ctx->a_tmp;
  double* scr = ctx->a_out;
  auto U0 = [&](int q) { return ctx->rec_seg + (size_t)(3 * q) * n5; };
  auto U1 = [&](int q) { return ctx->rec_seg + (size_t)(3 * q + 1) * n5; };
  auto U2 = [&](int q) { return ctx->rec_seg + (size_t)(3 * q + 2) * n5; };
  if ((st = copy_in(ctx, g, gU_final, on_device != 0)) != IDP_OK) return st;
  int64_t launches = 0;
  const bool stored = ctx->rec_snap != nullptr;
  for (int c = n_ckpt - 1; c >= 0; --c) {
    const int first = c * every;
    const int len = n_steps - first < every ? n_steps - first : every;
    // recompute the segment's step inputs and first two stage states (with
    // stored traces: every stage traced into its own buffers, once)
    IDP_CUDA(ctx, cudaMemcpyAsync(U0(0), ctx->rec_ckpt + (size_t)c * n5, bytes, cudaMemcpyDeviceToDevice, s));
    for (int q = 0; q < len; ++q) {
      if (stored) {
        launches += launch_traced(ctx, snapshot_set(ctx, 3 * q), U0(q), U1(q), U0(q), idp::kBlendNone, 0, s,
                                  &ctx->prof);
        launches += launch_traced(ctx, snapshot_set(ctx, 3 * q + 1), U1(q), U2(q), U0(q), idp::kBlendStage2, 1, s,
                                  &ctx->prof);
        launches += launch_traced(ctx, snapshot_set(ctx, 3 * q + 2), U2(q), q + 1 < len ? U0(q + 1) : scr, U0(q),
                                  idp::kBlendStage3, 1, s, &ctx->prof);
        continue;
      }
      launches += launch(ctx, U0(q), U1(q), U0(q), idp::kBlendNone, 0, false, false, false, s, &ctx->prof);
      launches += launch(ctx, U1(q), U2(q), U0(q), idp::kBlendStage2, 1, false, false, false, s, &ctx->prof);
      if (q + 1 < len)
        launches += launch(ctx, U2(q), U0(q + 1), U0(q), idp::kBlendStage3, 1, false, false, false, s, &ctx->prof);
    }
    for (int q = len - 1; q >= 0; --q) {
      IDP_CUDA(ctx, cudaMemcpyAsync(G.tau, ctx->rec_tau + first + q, sizeof(double), cudaMemcpyDeviceToDevice, s));
      IDP_CUDA(ctx, cudaMemsetAsync(ctx->A.gtau, 0, 2 * sizeof(double), s));
      const idp::StageBuffers B1 = stored ? snapshot_set(ctx, 3 * q) : B;
      const idp::StageBuffers B2 = stored ? snapshot_set(ctx, 3 * q + 1) : B;
      const idp::StageBuffers B3 = stored ? snapshot_set(ctx, 3 * q + 2) : B;
      // stage 3: U^{n+1} = U^n/3 + 2/3 E(U2)
      if (!stored) launches += launch(ctx, U2(q), scr, U2(q), idp::kBlendNone, 1, false, false, true, s, &ctx->prof);
      idp::launch_axpby(gE, 2.0 / 3.0, g, 0.0, nullptr, (int64_t)n5, s);
      idp::launch_axpby(acc, 1.0 / 3.0, g, 0.0, nullptr, (int64_t)n5, s);
      launches += idp::launch_adjoint_stage(G, B3, ctx->A, ctx->C, U2(q), gE, tmp, false, s, &ctx->prof);
      // stage 2: U2 = 3/4 U^n + 1/4 E(U1)
      if (!stored) launches += launch(ctx, U1(q), scr, U1(q), idp::kBlendNone, 1, false, false, true, s, &ctx->prof);
      idp::launch_axpby(gE, 0.25, tmp, 0.0, nullptr, (int64_t)n5, s);
      idp::launch_axpby(acc, 0.75, tmp, 1.0, acc, (int64_t)n5, s);
      launches += idp::launch_adjoint_stage(G, B2, ctx->A, ctx->C, U1(q), gE, tmp, false, s, &ctx->prof);
      // stage 1: U1 = E(U^n), tau_n computed here
      if (!stored) launches += launch(ctx, U0(q), scr, U0(q), idp::kBlendNone, 0, false, false, true, s, &ctx->prof);
      launches += idp::launch_adjoint_stage(G, B1, ctx->A, ctx->C, U0(q), tmp, gE, true, s, &ctx->prof);
      idp::launch_axpby(g, 1.0, gE, 1.0, acc, (int64_t)n5, s);
      launches += 5;  // the blends
    }
  }
  IDP_CUDA(ctx, cudaMemcpyAsync(G.tau, ctx->rec_tau + n_steps - 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
  IDP_CUDA(ctx, cudaGetLastError());
  if ((st = copy_out(ctx, gU_initial, g, on_device != 0)) != IDP_OK) return st;
  ctx->launches = launches;
  return device_status(ctx, true);
}

}  // extern "C"
