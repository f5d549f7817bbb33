// Device-side data of one context and the stage launcher.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "idp_device.cuh"
#include "idp_internal.h"

namespace idp {

// Read-only graph: sliced-ELL matrices (slot = slice_ptr[r/32] + 32 k + r%32)
// and per-row data, in the library's row order.
struct DeviceGraph {
  int64_t n;
  int64_t n_slots;
  // Rows that the per-step kernels of Steps 2-6 compute: [row0, row1), all
  // rows unless the context is a shard (whose ghost rows need Steps 0-1 only)
  int64_t row0, row1;
  const int32_t* slice_ptr;
  const int32_t* row_len;
  const int32_t* col;
  const int32_t* tpos;
  const uint8_t* flags;
  const double* cx;
  const double* cy;
  const double* cz;
  const double* mij;
  const double* cn;      // |c_ij|
  const double* inv_cn;  // 1/|c_ij|
  const double* csx;     // row sums of c_ij
  const double* csy;
  const double* csz;
  const double* mi;
  const double* inv_mi;
  const double* lam;
  const int32_t* bc;
  const double* relax;  // per-row bound relaxation r_i, or nullptr (off)
  // Row patterns of the FP64 stage (nullptr: the col, tpos and flags streams):
  // rows whose entries k have the same column offset j - r, the same index k'
  // of the transposed entry in row j and the same flags share a pattern; rpat[r]
  // is row r's and ptab[rpat[r] * pwidth + k] holds entry k as (j - r, k' |
  // flags << 8).  Built at upload when the mesh has at most 4096 patterns.
  const uint16_t* rpat;
  const uint2* ptab;
  int pwidth;
  // Row order (idp_config.renumber): caller node of each row and row of each
  // caller node, or nullptr for the caller's order.  Read where a result
  // depends on the order of rows (the adjoint's fixed-order sum of the tau
  // adjoint and its CFL arg-min tie rule), so that it is the same either way.
  const int64_t* node_of_row;
  const int64_t* row_of_node;
  // Independent instances (node ranges without entries between them): each
  // has its own tau_n and time.  inst[r] is the instance of row r (nullptr:
  // one instance).  The per-instance arrays below are device state written
  // by the kernels, not part of the read-only graph.
  int64_t n_inst;
  const int32_t* inst;
  double* tau;                   // tau_n of the current RK step
  double* time;                  // accumulated simulated time
  double* tau_max;               // min_i m_i / (-2 d_ii) of the last stage
  unsigned long long* tau_min;   // atomicMin accumulator (bits of positive doubles)
};

__device__ __forceinline__ int instance_of(const DeviceGraph& G, int64_t r) { return G.inst ? G.inst[r] : 0; }

// Column, transposed slot and flags of entry k (slot p) of row r, from the
// row's pattern or from the per-slot streams.
struct Slot64 {
  int64_t j;
  int64_t pt;
  unsigned int fl;
};

__device__ __forceinline__ const uint2* row_pattern64(const DeviceGraph& G, int64_t r) {
  return G.rpat ? G.ptab + (int64_t)G.rpat[r] * G.pwidth : nullptr;
}

__device__ __forceinline__ Slot64 slot64(const DeviceGraph& G, const uint2* pat, int64_t r, int k, int64_t p) {
  Slot64 e;
  if (pat) {
    const uint2 w = __ldg(&pat[k]);
    e.j = r + (int32_t)w.x;
    e.pt = (int64_t)G.slice_ptr[e.j >> 5] + (e.j & 31) + 32 * (int64_t)(w.y & 0xffu);
    e.fl = (w.y >> 8) & 0xffu;
  } else {
    e.j = G.col[p];
    e.pt = G.tpos[p];
    e.fl = G.flags[p];
  }
  return e;
}

// Rows of the per-step kernels of Steps 2-6: [row0, row1), launched from the
// start of row0's slice so that a warp's rows share one slice.
__device__ __forceinline__ int64_t row_start(const DeviceGraph& G) { return G.row0 & ~(int64_t)(kSlice - 1); }
__device__ __forceinline__ bool computes_row(const DeviceGraph& G, int64_t r) { return r >= G.row0 && r < G.row1; }

// Device status bits latched by the kernels.
enum : int {
  kStatusNotAdmissible = 1,
  kStatusCfl = 2,
  kStatusNonFinite = 4,
  kStatusTimeout = 8
};

// Device scalars of a context.
struct DeviceScalars {
  int status;
};

// Work buffers of the stage (all device memory owned by the context).
struct StageBuffers {
  double* U;     // U^n, 5n
  double* Us;    // RK stage state, 5n
  double* node;  // kNodeQ * n
  double* d;     // n_slots
  double* dinv;  // n_slots: 1/(2 d_ij)
  double* alpha; // n
  double* UL;    // 5n
  double* R;     // 5n
  double* bnd;   // 3n
  double* P;     // 5 * n_slots (holds (f_j - f_i).c_ij from Step 1 to Step 3)
  double* l[2];  // n_slots each
  double* Uw[2]; // 5n each
  double* Ulast; // 5n: output of the last stage after its last limiter pass, before boundary values and
                 // the RK blend (what the local bounds of that stage constrain); nullptr: not kept
  DeviceScalars* scal;
  // trace copies (allocated on first traced stage)
  double* tP;
  double* tl4;
  double* tU5;
  double* tl5;
  double* tUlim;
  double* tab;  // 6n: a_i and b_i (5) of the indicator, as Step 2 formed them
  double* tdF;  // 5 n_slots: (f_j - f_i).c_ij of Step 1 (a traced stage keeps them here instead of in P)
};

struct StageConfig {
  double cfl;
  int limiter_passes;
  LimiterParams lim;
  double inflow[5];
  long long spin_limit;  // bound on the polls of a grid-barrier wait
};

enum Blend : int { kBlendNone = 0, kBlendStage2 = 1, kBlendStage3 = 2 };

// Largest block size the stage kernels are compiled for.
constexpr int kMaxBlock = 256;

// tau of row r's instance: c_cfl times the CFL bound in the first RK stage,
// the stored tau_n in the later ones.
// (The reduction word is read through L2: in a persistent launch other
// blocks updated it with atomics after this block may have touched it.)
__device__ __forceinline__ double stage_tau(const DeviceGraph& G, int ins, int tau_mode, double cfl) {
  return tau_mode == 0 ? cfl * __longlong_as_double((long long)__ldcg(&G.tau_min[ins])) : G.tau[ins];
}

// Thread r < n_inst keeps instance r's books after the CFL reduction: the
// bound, tau_n and the time in the first stage, the CFL check in the others.
__device__ __forceinline__ void instance_books(const DeviceGraph& G, int64_t r, int tau_mode, double cfl,
                                               int accumulate_time, DeviceScalars* scal) {
  if (r >= G.n_inst) return;
  const double tmax = __longlong_as_double((long long)__ldcg(&G.tau_min[r]));
  G.tau_max[r] = tmax;
  if (tau_mode == 0) {
    const double tau = cfl * tmax;
    G.tau[r] = tau;
    if (accumulate_time) G.time[r] += tau;
  } else if (G.tau[r] > tmax) {
    atomicOr(&scal->status, kStatusCfl);
  }
}

// min-reduction of the CFL candidates into their instances' accumulators:
// one atomic per warp when the warp's rows share an instance.
__device__ __forceinline__ void reduce_tau_candidate(const DeviceGraph& G, int64_t r, double cand) {
  const bool valid = r < G.n;
  const int ins = valid ? instance_of(G, r) : -1;
  const int ins0 = __shfl_sync(0xffffffffu, ins, 0);
  const bool uniform = __all_sync(0xffffffffu, !valid || ins == ins0);
  if (uniform) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cand = fmin(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    if ((threadIdx.x & 31) == 0 && ins0 >= 0 && cand < INFINITY)
      atomicMin(&G.tau_min[ins0], (unsigned long long)__double_as_longlong(cand));
  } else if (valid && cand < INFINITY) {
    atomicMin(&G.tau_min[ins], (unsigned long long)__double_as_longlong(cand));
  }
}

// Grid-wide barrier of a cooperative (co-resident) launch.  Thread 0 of each
// block arrives on a counter in device memory; the last arrival resets it
// and advances the generation, the others poll the generation at most
// spin_limit times.  A wait that runs out sets the abort flag and
// kStatusTimeout; every block then leaves at its next barrier.  Returns
// false once the launch is aborted.  count and abort start at zero.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int abort;
  unsigned int tile[12];  // next row tile of each phase (dynamic work list)
};

__device__ __forceinline__ bool grid_barrier(GridBarrier* b, long long spin_limit, DeviceScalars* scal) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &b->gen;
    volatile int* vabort = &b->abort;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long polls = 0;
      while (*vgen == g) {
        if (*vabort || ++polls > spin_limit) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!ok && !*vabort) {
      atomicExch(&b->abort, 1);
      atomicOr(&scal->status, kStatusTimeout);
    }
    __threadfence();
    s_go = ok && !*vabort;
  }
  __syncthreads();
  return s_go != 0;
}

// Dynamic work list of a persistent phase: each warp takes the next tile of
// 32 rows (one sliced-ELL slice) from the phase's counter until none are
// left, so blocks that drew cheap rows take more tiles.  f(r) is called by
// all 32 lanes of the warp, also for r >= n (padding rows of the last tile).
template <typename F>
__device__ __forceinline__ void for_each_row_tile(unsigned int* counter, int64_t n, F&& f) {
  const int64_t tiles = (n + 31) >> 5;
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= tiles) break;
    f(((int64_t)t << 5) + lane);
  }
}

// Arguments of the persistent (one launch per euler_step) kernel.
struct PersistentStage {
  DeviceGraph G;
  StageConfig C;
  StageBuffers B;
  const double* Uin;
  double* Uout;
  const double* Un;
  GridBarrier* bar;
  int blend, tau_mode, accumulate_time, skip_write_on_error;
};

// Kernel ids of one euler_step (also the order of idp_profile_read).
enum KernelId : int {
  kKNode = 0,
  kKEdge,
  kKDiag,
  kKLowOrder,
  kKFluxLimit,
  kKLimiterPass,
  kKFinal,
  // reverse mode
  kKAdjFinal,
  kKAdjPass,
  kKAdjFlux,
  kKAdjLow,
  kKAdjTau,
  kKAdjDiag,
  kKAdjEdge,
  kKAdjGather,
  kNumKernels
};

// Optional per-kernel timing: CUDA events recorded on the launch stream
// around each kernel; read back (and synchronised) by the owner.
struct Profiler {
  bool enabled = false;
  std::vector<cudaEvent_t> ev;     // begin/end pairs
  std::vector<int> kernel;         // kernel id per pair
  cudaEvent_t take();
  void begin(int id, cudaStream_t s);
  void end(cudaStream_t s);
  void clear();
};

// Enqueues one euler_step (Alg. 1) on stream s:
//   Uin -> Uout with boundary post-processing and the RK blend with Un.
// tau_mode 0: tau = c_cfl min m_i/(-2 d_ii) is computed and stored (stage 1);
// tau_mode 1: the stored tau is used and checked (stages 2, 3, fixed tau).
// accumulate_time adds tau to the simulated time (once per RK step).
// Returns the number of kernel launches.
// persistent (with bar, device memory): the whole euler_step as one
// cooperative launch of k_stage_persistent (not with trace or profiling,
// which take the per-step kernels).
int launch_euler_step(const DeviceGraph& G, const StageBuffers& B, const StageConfig& C, const double* Uin,
                      double* Uout, const double* Un, int blend, int tau_mode, bool accumulate_time,
                      bool skip_write_on_error, bool trace, cudaStream_t s, Profiler* prof = nullptr,
                      int block = 128, GridBarrier* bar = nullptr);

// One euler_step in phases, for a caller that interleaves the phases of
// several contexts (the sharded stage) and exchanges, between two phases, the
// values that the next phase reads at rows of other shards:
//   phase 0             Steps 0-2: node quantities, d_ij, alpha_i, CFL bound
//                       (then: alpha_j and the tau reduction)
//   phase 1             Step 3: U^L, R_i, bounds (then: R_j)
//   phase 2             Step 4: P_ij, l_ij (then: l_ji, in phase_l_buffer)
//   phase 2 + p         limiter pass p = 1 .. passes-1 of Step 5 (then: l_ji)
//   phase 2 + passes    Step 6: last pass, boundary values, RK blend (then: U)
// The kernels and arguments are those of launch_euler_step's per-step
// schedule.  Returns the number of launches.
int euler_phase_count(const StageConfig& C);
int launch_euler_phase(const DeviceGraph& G, const StageBuffers& B, const StageConfig& C, const double* Uin,
                       double* Uout, const double* Un, int blend, int tau_mode, bool accumulate_time,
                       bool skip_write_on_error, int phase, cudaStream_t s, int block);
// The limiter-value buffer that phase 2 + p (p >= 0) writes.
double* phase_l_buffer(const StageBuffers& B, int phase);
// Own-row grid of Steps 2-6 ([row0, row1) from the start of row0's slice,
// at least n_inst threads for the instance books).
inline unsigned own_row_grid(const DeviceGraph& G, int block) {
  int64_t own = G.row1 - (G.row0 & ~(int64_t)(kSlice - 1));
  if (own < G.n_inst) own = G.n_inst;
  return (unsigned)((own + block - 1) / block);
}

// Blocks of the persistent stage kernel that fit on the device at once.
int persistent_grid_limit(int block, bool mixed);
// The FP32-mixed persistent stage kernel (idp_mixed.cu).
const void* persistent_kernel_mixed();
// Grid-barrier self-test (cooperative launch of `blocks` blocks, `rounds`
// barriers, optionally with block 0 absent); passes counts block passes.
cudaError_t launch_barrier_selftest(GridBarrier* bar, long long spin_limit, int blocks, int rounds, int skip_block0,
                                    unsigned int* passes, DeviceScalars* scal, cudaStream_t s);

// Counts nodes with rho <= 0, epsilon <= 0, non-finite values; writes
// {count_rho, count_eps, count_nonfinite} as doubles plus rho_min, eps_min
// into out[0..4] (device memory); acc is 5 words of device scratch.
void launch_check_state(const double* U, int64_t n, double* out, unsigned long long* acc, cudaStream_t s);
// Local bounds (Sec. 3.9) of a state U against per-row bounds bnd (rho_min,
// rho_max, phi_min; 3n): out = {rows, n_rho_below, n_rho_above, n_phi_below,
// worst rho_min, rho_max and phi_min relative violations}; acc: 7 words.
void launch_check_local(const double* U, const double* bnd, int64_t n, double slack_rho, double slack_phi,
                        double* out, unsigned long long* acc, cudaStream_t s);

}  // namespace idp
