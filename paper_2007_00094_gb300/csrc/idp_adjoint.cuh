// Reverse mode (discrete adjoint) of the FP64 euler_step: buffers and launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "idp_stage.cuh"

namespace idp {

// Adjoint work buffers (device memory owned by the context).  "own" arrays
// hold a row's adjoint of its own quantities; "tr" arrays hold, at entry
// (i, j), row i's contribution to the adjoint of a quantity of row j, which
// row j gathers through the transposed entry.
// Blocks of the first level of the fixed-order sum of the tau adjoint.
constexpr int kTauBlocks = 1024;

struct AdjointBuffers {
  double* gU5;       // 5n: adjoint of the state after the first limiter pass
  double* gUL;       // 5n: adjoint of U^L
  double* gR_own;    // 5n: adjoint of R_i from row i's own P_ij
  double* gU_own;    // 5n: adjoint of the stage input U_i (own part)
  double* gbnd;      // 3n: adjoint of rho_min, rho_max, phi_min
  double* ga_own;    // n: adjoint of alpha_i (own part)
  double* gtau_part; // n: per-row adjoint of tau_n
  double* gPp;       // 5 n_slots: adjoint of P_ij after the first pass
  double* gP;        // 5 n_slots: adjoint of P_ij of Step 4
  double* gR_tr;     // 5 n_slots
  double* gU_tr;     // 5 n_slots
  double* gdF;       // 5 n_slots: adjoint of (f_j - f_i).c_ij
  double* gl5_own;   // n_slots: adjoint of the first pass's l_ij
  double* gl5_tr;
  double* gl4_own;   // n_slots: adjoint of Step 4's l_ij
  double* gl4_tr;
  double* gd;        // n_slots: adjoint of d_ij as row i uses it
  double* ga_tr;     // n_slots
  double* gphi_tr;   // n_slots
  double* gtau_blk;  // kTauBlocks: partial sums of gtau_part over contiguous ranges of caller nodes
  double* gtau;      // 2: [0] carried over the stages of an RK step, [1] total of the first stage
  unsigned long long* argmin;  // 2: [0] bits of the CFL minimum, [1] first row attaining it
  // The entries whose limiter derivative is evaluated (off the diagonal,
  // adjoint of l_ij non-zero, 0 < l_ij < 1), listed in any order; each
  // listed entry's contributions to its row are kept at the entry and summed
  // by the row in slot order.
  int32_t* lim_slot;    // n_slots: listed entries
  int32_t* lim_row;     // n_slots: their rows
  unsigned int* lim_count;  // 1: length of the list
  uint8_t* lim_flag;    // n_slots: 1 where listed
  double* lim_gl;       // n_slots: adjoint of l_ij at listed entries
  double* lim_gU;       // 5 n_slots: contribution to the adjoint of the row state
  double* lim_gb;       // 3 n_slots: contribution to the adjoint of the row's bounds
};

// Enqueues the reverse of one traced euler_step with two limiter passes:
// given the adjoint gE of its output (before any RK blend), writes the
// adjoint of its input Uin to gIn.  B must hold the trace of the forward
// evaluation of this stage (launch_euler_step with trace = true from Uin).
// tau_computed: the stage computed tau_n (first RK stage); the adjoint of
// tau_n collected over the RK step (A.gtau[0] plus this stage's part) is
// then routed to d_kk of the first row k attaining the CFL minimum.
// Otherwise this stage's adjoint of tau_n is added to A.gtau[0].
// Returns the number of kernel launches.
int launch_adjoint_stage(const DeviceGraph& G, const StageBuffers& B, const AdjointBuffers& A, const StageConfig& C,
                         const double* Uin, const double* gE, double* gIn, bool tau_computed, cudaStream_t s,
                         Profiler* prof = nullptr);

// out = a x + b y over count doubles (y may be null: out = a x).
void launch_axpby(double* out, double a, const double* x, double b, const double* y, int64_t count, cudaStream_t s);

}  // namespace idp
