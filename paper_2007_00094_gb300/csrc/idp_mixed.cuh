// FP32-mixed stage: FP32 copies of the per-entry matrices and FP32 work
// buffers next to the FP64 state buffers of StageBuffers.
#pragma once
#include "idp_stage.cuh"

namespace idp {

struct MixedGraph {
  const float* cx;
  const float* cy;
  const float* cz;
  const float* mij;
  const float* cn;
  const float* inv_cn;
  const float* inv_mi;  // per node
};

struct MixedBuffers {
  float* Uf;     // 5n: FP32 copy of the stage input
  float* Q;      // kNodeQ * n per-node quantities
  float* d;      // n_slots
  float* dinv;   // n_slots
  float* P;      // 5 * n_slots (flux differences from Step 1 to Step 3, then P_ij)
  float* l[2];   // n_slots each
  float* alpha;  // n
  float* R;      // 5n
};

// Same contract as launch_euler_step (idp_stage.cuh) with FP32 candidates.
int launch_euler_step_mixed(const DeviceGraph& G, const MixedGraph& M, const StageBuffers& B, const MixedBuffers& X,
                            const StageConfig& C, const double* Uin, double* Uout, const double* Un, int blend,
                            int tau_mode, bool accumulate_time, bool skip_write_on_error, bool trace, cudaStream_t s,
                            Profiler* prof, int block = 128, GridBarrier* bar = nullptr);

}  // namespace idp
