// FP32-mixed stage: FP32 copies of the per-entry matrices and FP32 work
// buffers next to the FP64 state buffers of StageBuffers.
#pragma once
#include <vector>

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
  // Entry table (nullptr: per-entry arrays above): slot p holds the index
  // ecode[p] of its values (cx, cy, cz, m_ij) = etab[2 ecode[p]],
  // (|c|, 1/|c|, 0, 0) = etab[2 ecode[p] + 1].
  const uint16_t* ecode;
  const float4* etab;
  // Row patterns (nullptr: per-slot arrays).  On a structured grid most rows
  // differ from others only by a shift of their column indices: rows whose
  // entries k have the same column offset j - r, the same index k' of the
  // transposed entry in row j, the same flags and the same entry-table code
  // share a pattern, rpat[r] is row r's, and ptab[rpat[r] * pwidth + k]
  // holds entry k as (j - r, k' | flags << 8 | code << 16).  The kernels
  // (all but Step 3's) then read one record per entry from a table that
  // stays in L1 instead of the column, transpose, flag and code streams.
  const uint16_t* rpat;
  const uint2* ptab;
  int pwidth;
};

constexpr int kEntryTableMax = 4096;
constexpr int kRowPatternMax = 4096;

// Host-side FP32 copies of the per-slot entries (SELL order).
struct HostEntriesF {
  std::vector<float> cx, cy, cz, m, cn, inv_cn;
};

// FP32 values of stored entry p (Sec. 3.1 matrices) from the table or the
// per-entry arrays; the compiler drops the loads of unused fields.
struct EntryF {
  float cx, cy, cz, m, cn, inv_cn;
};

__device__ __forceinline__ EntryF entry_f_code(const MixedGraph& M, int64_t p, int c) {
  EntryF e;
  if (M.ecode) {
    const float4 a = __ldg(&M.etab[2 * c]), b = __ldg(&M.etab[2 * c + 1]);
    e.cx = a.x;
    e.cy = a.y;
    e.cz = a.z;
    e.m = a.w;
    e.cn = b.x;
    e.inv_cn = b.y;
  } else {
    e.cx = M.cx[p];
    e.cy = M.cy[p];
    e.cz = M.cz[p];
    e.m = M.mij[p];
    e.cn = M.cn[p];
    e.inv_cn = M.inv_cn[p];
  }
  return e;
}

__device__ __forceinline__ EntryF entry_f(const MixedGraph& M, int64_t p) {
  return entry_f_code(M, p, M.ecode ? (int)M.ecode[p] : 0);
}

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

// The phases of launch_euler_phase (idp_stage.cuh) for the FP32-mixed stage,
// whose Step 2 runs inside Step 1: phase 0 = Steps 0-2 (node quantities of
// all rows, then d_ij, alpha_i and the CFL bound of the own rows), then
// Step 3, Step 4, the limiter passes and Step 6 as there; alpha, R and l are
// FP32 arrays of MixedBuffers.
int launch_euler_phase_mixed(const DeviceGraph& G, const MixedGraph& M, const StageBuffers& B,
                             const MixedBuffers& X, const StageConfig& C, const double* Uin, double* Uout,
                             const double* Un, int blend, int tau_mode, bool accumulate_time,
                             bool skip_write_on_error, int phase, cudaStream_t s, int block);

}  // namespace idp
