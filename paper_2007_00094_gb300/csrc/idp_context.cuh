// The context behind the opaque idp_ctx of include/idp.h: host copies of the
// matrices, the sliced-ELL layout, device graph and buffers, schedule and
// reverse-mode state.  Shared by the translation units that drive stages.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "idp.h"
#include "idp_adjoint.cuh"
#include "idp_internal.h"
#include "idp_mixed.cuh"
#include "idp_stage.cuh"

struct idp_ctx {
  idp_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  bool has_mesh = false, has_state = false, has_trace = false;
  bool stage_ran = false;
  // > 0: the largest |c_ij| of the whole mesh, for the FP32 copies of the
  // mixed stage (a shard's context sees part of the mesh); 0: its own
  double c_scale = 0.0;  // B.Ulast and B.bnd hold the output and bounds of one stage of the current state
  idp::HostMatrices M;
  idp::SellLayout L;
  idp::DeviceGraph G{};
  idp::StageBuffers B{};
  idp::StageConfig C{};
  idp::MixedGraph MG{};
  int64_t n_entry_values = 0;  // size of the mixed stage's entry table (0: per-entry arrays)
  int64_t n_row_patterns = 0;  // row patterns of the mixed stage (0: per-slot column and transpose arrays)
  // row order (idp_config.renumber): library row of each caller node and back,
  // on the device, and a 5n buffer for reordering states at the interface
  bool renumbered = false;
  int64_t *d_perm = nullptr, *d_iperm = nullptr;
  double* perm_buf = nullptr;
  idp::MixedBuffers MB{};
  bool mixed = false;
  std::vector<void*> allocations;
  double* check = nullptr;  // 12 doubles: state check (5), local-bound check (7)
  unsigned long long* check_acc = nullptr;  // 12 words
  int64_t launches = 0;
  idp::Profiler prof;
  // per-instance device state (one instance unless idp_set_instances)
  std::vector<void*> inst_allocs;
  // schedule: block size of the stage kernels and CUDA-graph replay of idp_step
  int block = 64;  // measured fastest of 64, 128, 256 on the benchmark workloads
  bool use_graph = false;
  bool persistent = false;            // one cooperative launch per euler_step
  idp::GridBarrier* bar = nullptr;   // its grid barrier (device)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;
  // reverse mode: adjoint buffers and scratch states (allocated on first use)
  bool has_adjoint = false;
  idp::AdjointBuffers A{};
  double *a_in = nullptr, *a_out = nullptr, *a_g = nullptr, *a_acc = nullptr, *a_e = nullptr, *a_tmp = nullptr;
  // recorded forward run: checkpoints every rec_every steps, tau_n per step,
  // and the states of one segment (U^n, stage 1, stage 2 of each step)
  std::vector<void*> rec_allocs;
  int rec_steps = 0, rec_every = 0;
  double *rec_ckpt = nullptr, *rec_tau = nullptr, *rec_seg = nullptr;
  double* rec_snap = nullptr;  // stage traces of one checkpoint segment (adjoint_store_stages), or nullptr
};
