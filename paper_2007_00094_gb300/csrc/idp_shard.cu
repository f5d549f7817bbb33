// Sharded stage (Sec. 4.1, Fig. 1-2): the rows split into contiguous ranges,
// one context per shard holding its rows and one ghost layer, all on the
// caller's stream.  Each euler_step runs phase by phase over every shard;
// between phases the shards exchange what the next phase reads at rows they
// do not own, at the synchronisation points of Fig. 2:
//
//   after Steps 0-2   alpha_j of ghost rows, and a min-reduction of the CFL
//                     bound over the shards (tau_n is global)
//   after Step 3      R_j of ghost rows
//   after Step 4      l_ji of ghost rows' entries into own rows
//   after each pass   l_ji again (the pass recomputes it)
//   after Step 6      the stage output U_j of ghost rows
//
// Ghost rows run Steps 0 and 1, on their entries inside the shard, and are
// exact there: node values, and the pair values of the pairs a ghost row
// evaluates (d_ij, 1/(2 d_ij), the flux differences and m_j.c_ij), which an
// own row reads through its lower entries.  Steps 2-6 run on own rows only;
// what they read at ghost rows arrives by the exchanges.  Every own row
// therefore computes what it computes unsharded, in the same order, and the
// result is bitwise the same.
//
// Each shard runs on a stream of its own, as it would on its own GPU; the
// exchanges and the tau reduction order the shards by events.  An exchange
// is pack (a gather kernel on the sender's stream), one cudaMemcpyAsync of
// the packed buffer into the receiver's buffer (with one GPU per shard, the
// transfer between GPUs), and unpack (a scatter kernel on the receiver's
// stream).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "idp.h"
#include "idp_context.cuh"
#include "idp_shard.h"

struct idp_shard_plan {
  idp::ShardPlan P;
};

struct idp_shards {
  cudaStream_t stream = nullptr;  // the caller's stream
  std::string err;
  idp::ShardPlan P;
  std::vector<idp_ctx*> ctx;
  // Each shard works on a stream of its own, as it would on a GPU of its
  // own; what one shard needs from another is ordered by events.
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;  // every event the group created
  std::vector<cudaEvent_t> ev_phase, ev_end;  // per shard
  cudaEvent_t ev_start = nullptr, ev_tau = nullptr;
  // one link per ordered pair of shards with values to exchange
  struct Link {
    int src = 0, dst = 0;
    int64_t nn = 0, ne = 0;                  // node and entry values per field
    int64_t *sn = nullptr, *dn = nullptr;    // sender / receiver local node ids
    int64_t *ss = nullptr, *ds = nullptr;    // sender / receiver slots
    double* send = nullptr;                  // packed buffer of the sender (max(5 nn, ne) doubles)
    double* recv[2] = {nullptr, nullptr};    // receiver's buffers, alternating between exchanges
    cudaEvent_t copied = nullptr;            // the sender's copy of the current exchange is done
    cudaEvent_t unpacked[2] = {nullptr, nullptr};  // the receiver has emptied recv[k]
  };
  std::vector<Link> links;
  int64_t exchanges = 0;  // parity of the receive buffers
  cudaError_t enqueue_error = cudaSuccess;  // first failed copy or event call of the last step
  unsigned long long** words = nullptr;  // device: each shard's CFL reduction word
  std::vector<void*> allocs;
  bool has_state = false;
  int64_t launches = 0;
};

namespace {

constexpr int kXBlock = 256;

idp_status sfail(idp_shards* sh, idp_status st, const std::string& msg) {
  if (sh) sh->err = msg;
  return st;
}

#define SH_CUDA(sh, expr)                                                                         \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess) return sfail(sh, IDP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
idp_status salloc(idp_shards* sh, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(sh, IDP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  sh->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return IDP_OK;
}

template <typename T>
idp_status supload(idp_shards* sh, T** p, const std::vector<T>& v) {
  idp_status st = salloc(sh, p, v.size());
  if (st != IDP_OK) return st;
  if (!v.empty()) SH_CUDA(sh, cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return IDP_OK;
}

// buf[c m + k] = X[c n + idx[k]] for comps fields of a node array
template <typename T>
__global__ void k_pack_nodes(const T* __restrict__ X, int64_t n, int comps, const int64_t* __restrict__ idx,
                             int64_t m, T* __restrict__ buf) {
  const int64_t total = (int64_t)comps * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / m, k = t - c * m;
    buf[t] = X[c * n + idx[k]];
  }
}

template <typename T>
__global__ void k_unpack_nodes(T* __restrict__ X, int64_t n, int comps, const int64_t* __restrict__ idx, int64_t m,
                               const T* __restrict__ buf) {
  const int64_t total = (int64_t)comps * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / m, k = t - c * m;
    X[c * n + idx[k]] = buf[t];
  }
}

// buf[k] = X[idx[k]] for a per-slot array, and back
template <typename T>
__global__ void k_pack_slots(const T* __restrict__ X, const int64_t* __restrict__ idx, int64_t m,
                             T* __restrict__ buf) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    buf[k] = X[idx[k]];
}

template <typename T>
__global__ void k_unpack_slots(T* __restrict__ X, const int64_t* __restrict__ idx, int64_t m,
                               const T* __restrict__ buf) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    X[idx[k]] = buf[k];
}

// The global CFL bound: the minimum of the shards' reduction words (the bits
// of positive doubles order like the doubles), written back to every shard.
__global__ void k_tau_allreduce(unsigned long long* const* words, int n_shards) {
  unsigned long long m = ~0ull;
  for (int s = 0; s < n_shards; ++s) m = min(m, *words[s]);
  for (int s = 0; s < n_shards; ++s) *words[s] = m;
}

unsigned grid_for(int64_t work) {
  const int64_t b = (work + kXBlock - 1) / kXBlock;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// Keeps the first error of an enqueued copy or event call for idp_shards_step.
void note(idp_shards* sh, cudaError_t e) {
  if (e != cudaSuccess && sh->enqueue_error == cudaSuccess) sh->enqueue_error = e;
}

// One exchange over every link: pack(k) enqueues the sender's gather of
// link k into its send buffer, unpack(k, buf) the receiver's scatter.  The
// sender copies into the receiver's buffer of this exchange's parity once
// the receiver has emptied it (two exchanges back), and the receiver waits
// for the copy.  bytes(k) is the size of link k's message.
template <typename Pack, typename Unpack, typename Bytes>
int exchange(idp_shards* sh, Pack&& pack, Unpack&& unpack, Bytes&& bytes) {
  const int par = (int)(sh->exchanges++ & 1);
  int launches = 0;
  for (idp_shards::Link& k : sh->links) {
    const size_t b = bytes(k);
    if (b == 0) continue;
    cudaStream_t s = sh->streams[k.src];
    pack(k, s);
    note(sh, cudaStreamWaitEvent(s, k.unpacked[par], 0));
    note(sh, cudaMemcpyAsync(k.recv[par], k.send, b, cudaMemcpyDeviceToDevice, s));
    note(sh, cudaEventRecord(k.copied, s));
    ++launches;
  }
  for (idp_shards::Link& k : sh->links) {
    if (bytes(k) == 0) continue;
    cudaStream_t s = sh->streams[k.dst];
    note(sh, cudaStreamWaitEvent(s, k.copied, 0));
    unpack(k, k.recv[par], s);
    note(sh, cudaEventRecord(k.unpacked[par], s));
    ++launches;
  }
  return launches;
}

// A node array of comps fields (stride n of each shard); field(s) gives
// shard s's array.
template <typename T, typename F>
int exchange_nodes(idp_shards* sh, int comps, F&& field) {
  return exchange(
      sh,
      [&](const idp_shards::Link& k, cudaStream_t s) {
        k_pack_nodes<T><<<grid_for(comps * k.nn), kXBlock, 0, s>>>(field(k.src), sh->ctx[k.src]->G.n, comps, k.sn,
                                                                    k.nn, reinterpret_cast<T*>(k.send));
      },
      [&](const idp_shards::Link& k, const double* buf, cudaStream_t s) {
        k_unpack_nodes<T><<<grid_for(comps * k.nn), kXBlock, 0, s>>>(field(k.dst), sh->ctx[k.dst]->G.n, comps, k.dn,
                                                                      k.nn, reinterpret_cast<const T*>(buf));
      },
      [&](const idp_shards::Link& k) { return sizeof(T) * (size_t)comps * (size_t)k.nn; });
}

// A per-slot array.
template <typename T, typename F>
int exchange_slots(idp_shards* sh, F&& field) {
  return exchange(
      sh,
      [&](const idp_shards::Link& k, cudaStream_t s) {
        k_pack_slots<T><<<grid_for(k.ne), kXBlock, 0, s>>>(field(k.src), k.ss, k.ne, reinterpret_cast<T*>(k.send));
      },
      [&](const idp_shards::Link& k, const double* buf, cudaStream_t s) {
        k_unpack_slots<T><<<grid_for(k.ne), kXBlock, 0, s>>>(field(k.dst), k.ds, k.ne,
                                                              reinterpret_cast<const T*>(buf));
      },
      [&](const idp_shards::Link& k) { return sizeof(T) * (size_t)k.ne; });
}

// One euler_step of every shard (the roles of U^n, the stage state and the
// blend as in the unsharded SSP-RK3 step).  The FP32-mixed stage exchanges
// its FP32 alpha, R and l.
int sharded_stage(idp_shards* sh, int stage) {
  const int S = (int)sh->ctx.size();
  const idp::StageConfig& C0 = sh->ctx[0]->C;
  const bool mixed = sh->ctx[0]->mixed;
  const int phases = idp::euler_phase_count(C0);
  const int passes = C0.limiter_passes;
  int launches = 0;
  for (int ph = 0; ph < phases; ++ph) {
    for (int s = 0; s < S; ++s) {
      idp_ctx* c = sh->ctx[s];
      idp::StageBuffers& B = c->B;
      c->stage_ran = true;
      const double* Uin = stage == 0 ? B.U : B.Us;
      double* Uout = stage == 2 ? B.U : B.Us;
      const int blend = stage == 0 ? idp::kBlendNone : (stage == 1 ? idp::kBlendStage2 : idp::kBlendStage3);
      if (mixed)
        launches += idp::launch_euler_phase_mixed(c->G, c->MG, B, c->MB, c->C, Uin, Uout, B.U, blend,
                                                  stage == 0 ? 0 : 1, stage == 0, stage == 2, ph, sh->streams[s],
                                                  c->block);
      else
        launches += idp::launch_euler_phase(c->G, B, c->C, Uin, Uout, B.U, blend, stage == 0 ? 0 : 1, stage == 0,
                                            stage == 2, ph, sh->streams[s], c->block);
    }
    if (S == 1) continue;
    if (ph == 0) {
      // tau_n is global: the minimum of every shard's CFL bound, formed on
      // shard 0's stream once every shard has its own
      for (int s = 0; s < S; ++s) {
        note(sh, cudaEventRecord(sh->ev_phase[s], sh->streams[s]));
        note(sh, cudaStreamWaitEvent(sh->streams[0], sh->ev_phase[s], 0));
      }
      k_tau_allreduce<<<1, 1, 0, sh->streams[0]>>>(sh->words, S);
      note(sh, cudaEventRecord(sh->ev_tau, sh->streams[0]));
      for (int s = 1; s < S; ++s) note(sh, cudaStreamWaitEvent(sh->streams[s], sh->ev_tau, 0));
      ++launches;
      if (mixed)
        launches += exchange_nodes<float>(sh, 1, [&](int s) { return sh->ctx[s]->MB.alpha; });
      else
        launches += exchange_nodes<double>(sh, 1, [&](int s) { return sh->ctx[s]->B.alpha; });
    } else if (ph == 1) {
      if (mixed)
        launches += exchange_nodes<float>(sh, 5, [&](int s) { return sh->ctx[s]->MB.R; });
      else
        launches += exchange_nodes<double>(sh, 5, [&](int s) { return sh->ctx[s]->B.R; });
    } else if (ph < 2 + passes) {
      if (mixed)
        launches += exchange_slots<float>(sh, [&](int s) { return sh->ctx[s]->MB.l[(ph - 2) & 1]; });
      else
        launches += exchange_slots<double>(sh, [&](int s) { return idp::phase_l_buffer(sh->ctx[s]->B, ph); });
    } else {
      launches +=
          exchange_nodes<double>(sh, 5, [&](int s) { return stage == 2 ? sh->ctx[s]->B.U : sh->ctx[s]->B.Us; });
    }
  }
  return launches;
}

// Waits (on the host) for every shard's stream.
idp_status sync_all(idp_shards* sh) {
  for (cudaStream_t s : sh->streams) SH_CUDA(sh, cudaStreamSynchronize(s));
  return IDP_OK;
}

idp_status new_event(idp_shards* sh, cudaEvent_t* e) {
  SH_CUDA(sh, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  sh->events.push_back(*e);
  return IDP_OK;
}

}  // namespace

extern "C" {

idp_status idp_shard_plan_create(int64_t n_nodes, const int64_t* rowptr, const int64_t* col, int n_shards,
                                 const int64_t* row_begin, idp_shard_plan** out) {
  if (!out) return IDP_ERR_ARG;
  *out = nullptr;
  if (n_nodes <= 0 || n_shards < 1 || n_shards > n_nodes || !rowptr || !col) return IDP_ERR_ARG;
  std::vector<int64_t> rb(n_shards + 1);
  if (row_begin) {
    rb.assign(row_begin, row_begin + n_shards + 1);
  } else {  // equal ranges
    for (int s = 0; s <= n_shards; ++s) rb[s] = n_nodes * s / n_shards;
  }
  idp_shard_plan* p = new (std::nothrow) idp_shard_plan;
  if (!p) return IDP_ERR_OOM;
  if (!idp::build_shard_plan(n_nodes, rowptr, col, n_shards, rb.data(), p->P).empty()) {
    delete p;
    return IDP_ERR_ARG;
  }
  *out = p;
  return IDP_OK;
}

void idp_shard_plan_destroy(idp_shard_plan* plan) { delete plan; }

idp_status idp_shard_plan_info(const idp_shard_plan* plan, int shard, int64_t* n_local, int64_t* own_begin,
                               int64_t* own_end, int64_t* nnz_local) {
  if (!plan || shard < 0 || shard >= plan->P.n_shards) return IDP_ERR_ARG;
  const idp::ShardLocal& S = plan->P.shard[shard];
  if (n_local) *n_local = (int64_t)S.nodes.size();
  if (own_begin) *own_begin = S.own_lo;
  if (own_end) *own_end = S.own_hi;
  if (nnz_local) *nnz_local = (int64_t)S.col.size();
  return IDP_OK;
}

idp_status idp_shard_plan_nodes(const idp_shard_plan* plan, int shard, int64_t* nodes) {
  if (!plan || shard < 0 || shard >= plan->P.n_shards || !nodes) return IDP_ERR_ARG;
  const idp::ShardLocal& S = plan->P.shard[shard];
  std::copy(S.nodes.begin(), S.nodes.end(), nodes);
  return IDP_OK;
}

idp_status idp_shard_plan_csr(const idp_shard_plan* plan, int shard, int64_t* rowptr, int64_t* col, int64_t* entry) {
  if (!plan || shard < 0 || shard >= plan->P.n_shards) return IDP_ERR_ARG;
  const idp::ShardLocal& S = plan->P.shard[shard];
  if (rowptr) std::copy(S.rowptr.begin(), S.rowptr.end(), rowptr);
  if (col) std::copy(S.col.begin(), S.col.end(), col);
  if (entry) std::copy(S.entry.begin(), S.entry.end(), entry);
  return IDP_OK;
}

idp_status idp_shard_plan_list(const idp_shard_plan* plan, int shard, int peer, int kind, int64_t* count,
                               int64_t* ids) {
  if (!plan || shard < 0 || shard >= plan->P.n_shards || peer < 0 || peer >= plan->P.n_shards || kind < 0 ||
      kind > 3)
    return IDP_ERR_ARG;
  const idp::ShardLocal& S = plan->P.shard[shard];
  const std::vector<int64_t>& v = kind == IDP_SEND_NODES     ? S.send_nodes[peer]
                                  : kind == IDP_RECV_NODES   ? S.recv_nodes[peer]
                                  : kind == IDP_SEND_ENTRIES ? S.send_entries[peer]
                                                             : S.recv_entries[peer];
  if (count) *count = (int64_t)v.size();
  if (ids) std::copy(v.begin(), v.end(), ids);
  return IDP_OK;
}

void idp_shards_destroy(idp_shards* sh) {
  if (!sh) return;
  for (cudaStream_t s : sh->streams) cudaStreamSynchronize(s);
  for (idp_ctx* c : sh->ctx) idp_destroy(c);
  for (void* p : sh->allocs) cudaFree(p);
  for (cudaEvent_t e : sh->events) cudaEventDestroy(e);
  for (cudaStream_t s : sh->streams) cudaStreamDestroy(s);
  delete sh;
}

const char* idp_shards_last_error(const idp_shards* sh) { return sh ? sh->err.c_str() : "no sharded stage"; }

idp_status idp_shards_create(const idp_config* cfg_in, void* cuda_stream, const idp_shard_plan* plan,
                             const double* mij, const double* cij, const double* mi, const int32_t* node_bc,
                             const double* inflow_state, idp_shards** out) {
  if (!out) return IDP_ERR_ARG;
  *out = nullptr;
  if (!plan || !mij || !cij) return IDP_ERR_ARG;
  idp_config cfg;
  if (cfg_in) {
    cfg = *cfg_in;
  } else {
    idp_config_default(&cfg);
  }
  // FP64 per-step kernels in the caller's row order; the bound relaxation
  // scales by the volume of the whole domain, which no shard sees
  if ((cfg.precision != IDP_PRECISION_FP64 && cfg.precision != IDP_PRECISION_MIXED) || cfg.relax != 0 ||
      cfg.renumber != 0)
    return IDP_ERR_ARG;
  idp_shards* sh = new (std::nothrow) idp_shards;
  if (!sh) return IDP_ERR_OOM;
  sh->stream = static_cast<cudaStream_t>(cuda_stream);
  sh->P = plan->P;
  const idp::ShardPlan& P = sh->P;
  const int S = P.n_shards;
  const int64_t n = P.n, nnz = P.nnz;
  // lumped masses of the whole mesh (a ghost row's own sum covers only its
  // entries inside the shard); without the caller's, the row sums of m_ij in
  // column order, as an unsharded context forms them
  std::vector<double> m_all(n);
  if (mi) {
    std::copy(mi, mi + n, m_all.begin());
  } else {
    // the plan keeps only the local patterns; the global row of node g is the
    // local row of g in the shard that owns it
    for (int s = 0; s < S; ++s) {
      const idp::ShardLocal& L = P.shard[s];
      for (int64_t l = L.own_lo; l < L.own_hi; ++l) {
        double m = 0.0;
        for (int64_t e = L.rowptr[l]; e < L.rowptr[l + 1]; ++e) m += mij[L.entry[e]];
        m_all[L.nodes[l]] = m;
      }
    }
  }
  // the FP32 copies of c_ij take exact zeros relative to the largest |c_ij|
  // of the whole mesh, as an unsharded context does
  double c_scale = 0.0;
  for (int64_t e = 0; e < nnz; ++e) {
    const double x = cij[e], y = cij[nnz + e], z = cij[2 * nnz + e];
    c_scale = std::fmax(c_scale, std::sqrt(x * x + y * y + z * z));
  }
  idp_status st = IDP_OK;
  for (int s = 0; s < S && st == IDP_OK; ++s) {
    cudaStream_t q = nullptr;
    if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = sfail(sh, IDP_ERR_CUDA, "cudaStreamCreateWithFlags failed");
      break;
    }
    sh->streams.push_back(q);
    cudaEvent_t a = nullptr, b = nullptr;
    if ((st = new_event(sh, &a)) || (st = new_event(sh, &b))) break;
    sh->ev_phase.push_back(a);
    sh->ev_end.push_back(b);
  }
  if (st == IDP_OK && (st = new_event(sh, &sh->ev_start)) == IDP_OK) st = new_event(sh, &sh->ev_tau);
  for (int s = 0; s < S && st == IDP_OK; ++s) {
    const idp::ShardLocal& L = P.shard[s];
    const int64_t nl = (int64_t)L.nodes.size(), el = (int64_t)L.col.size();
    std::vector<double> lm(el), lc(3 * el), lmi(nl);
    std::vector<int32_t> lbc(nl, 0);
    for (int64_t e = 0; e < el; ++e) {
      const int64_t g = L.entry[e];
      lm[e] = mij[g];
      for (int d = 0; d < 3; ++d) lc[d * el + e] = cij[d * nnz + g];
    }
    for (int64_t l = 0; l < nl; ++l) {
      lmi[l] = m_all[L.nodes[l]];
      if (node_bc) lbc[l] = node_bc[L.nodes[l]];
    }
    idp_ctx* c = nullptr;
    st = idp_create(&cfg, sh->streams[s], &c);
    if (st != IDP_OK) break;
    sh->ctx.push_back(c);
    c->c_scale = c_scale;
    st = idp_upload_sparsity(c, nl, L.rowptr.data(), L.col.data(), lm.data(), lc.data(), lmi.data(), lbc.data(),
                             inflow_state);
    if (st != IDP_OK) {
      sh->err = std::string("shard ") + std::to_string(s) + ": " + idp_last_error(c);
      break;
    }
    // ghost rows take Steps 0-1 only: what they compute after that is
    // overwritten by the exchanges before an own row reads it
    c->G.row0 = L.own_lo;
    c->G.row1 = L.own_hi;
  }
  // links: the sender's lists index its own rows, the receiver's its ghosts;
  // entries become slots of each side's layout
  for (int a = 0; a < S && st == IDP_OK; ++a)
    for (int b = 0; b < S && st == IDP_OK; ++b) {
      if (a == b) continue;
      const idp::ShardLocal &A = P.shard[a], &B = P.shard[b];
      const std::vector<int64_t>&sn = A.send_nodes[b], &dn = B.recv_nodes[a];
      const std::vector<int64_t>&se = A.send_entries[b], &de = B.recv_entries[a];
      if (sn.empty() && se.empty()) continue;
      idp_shards::Link k;
      k.src = a;
      k.dst = b;
      k.nn = (int64_t)sn.size();
      k.ne = (int64_t)se.size();
      std::vector<int64_t> ss(se.size()), ds(de.size());
      for (size_t q = 0; q < se.size(); ++q) ss[q] = sh->ctx[a]->L.slot_of_entry[se[q]];
      for (size_t q = 0; q < de.size(); ++q) ds[q] = sh->ctx[b]->L.slot_of_entry[de[q]];
      const size_t buf = (size_t)std::max<int64_t>(5 * k.nn, k.ne);
      if ((st = supload(sh, &k.sn, sn)) || (st = supload(sh, &k.dn, dn)) || (st = supload(sh, &k.ss, ss)) ||
          (st = supload(sh, &k.ds, ds)) || (st = salloc(sh, &k.send, buf)) || (st = salloc(sh, &k.recv[0], buf)) ||
          (st = salloc(sh, &k.recv[1], buf)) || (st = new_event(sh, &k.copied)) ||
          (st = new_event(sh, &k.unpacked[0])) || (st = new_event(sh, &k.unpacked[1])))
        break;
      sh->links.push_back(k);
    }
  if (st == IDP_OK) {
    std::vector<unsigned long long*> w(S);
    for (int s = 0; s < S; ++s) w[s] = sh->ctx[s]->G.tau_min;
    st = supload(sh, &sh->words, w);
  }
  if (st != IDP_OK) {
    idp_shards_destroy(sh);
    return st;
  }
  *out = sh;
  return IDP_OK;
}

idp_status idp_shards_context(idp_shards* sh, int shard, idp_ctx** out) {
  if (!sh || !out || shard < 0 || shard >= (int)sh->ctx.size()) return IDP_ERR_ARG;
  *out = sh->ctx[shard];
  return IDP_OK;
}

idp_status idp_shards_init_state(idp_shards* sh, const double* U) {
  if (!sh || !U) return IDP_ERR_ARG;
  idp_status st0 = sync_all(sh);
  if (st0 != IDP_OK) return st0;
  const int64_t n = sh->P.n;
  for (size_t s = 0; s < sh->ctx.size(); ++s) {
    const idp::ShardLocal& L = sh->P.shard[s];
    const int64_t nl = (int64_t)L.nodes.size();
    std::vector<double> u(5 * nl);
    for (int f = 0; f < 5; ++f)
      for (int64_t l = 0; l < nl; ++l) u[f * nl + l] = U[f * n + L.nodes[l]];
    const idp_status st = idp_init_state(sh->ctx[s], u.data(), 0);
    if (st != IDP_OK) return sfail(sh, st, idp_last_error(sh->ctx[s]));
  }
  sh->has_state = true;
  return IDP_OK;
}

idp_status idp_shards_get_state(idp_shards* sh, double* U) {
  if (!sh || !U) return IDP_ERR_ARG;
  if (!sh->has_state) return sfail(sh, IDP_ERR_STATE, "no state");
  idp_status st0 = sync_all(sh);
  if (st0 != IDP_OK) return st0;
  const int64_t n = sh->P.n;
  for (size_t s = 0; s < sh->ctx.size(); ++s) {
    const idp::ShardLocal& L = sh->P.shard[s];
    const int64_t nl = (int64_t)L.nodes.size();
    std::vector<double> u(5 * nl);
    const idp_status st = idp_get_state(sh->ctx[s], u.data(), 0);
    if (st != IDP_OK) return sfail(sh, st, idp_last_error(sh->ctx[s]));
    for (int f = 0; f < 5; ++f)
      for (int64_t l = L.own_lo; l < L.own_hi; ++l) U[f * n + L.nodes[l]] = u[f * nl + l];
  }
  return IDP_OK;
}

idp_status idp_shards_step(idp_shards* sh, int n_steps) {
  if (!sh || n_steps < 0) return IDP_ERR_ARG;
  if (!sh->has_state) return sfail(sh, IDP_ERR_STATE, "no state");
  // the shards' streams start after what the caller enqueued before, and
  // the caller's stream continues once every shard is done
  SH_CUDA(sh, cudaEventRecord(sh->ev_start, sh->stream));
  for (cudaStream_t s : sh->streams) SH_CUDA(sh, cudaStreamWaitEvent(s, sh->ev_start, 0));
  int64_t launches = 0;
  sh->enqueue_error = cudaSuccess;
  for (int k = 0; k < n_steps; ++k)
    for (int stage = 0; stage < 3; ++stage) launches += sharded_stage(sh, stage);
  if (sh->enqueue_error != cudaSuccess)
    return sfail(sh, IDP_ERR_CUDA, std::string("sharded exchange: ") + cudaGetErrorString(sh->enqueue_error));
  for (size_t s = 0; s < sh->streams.size(); ++s) {
    SH_CUDA(sh, cudaEventRecord(sh->ev_end[s], sh->streams[s]));
    SH_CUDA(sh, cudaStreamWaitEvent(sh->stream, sh->ev_end[s], 0));
  }
  sh->launches = launches;
  SH_CUDA(sh, cudaGetLastError());
  return IDP_OK;
}

idp_status idp_shards_synchronize(idp_shards* sh) {
  if (!sh) return IDP_ERR_ARG;
  idp_status first = IDP_OK;
  for (size_t s = 0; s < sh->ctx.size(); ++s) {
    const idp_status st = idp_synchronize(sh->ctx[s]);
    if (st != IDP_OK && first == IDP_OK) {
      first = st;
      sh->err = std::string("shard ") + std::to_string(s) + ": " + idp_last_error(sh->ctx[s]);
    }
  }
  return first;
}

idp_status idp_shards_get_time(idp_shards* sh, double* t, double* last_tau) {
  if (!sh || sh->ctx.empty()) return IDP_ERR_ARG;
  return idp_get_time(sh->ctx[0], t, last_tau);
}

idp_status idp_shards_halo_size(const idp_shards* sh, int64_t* node_values, int64_t* entry_values,
                                int64_t* launches) {
  if (!sh) return IDP_ERR_ARG;
  int64_t a = 0, b = 0;
  for (const idp_shards::Link& k : sh->links) {
    a += k.nn;
    b += k.ne;
  }
  if (node_values) *node_values = a;
  if (entry_values) *entry_values = b;
  if (launches) *launches = sh->launches;
  return IDP_OK;
}

}  // extern "C"
