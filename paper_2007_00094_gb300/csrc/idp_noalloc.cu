// idp_tau_max_noalloc: the admissible time-step bound of a state, computed
// without allocating device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree itself, e.g. a
// host framework that hands out all device memory from its own pool (an
// allocation behind its back escapes its accounting and can fail under its
// memory cap), or a long-running service that allocates everything at
// start-up and forbids allocation afterwards.  Such callers cannot create an
// idp_ctx (which allocates), but they can hand over their own device arrays:
// CSR matrices (as returned by idp_get_matrices), lumped masses and a state.
//
// The bound is tau_max = min_i m_i / (-2 d_ii) with d_ii = -sum_{j != i} d_ij
// and d_ij the larger of the two orientations of the two-rarefaction
// wavespeed bound times |c|.  The reduction needs scratch memory; here it is a
// file-scope device array of fixed size instead of an allocation.
#include <cuda_runtime.h>

#include "idp.h"
#include "idp_device.cuh"

namespace idp {
namespace {

constexpr int kNaBlock = 128;
constexpr int kNaMaxBlocks = (int)(IDP_NOALLOC_MAX_NODES / kNaBlock);

// Scratch shared by every call on a device: one partial minimum per block and
// the ticket that elects the block doing the final reduction.
struct NoallocScratch {
  double partial[kNaMaxBlocks];
  unsigned int ticket;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, not a device address, so it
// is looked up (cudaGetSymbolAddress, which allocates nothing) on every call:
// the address stays right after a device reset or a new primary context.
cudaError_t scratch_address(NoallocScratch** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<NoallocScratch*>(p);
  return cudaSuccess;
}

// Minimum that keeps a NaN: fmin would drop it, and a NaN partial means a
// row whose state is not admissible.
__device__ __forceinline__ double min_keep_nan(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }
__device__ __forceinline__ double max_keep_nan(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }

__device__ __forceinline__ Side side_of(const double* U, int64_t n, int64_t i) {
  Side s;
  s.rho = U[i];
  s.mx = U[n + i];
  s.my = U[2 * n + i];
  s.mz = U[3 * n + i];
  s.inv_rho = 1.0 / s.rho;
  const double eps = U[4 * n + i] - 0.5 * (s.mx * s.mx + s.my * s.my + s.mz * s.mz) * s.inv_rho;
  s.p = 0.4 * eps;
  s.c = sqrt(1.4 * s.p * s.inv_rho);
  s.pm = inv_root<7>(s.p);
  s.inv_p = 1.0 / s.p;
  return s;
}

__global__ void __launch_bounds__(kNaBlock)
k_tau_max_noalloc(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ col,
                  const double* __restrict__ cij, const double* __restrict__ mi, const double* __restrict__ U,
                  NoallocScratch* scratch, double* tau_out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double cand = INFINITY;
  if (r < n) {
    const Side si = side_of(U, n, r);
    // rho > 0 and epsilon > 0 (p = (gamma - 1) epsilon); otherwise the row
    // yields NaN, which the reduction carries to tau_max
    const bool admissible = si.rho > 0.0 && si.p > 0.0;
    double sum = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      const int64_t j = col[k];
      if (j == r) continue;
      // position of entry (j, r): columns are sorted within each row
      int64_t lo = rowptr[j], hi = rowptr[j + 1] - 1, kt = -1;
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t cm = col[mid];
        if (cm == r) {
          kt = mid;
          break;
        }
        if (cm < r) lo = mid + 1; else hi = mid - 1;
      }
      const Side sj = side_of(U, n, j);
      const double cx = cij[k], cy = cij[nnz + k], cz = cij[2 * nnz + k];
      const double nc = sqrt(cx * cx + cy * cy + cz * cz);
      double dij = 0.0;
      if (nc > 0.0) dij = lambda_max(cx / nc, cy / nc, cz / nc, si, sj) * nc;
      if (kt >= 0) {
        const double tx = cij[kt], ty = cij[nnz + kt], tz = cij[2 * nnz + kt];
        const double nt = sqrt(tx * tx + ty * ty + tz * tz);
        if (nt > 0.0) dij = max_keep_nan(dij, lambda_max(tx / nt, ty / nt, tz / nt, sj, si) * nt);
      }
      sum += dij;
    }
    cand = admissible ? mi[r] / (2.0 * sum) : NAN;
  }
  // block minimum, then the last block to finish reduces the partials
  __shared__ double red[kNaBlock / 32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) cand = min_keep_nan(cand, __shfl_xor_sync(0xffffffffu, cand, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cand;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = red[0];
    for (int w = 1; w < kNaBlock / 32; ++w) v = min_keep_nan(v, red[w]);
    scratch->partial[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = INFINITY;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) v = min_keep_nan(v, __ldcg(&scratch->partial[b]));
  for (int o = 16; o > 0; o >>= 1) v = min_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kNaBlock / 32; ++w) v = min_keep_nan(v, red[w]);
    v = min_keep_nan(v, red[0]);
    *tau_out = v;
    scratch->ticket = 0u;
  }
}

}  // namespace
}  // namespace idp

extern "C" idp_status idp_tau_max_noalloc(int64_t n_nodes, int64_t nnz, const int64_t* rowptr, const int64_t* col,
                                          const double* cij, const double* mi, const double* U, double* tau_max,
                                          void* cuda_stream) {
  if (n_nodes <= 0 || nnz <= 0 || !rowptr || !col || !cij || !mi || !U || !tau_max) return IDP_ERR_ARG;
  if (n_nodes > IDP_NOALLOC_MAX_NODES) return IDP_ERR_ARG;
  idp::NoallocScratch* scratch = nullptr;
  if (idp::scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return IDP_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the ticket must start at zero; the partials are overwritten by every call
  if (cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
    cudaGetLastError();
    return IDP_ERR_CUDA;
  }
  const unsigned grid = (unsigned)((n_nodes + idp::kNaBlock - 1) / idp::kNaBlock);
  idp::k_tau_max_noalloc<<<grid, idp::kNaBlock, 0, s>>>(n_nodes, nnz, rowptr, col, cij, mi, U, scratch, tau_max);
  if (cudaGetLastError() != cudaSuccess) return IDP_ERR_CUDA;
  return IDP_OK;
}
