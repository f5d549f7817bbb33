// idp_probe_fp64_peak: the FP64 fused multiply-add rate of the current GPU,
// the denominator of the FP64 stage's roofline.  The stage's heavy kernels
// are bound by the FP64 pipe (nothing in them is a dense contraction), and
// neither the vendor's peak tables nor a copy or GEMM benchmark measure that
// pipe, so the library measures it itself: every thread runs kChains
// independent FMA recurrences, enough to cover the pipe's latency, on a grid
// of several blocks per SM.
#include <cuda_runtime.h>

#include "idp.h"

namespace {

constexpr int kChains = 16;
constexpr int kProbeBlock = 256;

__device__ double g_probe_sink;

// The trip counter is 32-bit and the loop unrolled: on this GPU 64-bit integer
// compares issue on the FP64 pipe and would be counted against it.
__global__ void __launch_bounds__(kProbeBlock) k_fp64_fma_stream(int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  // x <- x * b + e with b slightly below 1 stays bounded: a fixed point near
  // e / (1 - b); nothing overflows or becomes subnormal
  const double b = 0.999999, e = 1e-6;
#pragma unroll 4
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, e);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) g_probe_sink = s;  // keeps the chains alive; never true for these values
}

}  // namespace

extern "C" idp_status idp_probe_fp64_peak(void* cuda_stream, int64_t fma_per_thread, double* tflops, double* ms) {
  if (!tflops || fma_per_thread < kChains) return IDP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_stream, kProbeBlock, 0)) {
    cudaGetLastError();
    return IDP_ERR_CUDA;
  }
  const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  if (fma_per_thread / kChains > (int64_t)1 << 30) return IDP_ERR_ARG;
  const int iters = (int)(fma_per_thread / kChains);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    return IDP_ERR_CUDA;
  }
  k_fp64_fma_stream<<<grid, kProbeBlock, 0, s>>>(iters / 8, 0.5);  // warm-up
  cudaEventRecord(a, s);
  k_fp64_fma_stream<<<grid, kProbeBlock, 0, s>>>(iters, 0.5);
  cudaEventRecord(b, s);
  float t = 0.0f;
  const cudaError_t e = cudaEventSynchronize(b);
  if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || t <= 0.0f) return IDP_ERR_CUDA;
  const double flops = 2.0 * (double)grid * kProbeBlock * kChains * (double)iters;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return IDP_OK;
}
