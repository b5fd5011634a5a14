// FP64 fused multiply-add throughput of the current device (a measurement aid, not part of the
// method).  The residual-side kernels of this library are bound by the FP64 pipes, whose rate
// no vendor figure for this part states reliably; the roofline of those kernels is taken
// against this measured rate.
//
// Every thread advances kChains independent recurrences x <- x a + b (one DFMA each per
// round), so that the pipes, not the ~70-cycle DFMA latency, set the pace; the grid holds
// kBlocksPerSM CTAs of kThreads threads per SM.  The result is written only when it equals a
// value it cannot reach, which keeps the compiler from removing the loop.
#include <cuda_runtime.h>

#include "../../include/cs.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kBlocksPerSM = 4;

__device__ double g_dfma_sink;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(int rounds, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) g_dfma_sink = s;   // every x stays positive: never taken
}

}  // namespace

extern "C" cs_status cs_measure_fp64_rate(void* cuda_stream, double* gflops_out) {
  if (!gflops_out) return CS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CS_ERR_CUDA;
  const int grid = sms * kBlocksPerSM;
  const int rounds = 16384;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CS_ERR_CUDA;
  }
  float best = 0.0f;
  cs_status status = CS_OK;
  for (int rep = 0; rep < 4 && status == CS_OK; ++rep) {   // the first launch is a warm-up
    cudaEventRecord(e0, st);
    k_dfma_rate<<<grid, kThreads, 0, st>>>(rounds, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = CS_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != CS_OK) return status;
  const double flop = 2.0 * kChains * (double)rounds * kThreads * (double)grid;
  *gflops_out = flop / (best * 1e-3) / 1e9;
  return CS_OK;
}
