// Residual norms without any device allocation.
//
// Some callers cannot allocate device memory: a host application that has already claimed the
// device's memory for its own pool, a monitor that must not let cudaMalloc / cudaFree
// synchronise the device while a solver is running, or a process whose allocator is locked
// down.  For them this file computes the two residual monitors of cs_residual
// (r_species = sqrt(sum_cells sum_s (R_s/V)^2), r_energy = sqrt(sum_cells (R_E/V)^2)) from a
// residual and the cell volumes the caller already holds, using a scratch buffer that is a
// file-scope static device array instead of memory the library allocates.
//
// The scratch array is CS_NORMS_STATIC_MAX_BLOCKS x 2 doubles (256 KiB) and stays resident on
// every GPU that loads the library until the process exits.  All calls share it and it keeps
// the contents of the last call; every call rewrites every slot it reads, so nothing needs
// clearing.  Calls that overlap on the GPU (different streams, or several host threads) race
// on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include "../../include/cs.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = CS_NORMS_STATIC_MAX_CELLS / kThreads;

// per-block partial sums [block][2], followed by the two final sums
static __device__ __align__(256) double g_norm_scratch[2 * kMaxBlocks + 2];

__global__ void __launch_bounds__(kThreads) k_norm_partials(const double* R, const double* V,
                                                            int N, int ns, int iE,
                                                            double* scratch) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rs = 0.0, re = 0.0;
  if (c < N) {
    const double iV = 1.0 / V[c];
    for (int s = 0; s < ns; ++s) {
      const double r = R[(size_t)s * N + c] * iV;
      rs += r * r;
    }
    const double r = R[(size_t)iE * N + c] * iV;
    re = r * r;
  }
  __shared__ double sh[2][kThreads];
  sh[0][threadIdx.x] = rs;
  sh[1][threadIdx.x] = re;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = sh[0][0];
    scratch[2 * blockIdx.x + 1] = sh[1][0];
  }
}

__global__ void __launch_bounds__(kThreads) k_norm_final(double* scratch, int nblocks) {
  __shared__ double sh[2][kThreads];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kThreads) {
    a += scratch[2 * k];
    b += scratch[2 * k + 1];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * kMaxBlocks] = sqrt(sh[0][0]);
    scratch[2 * kMaxBlocks + 1] = sqrt(sh[1][0]);
  }
}

// Device address of the scratch array in the current context.  The address belongs to the
// context, not to the device ordinal (it changes after cudaDeviceReset or under another context
// on the same device), so it is looked up on every call: cudaGetSymbolAddress allocates
// nothing.  The first lookup in a context may load the module, which is why the first call
// should come before any stream capture.
cudaError_t scratch_for_current_context(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" cs_status cs_residual_norms_static(const double* R_dev, const double* V_dev, int ncell,
                                              int nspecies, int ndim, void* cuda_stream,
                                              double norms_host[2]) {
  if (!R_dev || !V_dev || !norms_host) return CS_ERR_ARG;
  if (ncell < 1 || ncell > CS_NORMS_STATIC_MAX_CELLS) return CS_ERR_ARG;
  if (nspecies < 1 || (ndim != 2 && ndim != 3)) return CS_ERR_ARG;
  double* scratch = nullptr;
  if (scratch_for_current_context(&scratch) != cudaSuccess) return CS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (ncell + kThreads - 1) / kThreads;
  k_norm_partials<<<nb, kThreads, 0, st>>>(R_dev, V_dev, ncell, nspecies, nspecies + ndim, scratch);
  k_norm_final<<<1, kThreads, 0, st>>>(scratch, nb);
  if (cudaGetLastError() != cudaSuccess) return CS_ERR_CUDA;
  if (cudaMemcpyAsync(norms_host, scratch + 2 * kMaxBlocks, 2 * sizeof(double),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CS_ERR_CUDA;
  return CS_OK;
}
