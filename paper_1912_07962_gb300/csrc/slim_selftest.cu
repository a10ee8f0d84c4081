// Self-test of the bounded device waits: a grid barrier that one CTA never
// reaches.  The waiting CTA gives up after its poll limit, records
// SLIM_ETIMEOUT and returns, so the kernel ends and the context stays usable.
#include <cuda_runtime.h>

#include "slim.h"
#include "slim_grid.cuh"

namespace slim {
namespace {

__global__ void barrier_timeout_kernel(unsigned* bar, int* status) {
  __shared__ int s_flag;
  if (blockIdx.x == 1) return;   // this CTA never arrives at the barrier
  grid_barrier(bar, status, &s_flag);
}

}  // namespace
}  // namespace slim

extern "C" slim_status slim_selftest_wait(void* cuda_stream) {
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* bar = nullptr;
  int* status = nullptr;
  if (cudaMalloc(&bar, 2 * sizeof(unsigned)) != cudaSuccess) return SLIM_ENOMEM;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(bar);
    return SLIM_ENOMEM;
  }
  int st = SLIM_ECUDA;
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    // cooperative: both CTAs resident, so only the missing arrival holds the wait
    void* params[] = {&bar, &status};
    e = cudaLaunchCooperativeKernel((const void*)slim::barrier_timeout_kernel, dim3(2), dim3(32),
                                    params, 0, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bar);
  cudaFree(status);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLIM_ECUDA;
  }
  return (slim_status)st;
}
