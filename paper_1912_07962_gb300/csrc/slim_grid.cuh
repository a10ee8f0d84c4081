// Bounded grid-wide barrier for cooperative persistent launches (every CTA
// resident).  A wait that runs out records SLIM_ETIMEOUT and returns false;
// the CTA then leaves its kernel, and the others run out at their next
// barrier, so the context stays usable.
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"

namespace slim {

constexpr unsigned kGridSpin = 1u << 22;   // polls of a barrier before giving up (about a second)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// bar[0] counts arrivals, bar[1] is the generation (both zero before the
// launch's first barrier).  s_flag: a shared int of the CTA.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* status, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) + 1 == gridDim.x) {
      bar[0] = 0;
      __threadfence();
      st_release_u32(bar + 1, gen + 1);
    } else {
      unsigned it = 0;
      while (ld_acquire_u32(bar + 1) == gen) {
        if (++it > kGridSpin) {
          set_status(status, SLIM_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

}  // namespace slim
