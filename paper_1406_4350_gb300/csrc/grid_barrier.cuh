// Grid-wide barrier of the cooperative Jacobi sweep, shared with the self-test of the
// library's bounded waits.
#pragma once

#include <stdint.h>

#include "../../include/chebfi.h"

namespace chebfi {

__device__ __forceinline__ void barrier_flag(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all blocks resident).  The wait is bounded:
// after limit_ns it records CHEBFI_ERR_CUDA and lets the block go on.
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* status,
                                             unsigned long long limit_ns = 1000000000ull) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned long long t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      // poll with plain acquire loads: read-modify-write polls from every waiting block
      // would queue behind each other (and behind the arrivals) on the one L2 line
      while (ld_acquire(gen) == g) {
        __nanosleep(32);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
          barrier_flag(status, CHEBFI_ERR_CUDA);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace chebfi
