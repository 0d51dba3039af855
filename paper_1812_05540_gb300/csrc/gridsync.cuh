// Bounded grid-wide barrier for cooperative launches (every CTA of the grid co-resident).  The counter
// only grows: the p-th barrier of a launch waits for p * gridDim.x arrivals past the launch's base, so
// nothing has to be reset between barriers.  Every wait polls at most `limit` times; on expiry (or when
// another CTA has already given up, seen through *err) it sets *err and returns false, and the kernel
// returns without touching the barrier again.
#pragma once
#include <stdint.h>

namespace ps_internal {

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// all CTAs arrive, then wait until the counter reaches target; false (and *err set) when the
// wait gives up after limit polls or another CTA has already given up
__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned long long target, int64_t limit,
                                             int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add(ctr, 1ull);
    int good = 1;
    int64_t it = 0;
    while (ld_acquire_u64(ctr) < target) {
      if (++it > limit || ((it & 255) == 0 && *(volatile int*)err)) {
        good = 0;
        atomicExch(err, 1);
        break;
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace ps_internal
