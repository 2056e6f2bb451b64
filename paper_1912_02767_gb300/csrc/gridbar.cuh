// gridbar.cuh -- bounded grid-wide barrier of the cooperative kernels:
// generation counter with two-level arrival (CTAs in groups of 16, the last
// of each group at the top, the last group bumps the generation); every
// wait is bounded in time (GridBar::limit_ns, else kWaitLimitNs), after
// which GridBar::err is set and every caller returns false.  Data written by other CTAs before a barrier
// must be read after it past L1 (__ldcg): L1 is not coherent across SMs.
#pragma once
#include "common.cuh"

namespace sdpg {

__device__ __forceinline__ bool gbar(GridBar* b) {
  // two-level arrival: CTAs count in groups of 16, the last of each group
  // counts at the top, the last group bumps the generation everybody waits on
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    const unsigned nb = gridDim.x, g = blockIdx.x >> 4, ng = (nb + 15) >> 4;
    const unsigned gs = (g + 1 < ng) ? 16u : nb - 16u * g;
    unsigned gen0 = *vgen;
    __threadfence();
    ok = 1;
    bool last = false;
    if (atomicAdd(&b->grp[g], 1u) == gs - 1) {
      atomicExch(&b->grp[g], 0u);
      __threadfence();
      if (atomicAdd(&b->top, 1u) == ng - 1) {
        atomicExch(&b->top, 0u);
        __threadfence();
        atomicAdd(&b->gen, 1u);
        last = true;
      }
    }
    if (!last) {
      const unsigned long long lim = b->limit_ns ? b->limit_ns : kWaitLimitNs;
      const unsigned long long t0 = globaltimer_ns();
      while (*vgen == gen0) {
        if (*(volatile int*)&b->err || globaltimer_ns() - t0 > lim) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (*(volatile int*)&b->err) ok = 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace sdpg
