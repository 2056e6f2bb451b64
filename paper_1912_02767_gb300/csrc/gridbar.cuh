// gridbar.cuh -- bounded grid-wide barrier of the cooperative kernels:
// generation counter with one arrival counter (the last arrival bumps the
// generation); every
// wait is bounded in time (GridBar::limit_ns, else kWaitLimitNs), after
// which GridBar::err is set and every caller returns false.  Data written by other CTAs before a barrier
// must be read after it past L1 (__ldcg): L1 is not coherent across SMs.
#pragma once
#include "common.cuh"

namespace sdpg {

__device__ __forceinline__ bool gbar(GridBar* b) {
  // one arrival counter: the last of the G arrivals resets it and bumps the
  // generation everybody waits on (three L2 atomics on the critical path;
  // at this grid size the contention of a single counter costs less than a
  // second level of arrivals)
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    const unsigned gen0 = *vgen;
    __threadfence();
    ok = 1;
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long lim = b->limit_ns ? b->limit_ns : kWaitLimitNs;
      const unsigned long long t0 = globaltimer_ns();
      unsigned polls = 0;
      while (*vgen == gen0) {
        // the clock is read every 16th poll, every poll under a short test limit
        if ((lim < 1000000ull || (++polls & 15u) == 0) &&
            (*(volatile int*)&b->err || globaltimer_ns() - t0 > lim)) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
      }
    }
    if (*(volatile int*)&b->err) ok = 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace sdpg
