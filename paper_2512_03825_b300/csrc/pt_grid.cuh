// pt_grid.cuh -- the bounded grid barrier of the cooperative (persistent) kernels.
#pragma once
#include <stdint.h>

#include "pt.h"
#include "pt_device.cuh"

namespace ptb {

// Every CTA arrives once; returns false when the wait gave up (time limit or a status set
// by another CTA): the caller leaves the kernel. Thread 0 polls the counter with relaxed
// loads and orders the CTA's later reads with one fence after the wait. A grid of one CTA
// that waits for no extra arrival (`stalled`: the test hook that makes a wait run out) has
// no one to wait for: the block barrier and one fence give the same ordering.
__device__ inline bool grid_barrier(unsigned* bar, unsigned target, int* status,
                                    uint64_t limit_ns, int* ok_s, bool stalled = false) {
  if (gridDim.x == 1 && !stalled) {
    __syncthreads();
    if (threadIdx.x == 0) __threadfence();
    __syncthreads();
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();  // the CTA's writes (ordered before by the block barrier) go first
    atomicAdd(bar, 1u);
    const uint64_t t0 = global_ns();
    // the status word and the clock are looked at every 16th poll only: each is a round
    // trip of its own, and between them the counter poll is the whole loop
    for (unsigned polls = 1; (int)(ld_relaxed_u32(bar) - target) < 0; ++polls) {
      if ((polls & 15u) != 0) continue;
      if (*(volatile int*)status != 0) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns) {
        atomicCAS(status, 0, PT_ETIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

}  // namespace ptb
