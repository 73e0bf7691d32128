// sph_grid.cuh -- grid-wide barrier for cooperative launches (every block of
// the grid is resident at once, so a block that waits only waits on blocks
// that are running).
//
// The barrier words live in device memory and start at zero.  Barrier k
// (1, 2, ... within one launch) waits until k x gridDim.x arrivals have been
// counted.  Each wait is bounded: when it runs out, the block sets
// SPH_ERR_TIMEOUT in the status word and the abort flag, which the other
// blocks' waits read, and the caller skips its remaining work.  The last
// block to leave (grid_leave) resets the words for the next launch.
#pragma once
#include <cstdint>

#include "sph.h"

namespace sphk {

struct GridBarrier {
  uint32_t arrive;  // arrivals of this launch (monotonic)
  uint32_t leave;   // blocks that have finished
  uint32_t abort;   // set when a wait ran out
  uint32_t word;    // one free word for the launch's own use (reset too)
};

constexpr uint32_t kGridSpinLimit = 1u << 20;  // polls of one wait: well under a second

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// barrier number k of this launch; false when the launch was aborted.
// s_ok is a __shared__ int of the calling block.  The arrival is a
// release add and the wait an acquire load at GPU scope; with the block
// barriers on both sides, every write made before the barrier by any thread
// of any block is visible to every thread after it.
__device__ __forceinline__ bool grid_sync(GridBarrier *g, uint32_t k, int32_t *status, int *s_ok,
                                          uint32_t spin_limit = kGridSpinLimit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t target = k * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&g->arrive), "r"(1u) : "memory");
    uint32_t it = 0;
    while (ld_acquire_u32(&g->arrive) < target) {
      if (ld_relaxed_u32(&g->abort)) {
        ok = 0;
        break;
      }
      if (++it > spin_limit) {
        atomicExch(&g->abort, 1u);
        atomicCAS(status, 0, SPH_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      if (it > 64) __nanosleep(64);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// every block calls this once, after its last barrier
__device__ __forceinline__ void grid_leave(GridBarrier *g) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&g->leave, 1u) == gridDim.x - 1u) {
      g->arrive = 0u;
      g->leave = 0u;
      g->abort = 0u;
      g->word = 0u;
      __threadfence();
    }
  }
}

}  // namespace sphk
