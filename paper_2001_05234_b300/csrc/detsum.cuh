// Run-to-run reproducible sums of one double per block of a 1-D grid.
//
// Floating-point addition is not associative, so a total assembled with atomicAdd depends on the
// order in which the blocks finish, and a result built from it (the mean of the singular solution, the
// constant-flow-rate forcing) changes in its last bits from one run to the next.  Here each block
// stores its value in its own slot; the block that arrives last (found with an atomic counter, no
// waiting on other blocks) adds the slots in index order and writes the total, then resets the
// counter for the next use.  The total depends only on the values and on the launch shape.
#pragma once
#include <cuda_runtime.h>

namespace cans {

struct DetSum {
  double* slots = nullptr;    // at least gridDim.x entries
  unsigned* count = nullptr;  // 0 between uses (the last block resets it)
  double* out = nullptr;      // the total, overwritten; nullptr: no sum wanted
};

// Sum of v over the block, valid in thread 0 (blockDim.x a multiple of 32; every thread calls it).
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // a previous call's readers are done with red
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;
}

// Every thread of the block calls this; v (the block's value) is read from thread 0.
__device__ __forceinline__ void det_sum_finish(double v, const DetSum& d) {
  __shared__ unsigned last;
  if (threadIdx.x == 0) {
    d.slots[blockIdx.x] = v;
    __threadfence();  // the slot is visible before the arrival is counted
    last = (atomicAdd(d.count, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;  // uniform over the block
  __threadfence();
  double s = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(d.slots + b);
  s = block_sum_d(s);
  if (threadIdx.x == 0) {
    *d.out = s;
    *d.count = 0u;
  }
}

}  // namespace cans
