// Deterministic block-wide scans and reductions (integer and float) built from
// warp shuffles in a fixed order: no atomics, the result does not depend on
// scheduling.
#pragma once
#include <cuda_runtime.h>

namespace sift {

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Exclusive scan over the block; *total receives the block sum. `tmp` needs
// blockDim.x / 32 + 1 ints of shared memory. All threads must call it.
__device__ __forceinline__ int block_excl_scan(int v, int *tmp, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int incl = warp_incl_scan(v);
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? tmp[lane] : 0;
    const int wi = warp_incl_scan(w);
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1) tmp[nw] = wi;
  }
  __syncthreads();
  const int r = tmp[warp] + incl - v;
  *total = tmp[nw];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_sum(int v, int *tmp) {
  int total;
  block_excl_scan(v, tmp, &total);
  return total;
}

}  // namespace sift
