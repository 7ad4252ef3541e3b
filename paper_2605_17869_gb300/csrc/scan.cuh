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

// Exclusive scan of cnt[0, n) into off[0, n) by one warp; every lane returns
// the total. Each lane issues 8 loads ahead of the 8 warp scans they feed.
__device__ __forceinline__ int warp_excl_scan_array(const int *cnt, int *off, int n) {
  const int lane = threadIdx.x & 31;
  int carry = 0;
  for (int base = 0; base < n; base += 256) {
    int v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int i = base + k * 32 + lane;
      v[k] = i < n ? cnt[i] : 0;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int incl = warp_incl_scan(v[k]);
      const int i = base + k * 32 + lane;
      if (i < n) off[i] = carry + incl - v[k];
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  return carry;
}

// Exclusive scan of v[0, n) (shared or global) into out[0, n) by one warp;
// out[n] receives the total.
__device__ __forceinline__ void warp_excl_scan_small(const int *v, int *out, int n) {
  const int lane = threadIdx.x & 31;
  int flat = 0;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int b = b0 + lane;
    const int x = b < n ? v[b] : 0;
    const int incl = warp_incl_scan(x);
    if (b < n) out[b] = flat + incl - x;
    flat += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) out[n] = flat;
}

__device__ __forceinline__ int block_sum(int v, int *tmp) {
  int total;
  block_excl_scan(v, tmp, &total);
  return total;
}

}  // namespace sift
