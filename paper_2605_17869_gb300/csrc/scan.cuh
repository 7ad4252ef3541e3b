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

// ------------------------------------------------ single-pass chunked scan
//
// Exclusive prefix sums over the chunks of a list in one kernel, by decoupled
// look-back: each chunk publishes its count (an aggregate) as soon as it is
// known, then its inclusive prefix once it has summed its predecessors'
// aggregates back to the nearest published inclusive prefix. A status is one
// 64-bit word written by one store: bits 63-62 the kind (1 aggregate, 2
// inclusive), bits 61-32 the run's epoch, bits 31-0 the value. A word of
// another epoch is a leftover of an earlier run and counts as unpublished, so
// the status arrays need no clearing between runs. The values are integers,
// so the prefix does not depend on the order in which they are added.
//
// Waits are bounded: after `spins` polls without a status the wait gives up,
// records the run's epoch in *err (read back by the host) and counts the
// missing chunk as empty; every write stays within its capacity, so a lost
// wait costs correctness of that run's counts, never memory safety or a hang.
// A chunk only ever waits for chunks of lower index, and a block takes its
// chunks in increasing order, so the lowest unfinished chunk never waits.
constexpr unsigned long long kLbAgg = 1ull << 62, kLbInc = 2ull << 62;
constexpr unsigned kLbEpochMask = 0x3fffffffu;

struct LookbackCfg {
  unsigned epoch;   // 1 .. kLbEpochMask
  int spins;        // poll limit of one wait
  int hold;         // test hook: this chunk never publishes (-1: none)
  unsigned long long *err;
};

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long lb_word(unsigned long long kind, unsigned epoch,
                                                      int v) {
  return kind | ((unsigned long long)(epoch & kLbEpochMask) << 32) | (unsigned)v;
}
__device__ __forceinline__ bool lb_current(unsigned long long w, unsigned epoch) {
  return (w >> 62) != 0 && (unsigned)((w >> 32) & kLbEpochMask) == epoch;
}

// Warp-wide wait until st[idx] holds a status of this run on every lane with
// want set (lanes without want are ready). Returns false if it gave up.
__device__ __forceinline__ bool lb_wait(const unsigned long long *st, int idx, bool want,
                                        const LookbackCfg &cfg, unsigned long long *w) {
  for (int k = 0;; k++) {
    if (want) *w = lb_load(st + idx);
    const bool ready = !want || lb_current(*w, cfg.epoch);
    if (__all_sync(0xffffffffu, ready)) return true;
    if (k >= cfg.spins) {
      if (!ready) *w = 0;
      if ((threadIdx.x & 31) == 0) lb_store(cfg.err, cfg.epoch);
      return false;
    }
    __nanosleep(128);
  }
}

// Called by one full warp for chunk c of a list whose chunks of this image
// are [c0, c): returns (to every lane) the sum of the counts of chunks c0 ..
// c - 1 and publishes chunk c's statuses, given its count agg.
__device__ __forceinline__ int lb_exclusive(unsigned long long *st, int c0, int c, int agg,
                                            const LookbackCfg &cfg) {
  const int lane = threadIdx.x & 31;
  const bool pub = c != cfg.hold;
  if (c == c0) {
    if (lane == 0 && pub) lb_store(st + c, lb_word(kLbInc, cfg.epoch, agg));
    return 0;
  }
  if (lane == 0 && pub) lb_store(st + c, lb_word(kLbAgg, cfg.epoch, agg));
  int excl = 0;
  for (int j = c - 1;; j -= 32) {
    // Lane l looks at chunk j - l; chunks before c0 act as an inclusive 0.
    const int idx = j - lane;
    const bool valid = idx >= c0;
    unsigned long long w = 0;
    lb_wait(st, idx, valid, cfg, &w);
    const bool have = valid && lb_current(w, cfg.epoch);
    // The nearest lane holding an inclusive prefix (or past the image start,
    // or given up on) ends the look-back; lanes up to it contribute.
    const bool stop = !have || (w >> 62) == 2;
    const unsigned m = __ballot_sync(0xffffffffu, stop);
    const int last = m ? __ffs(m) - 1 : 31;
    int v = (lane <= last && have) ? (int)(unsigned)(w & 0xffffffffu) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (m) break;
  }
  if (lane == 0 && pub) lb_store(st + c, lb_word(kLbInc, cfg.epoch, excl + agg));
  return excl;
}

// One warp: wait for the per-image totals img_st[0, n) of this run and write
// their exclusive prefix to out[0, n] (out[n] the sum). A total that never
// arrives counts as 0 (and is recorded in *cfg.err).
__device__ __forceinline__ void lb_image_prefix(const unsigned long long *img_st, int n,
                                                const LookbackCfg &cfg, int *out) {
  const int lane = threadIdx.x & 31;
  int flat = 0;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int b = b0 + lane;
    unsigned long long w = 0;
    lb_wait(img_st, b, b < n, cfg, &w);
    const int x = (b < n && lb_current(w, cfg.epoch)) ? (int)(unsigned)(w & 0xffffffffu) : 0;
    const int incl = warp_incl_scan(x);
    if (b < n) out[b] = flat + incl - x;
    flat += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) out[n] = flat;
}

}  // namespace sift
