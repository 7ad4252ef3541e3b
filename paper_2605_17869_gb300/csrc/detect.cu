// Detection (§3.2): DoG subtraction fused with the 26-neighbour extremum test
// and the contrast gate, compaction of candidates in canonical order, and
// sub-pixel refinement by a 3-D Taylor expansion solved with Cramer's rule.
//
// The DoG is never stored: every consumer recomputes D = G[i+1] - G[i] with the
// same single FP32 subtraction, so all stages see identical values.
//
// Candidates are first marked in a bitmap (one warp ballot per 32 pixels and
// layer), then compacted by a two-level prefix scan over bitmap words. The
// bitmap's memory order is (octave, layer, row, column), so the candidate list
// comes out in that canonical order independently of tile shapes or batch
// composition.
#include <algorithm>

#include "scan.cuh"
#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kThreads = 256;
constexpr int kExtThreads = 128;  // extrema scan: four warps per block, five blocks per SM

// ------------------------------------------------------------ extrema scan

// 3-input maximum / minimum (one instruction on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// One row of DoG values as the scan holds it, for the lane's column x: the
// maximum and minimum over columns x - 1 .. x + 1 of each of the S + 2 DoG
// layers, and for the tested layers 1 .. S the value itself and the larger and
// smaller of its left and right neighbours.
template <int S> struct ExtRow {
  float hx[S + 2], hn[S + 2];
  float c[S], lrx[S], lrn[S];
};

// DoG (one FP32 subtraction per value, as in every other stage) of one row
// from its S + 3 Gaussian levels, and the row's three-column maxima / minima
// (neighbours by warp shuffle; lanes 0 and 31 get meaningless values there,
// they only supply neighbours).
template <int S>
__device__ __forceinline__ void ext_row(ExtRow<S> &R, const float (&g)[S + 3]) {
#pragma unroll
  for (int l = 0; l < S + 2; l++) {
    const float v = g[l + 1] - g[l];
    const float lf = __shfl_up_sync(0xffffffffu, v, 1);
    const float rt = __shfl_down_sync(0xffffffffu, v, 1);
    R.hx[l] = max3f(lf, v, rt);
    R.hn[l] = min3f(lf, v, rt);
    if (l >= 1 && l <= S) {
      R.c[l - 1] = v;
      R.lrx[l - 1] = fmaxf(lf, rt);
      R.lrn[l - 1] = fminf(lf, rt);
    }
  }
}

// The rows a warp has in flight: a ring of kExtRing rows x (S + 3) levels x
// 32 lanes in shared memory, filled by 4-byte asynchronous copies (each lane
// copies its own column) so that kExtRing - 1 rows are on their way while
// one is consumed.
constexpr int kExtRing = 4;  // a power of two

__device__ __forceinline__ void cp_async4_ca(float *dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy the S + 3 levels of one image row at the lane's column into a ring
// slot (lp[l]: level l at row 0 and the lane's column; row_off: the row's
// offset, the same for the whole warp).
template <int S>
__device__ __forceinline__ void ext_issue(float *slot, const float *const (&lp)[S + 3],
                                          long long row_off) {
#pragma unroll
  for (int l = 0; l < S + 3; l++) cp_async4_ca(slot + l * 32, lp[l] + row_off);
}

// Test row y (P, C, N: rows y - 1, y, y + 1) and write its bitmap words:
// pixel x of layer s is a candidate when it lies inside the border, |D|
// exceeds the pre-gate, and D is strictly above the maximum, or strictly
// below the minimum, of its 26 neighbours. Those extrema are separable: the
// 9 values of layer s +- 1 reduce to max(hx(y - 1), hx(y), hx(y + 1)), the 8
// of layer s to max(hx(y - 1), hx(y + 1), left, right).
template <int S>
__device__ __forceinline__ void ext_test(const ExtRow<S> &P, const ExtRow<S> &C,
                                         const ExtRow<S> &N, bool inb, float thr, int lane,
                                         uint32_t *word) {
  // Rows where no pixel of the strip passes the border and pre-gate tests
  // in any layer have no candidate: skip the neighbour comparisons.
  float amax = fabsf(C.c[0]);
#pragma unroll
  for (int s = 2; s <= S; s++) amax = fmaxf(amax, fabsf(C.c[s - 1]));
  if (!__any_sync(0xffffffffu, inb && amax > thr)) {
    if (lane < S) *word = 0u;
    return;
  }
  float vx[S + 2], vn[S + 2];
#pragma unroll
  for (int l = 0; l < S + 2; l++) {
    vx[l] = max3f(P.hx[l], C.hx[l], N.hx[l]);
    vn[l] = min3f(P.hn[l], C.hn[l], N.hn[l]);
  }
  unsigned mine = 0u;
#pragma unroll
  for (int s = 1; s <= S; s++) {
    const float c = C.c[s - 1];
    const float mx = max3f(vx[s - 1], vx[s + 1], max3f(P.hx[s], N.hx[s], C.lrx[s - 1]));
    const float mn = min3f(vn[s - 1], vn[s + 1], min3f(P.hn[s], N.hn[s], C.lrn[s - 1]));
    // |c| > thr and (c > mx or c < mn), as one comparison with zero: the
    // differences of distinct finite FP32 values are never zero (gradual
    // underflow) and keep their sign, so each difference is positive exactly
    // when its comparison holds, and the minimum / maximum combine them. The
    // subtractions run on the FMA pipe, leaving the ALU pipe (the scan's
    // bound) three instructions instead of five.
    const float margin = fminf(fabsf(c) - thr, fmaxf(c - mx, mn - c));
    const bool ok = inb && margin > 0.f;
    const unsigned bits = __ballot_sync(0xffffffffu, ok);
    mine = lane == s - 1 ? bits : mine;
  }
  if (lane < S) *word = mine >> 1;  // lanes 1 .. 30 -> bits 0 .. 29
}

// A warp owns a strip of kBmCols = 30 columns x kExtTH rows: lane l holds
// column 30 tx - 1 + l, so lanes 1 .. 30 are the strip and lanes 0 and 31 its
// neighbours, and one bitmap word covers the strip's row. The warp streams
// down the strip: each image row's S + 3 levels are loaded once (the next
// row's loads are in flight while the current row is tested) and every test
// is done from registers. The candidate decisions are exact comparisons of
// the same FP32 values, so they do not depend on the tiling. Bitmap words are
// written by ballots; no atomics.
// HALF: the octave's levels are binary16 (fp16 storage mode). cp.async has no
// 2-byte copy, so each lane copies the 32-bit word that holds its column's
// value (4-byte aligned: rows start on 64-byte boundaries) and takes the low
// or the high half of it, widened to FP32, when it reads the row.
template <int S, bool HALF>
__global__ void __launch_bounds__(kExtThreads, 5) k_extrema(const Desc *__restrict__ d, int oct) {
  constexpr int WPB = kExtThreads / 32;
  constexpr int SLOT = (S + 3) * 32;
  __shared__ float ring[WPB][kExtRing * SLOT];
  const int n = d->n_img;
  const int *pre = d->tile_pre[TK_EXT][oct];
  const int total = pre[n];
  const int lane = threadIdx.x & 31;
  float *my = ring[threadIdx.x >> 5];
  const float thr = d->prefilter;
  const int bord = d->border;
  pdl_wait();
  for (int t = blockIdx.x * WPB + (threadIdx.x >> 5); t < total; t += gridDim.x * WPB) {
    if (t + gridDim.x * WPB >= total) pdl_trigger();  // this warp's last tile
    const int b = find_owner(pre, n, t);
    const OctDev od = d->oct[b * kMaxOct + oct];  // image b's octaves sit at fixed slots
    const int H = od.H, W = od.W;
    const long long pitch = od.pitch, ls = od.lstride;
    const int lt = t - pre[b];
    const int ty = lt / od.wpr, tx = lt - ty * od.wpr;
    const int x = tx * kBmCols - 1 + lane;
    const int y0 = ty * kExtTH, y1 = min(y0 + kExtTH, H);
    // lp[l]: the 32-bit word of level l, row 0, that holds the lane's column
    // (binary16 levels: the word of halves xc & ~1 and its neighbour); a row's
    // words are rstride apart.
    const float *lp[S + 3];
    const int xc = min(max(x, 0), W - 1);
    const bool hi_half = HALF && (xc & 1);
    const long long rstride = HALF ? pitch / 2 : pitch;
    {
      const float *G = HALF ? reinterpret_cast<const float *>(
                                  reinterpret_cast<const __half *>(d->pyr + od.lvl) + (xc & ~1))
                            : d->pyr + od.lvl + xc;
#pragma unroll
      for (int l = 0; l < S + 3; l++) lp[l] = G + l * (HALF ? ls / 2 : ls);
    }
    float *mine_ring = my + lane;
    const bool xin = lane >= 1 && lane <= kBmCols && x >= bord && x < W - bord;
    uint32_t *bmw = d->bm + od.bm + (long long)lane * H * od.wpr + tx;
    // Row k of the strip's sequence is image row y0 - 1 + k (clamped), k = 0 ..
    // n_rows - 1; it lives in ring slot k % kExtRing. One commit group per
    // row, empty past the end, so that the number of pending groups is fixed.
    const int n_rows = y1 - y0 + 2;
    auto issue = [&](int k) {
      if (k < n_rows) {
        const int row = min(max(y0 - 1 + k, 0), H - 1);
        ext_issue<S>(mine_ring + (k & (kExtRing - 1)) * SLOT, lp, row * rstride);
      }
      cp_async_commit();
    };
    auto consume = [&](ExtRow<S> &R, int k) {
      cp_async_wait<kExtRing - 1>();  // row k's group is complete
      const float *slot = mine_ring + (k & (kExtRing - 1)) * SLOT;
      float g[S + 3];
#pragma unroll
      for (int l = 0; l < S + 3; l++) {
        if (HALF) {
          const unsigned w = __float_as_uint(slot[l * 32]);
          g[l] = __half2float(__ushort_as_half((unsigned short)(hi_half ? w >> 16 : w & 0xffffu)));
        } else {
          g[l] = slot[l * 32];
        }
      }
      ext_row<S>(R, g);
      issue(k + kExtRing);  // into the slot just read (each lane rewrites only its own words)
    };
#pragma unroll
    for (int k = 0; k < kExtRing; k++) issue(k);
    ExtRow<S> A, B, C;
    consume(A, 0);
    consume(B, 1);
    // Rows rotate through A, B, C (previous, current, next) without copies.
    auto step = [&](ExtRow<S> &Pr, ExtRow<S> &Cu, ExtRow<S> &Nx, int y) {
      consume(Nx, y - y0 + 2);                                    // image row y + 1 (clamped)
      const bool inb = xin && y >= bord && y < H - bord;
      ext_test<S>(Pr, Cu, Nx, inb, thr, lane, bmw + (long long)y * od.wpr);
    };
    for (int y = y0; y < y1; y += 3) {
      step(A, B, C, y);
      if (y + 1 >= y1) break;
      step(B, C, A, y + 1);
      if (y + 2 >= y1) break;
      step(C, A, B, y + 2);
    }
    cp_async_wait<0>();  // no copy of this strip outlives it
    __syncwarp();
  }
}

// ----------------------------------------------------- bitmap compaction

// Candidate list of every image in canonical order (octave, layer, row,
// column), in one pass. Block g of G takes the contiguous range of bitmap
// chunks [C g / G, C (g + 1) / G):
//  1. it counts the set bits of its chunks (per chunk and warp, kept in
//     shared memory);
//  2. it takes the count of everything before its range from the
//     single-pass scan over blocks, so it only ever waits for blocks of lower
//     index, and at once publishes the global offset of every image that
//     starts in its range;
//  3. it writes its candidates chunk by chunk, each image's slots counted
//     from that image's start (published by the block that holds the image's
//     first chunk).
// The block with an image's last chunk writes the image's totals, and the
// last block forms the prefix of the candidate counts over the images.
constexpr int kCmpWarps = kThreads / 32;
constexpr int kMaxCh = 256;  // chunks per block whose counts are kept (more are recounted)

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int bm_chunk_words(const Desc *__restrict__ d, const ImgDev &im, int c,
                                              int c0, uint32_t (&words)[kChunk / kThreads],
                                              long long *w0_out) {
  constexpr int WPT = kChunk / kThreads;
  const long long w0 = (long long)(c - c0) * kChunk + threadIdx.x * WPT;
  const uint32_t *bm = d->bm + im.bm_begin;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    words[k] = (w0 + k < im.bm_words) ? bm[w0 + k] : 0u;
    cnt += __popc(words[k]);
  }
  *w0_out = w0;
  return cnt;
}

__global__ void __launch_bounds__(kThreads) k_bm_compact(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int tmp[kThreads / 32 + 1];
  __shared__ int s_w[kMaxCh][kCmpWarps];  // set bits per kept chunk and warp
  __shared__ int s_val;
  constexpr int WPT = kChunk / kThreads;  // words per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = d->n_img, C = d->n_bm_chunks, G = gridDim.x, g = blockIdx.x;
  const LookbackCfg cfg{d->lb_epoch, d->lb_spins, d->lb_hold, d->lb_err};
  const int ca = (int)((long long)C * g / G), cb = (int)((long long)C * (g + 1) / G);
  const int kept = min(cb - ca, kMaxCh);
  // Owners of the range's chunks: found once, then advanced (the chunks are
  // contiguous and images are in order).
  const int b_lo = ca < cb ? find_owner(d->bmc_pre, n, ca) : 0;
  uint32_t words[WPT];
  long long w0;
  // 1. Counts.
  int over = 0;
  for (int c = ca, b = b_lo; c < cb; c++) {
    while (c >= d->bmc_pre[b + 1]) b++;
    const int cnt = bm_chunk_words(d, d->img[b], c, d->bmc_pre[b], words, &w0);
    if (c - ca < kMaxCh) {
      const int ws = warp_sum_i(cnt);
      if (lane == 0) s_w[c - ca][warp] = ws;
    } else {
      over += cnt;
    }
  }
  __syncthreads();
  int part = over;
  for (int k = threadIdx.x; k < kept; k += kThreads)
#pragma unroll
    for (int w = 0; w < kCmpWarps; w++) part += s_w[k][w];
  const int agg = block_sum(part, tmp);
  // 2. Offset of the range; starts of the images beginning in it.
  if (threadIdx.x < 32) {
    const int ex = lb_exclusive(d->lb_bm, 0, g, agg, cfg);
    if (threadIdx.x == 0) s_val = ex;
  }
  __syncthreads();
  const int base = s_val;
  __syncthreads();
  {
    int acc = base;
    for (int c = ca, b = b_lo; c < cb; c++) {
      while (c >= d->bmc_pre[b + 1]) b++;
      if (c == d->bmc_pre[b] && threadIdx.x == 0)
        lb_store(d->lb_start + b, lb_word(kLbInc, cfg.epoch, acc));
      int t = 0;
      if (c - ca < kMaxCh) {
#pragma unroll
        for (int w = 0; w < kCmpWarps; w++) t += s_w[c - ca][w];
      } else {  // uniform over the block
        t = block_sum(bm_chunk_words(d, d->img[b], c, d->bmc_pre[b], words, &w0), tmp);
      }
      acc += t;
    }
  }
  // 3. Candidates.
  int carry = base;         // global offset of chunk c
  int cur = -1, start = 0;  // image of the previous chunk, global offset of its first slot
  for (int c = ca, b = b_lo; c < cb; c++) {
    while (c >= d->bmc_pre[b + 1]) b++;
    const ImgDev &im = d->img[b];
    const int c0 = d->bmc_pre[b];
    const int cnt = bm_chunk_words(d, im, c, c0, words, &w0);
    int pre, tot;
    if (c - ca < kMaxCh) {
      const int incl = warp_incl_scan(cnt);
      int wb = 0;
      tot = 0;
#pragma unroll
      for (int w = 0; w < kCmpWarps; w++) {
        const int x = s_w[c - ca][w];
        wb += w < warp ? x : 0;
        tot += x;
      }
      pre = wb + incl - cnt;
    } else {  // uniform over the block
      pre = block_excl_scan(cnt, tmp, &tot);
    }
    if (b != cur) {  // uniform over the block
      cur = b;
      if (c == c0) {
        start = carry;
      } else {  // the image began in a lower block's range (only the range's first image)
        if (threadIdx.x < 32) {
          unsigned long long w = 0;
          lb_wait(d->lb_start, b, threadIdx.x == 0, cfg, &w);
          if (threadIdx.x == 0) s_val = lb_current(w, cfg.epoch) ? (int)(unsigned)w : carry;
        }
        __syncthreads();
        start = s_val;
        __syncthreads();
      }
    }
    const int rel = carry - start;  // image-relative offset of chunk c
    int slot = rel + pre;
    if (cnt) {
      // Octave of the thread's words: found once and advanced (the words are
      // contiguous). Offsets within an octave's bitmap fit 32 bits.
      int o = 0;
      OctDev od = d->oct[im.oct0];
      for (int k = 0; k < WPT; k++) {
        uint32_t wv = words[k];
        if (!wv) continue;
        // Locate octave / layer / row / word of this bitmap word.
        const long long wa = im.bm_begin + w0 + k;
        while (o + 1 < im.n_oct && wa >= d->oct[im.oct0 + o + 1].bm) {
          o++;
          od = d->oct[im.oct0 + o];
        }
        const unsigned rel_w = (unsigned)(wa - od.bm);
        const unsigned lw = (unsigned)od.H * (unsigned)od.wpr;
        const unsigned li = rel_w / lw;
        const unsigned r2 = rel_w - li * lw;
        const int layer = (int)li + 1;
        const int y = (int)(r2 / (unsigned)od.wpr);
        const int wx = (int)(r2 - (unsigned)y * (unsigned)od.wpr);
        while (wv) {
          const int bit = __ffs(wv) - 1;
          wv &= wv - 1;
          if (slot >= 0 && slot < im.cand_cap)
            d->cand[im.cand_off + slot] = make_int4(o, layer, y, wx * kBmCols + bit);
          slot++;
        }
      }
    }
    if (threadIdx.x == 0 && c == d->bmc_pre[b + 1] - 1) {
      const int total = max(0, rel + tot);
      const int nc = min(total, im.cand_cap);
      ImgCounters &k = d->cnt[b];
      k.n_cand_raw = total;
      k.n_cand = nc;
      k.flags = total > im.cand_cap ? TF_CAND : 0;
      lb_store(d->lb_img + b, lb_word(kLbInc, cfg.epoch, nc));
    }
    carry += tot;
  }
  if (g == G - 1 && threadIdx.x < 32) lb_image_prefix(d->lb_img, n, cfg, d->cand_flat);
}

// ------------------------------------------------------------ refinement

__device__ __forceinline__ float det3(float a00, float a01, float a02, float a10, float a11,
                                      float a12, float a20, float a21, float a22) {
  return a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
         a02 * (a10 * a21 - a11 * a20);
}

__device__ __forceinline__ int round_half_away(float v) {
  const float a = floorf(fabsf(v) + 0.5f);
  return (int)(v >= 0.f ? a : -a);
}

// Levels s - 1 .. s + 2 at rows y - 1 .. y + 1 and columns x - 1 .. x + 1 of
// an octave's level stack G (FP32, or binary16 widened: HF).
template <bool HF>
__device__ __forceinline__ void refine_window(const float *__restrict__ G, int s, int y, int x,
                                              long long ls, int pitch, float (&g)[4][3][3]) {
  const long long base = (long long)(s - 1) * ls + (long long)(y - 1) * pitch + (x - 1);
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int bb = 0; bb < 3; bb++)
#pragma unroll
      for (int cc = 0; cc < 3; cc++) g[a][bb][cc] = lvl_ld(G, HF, base + a * ls + bb * pitch + cc);
}

__global__ void __launch_bounds__(kThreads) k_refine(const Desc *__restrict__ d) {
  pdl_wait();
  const int n = d->n_img;
  const int total = d->cand_flat[n];
  const int S = d->n_scales, bord = d->border, iters = d->max_iter;
  const float T = d->contrast_thr, er = d->edge_ratio;
  // Runs of 32 consecutive candidates go to the warps in turn, block first
  // (run c to block c % G, warp (c / G) % 8): a few thousand candidates still
  // spread over every SM, and the lanes of a warp refine neighbouring
  // candidates (canonical order: same layer, nearby rows), whose 3 x 3 x 3
  // windows share cache sectors.
  const int lane = threadIdx.x & 31;
  const int NW = gridDim.x * (blockDim.x >> 5);
  for (int run = blockIdx.x + gridDim.x * (threadIdx.x >> 5); run * 32 < total; run += NW) {
    const int t = run * 32 + lane;
    if (t >= total) continue;
    const int b = find_owner(d->cand_flat, n, t);
    const ImgDev &im = d->img[b];
    const long long slot = im.cand_off + (t - d->cand_flat[b]);
    const int4 cd = d->cand[slot];
    const int o = cd.x;
    int s = cd.y, y = cd.z, x = cd.w;
    const OctDev od = d->oct[im.oct0 + o];
    const float *G = d->pyr + od.lvl;
    const bool hf = od.half != 0;
    const long long ls = od.lstride;
    const int pitch = od.pitch;
    int code = RC_NOCONV;
    float dX = 0.f, dY = 0.f, dS = 0.f, gx = 0.f, gy = 0.f, gs = 0.f, c = 0.f;
    float hxx = 0.f, hyy = 0.f, hxy = 0.f;
    bool conv = false;
    for (int it = 0; it < iters; it++) {
      // The 3 x 3 x 3 DoG neighbourhood of layers s - 1 .. s + 1: the four
      // Gaussian levels s - 1 .. s + 2 are each loaded once (36 values), and
      // DoG layer k is level k + 1 minus level k, one FP32 subtraction.
      float g[4][3][3];
      if (hf)
        refine_window<true>(G, s, y, x, ls, pitch, g);
      else
        refine_window<false>(G, s, y, x, ls, pitch, g);
      float v[3][3][3];
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int bb = 0; bb < 3; bb++)
#pragma unroll
          for (int cc = 0; cc < 3; cc++) v[a][bb][cc] = g[a + 1][bb][cc] - g[a][bb][cc];
      c = v[1][1][1];
      gx = 0.5f * (v[1][1][2] - v[1][1][0]);
      gy = 0.5f * (v[1][2][1] - v[1][0][1]);
      gs = 0.5f * (v[2][1][1] - v[0][1][1]);
      hxx = v[1][1][2] + v[1][1][0] - 2.0f * c;
      hyy = v[1][2][1] + v[1][0][1] - 2.0f * c;
      const float hss = v[2][1][1] + v[0][1][1] - 2.0f * c;
      hxy = 0.25f * (v[1][2][2] - v[1][2][0] - v[1][0][2] + v[1][0][0]);
      const float hxs = 0.25f * (v[2][1][2] - v[2][1][0] - v[0][1][2] + v[0][1][0]);
      const float hys = 0.25f * (v[2][2][1] - v[2][0][1] - v[0][2][1] + v[0][0][1]);
      const float det = det3(hxx, hxy, hxs, hxy, hyy, hys, hxs, hys, hss);
      if (det == 0.f) { code = RC_SINGULAR; break; }
      // Cramer's rule for H delta = -g.
      dX = det3(-gx, hxy, hxs, -gy, hyy, hys, -gs, hys, hss) / det;
      dY = det3(hxx, -gx, hxs, hxy, -gy, hys, hxs, -gs, hss) / det;
      dS = det3(hxx, hxy, -gx, hxy, hyy, -gy, hxs, hys, -gs) / det;
      if (!isfinite(dX) || !isfinite(dY) || !isfinite(dS)) { code = RC_SINGULAR; break; }
      const float m = fmaxf(fabsf(dX), fmaxf(fabsf(dY), fabsf(dS)));
      if (m < 0.5f) { conv = true; break; }
      if (m > 1e7f) { code = RC_BOUNDS; break; }
      x += round_half_away(dX);
      y += round_half_away(dY);
      s += round_half_away(dS);
      if (s < 1 || s > S || x < bord || x >= od.W - bord || y < bord || y >= od.H - bord) {
        code = RC_BOUNDS;
        break;
      }
    }
    float resp = 0.f;
    if (conv) {
      const float contrast = c + 0.5f * (gx * dX + gy * dY + gs * dS);
      resp = fabsf(contrast);
      if (resp < T) {
        code = RC_CONTRAST;
      } else {
        const float tr = hxx + hyy;
        const float dt = hxx * hyy - hxy * hxy;
        code = (dt <= 0.f || tr * tr * er >= (er + 1.f) * (er + 1.f) * dt) ? RC_EDGE : RC_KEEP;
      }
    }
    RefRec r;
    r.o = o; r.s = s; r.y = y; r.x = x;
    r.dx = dX; r.dy = dY; r.ds = dS; r.resp = resp;
    d->ref[slot] = r;
    d->code[slot] = code;
  }
}

}  // namespace

cudaError_t extrema_set_attributes() { return cudaSuccess; }

int compact_max_ctas() {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bm_compact, kThreads, 0);
  if (e == cudaSuccess) e = cc_compact_occupancy(&b);
  return (e == cudaSuccess && a > 0 && b > 0) ? std::min(a, b) : 1;
}

int extrema_max_ctas(int n_scales) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (n_scales) {
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extrema<2, false>, kExtThreads, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extrema<3, false>, kExtThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extrema<4, false>, kExtThreads, 0); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extrema<5, false>, kExtThreads, 0); break;
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_extrema<6, false>, kExtThreads, 0); break;
    default: break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_extrema(const Desc *d, int oct, int n_scales, int grid, cudaStream_t s, bool pdl,
                           bool half) {
#define EXT_CASE(SS)                                                                       \
  case SS:                                                                                 \
    if (half)                                                                              \
      return pdl ? launch_pdl(k_extrema<SS, true>, grid, kExtThreads, 0, s, d, oct)          \
                 : launch_plain(k_extrema<SS, true>, grid, kExtThreads, 0, s, d, oct);       \
    return pdl ? launch_pdl(k_extrema<SS, false>, grid, kExtThreads, 0, s, d, oct)           \
               : launch_plain(k_extrema<SS, false>, grid, kExtThreads, 0, s, d, oct);
  switch (n_scales) {
    EXT_CASE(2)
    EXT_CASE(3)
    EXT_CASE(4)
    EXT_CASE(5)
    EXT_CASE(6)
    default: return cudaErrorInvalidValue;
  }
#undef EXT_CASE
}

cudaError_t launch_bm_compact(const Desc *d, int grid, cudaStream_t s) {
  return launch_pdl(k_bm_compact, grid, kThreads, 0, s, d);
}

cudaError_t launch_refine(const Desc *d, int grid, cudaStream_t s) {
  return launch_pdl(k_refine, grid, kThreads, 0, s, d);
}

}  // namespace sift
