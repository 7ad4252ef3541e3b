// Orientation and descriptor (§3.2), output cap, and the deterministic
// reduction scheme of §5 ("Bitwise Deterministic GPU Execution").
//
// Orientation takes one warp per keypoint, the descriptor one block of four
// warps. Threads sweep the sample window in a fixed order and accumulate
// into thread-private histogram columns in shared memory (a word is only ever
// touched by one thread at a time, in an order fixed by the code); the
// columns are then summed bin by bin in a fixed order. No atomics are used
// anywhere, so outputs are bitwise reproducible.
#include "scan.cuh"
#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr int kKpWarps = 4;  // warps per keypoint (orientation and descriptor)
constexpr int kThreads = 256;

__device__ __forceinline__ float sigma_of(const Desc *d, const RefRec &r) {
  return d->sigma0 * exp2f(((float)r.s + r.ds) / (float)d->n_scales);
}

// A pyramid level seen from one pixel: v[off] is the element off places
// (off = dy * pitch + dx) from it, FP32 or (HF) binary16 widened to FP32.
// The 64-bit address is formed once per keypoint; sample offsets are 32-bit.
template <bool HF>
struct LevelView {
  const void *p;
  __device__ __forceinline__ float operator[](int off) const {
    if (HF) return __half2float(__ldg(static_cast<const __half *>(p) + off));
    return __ldg(static_cast<const float *>(p) + off);
  }
};
template <bool HF>
__device__ __forceinline__ LevelView<HF> level_at(const float *L, long long lofs, int pitch, int x,
                                                  int y) {
  const long long e = lofs + (long long)y * pitch + x;
  if (HF) return {reinterpret_cast<const __half *>(L) + e};
  return {L + e};
}

// ------------------------------------------------------------ orientation

// One warp per kept candidate; a block holds kOriWarps independent warps.
// The warp sweeps the (2R + 1)^2 window as one flat list of samples, lane l
// taking samples l, l + 32, ...; lane l votes into its private column
// hist[bin][l], and bin k is the sum of the 32 columns in a fixed order, so
// the histogram is bitwise reproducible. MIXED: the pyramid has binary16
// octaves (fp16 storage mode) and the level type is chosen per keypoint.
constexpr int kOriWarps = 8;

// Nearest-bin vote of one gradient: weight wgt into bin floor(36 theta / 2 pi
// + 1/2) of lane's column.
__device__ __forceinline__ void ori_vote(float (*hist)[32], int lane, float dx, float dy,
                                         float wgt) {
  const float mag = sqrtf(dx * dx + dy * dy);
  float th = atan2f(dy, dx);
  if (th < 0.f) th += kTwoPi;
  int bin = (int)floorf(th * ((float)kOriBins / kTwoPi) + 0.5f);
  if (bin >= kOriBins) bin -= kOriBins;
  // |dx| = |dy|: theta is exactly 45 (2q + 1) degrees, a bin boundary the
  // nearest-bin rule floor(36 theta / 2 pi + 1/2) resolves upward; decided in
  // integers rather than left to the rounding of atan2f.
  if (fabsf(dx) == fabsf(dy) && dx != 0.f) {
    const int qd = dy > 0.f ? (dx > 0.f ? 0 : 1) : (dx < 0.f ? 2 : 3);
    bin = (kOriBins * (2 * qd + 1) + 4) / 8 % kOriBins;
  }
  hist[bin][lane] += wgt * mag;
}

// The window's samples, lane l taking samples l, l + 32, l + 64, ... in that
// order, three per step: the twelve loads of a step are issued before any of
// its votes, so that more loads are in flight per warp.
template <bool HF>
__device__ __forceinline__ void ori_sweep(const float *__restrict__ L, long long lofs, int pitch,
                                          int H, int W, int x0, int y0, int R, float ninv,
                                          float (*hist)[32], int lane) {
  const LevelView<HF> v = level_at<HF>(L, lofs, pitch, x0, y0);
  const int side = 2 * R + 1, nsamp = side * side;
  // Sample q = jj * side + c; advancing q by 32 adds dr rows and dc columns.
  const int dr = 32 / side, dc = 32 - dr * side;
  int jj = lane / side, c = lane - jj * side;
  auto advance = [&]() {
    c += dc;
    jj += dr;
    if (c >= side) {
      c -= side;
      jj++;
    }
  };
  // Inside the window with a full 3 x 3 neighbourhood in the level.
  auto inside = [&](int q, int i, int j) {
    const int px = x0 + i, py = y0 + j;
    return q < nsamp && px >= 1 && px <= W - 2 && py >= 1 && py <= H - 2;
  };
  // Without branches: a sample outside the window or the image reads the
  // keypoint's own pixel neighbourhood (always inside: keypoints keep the
  // border) and votes with weight 0, which leaves its bin unchanged.
  constexpr int NS = 3;
  for (int q = lane; q < nsamp; q += 32 * NS) {
    int ii[NS], jv[NS], off[NS];
    bool ok[NS];
#pragma unroll
    for (int k = 0; k < NS; k++) {
      ii[k] = c - R;
      jv[k] = jj - R;
      advance();
      ok[k] = inside(q + 32 * k, ii[k], jv[k]);
      off[k] = ok[k] ? jv[k] * pitch + ii[k] : 0;
    }
    float gx[NS], gy[NS];
#pragma unroll
    for (int k = 0; k < NS; k++) {
      gx[k] = v[off[k] + 1] - v[off[k] - 1];
      gy[k] = v[off[k] + pitch] - v[off[k] - pitch];
    }
#pragma unroll
    for (int k = 0; k < NS; k++) {
      const float w = expf((float)(ii[k] * ii[k] + jv[k] * jv[k]) * ninv);
      ori_vote(hist, lane, gx[k], gy[k], ok[k] ? w : 0.f);
    }
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(kOriWarps * 32, 4) k_orientation(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ float s_hist[kOriWarps][kOriBins][32];
  __shared__ float s_sum[kOriWarps][kOriBins];
  __shared__ float s_sm[kOriWarps][kOriBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float(*hist)[32] = s_hist[warp];
  float *hsum = s_sum[warp], *hsm = s_sm[warp];
  const int n = d->n_img;
  const int total = d->cand_flat[n];
  const bool upright = d->upright != 0;
  // Warp g of NW takes the candidate slots g, g + NW, g + 2 NW, ..., 32 at a
  // time (lane l looks at the l-th of them): the lanes settle the rejected
  // slots (no peak) and, in upright mode, the kept ones (one peak at angle
  // 0); the kept slots are then taken one at a time by the whole warp. The
  // interleave spreads the kept candidates evenly over the warps.
  const int NW = gridDim.x * kOriWarps;
  for (int g0 = blockIdx.x + gridDim.x * warp; g0 < total; g0 += 32 * NW) {
    const int tl = g0 + lane * NW;
    int bl = 0;
    long long sl = 0;
    bool keep = false;
    if (tl < total) {
      bl = find_owner(d->cand_flat, n, tl);
      sl = d->img[bl].cand_off + (tl - d->cand_flat[bl]);
      keep = d->code[sl] == RC_KEEP;
      if (!keep || upright) {
        d->npk[sl] = keep ? 1 : 0;
        if (keep) d->angs[sl * kMaxPeaks] = 0.f;
      }
    }
    unsigned todo = upright ? 0u : __ballot_sync(0xffffffffu, keep);
    while (todo) {
      const int kl = __ffs(todo) - 1;
      todo &= todo - 1;
      const int b = __shfl_sync(0xffffffffu, bl, kl);
      const long long slot = __shfl_sync(0xffffffffu, sl, kl);
      const ImgDev &im = d->img[b];
      const RefRec r = d->ref[slot];
      const OctDev od = d->oct[im.oct0 + r.o];
      const float *L = d->pyr + od.lvl;
      const long long lofs = (long long)r.s * od.lstride;
      const float sw = 1.5f * sigma_of(d, r);
      const int R = (int)floorf(3.0f * sw + 0.5f);
      const float ninv = -1.0f / (2.0f * sw * sw);
#pragma unroll 4
      for (int k = 0; k < kOriBins; k++) hist[k][lane] = 0.f;
      if (MIXED && od.half != 0)
        ori_sweep<true>(L, lofs, od.pitch, od.H, od.W, r.x, r.y, R, ninv, hist, lane);
      else
        ori_sweep<false>(L, lofs, od.pitch, od.H, od.W, r.x, r.y, R, ninv, hist, lane);
      __syncwarp();
      // Bin k: the 32 columns in the order k, k + 1, ... (mod 32); the rotated
      // start puts the lanes on distinct banks.
      for (int k = lane; k < kOriBins; k += 32) {
        float sacc = 0.f;
#pragma unroll 8
        for (int q = 0; q < 32; q++) sacc += hist[k][(q + k) & 31];
        hsum[k] = sacc;
      }
      __syncwarp();
      for (int k = lane; k < kOriBins; k += 32) {
        const float hm = hsum[(k + kOriBins - 1) % kOriBins];
        const float hp = hsum[(k + 1) % kOriBins];
        hsm[k] = 0.25f * hm + 0.5f * hsum[k] + 0.25f * hp;
      }
      __syncwarp();
      float hmax = 0.f;
      for (int k = lane; k < kOriBins; k += 32) hmax = fmaxf(hmax, hsm[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
      const float thr = d->ori_peak_ratio * hmax;
      int base = 0;
      for (int k0 = 0; k0 < kOriBins; k0 += 32) {
        const int k = k0 + lane;
        bool peak = false;
        float ang = 0.f;
        if (k < kOriBins) {
          const float hk = hsm[k];
          const float hm = hsm[(k + kOriBins - 1) % kOriBins];
          const float hp = hsm[(k + 1) % kOriBins];
          if (hk > hm && hk > hp && hk >= thr) {
            peak = true;
            float kf = (float)k + 0.5f * (hm - hp) / (hm - 2.0f * hk + hp);
            if (kf < 0.f) kf += (float)kOriBins;
            if (kf >= (float)kOriBins) kf -= (float)kOriBins;
            ang = kf * (360.0f / (float)kOriBins);
            if (ang >= 360.0f) ang -= 360.0f;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, peak);
        if (peak) d->angs[slot * kMaxPeaks + base + __popc(m & ((1u << lane) - 1u))] = ang;
        base += __popc(m);
      }
      if (lane == 0) d->npk[slot] = base;
      __syncwarp();  // the next keypoint rewrites this warp's histogram
    }
  }
}

// --------------------------------------------- oriented keypoint compaction

// The oriented keypoints of every image in canonical order (candidate slot,
// then peak), in one pass over chunks of kChunk candidate slots, organised as
// k_bm_compact (contiguous chunk ranges per block, counts kept per chunk and
// warp, one scan over blocks, image starts published right after it). The
// block with an image's last chunk writes the image's oriented, capped and
// final counts (and the caller's count output); the last block forms the
// prefix of the final counts over the images.
constexpr int kCmpWarps = kThreads / 32;
constexpr int kMaxCh = 256;

__device__ __forceinline__ int cc_chunk_peaks(const Desc *__restrict__ d, const ImgDev &im, int nc,
                                              int c, int c0, int (&np)[kChunk / kThreads],
                                              int *s0_out) {
  constexpr int SPT = kChunk / kThreads;
  const int s0 = (c - c0) * kChunk + threadIdx.x * SPT;
  int v = 0;
#pragma unroll
  for (int k = 0; k < SPT; k++) {
    np[k] = (s0 + k < nc) ? d->npk[im.cand_off + s0 + k] : 0;
    v += np[k];
  }
  *s0_out = s0;
  return v;
}

__global__ void __launch_bounds__(kThreads) k_cc_compact(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int tmp[kThreads / 32 + 1];
  __shared__ int s_w[kMaxCh][kCmpWarps];
  __shared__ int s_val;
  __shared__ int s_act[kMaxImg + 1];
  constexpr int SPT = kChunk / kThreads;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = d->n_img, g = blockIdx.x;
  const LookbackCfg cfg{d->lb_epoch, d->lb_spins, d->lb_hold, d->lb_err};
  // Only the chunks that hold candidates are scanned: image b's n_cand
  // candidates fill its first ceil(n_cand / kChunk) chunks (at least one, so
  // that every image has a chunk whose block writes its totals). s_act is the
  // prefix of those counts over the images; the blocks beyond the number of
  // active chunks take no part.
  if (warp == 0) {
    int flat = 0;
    for (int b0 = 0; b0 < n; b0 += 32) {
      const int b = b0 + lane;
      const int a = b < n ? max(1, (d->cnt[b].n_cand + kChunk - 1) / kChunk) : 0;
      const int incl = warp_incl_scan(a);
      if (b < n) s_act[b + 1] = flat + incl;
      flat += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) s_act[0] = 0;
  }
  __syncthreads();
  const int C = s_act[n], G = min((int)gridDim.x, C);
  if (g >= G) return;
  const int ca = (int)((long long)C * g / G), cb = (int)((long long)C * (g + 1) / G);
  const int kept = min(cb - ca, kMaxCh);
  // Owners of the range's chunks: found once, then advanced (the chunks are
  // contiguous and images are in order).
  const int b_lo = ca < cb ? find_owner(s_act, n, ca) : 0;
  int np[SPT];
  int s0;
  int over = 0;
  for (int c = ca, b = b_lo; c < cb; c++) {
    while (c >= s_act[b + 1]) b++;
    const int v = cc_chunk_peaks(d, d->img[b], d->cnt[b].n_cand, c, s_act[b], np, &s0);
    if (c - ca < kMaxCh) {
      int ws = v;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
      if (lane == 0) s_w[c - ca][warp] = ws;
    } else {
      over += v;
    }
  }
  __syncthreads();
  int part = over;
  for (int k = threadIdx.x; k < kept; k += kThreads)
#pragma unroll
    for (int w = 0; w < kCmpWarps; w++) part += s_w[k][w];
  const int agg = block_sum(part, tmp);
  if (threadIdx.x < 32) {
    const int ex = lb_exclusive(d->lb_cc, 0, g, agg, cfg);
    if (threadIdx.x == 0) s_val = ex;
  }
  __syncthreads();
  const int base = s_val;
  __syncthreads();
  unsigned long long *starts = d->lb_start + kMaxImg;
  {
    int acc = base;
    for (int c = ca, b = b_lo; c < cb; c++) {
      while (c >= s_act[b + 1]) b++;
      if (c == s_act[b] && threadIdx.x == 0) lb_store(starts + b, lb_word(kLbInc, cfg.epoch, acc));
      int t = 0;
      if (c - ca < kMaxCh) {
#pragma unroll
        for (int w = 0; w < kCmpWarps; w++) t += s_w[c - ca][w];
      } else {  // uniform over the block
        t = block_sum(cc_chunk_peaks(d, d->img[b], d->cnt[b].n_cand, c, s_act[b], np, &s0), tmp);
      }
      acc += t;
    }
  }
  int carry = base;
  int cur = -1, start = 0;
  for (int c = ca, b = b_lo; c < cb; c++) {
    while (c >= s_act[b + 1]) b++;
    const ImgDev &im = d->img[b];
    const int c0 = s_act[b];
    const int v = cc_chunk_peaks(d, im, d->cnt[b].n_cand, c, c0, np, &s0);
    int pre, tot;
    if (c - ca < kMaxCh) {
      const int incl = warp_incl_scan(v);
      int wb = 0;
      tot = 0;
#pragma unroll
      for (int w = 0; w < kCmpWarps; w++) {
        const int x = s_w[c - ca][w];
        wb += w < warp ? x : 0;
        tot += x;
      }
      pre = wb + incl - v;
    } else {  // uniform over the block
      pre = block_excl_scan(v, tmp, &tot);
    }
    if (b != cur) {  // uniform over the block
      cur = b;
      if (c == c0) {
        start = carry;
      } else {
        if (threadIdx.x < 32) {
          unsigned long long w = 0;
          lb_wait(starts, b, threadIdx.x == 0, cfg, &w);
          if (threadIdx.x == 0) s_val = lb_current(w, cfg.epoch) ? (int)(unsigned)w : carry;
        }
        __syncthreads();
        start = s_val;
        __syncthreads();
      }
    }
    const int rel = carry - start;
    int j = rel + pre;
    if (v) {
#pragma unroll
      for (int k = 0; k < SPT; k++) {
        if (!np[k]) continue;
        const long long slot = im.cand_off + s0 + k;
        const uint32_t key = __float_as_uint(d->ref[slot].resp);
        for (int p = 0; p < np[k]; p++, j++) {
          if (j >= 0 && j < im.ori_cap) {
            d->ori[im.ori_off + j] = make_int2(s0 + k, p);
            d->okey[im.ori_off + j] = key;
          }
        }
      }
    }
    if (threadIdx.x == 0 && c == s_act[b + 1] - 1) {
      const int total = max(0, rel + tot);
      const int no = min(total, im.ori_cap);
      const int nf = min(no, im.kcap);
      ImgCounters &k = d->cnt[b];
      k.n_ori_raw = total;
      k.n_ori = no;
      k.n_fin = nf;
      k.flags |= (total > im.ori_cap ? TF_ORI : 0) | (no > im.kcap ? TF_TOPK : 0);
      if (im.ocount) *im.ocount = nf;
      lb_store(d->lb_img + kMaxImg + b, lb_word(kLbInc, cfg.epoch, nf));
    }
    carry += tot;
  }
  if (g == G - 1 && threadIdx.x < 32) lb_image_prefix(d->lb_img + kMaxImg, n, cfg, d->fin_flat);
}

// --------------------------------------------------------- top-K cap

// Per image (one block): if more than kcap oriented keypoints, keep the kcap
// largest responses, ties broken by canonical order, and list the kept indices
// in canonical order. The threshold is found by a bitwise search on the
// response bits (responses are non-negative, so bit order = value order).
// With binary16 octaves (fp16 storage mode) the block also counts the kept
// keypoints of octave 0 (n_fin0), which the descriptor's two launches split on.
__global__ void __launch_bounds__(1024) k_select(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int tmp[1024 / 32 + 1];
  const int n_img = d->n_img;
  for (int b = blockIdx.x; b < n_img; b += gridDim.x) {
    const ImgDev &im = d->img[b];
    const int n = d->cnt[b].n_ori;
    const int K = im.kcap;
    auto count_octave0 = [&]() {  // uniform over the block
      if (!d->fp16) return;
      const int nf = min(n, K);
      int c = 0;
      for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const int oi = n > K ? d->fin[im.fin_off + j] : j;
        c += d->ref[im.cand_off + d->ori[im.ori_off + oi].x].o == 0;
      }
      const int c0 = block_sum(c, tmp);
      if (threadIdx.x == 0) d->cnt[b].n_fin0 = c0;
    };
    if (n <= K) {
      count_octave0();
      continue;
    }
    const uint32_t *key = d->okey + im.ori_off;
    uint32_t thr = 0;
    for (int bit = 31; bit >= 0; bit--) {
      const uint32_t cand = thr | (1u << bit);
      int c = 0;
      for (int j = threadIdx.x; j < n; j += blockDim.x) c += key[j] >= cand;
      if (block_sum(c, tmp) >= K) thr = cand;
    }
    int cg = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) cg += key[j] > thr;
    const int need_eq = K - block_sum(cg, tmp);
    int out = 0, eq_seen = 0;
    for (int base = 0; base < n; base += blockDim.x) {
      const int j = base + threadIdx.x;
      const uint32_t kv = j < n ? key[j] : 0u;
      const int is_eq = (j < n && kv == thr) ? 1 : 0;
      int eq_tot;
      const int eq_rank = eq_seen + block_excl_scan(is_eq, tmp, &eq_tot);
      const int keep = (j < n && (kv > thr || (is_eq && eq_rank < need_eq))) ? 1 : 0;
      int k_tot;
      const int pos = out + block_excl_scan(keep, tmp, &k_tot);
      if (keep) d->fin[im.fin_off + pos] = j;
      out += k_tot;
      eq_seen += eq_tot;
    }
    __syncthreads();  // the kept list, before it is read back
    count_octave0();
  }
}

// ------------------------------------------------------------- descriptor

// Histogram columns of the descriptor: kDescCols per warp, column lane % 16,
// layout [bin][column] with bin = cell * 8 + orientation. Each sample votes
// into at most 4 cells and into the two orientation bins around its angle, of
// which one is even and one odd. Lanes l and l + 16 share a column and commit
// in two passes: in pass 0 the lower half-warp adds its even-orientation votes
// while the upper half adds its odd ones, in pass 1 the other way round. Two
// lanes of one pass then never touch the same word (different column, or
// different orientation parity), every lane is busy in both passes, and the
// order in which a word receives its votes is fixed by the code.
constexpr int kDescCols = 16;
// Floats of one warp's histogram block: 128 bins x 16 columns.
constexpr int kDescWarpFloats = kDescLen * kDescCols;

// The trilinear targets of one gradient sample at bin coordinates (rx, ry)
// from the keypoint, (u, v) = (rx, ry) + 3/2: weight m * exp(-(rx^2 + ry^2) /
// 8), orientation relative to th. Cells outside the 4 x 4 grid get -1.
struct Vote {
  int cell[4];    // (v * 4 + u) * 8 * kDescCols (the cell's first histogram word), or -1
  float w[4];     // spatial weights times the magnitude-Gaussian weight
  int oe, oo;     // the even and the odd orientation bin, times kDescCols
  float fe, fo;   // their orientation weights
};

// ok false: the lane has no sample (its coordinates may lie anywhere); all
// four of its cells are then -1, so that the commit skips it without a
// branch around this function.
__device__ __forceinline__ void desc_targets(Vote &v, float rx, float ry, float gx, float gy,
                                             float th, bool ok = true) {
  const float u = rx + 1.5f, vv0 = ry + 1.5f;
  const float mag = sqrtf(gx * gx + gy * gy);
  float phi = atan2f(gy, gx) - th;
  if (phi < 0.f) phi += kTwoPi;
  if (phi < 0.f) phi += kTwoPi;
  if (phi >= kTwoPi) phi -= kTwoPi;
  const float ob = phi * (8.0f / kTwoPi);
  const float wt = mag * expf(-(rx * rx + ry * ry) * 0.125f);
  const float u0f = floorf(u), v0f = floorf(vv0), o0f = floorf(ob);
  const float fu = u - u0f, fv = vv0 - v0f, f1 = ob - o0f;
  const int u0 = (int)u0f, v0 = (int)v0f, o0 = (int)o0f & 7, o1 = (o0 + 1) & 7;
  const bool even0 = (o0 & 1) == 0;
  v.oe = (even0 ? o0 : o1) * kDescCols;
  v.oo = (even0 ? o1 : o0) * kDescCols;
  v.fe = even0 ? 1.f - f1 : f1;
  v.fo = even0 ? f1 : 1.f - f1;
  // u0, v0 lie in [-1, 3] (u, v in (-1, 4)): cell u0 + du exists iff u0 >= 0
  // (du = 0) or u0 <= 2 (du = 1), and the same for v.
  const bool uok[2] = {ok && u0 >= 0, ok && u0 <= 2}, vok[2] = {v0 >= 0, v0 <= 2};
  const int c00 = (v0 * 4 + u0) * 8;
#pragma unroll
  for (int dv = 0; dv < 2; dv++) {
    const float wv = wt * (dv ? fv : 1.f - fv);
#pragma unroll
    for (int du = 0; du < 2; du++) {
      const float wu = du ? fu : 1.f - fu;
      v.cell[dv * 2 + du] = (uok[du] && vok[dv]) ? (c00 + (dv * 4 + du) * 8) * kDescCols : -1;
      v.w[dv * 2 + du] = wv * wu;
    }
  }
}

// Add the votes of the warp's lanes to the warp's columns in the two passes
// described above; a vote without a target (a cell outside the grid) is
// skipped. Every lane of the warp must call it.
__device__ __forceinline__ void desc_commit(float *hist, int lane, const Vote &v) {
  float *col = hist + (lane & (kDescCols - 1));
  const bool upper = lane >= 16;
#pragma unroll
  for (int pass = 0; pass < 2; pass++) {
    const bool even = (pass == 0) != upper;
    const int o = even ? v.oe : v.oo;
    const float f = even ? v.fe : v.fo;
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (v.cell[k] >= 0) col[v.cell[k] + o] += v.w[k] * f;
    __syncwarp();
  }
}

// DSP-SIFT pooling (§3.2): relative scales of the descriptor's bin width.
__constant__ float kDspScale[5] = {0.5f, 0.70710678118654752f, 1.0f, 1.41421356237309505f, 2.0f};

// The sample sweeps of one keypoint (plain or DSP), instantiated once per
// storage type of the level (HF: binary16) so that no load tests it.
template <bool HF>
__device__ __forceinline__ void desc_sweep(const Desc *__restrict__ d, const RefRec &r,
                                           const OctDev &od, const float *L, long long lofs,
                                           float wbin, float inv_w, float th, float st,
                                           float ct, int R, float *hist, int lane, int warp,
                                           int (*s_lo)[32], int (*s_pre)[33]) {
  const int tid = threadIdx.x;
  const int pitch = od.pitch;
  const LevelView<HF> lv = level_at<HF>(L, lofs, pitch, r.x, r.y);
    if (!d->dsp) {
      // Samples: integer offsets (i, jy) in [-R, R]^2 inside the image whose
      // rotated bin coordinates fall in (-1, 4)^2, i.e. inside a square of half
      // side h = 2.5 bins around the keypoint. Warp w takes rows jlo + w,
      // jlo + w + 4, ... (at most 32 of them, one per lane): each lane cuts its
      // row to an interval, a superset of the square's chord widened by 2
      // pixels so that rounding can only add candidates, and a warp scan lays
      // the intervals end to end. The warp then sweeps that list 32 samples at
      // a time, and the exact test below decides, so the sample set is the
      // same as a sweep of the whole window.
      const float h = 2.5f * wbin;
      const int ilo = max(-R, 1 - r.x), ihi = min(R, od.W - 2 - r.x);
      const int jlo = max(-R, 1 - r.y), jhi = min(R, od.H - 2 - r.y);
      const float ica = fabsf(ct) * (float)(R + 1) < 1.0f ? 0.f : 1.0f / ct;
      const float isa = fabsf(st) * (float)(R + 1) < 1.0f ? 0.f : -1.0f / st;
      // Rows per warp are at most (2R + 1) / 4 + 1, i.e. 20 for the largest
      // octave-relative scale of the default parameters; larger windows take
      // several rounds of 32 rows.
      for (int rb = 0; jlo + warp + kKpWarps * rb <= jhi; rb += 32) {
        int len = 0, a0 = 0;
        {
          const int jy = jlo + warp + kKpWarps * (rb + lane);
          if (jy <= jhi) {
            const float oy = (float)jy - r.dy;
            float lo = -1e30f, hi = 1e30f;
            // slab a * ox + b in (-h, h) for (a, b) = (ct, st * oy), (-st, ct * oy)
#pragma unroll
            for (int k = 0; k < 2; k++) {
              const float ia = k ? isa : ica, b = k ? ct * oy : st * oy;
              if (ia == 0.f) {
                if (fabsf(b) >= h + 2.0f) hi = -1e30f;  // |a * ox| < 1: the row misses the slab
              } else {
                const float e0 = (-h - b) * ia, e1 = (h - b) * ia;
                lo = fmaxf(lo, fminf(e0, e1));
                hi = fminf(hi, fmaxf(e0, e1));
              }
            }
            int a1 = ihi;
            a0 = ilo;
            if (hi < lo) {
              a1 = a0 - 1;
            } else {
              if (lo + r.dx > (float)ilo) a0 = max(ilo, (int)floorf(lo + r.dx) - 2);
              if (hi + r.dx < (float)ihi) a1 = min(ihi, (int)ceilf(hi + r.dx) + 2);
            }
            len = max(0, a1 - a0 + 1);
          }
        }
        // Exclusive scan of the interval lengths over the warp's rows.
        int pre = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, pre, o);
          if (lane >= o) pre += v;
        }
        const int tot = __shfl_sync(0xffffffffu, pre, 31);
        pre -= len;
        int *wlo = s_lo[warp], *wpre = s_pre[warp];
        wlo[lane] = a0;
        wpre[lane] = pre;
        if (lane == 31) wpre[32] = tot;
        __syncwarp();
        int row = 0;
        // Sample q of the list: bin coordinates, whether it lies in the
        // square, and its offset from the keypoint pixel (0, the keypoint's
        // own in-image neighbourhood, when it does not).
        auto locate = [&](int q, float &rx, float &ry, int &off) {
          if (q >= tot) return false;
          while (wpre[row + 1] <= q) row++;
          const int jy = jlo + warp + kKpWarps * (rb + row);
          const int i = wlo[row] + (q - wpre[row]);
          const float ox = (float)i - r.dx, oy = (float)jy - r.dy;
          rx = (ct * ox + st * oy) * inv_w;
          ry = (-st * ox + ct * oy) * inv_w;
          const float u = rx + 1.5f, v = ry + 1.5f;
          const bool in = u > -1.f && u < 4.f && v > -1.f && v < 4.f;
          off = in ? jy * pitch + i : 0;
          return in;
        };
        // Two samples per lane per step, q and q + 32 (the lane's samples in
        // increasing order, as one per step would take them): the eight loads
        // of both are issued before either votes. Warp-uniform trip count:
        // every lane reaches the commits' __syncwarp.
        for (int q0 = 0; q0 < tot; q0 += 64) {
          float rxa = 0.f, rya = 0.f, rxb = 0.f, ryb = 0.f;
          int oa = 0, ob = 0;
          const bool oka = locate(q0 + lane, rxa, rya, oa);
          const bool okb = locate(q0 + 32 + lane, rxb, ryb, ob);
          const float ga = lv[oa + 1] - lv[oa - 1], ha = lv[oa + pitch] - lv[oa - pitch];
          const float gb = lv[ob + 1] - lv[ob - 1], hb = lv[ob + pitch] - lv[ob - pitch];
          Vote vt;
          desc_targets(vt, rxa, rya, ga, ha, th, oka);
          desc_commit(hist, lane, vt);
          desc_targets(vt, rxb, ryb, gb, hb, th, okb);
          desc_commit(hist, lane, vt);
        }
        __syncwarp();  // the next round rewrites this warp's interval table
      }
    } else {
      for (int f = 0; f < 5; f++) {
        const float wb = wbin * kDspScale[f];
        for (int idx = tid; idx < 32 * 32; idx += kKpWarps * 32) {
          const float rx = ((float)(idx & 31) + 0.5f) * 0.125f - 2.0f;
          const float ry = ((float)(idx >> 5) + 0.5f) * 0.125f - 2.0f;
          const float xr = r.dx + wb * (ct * rx - st * ry);  // relative to pixel (r.x, r.y)
          const float yr = r.dy + wb * (st * rx + ct * ry);
          const float xf = floorf(xr), yf = floorf(yr);
          const int ix = (int)xf, iy = (int)yf;
          const int x0 = r.x + ix, y0 = r.y + iy;
          const bool ok = !(x0 < 1 || x0 > od.W - 3 || y0 < 1 || y0 > od.H - 3);
          Vote vt;
          if (!ok) {  // (1024 samples per scale: the trip count is warp-uniform)
#pragma unroll
            for (int k = 0; k < 4; k++) vt.cell[k] = -1;
            desc_commit(hist, lane, vt);
            continue;
          }
          const float fx = xr - xf, fy = yr - yf, gx1 = 1.f - fx, gy1 = 1.f - fy;
          const int p = iy * pitch + ix;
          const int pm = p - pitch, pp = p + pitch, p2 = pp + pitch;
          auto at = [&](int i) { return lv[i]; };
          // L(x + 1, y) - L(x - 1, y) and L(x, y + 1) - L(x, y - 1), bilinear
          const float xp = gy1 * (gx1 * at(p + 1) + fx * at(p + 2)) +
                           fy * (gx1 * at(pp + 1) + fx * at(pp + 2));
          const float xm = gy1 * (gx1 * at(p - 1) + fx * at(p)) +
                           fy * (gx1 * at(pp - 1) + fx * at(pp));
          const float yp = gy1 * (gx1 * at(pp) + fx * at(pp + 1)) +
                           fy * (gx1 * at(p2) + fx * at(p2 + 1));
          const float ym = gy1 * (gx1 * at(pm) + fx * at(pm + 1)) +
                           fy * (gx1 * at(p) + fx * at(p + 1));
          desc_targets(vt, rx, ry, xp - xm, yp - ym, th);
          desc_commit(hist, lane, vt);
        }
      }
    }
}

// One block of kKpWarps warps per output keypoint; same lane-private
// histogram scheme as the orientation (merge order: warp, then lane).
// Plain mode samples the pixel grid around the keypoint. DSP mode samples, for
// each of the 5 scales, a 32 x 32 grid at bin coordinates (a + 1/2)/8 - 2 in
// the keypoint's rotated frame (bin width 3 sigma x scale) and takes the
// gradient as central differences of the bilinearly interpolated level; all
// scales vote into the same histogram (pooling before normalisation).
// Positions are kept relative to the integer keypoint pixel, so the
// interpolation weights keep full FP32 precision in large octaves.
// PART: which keypoints a launch describes. 0: all of them (every octave
// FP32); with binary16 octaves (fp16 storage mode) two launches, 1 for the
// keypoints of octave 0 (FP32) and 2 for those of the binary16 octaves, each
// over its own index ranges (k_select's n_fin0) and with only its own sample
// sweep compiled in (one kernel carrying both sweeps ran a third slower per
// keypoint).
template <int PART>
__global__ void __launch_bounds__(kKpWarps * 32, 6) k_descriptor(const Desc *__restrict__ d) {
  pdl_wait();
  extern __shared__ __align__(16) float dsm[];
  __shared__ float s_bins[kDescLen];
  __shared__ int s_lo[kKpWarps][32], s_pre[kKpWarps][33];
  // The prefix over the images of the keypoints this launch describes: all
  // (PART 0), image b's first n_fin0 (PART 1) or the rest (PART 2); j0 is
  // where image b's share starts in its list.
  __shared__ int s_fin[kMaxImg + 1], s_j0[kMaxImg];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float *hist = dsm + warp * kDescWarpFloats;
  const int n = d->n_img;
  if (PART == 0) {
    for (int i = tid; i <= n; i += kKpWarps * 32) s_fin[i] = d->fin_flat[i];
    for (int i = tid; i < n; i += kKpWarps * 32) s_j0[i] = 0;
  } else if (warp == 0) {
    int flat = 0;
    for (int b0 = 0; b0 < n; b0 += 32) {
      const int b = b0 + lane;
      int c = 0;
      if (b < n) {
        const int f = d->fin_flat[b + 1] - d->fin_flat[b], f0 = d->cnt[b].n_fin0;
        c = PART == 1 ? f0 : f - f0;
        s_j0[b] = PART == 1 ? 0 : f0;
      }
      const int incl = warp_incl_scan(c);
      if (b < n) s_fin[b] = flat + incl - c;
      flat += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) s_fin[n] = flat;
  }
  __syncthreads();
  const int total = s_fin[n];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(s_fin, n, t);  // in shared memory: no chain of global loads
    const ImgDev &im = d->img[b];
    const int j = s_j0[b] + (t - s_fin[b]);
    const int oi = (d->cnt[b].n_ori > im.kcap) ? d->fin[im.fin_off + j] : j;
    const int2 e = d->ori[im.ori_off + oi];
    const long long slot = im.cand_off + e.x;
    const RefRec r = d->ref[slot];
    const float angle = d->angs[slot * kMaxPeaks + e.y];
    const OctDev od = d->oct[im.oct0 + r.o];
    const float sig = sigma_of(d, r);
    if (tid == 0) {
      const float sc = ldexpf(im.up ? 0.5f : 1.0f, r.o);
      im.ox[j] = ((float)r.x + r.dx) * sc;
      im.oy[j] = ((float)r.y + r.dy) * sc;
      im.osig[j] = sig * sc;
      im.oang[j] = angle;
      im.oresp[j] = r.resp;
      im.ooct[j] = r.o;
      im.olay[j] = r.s;
    }
    // Level r.s of the keypoint's octave: FP32, or binary16 (od.half, PART 2).
    const float *L = d->pyr + od.lvl;
    const long long lofs = (long long)r.s * od.lstride;
    const float wbin = 3.0f * sig;
    const float inv_w = 1.0f / wbin;
    const int R = (int)floorf(wbin * 1.41421356237f * 2.5f + 0.5f);
    const float th = angle * (kTwoPi / 360.0f);
    float st, ct;
    sincosf(th, &st, &ct);
    {
      float4 *h4 = reinterpret_cast<float4 *>(hist);
#pragma unroll 8
      for (int k = lane; k < kDescLen * kDescCols / 4; k += 32) h4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    desc_sweep<PART == 2>(d, r, od, L, lofs, wbin, inv_w, th, st, ct, R, hist, lane, warp, s_lo, s_pre);
    __syncthreads();
    // Bin tid: per warp, the 16 columns starting at column (tid / 2) % 16 (with
    // the layout [bin][16], the 32 threads of a warp then read 32 distinct
    // banks), then the warp partials in warp order.
    float pw[kKpWarps];
#pragma unroll
    for (int w = 0; w < kKpWarps; w++) {
      const float *h = dsm + w * kDescWarpFloats + tid * kDescCols;
      float s = 0.f;
#pragma unroll
      for (int l = 0; l < kDescCols; l++) s += h[(l + (tid >> 1)) & (kDescCols - 1)];
      pw[w] = s;
    }
    float val = pw[0];
#pragma unroll
    for (int w = 1; w < kKpWarps; w++) val += pw[w];
    s_bins[tid] = val;
    __syncthreads();
    // Normalisation by warp 0 alone (lane l: bins l, l + 32, l + 64, l + 96;
    // sums in that order, then across lanes by a butterfly), so that the
    // other warps go on to the next keypoint without waiting. Warp 0 reads
    // the bins before it reaches the next keypoint's barrier, the only point
    // after which they are rewritten.
    if (warp == 0) {
      float bv[4];
#pragma unroll
      for (int k = 0; k < 4; k++) bv[k] = s_bins[lane + 32 * k];
      auto warp_total = [&](float x) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
      };
      const float sq = warp_total(bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2] + bv[3] * bv[3]);
      if (sq > 0.f) {
        const float n1 = sqrtf(sq);
#pragma unroll
        for (int k = 0; k < 4; k++) bv[k] = fminf(bv[k] / n1, 0.2f);
        const float n2 =
            sqrtf(warp_total(bv[0] * bv[0] + bv[1] * bv[1] + bv[2] * bv[2] + bv[3] * bv[3]));
#pragma unroll
        for (int k = 0; k < 4; k++) bv[k] = bv[k] / n2;
        if (d->rootsift) {
          const float l1 = warp_total(bv[0] + bv[1] + bv[2] + bv[3]);
#pragma unroll
          for (int k = 0; k < 4; k++) bv[k] = sqrtf(bv[k] / l1);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++) bv[k] = 0.f;
      }
      float *out = im.odesc + (long long)j * kDescLen;
#pragma unroll
      for (int k = 0; k < 4; k++) out[lane + 32 * k] = bv[k];
    }
  }
}

// Outputs of a batch packed into one block: the N x 128 descriptors, then x,
// y, sigma, angle, response, octave, layer (N entries each), N = fin_flat[n],
// images in batch order. One thread per float4 of descriptor, then one per
// keypoint for the scalar fields.
__global__ void __launch_bounds__(kThreads) k_pack(PackSrc src, float4 *__restrict__ dst) {
  // The parts' images in batch order: part p's keypoints start at first[p].
  int first[5];
  first[0] = 0;
  for (int p = 0; p < 4; p++)
    first[p + 1] = first[p] + (p < src.n ? src.d[p]->fin_flat[src.d[p]->n_img] : 0);
  const int N = first[4];
  auto locate = [&](int t, const ImgDev *&im, int &j) {
    int p = 0;
    while (p + 1 < src.n && t >= first[p + 1]) p++;
    const Desc *d = src.d[p];
    const int u = t - first[p];
    const int b = find_owner(d->fin_flat, d->n_img, u);
    im = &d->img[b];
    j = u - d->fin_flat[b];
  };
  const int stride = gridDim.x * blockDim.x;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  for (int q = g; q < N * (kDescLen / 4); q += stride) {
    const int t = q / (kDescLen / 4), c = q - t * (kDescLen / 4);
    const ImgDev *im;
    int j;
    locate(t, im, j);
    dst[q] = reinterpret_cast<const float4 *>(im->odesc + (long long)j * kDescLen)[c];
  }
  float *f = reinterpret_cast<float *>(dst + (long long)N * (kDescLen / 4));
  int *oi = reinterpret_cast<int *>(f + 5LL * N);
  for (int t = g; t < N; t += stride) {
    const ImgDev *im;
    int j;
    locate(t, im, j);
    f[t] = im->ox[j];
    f[N + t] = im->oy[j];
    f[2LL * N + t] = im->osig[j];
    f[3LL * N + t] = im->oang[j];
    f[4LL * N + t] = im->oresp[j];
    oi[t] = im->ooct[j];
    oi[N + t] = im->olay[j];
  }
}

}  // namespace

cudaError_t launch_pack(PackSrc src, void *dst, int n_sm, cudaStream_t s) {
  return launch_plain(k_pack, n_sm * 4, kThreads, 0, s, src, static_cast<float4 *>(dst));
}

cudaError_t launch_orientation(const Desc *d, int grid, cudaStream_t s, bool mixed) {
  if (mixed) return launch_pdl(k_orientation<true>, grid, kOriWarps * 32, 0, s, d);
  return launch_pdl(k_orientation<false>, grid, kOriWarps * 32, 0, s, d);
}

cudaError_t launch_ori_compact(const Desc *d, int grid, cudaStream_t s) {
  return launch_pdl(k_cc_compact, grid, kThreads, 0, s, d);
}

cudaError_t launch_select(const Desc *d, int grid, cudaStream_t s) {
  return launch_pdl(k_select, grid, 1024, 0, s, d);
}

int descriptor_smem_bytes() { return kKpWarps * kDescWarpFloats * (int)sizeof(float); }

cudaError_t cc_compact_occupancy(int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_cc_compact, kThreads, 0);
}

int orientation_max_ctas(bool mixed) {
  int nb = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, mixed ? k_orientation<true> : k_orientation<false>, kOriWarps * 32, 0);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

// Needs descriptor_set_attributes() first (the dynamic shared memory opt-in).
int descriptor_max_ctas(bool mixed) {
  int nb = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, mixed ? k_descriptor<2> : k_descriptor<0>, kKpWarps * 32,
      descriptor_smem_bytes());
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t descriptor_set_attributes() {
  cudaError_t e = cudaSuccess;
  for (const void *k : {reinterpret_cast<const void *>(k_descriptor<0>),
                        reinterpret_cast<const void *>(k_descriptor<1>),
                        reinterpret_cast<const void *>(k_descriptor<2>)})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, descriptor_smem_bytes());
  return e;
}

// With binary16 octaves (mixed) two launches: the keypoints of FP32 octaves,
// then those of binary16 octaves.
cudaError_t launch_descriptor(const Desc *d, int grid, cudaStream_t s, bool mixed) {
  if (!mixed) return launch_pdl(k_descriptor<0>, grid, kKpWarps * 32, descriptor_smem_bytes(), s, d);
  const cudaError_t e = launch_pdl(k_descriptor<1>, grid, kKpWarps * 32, descriptor_smem_bytes(), s, d);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_descriptor<2>, grid, kKpWarps * 32, descriptor_smem_bytes(), s, d);
}

}  // namespace sift
