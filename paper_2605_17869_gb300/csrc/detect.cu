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
#include "scan.cuh"
#include "sift_dev.cuh"

namespace sift {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------ extrema scan

// A warp owns a tile of 32 columns x kExtTH rows (lane = column). It issues
// the loads of all S+3 levels for the tile's rows plus one halo row above and
// below at once, forms the DoG values in registers (one FP32 subtraction each,
// as everywhere else), and tests each pixel in three steps:
//  1. the contrast gate |D| > 0.5 T;
//  2. a branch-free check against the four direct neighbours in its layer
//     (left / right by warp shuffle, up / down from the adjacent rows; lanes 0
//     and 31 skip their outer neighbour here, the exact test below covers it)
//     and the same column of rows r - 1 .. r + 1 in the two adjacent layers
//     (registers); 10 of the 26 neighbours in all;
//  3. for the few pixels that pass, the exact 26-neighbour test, done by the
//     whole warp per pixel (lane k < 26 compares one neighbour, then a vote).
// Only step 3 decides; steps 1-2 merely skip pixels that cannot pass it.
template <int S>
__global__ void __launch_bounds__(kThreads, 3) k_extrema(const Desc *__restrict__ d, int oct) {
  constexpr int ND = S + 2;
  constexpr int RR = kExtTH + 2;  // rows held: y0 - 1 .. y0 + kExtTH
  constexpr int WPB = kThreads / 32;
  const int n = d->n_img;
  const int *pre = d->tile_pre[TK_EXT][oct];
  const int total = pre[n];
  const int lane = threadIdx.x & 31;
  const float thr = d->prefilter;
  const int bord = d->border;
  // Neighbour k of the 26 (3x3x3 minus the centre), owned by lane k.
  const int jn = lane < 13 ? lane : lane + 1;
  const int nds = jn / 9 - 1, ndy = (jn / 3) % 3 - 1, ndx = jn % 3 - 1;
  pdl_wait();
  for (int t = blockIdx.x * WPB + (threadIdx.x >> 5); t < total; t += gridDim.x * WPB) {
    if (t + gridDim.x * WPB >= total) pdl_trigger();  // this warp's last tile
    const int b = find_owner(pre, n, t);
    const OctDev od = d->oct[b * kMaxOct + oct];  // image b's octaves sit at fixed slots
    const int H = od.H, W = od.W, pitch = od.pitch;
    const int lt = t - pre[b];
    const int ty = lt / od.wpr, tx = lt - ty * od.wpr;
    const int x = tx * 32 + lane, y0 = ty * kExtTH;
    const float *G = d->pyr + od.lvl;
    const long long ls = od.lstride;
    const int xc = min(x, W - 1);
    float D[RR][ND];
    {
      float g[RR][S + 3];
#pragma unroll
      for (int r = 0; r < RR; r++) {
        const int yc = min(max(y0 - 1 + r, 0), H - 1);
        const float *p = G + (long long)yc * pitch + xc;
#pragma unroll
        for (int l = 0; l < S + 3; l++) g[r][l] = __ldg(p + l * ls);
      }
#pragma unroll
      for (int r = 0; r < RR; r++)
#pragma unroll
        for (int l = 0; l < ND; l++) D[r][l] = g[r][l + 1] - g[r][l];
    }
    // Lane s < S writes layer s+1's word of each row.
    uint32_t *bmw = d->bm + od.bm + (long long)lane * H * od.wpr + tx;
    const bool xin = x >= bord && x < W - bord;
#pragma unroll
    for (int r = 1; r <= kExtTH; r++) {
      const int y = y0 + r - 1;
      if (y >= H) break;  // uniform over the warp
      const bool inb = xin && y >= bord && y < H - bord;
      bool gated = false;
#pragma unroll
      for (int s = 1; s <= S; s++) gated = gated || fabsf(D[r][s]) > thr;
      unsigned bits[S];
#pragma unroll
      for (int s = 0; s < S; s++) bits[s] = 0u;
      if (__any_sync(0xffffffffu, inb && gated)) {  // most rows skip everything below
#pragma unroll
        for (int s = 1; s <= S; s++) {
          const float cv = D[r][s];
          const float lf = __shfl_up_sync(0xffffffffu, cv, 1);
          const float rt = __shfl_down_sync(0xffffffffu, cv, 1);
          const float up = D[r - 1][s], dn = D[r + 1][s];
          // Same column in the adjacent layers, rows r - 1 .. r + 1 (registers).
          const float s0 = D[r][s - 1], s1 = D[r][s + 1];
          const float s2 = D[r - 1][s - 1], s3 = D[r + 1][s - 1];
          const float s4 = D[r - 1][s + 1], s5 = D[r + 1][s + 1];
          const float hi = fmaxf(fmaxf(fmaxf(up, dn), fmaxf(s0, s1)),
                                 fmaxf(fmaxf(s2, s3), fmaxf(s4, s5)));
          const float lo = fminf(fminf(fminf(up, dn), fminf(s0, s1)),
                                 fminf(fminf(s2, s3), fminf(s4, s5)));
          const bool pmax = cv > hi && (lane == 0 || cv > lf) && (lane == 31 || cv > rt);
          const bool pmin = cv < lo && (lane == 0 || cv < lf) && (lane == 31 || cv < rt);
          const bool ok = inb && fabsf(cv) > thr && (pmax || pmin);
          unsigned surv = __ballot_sync(0xffffffffu, ok);
          while (surv) {
            const int sl = __ffs(surv) - 1;
            surv &= surv - 1;
            const float sv = __shfl_sync(0xffffffffu, cv, sl);
            float nb = 0.f;
            if (lane < 26) {
              const long long q = (long long)(y + ndy) * pitch + (x - lane + sl + ndx);
              nb = __ldg(G + (s + nds + 1) * ls + q) - __ldg(G + (s + nds) * ls + q);
            }
            const bool ext = __all_sync(0xffffffffu, lane >= 26 || sv > nb) ||
                             __all_sync(0xffffffffu, lane >= 26 || sv < nb);
            if (ext) bits[s - 1] |= 1u << sl;
          }
        }
      }
      unsigned mine = bits[0];
#pragma unroll
      for (int s = 1; s < S; s++) mine = lane == s ? bits[s] : mine;
      if (lane < S) bmw[(long long)y * od.wpr] = mine;
    }
  }
}

// ----------------------------------------------------- bitmap compaction

__global__ void __launch_bounds__(kThreads) k_bm_count(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int tmp[kThreads / 32 + 1];
  const int n = d->n_img;
  for (int c = blockIdx.x; c < d->n_bm_chunks; c += gridDim.x) {
    const int b = find_owner(d->bmc_pre, n, c);
    const ImgDev &im = d->img[b];
    const long long w0 = (long long)(c - d->bmc_pre[b]) * kChunk + threadIdx.x * (kChunk / kThreads);
    const uint32_t *bm = d->bm + im.bm_begin;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kChunk / kThreads; k++)
      if (w0 + k < im.bm_words) cnt += __popc(bm[w0 + k]);
    const int tot = block_sum(cnt, tmp);
    if (threadIdx.x == 0) d->bm_cnt[c] = tot;
  }
}

// One block: per image (one warp each), exclusive scan of chunk counts and the
// candidate totals; then the prefix of candidate counts over images.
__global__ void __launch_bounds__(512) k_bm_scan(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int s_nc[kMaxImg];
  const int n = d->n_img, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = warp; b < n; b += 16) {
    const ImgDev &im = d->img[b];
    const int carry = warp_excl_scan_array(d->bm_cnt + im.bmc0, d->bm_off + im.bmc0, im.bmc_n);
    const int nc = min(carry, im.cand_cap);
    if (lane == 0) {
      ImgCounters &k = d->cnt[b];
      k.n_cand_raw = carry;
      k.n_cand = nc;
      k.flags = carry > im.cand_cap ? TF_CAND : 0;
      s_nc[b] = nc;
    }
  }
  __syncthreads();
  if (warp == 0) warp_excl_scan_small(s_nc, d->cand_flat, n);
}

__global__ void __launch_bounds__(kThreads) k_bm_emit(const Desc *__restrict__ d) {
  pdl_wait();
  __shared__ int tmp[kThreads / 32 + 1];
  constexpr int WPT = kChunk / kThreads;  // words per thread
  const int n = d->n_img;
  for (int c = blockIdx.x; c < d->n_bm_chunks; c += gridDim.x) {
    const int b = find_owner(d->bmc_pre, n, c);
    const ImgDev &im = d->img[b];
    const long long w0 = (long long)(c - d->bmc_pre[b]) * kChunk + threadIdx.x * WPT;
    const uint32_t *bm = d->bm + im.bm_begin;
    uint32_t words[WPT];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < WPT; k++) {
      words[k] = (w0 + k < im.bm_words) ? bm[w0 + k] : 0u;
      cnt += __popc(words[k]);
    }
    int tot;
    int slot = d->bm_off[c] + block_excl_scan(cnt, tmp, &tot);
    if (tot == 0) continue;
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
      const unsigned rel = (unsigned)(wa - od.bm);
      const unsigned lw = (unsigned)od.H * (unsigned)od.wpr;
      const unsigned li = rel / lw;
      const unsigned r2 = rel - li * lw;
      const int layer = (int)li + 1;
      const int y = (int)(r2 / (unsigned)od.wpr);
      const int wx = (int)(r2 - (unsigned)y * (unsigned)od.wpr);
      while (wv) {
        const int bit = __ffs(wv) - 1;
        wv &= wv - 1;
        if (slot < im.cand_cap) d->cand[im.cand_off + slot] = make_int4(o, layer, y, wx * 32 + bit);
        slot++;
      }
    }
  }
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

__global__ void __launch_bounds__(kThreads) k_refine(const Desc *__restrict__ d) {
  pdl_wait();
  const int n = d->n_img;
  const int total = d->cand_flat[n];
  const int S = d->n_scales, bord = d->border, iters = d->max_iter;
  const float T = d->contrast_thr, er = d->edge_ratio;
  // Candidate t goes to block t % G, thread (t / G) % blockDim.x: a few
  // thousand candidates spread over every SM instead of filling the first blocks.
  for (int t = blockIdx.x + gridDim.x * threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int b = find_owner(d->cand_flat, n, t);
    const ImgDev &im = d->img[b];
    const long long slot = im.cand_off + (t - d->cand_flat[b]);
    const int4 cd = d->cand[slot];
    const int o = cd.x;
    int s = cd.y, y = cd.z, x = cd.w;
    const OctDev od = d->oct[im.oct0 + o];
    const float *G = d->pyr + od.lvl;
    const long long ls = od.lstride;
    const int pitch = od.pitch;
    int code = RC_NOCONV;
    float dX = 0.f, dY = 0.f, dS = 0.f, gx = 0.f, gy = 0.f, gs = 0.f, c = 0.f;
    float hxx = 0.f, hyy = 0.f, hxy = 0.f;
    bool conv = false;
    for (int it = 0; it < iters; it++) {
      float v[3][3][3];
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const float *g0 = G + (long long)(s + a - 1) * ls;
        const float *g1 = g0 + ls;
#pragma unroll
        for (int bb = 0; bb < 3; bb++)
#pragma unroll
          for (int cc = 0; cc < 3; cc++) {
            const long long off = (long long)(y + bb - 1) * pitch + (x + cc - 1);
            v[a][bb][cc] = __ldg(g1 + off) - __ldg(g0 + off);
          }
      }
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

cudaError_t launch_extrema(const Desc *d, int oct, int n_scales, int grid, cudaStream_t s, bool pdl) {
#define EXT_CASE(SS)                                                               \
  case SS:                                                                         \
    if (pdl) return launch_pdl(k_extrema<SS>, grid, kThreads, 0, s, d, oct);        \
    return launch_plain(k_extrema<SS>, grid, kThreads, 0, s, d, oct);
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
  cudaError_t e = launch_pdl(k_bm_count, grid, kThreads, 0, s, d);
  if (e == cudaSuccess) e = launch_pdl(k_bm_scan, 1, 512, 0, s, d);
  if (e == cudaSuccess) e = launch_pdl(k_bm_emit, grid, kThreads, 0, s, d);
  return e;
}

cudaError_t launch_refine(const Desc *d, int grid, cudaStream_t s) {
  return launch_pdl(k_refine, grid, kThreads, 0, s, d);
}

}  // namespace sift
