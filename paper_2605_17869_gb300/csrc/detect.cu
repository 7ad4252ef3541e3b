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

template <int S>
__device__ __forceinline__ bool is_extremum(const float *__restrict__ G, long long ls, int pitch,
                                            int y, int x, int s, float c, const float *Dc) {
  bool mx = true, mn = true;
#pragma unroll
  for (int ds = -1; ds <= 1; ds++) {
    const float *g0 = G + (long long)(s + ds) * ls;
    const float *g1 = g0 + ls;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        if (ds == 0 && dy == 0 && dx == 0) continue;
        float nb;
        if (dy == 0 && dx == 0) {
          nb = Dc[s + ds];
        } else {
          const long long o = (long long)(y + dy) * pitch + (x + dx);
          nb = __ldg(g1 + o) - __ldg(g0 + o);
        }
        mx = mx && (c > nb);
        mn = mn && (c < nb);
        if (!mx && !mn) return false;
      }
    }
  }
  return true;
}

// One warp scans 32 adjacent columns of a row; a tile is 32 columns x kExtTH rows.
template <int S>
__global__ void __launch_bounds__(kThreads) k_extrema(const Desc *__restrict__ d, int oct) {
  const int n = d->n_img;
  const int *pre = d->tile_pre[TK_EXT][oct];
  const int total = pre[n];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float thr = d->prefilter;
  const int bord = d->border;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int b = find_owner(pre, n, t);
    const ImgDev &im = d->img[b];
    const OctDev od = d->oct[im.oct0 + oct];
    const int lt = t - pre[b];
    const int ty = lt / od.wpr, tx = lt - ty * od.wpr;
    const int x = tx * 32 + lane;
    const float *G = d->pyr + od.lvl;
    uint32_t *bm = d->bm + od.bm;
    const long long layer_words = (long long)od.H * od.wpr;
    for (int rr = warp; rr < kExtTH; rr += kThreads / 32) {
      const int y = ty * kExtTH + rr;
      if (y >= od.H) break;  // uniform over the warp
      const bool inb = x >= bord && x < od.W - bord && y >= bord && y < od.H - bord;
      bool cand[S];
#pragma unroll
      for (int s = 0; s < S; s++) cand[s] = false;
      if (inb) {
        float g[S + 3], Dc[S + 2];
        const long long o = (long long)y * od.pitch + x;
#pragma unroll
        for (int i = 0; i < S + 3; i++) g[i] = __ldg(G + i * od.lstride + o);
#pragma unroll
        for (int i = 0; i < S + 2; i++) Dc[i] = g[i + 1] - g[i];
#pragma unroll
        for (int s = 1; s <= S; s++) {
          const float c = Dc[s];
          if (fabsf(c) > thr) cand[s - 1] = is_extremum<S>(G, od.lstride, od.pitch, y, x, s, c, Dc);
        }
      }
#pragma unroll
      for (int s = 0; s < S; s++) {
        const unsigned bits = __ballot_sync(0xffffffffu, cand[s]);
        if (lane == 0) bm[s * layer_words + (long long)y * od.wpr + tx] = bits;
      }
    }
  }
}

// ----------------------------------------------------- bitmap compaction

__global__ void __launch_bounds__(kThreads) k_bm_count(const Desc *__restrict__ d) {
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

// One block: per image, exclusive scan of chunk counts; candidate totals and
// the prefix of candidate counts over images.
__global__ void __launch_bounds__(1024) k_bm_scan(const Desc *__restrict__ d) {
  __shared__ int tmp[1024 / 32 + 1];
  const int n = d->n_img;
  int flat = 0;
  for (int b = 0; b < n; b++) {
    const ImgDev &im = d->img[b];
    int carry = 0;
    for (int base = 0; base < im.bmc_n; base += blockDim.x) {
      const int i = base + threadIdx.x;
      const int v = i < im.bmc_n ? d->bm_cnt[im.bmc0 + i] : 0;
      int tot;
      const int ex = block_excl_scan(v, tmp, &tot);
      if (i < im.bmc_n) d->bm_off[im.bmc0 + i] = carry + ex;
      carry += tot;
    }
    const int nc = min(carry, im.cand_cap);
    if (threadIdx.x == 0) {
      ImgCounters &k = d->cnt[b];
      k.n_cand_raw = carry;
      k.n_cand = nc;
      k.flags = carry > im.cand_cap ? TF_CAND : 0;
      d->cand_flat[b] = flat;
    }
    flat += nc;
  }
  if (threadIdx.x == 0) d->cand_flat[n] = flat;
}

__global__ void __launch_bounds__(kThreads) k_bm_emit(const Desc *__restrict__ d) {
  __shared__ int tmp[kThreads / 32 + 1];
  constexpr int WPT = kChunk / kThreads;  // words per thread
  const int n = d->n_img;
  const int S = d->n_scales;
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
    for (int k = 0; k < WPT; k++) {
      uint32_t wv = words[k];
      if (!wv) continue;
      // Locate octave / layer / row / word of this bitmap word.
      const long long wa = im.bm_begin + w0 + k;
      int o = 0;
      OctDev od = d->oct[im.oct0];
      while (o + 1 < im.n_oct && wa >= d->oct[im.oct0 + o + 1].bm) {
        o++;
        od = d->oct[im.oct0 + o];
      }
      const long long rel = wa - od.bm;
      const long long lw = (long long)od.H * od.wpr;
      const int layer = (int)(rel / lw) + 1;
      const long long r2 = rel - (long long)(layer - 1) * lw;
      const int y = (int)(r2 / od.wpr);
      const int wx = (int)(r2 - (long long)y * od.wpr);
      while (wv) {
        const int bit = __ffs(wv) - 1;
        wv &= wv - 1;
        if (slot < im.cand_cap) d->cand[im.cand_off + slot] = make_int4(o, layer, y, wx * 32 + bit);
        slot++;
      }
    }
    (void)S;
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
  const int n = d->n_img;
  const int total = d->cand_flat[n];
  const int S = d->n_scales, bord = d->border, iters = d->max_iter;
  const float T = d->contrast_thr, er = d->edge_ratio;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
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

cudaError_t launch_extrema(const Desc *d, int oct, int n_scales, int grid, cudaStream_t s) {
  switch (n_scales) {
    case 2: k_extrema<2><<<grid, kThreads, 0, s>>>(d, oct); break;
    case 3: k_extrema<3><<<grid, kThreads, 0, s>>>(d, oct); break;
    case 4: k_extrema<4><<<grid, kThreads, 0, s>>>(d, oct); break;
    case 5: k_extrema<5><<<grid, kThreads, 0, s>>>(d, oct); break;
    case 6: k_extrema<6><<<grid, kThreads, 0, s>>>(d, oct); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bm_compact(const Desc *d, int grid, cudaStream_t s) {
  k_bm_count<<<grid, kThreads, 0, s>>>(d);
  k_bm_scan<<<1, 1024, 0, s>>>(d);
  k_bm_emit<<<grid, kThreads, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_refine(const Desc *d, int grid, cudaStream_t s) {
  k_refine<<<grid, kThreads, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace sift
