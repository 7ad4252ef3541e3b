// Host planner and launch sequencing for the extractor.
//
// Per call the host computes the octave geometry of every image, the
// flattened tile queues (one per octave and tile kind), the compaction chunk
// tables and the workspace slices, writes them into a pinned descriptor and
// copies it to the device on the caller's stream. The launch sequence itself
// (per octave: base blur or decimation, S+2 level blurs, extrema scan; then
// compaction, refinement, orientation, compaction, cap, descriptor) is a CUDA
// graph keyed only by the largest octave count of the batch, because every
// kernel reads its geometry from the descriptor and uses a persistent grid.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "engine.h"
#include "scan.cuh"

namespace sift {

namespace {
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
constexpr size_t kAlign = 256;
}  // namespace

static void fill_tap_pairs(BlurTaps *t) {
  for (int i = 0; i <= kMaxR; i++) {
    t->wp[i] = make_float2(t->w[2 * i], t->w[2 * i + 1]);
    t->wq[i] = make_float2(t->w[2 * i + 1], 2 * i + 2 <= 2 * kMaxR ? t->w[2 * i + 2] : 0.0f);
  }
  for (int j = 0; j <= 2 * kMaxR; j++) t->wd[j] = make_float2(t->w[j], t->w[j]);
}

int gaussian_taps(double sigma, BlurTaps *t) {
  std::memset(t, 0, sizeof(*t));
  if (!(sigma > 0.0)) {
    t->w[0] = 1.0f;
    fill_tap_pairs(t);
    return 0;
  }
  const int r = (int)std::ceil(4.0 * sigma);
  if (r > kMaxR) return -1;
  double w[2 * kMaxR + 1];
  double sum = 0.0;
  for (int k = -r; k <= r; k++) {
    w[k + r] = std::exp(-(double)k * k / (2.0 * sigma * sigma));
    sum += w[k + r];
  }
  for (int k = 0; k <= 2 * r; k++) t->w[k] = (float)(w[k] / sum);
  fill_tap_pairs(t);
  return r;
}

static double level_sigma(const sift_params &p, int i) {
  return (double)p.sigma0 * std::pow(2.0, (double)i / p.n_scales);
}

// Blur that brings the input (2x magnified when up) to sigma0.
static double base_sigma(const sift_params &p, bool up) {
  const double eff = (double)p.init_blur * (up ? 2.0 : 1.0);
  const double d = (double)p.sigma0 * p.sigma0 - eff * eff;
  return d > 0 ? std::sqrt(d) : 0.0;
}

sift_status validate_params(const sift_params &p, std::string *why) {
  auto bad = [&](const char *m) {
    if (why) *why = m;
    return SIFT_E_INVALID;
  };
  if (p.n_scales < 2 || p.n_scales > kMaxScales) return bad("n_scales must be in 2..6");
  if (!(p.sigma0 > 0.f)) return bad("sigma0 must be > 0");
  if (!(p.init_blur >= 0.f)) return bad("init_blur must be >= 0");
  if (!(p.contrast_thr > 0.f)) return bad("contrast_thr must be > 0");
  if (!(p.edge_ratio > 0.f)) return bad("edge_ratio must be > 0");
  if (!(p.prefilter_ratio >= 0.f)) return bad("prefilter_ratio must be >= 0");
  if (!(p.ori_peak_ratio > 0.f && p.ori_peak_ratio <= 1.f)) return bad("ori_peak_ratio in (0, 1]");
  if (p.border < 1) return bad("border must be >= 1");
  if (p.max_refine_iter < 1) return bad("max_refine_iter must be >= 1");
  if (p.max_kpts < 1) return bad("max_kpts must be >= 1");
  if (p.dsp != 0 && p.dsp != 1) return bad("dsp must be 0 or 1");
  if (p.upsample_max_px < 0) return bad("upsample_max_px must be >= 0");
  if (p.fp16_pyramid != 0 && p.fp16_pyramid != 1) return bad("fp16_pyramid must be 0 or 1");
  BlurTaps t;
  // Base blur of each mode in use: magnified first octaves when upsampling,
  // the input as is without upsampling or for images above upsample_max_px.
  int rmax = p.upsample ? gaussian_taps(base_sigma(p, true), &t) : 0;
  if (rmax >= 0 && (!p.upsample || p.upsample_max_px > 0)) {
    const int r0 = gaussian_taps(base_sigma(p, false), &t);
    rmax = r0 < 0 ? -1 : std::max(rmax, r0);
  }
  for (int i = 1; i <= p.n_scales + 2 && rmax >= 0; i++) {
    const double k = std::sqrt(level_sigma(p, i) * level_sigma(p, i) -
                               level_sigma(p, i - 1) * level_sigma(p, i - 1));
    const int r = gaussian_taps(k, &t);
    rmax = r < 0 ? -1 : std::max(rmax, r);
  }
  if (rmax < 0) return bad("sigma0 too large: blur radius above 16");
  if (p.min_octave_side < 16 || p.min_octave_side <= rmax || p.min_octave_side <= 2 * p.border)
    return bad("min_octave_side must be >= 16, above the blur radius and twice the border");
  return SIFT_OK;
}

Engine::Engine(const sift_params &p) : P_(p) {}

void lookback_config(int *spins, int *hold) {
  // A wait polls about every 0.2-1 us, so 2^19 polls give up after a fraction
  // of a second. Tests of the give-up path (no GPU fault, no hang) shorten
  // the limit and name a compaction block that never publishes its count
  // through these variables.
  *spins = 1 << 19;
  *hold = -1;
  if (const char *v = std::getenv("SIFT_TEST_LOOKBACK_SPINS")) *spins = std::max(1, std::atoi(v));
  if (const char *v = std::getenv("SIFT_TEST_LOOKBACK_HOLD")) *hold = std::atoi(v);
}

Engine::~Engine() {
  drop_graphs();
  if (ws_) cudaFree(ws_);
  if (lb_) cudaFree(lb_);
  if (ddesc_) cudaFree(ddesc_);
  for (int i = 0; i < kRing; i++) {
    if (hdesc_[i]) cudaFreeHost(hdesc_[i]);
    if (hevt_[i]) cudaEventDestroy(hevt_[i]);
  }
  if (done_) cudaEventDestroy(done_);
  if (cap_) cudaStreamDestroy(cap_);
  for (int k = 0; k < kSides; k++) {
    if (side_[k]) cudaStreamDestroy(side_[k]);
    if (join_ev_[k]) cudaEventDestroy(join_ev_[k]);
  }
  for (int o = 0; o < kMaxOct; o++)
    if (fork_ev_[o]) cudaEventDestroy(fork_ev_[o]);
}

sift_status Engine::init() {
  if (inited_) return SIFT_OK;
  std::string why;
  if (validate_params(P_, &why) != SIFT_OK) {
    err = why;
    return SIFT_E_INVALID;
  }
  cudaError_t e = cudaGetDevice(&dev_);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm_, cudaDevAttrMultiProcessorCount, dev_);
  if (e == cudaSuccess) e = blur_set_attributes();
  if (e == cudaSuccess) e = descriptor_set_attributes();
  if (e == cudaSuccess) e = extrema_set_attributes();
  if (e == cudaSuccess) e = cudaMalloc(&ddesc_, sizeof(Desc));
  for (int i = 0; i < kRing && e == cudaSuccess; i++) {
    e = cudaHostAlloc(&hdesc_[i], sizeof(Desc), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hevt_[i], cudaEventDisableTiming);
    if (e == cudaSuccess) std::memset(hdesc_[i], 0, sizeof(Desc));
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done_, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking);
  for (int k = 0; k < kSides && e == cudaSuccess; k++) {
    e = cudaStreamCreateWithFlags(&side_[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev_[k], cudaEventDisableTiming);
  }
  for (int o = 0; o < kMaxOct && e == cudaSuccess; o++)
    e = cudaEventCreateWithFlags(&fork_ev_[o], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    err = std::string("CUDA initialisation failed: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SIFT_E_OOM : SIFT_E_CUDA;
  }
  S_ = P_.n_scales;
  for (int m = 0; m < 2; m++) base_R_[m] = gaussian_taps(base_sigma(P_, m == 1), &base_t_[m]);
  for (int i = 1; i <= S_ + 2; i++) {
    const double k = std::sqrt(level_sigma(P_, i) * level_sigma(P_, i) -
                               level_sigma(P_, i - 1) * level_sigma(P_, i - 1));
    lvl_R_[i] = gaussian_taps(k, &lvl_t_[i]);
  }
  tun_ = default_tuning();
  lookback_config(&lb_spins_, &lb_hold_);
  ext_max_ = extrema_max_ctas(S_);
  ori_max_ = orientation_max_ctas(P_.fp16_pyramid != 0);
  desc_max_ = descriptor_max_ctas(P_.fp16_pyramid != 0);
  cmp_max_ = compact_max_ctas();
  inited_ = true;
  return SIFT_OK;
}

// Same set-up as init() minus every allocation: taps, SM count, tile tuning
// and kernel attributes only.
sift_status Engine::init_noalloc() {
  std::string why;
  if (validate_params(P_, &why) != SIFT_OK) {
    err = why;
    return SIFT_E_INVALID;
  }
  cudaError_t e = cudaGetDevice(&dev_);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm_, cudaDevAttrMultiProcessorCount, dev_);
  if (e != cudaSuccess) {
    err = std::string("CUDA device query failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  S_ = P_.n_scales;
  for (int m = 0; m < 2; m++) base_R_[m] = gaussian_taps(base_sigma(P_, m == 1), &base_t_[m]);
  for (int i = 1; i <= S_ + 2; i++) {
    const double k = std::sqrt(level_sigma(P_, i) * level_sigma(P_, i) -
                               level_sigma(P_, i - 1) * level_sigma(P_, i - 1));
    lvl_R_[i] = gaussian_taps(k, &lvl_t_[i]);
  }
  tun_ = default_tuning();
  lookback_config(&lb_spins_, &lb_hold_);
  ext_max_ = extrema_max_ctas(S_);
  ori_max_ = orientation_max_ctas(P_.fp16_pyramid != 0);
  desc_max_ = descriptor_max_ctas(P_.fp16_pyramid != 0);
  cmp_max_ = compact_max_ctas();
  return SIFT_OK;
}

bool Engine::magnify(int H, int W) const {
  return P_.upsample && (P_.upsample_max_px <= 0 || (long long)H * W <= P_.upsample_max_px);
}

int Engine::octave_sizes(int H, int W, int *hs, int *ws) const {
  const bool up = magnify(H, W);
  int h = up ? 2 * H : H, w = up ? 2 * W : W;
  int n = 0;
  while (std::min(h, w) >= P_.min_octave_side && n < kMaxOct) {
    if (hs) hs[n] = h;
    if (ws) ws[n] = w;
    n++;
    h /= 2;
    w /= 2;
  }
  return n;
}

bool Engine::addressable(int H, int W) const {
  const bool up = magnify(H, W);
  const unsigned long long h = up ? 2ull * H : (unsigned long long)H;
  const unsigned long long w = up ? 2ull * W : (unsigned long long)W;
  const unsigned long long pitch = (w + 31) / 32 * 32;
  return (unsigned long long)(P_.n_scales + 3) * h * pitch <= 0xffffffffull;
}

namespace {
// Candidate slots per image: one per 32 octave pixels, at least 8192.
int cand_capacity(long long octave_px) {
  long long c = octave_px / 32;
  c = std::max<long long>(c, 8192);
  c = std::min<long long>(c, 1 << 22);
  return (int)((c + kChunk - 1) / kChunk * kChunk);
}
int tile_h_of(int kind) { return kind == TK_BLUR16 ? 16 : kind == TK_BLUR64 ? 64 : 32; }
}  // namespace

size_t Engine::workspace_bytes(int n, const int *H, const int *W) const {
  size_t pyr = 0, bm = 0, cand = 0, ori = 0, fin = 0, chunks = 0;
  for (int b = 0; b < n; b++) {
    int hs[kMaxOct], ws[kMaxOct];
    const int no = octave_sizes(H[b], W[b], hs, ws);
    long long px = 0, words = 0;
    for (int o = 0; o < no; o++) {
      const long long pitch = align_up(ws[o], 32);
      pyr += (size_t)(S_ + 3) * hs[o] * pitch / (half_octave(o) ? 2 : 1);
      words += (long long)S_ * hs[o] * div_up(ws[o], kBmCols);
      px += (long long)hs[o] * ws[o];
    }
    bm += words;
    const int cc = cand_capacity(px);
    cand += cc;
    ori += 2 * (size_t)cc;
    fin += P_.max_kpts;
    chunks += div_up(words, kChunk) + cc / kChunk;
  }
  return pyr * 4 + bm * 4 + cand * (16 + sizeof(RefRec) + 8 + 4 * kMaxPeaks) + ori * 12 +
         fin * 4 + chunks * 8 + 16 * kAlign + kMaxImg * 48;
}

sift_status Engine::fill_plan(int n, const ImgIn *in, Desc &hd, WsLayout &L, int *max_oct) const {
  hd.n_img = n;
  hd.n_scales = S_;
  hd.upsample = P_.upsample ? 1 : 0;
  hd.sigma0 = P_.sigma0;
  hd.contrast_thr = P_.contrast_thr;
  hd.prefilter = (float)((double)P_.prefilter_ratio * (double)P_.contrast_thr);
  hd.edge_ratio = P_.edge_ratio;
  hd.border = P_.border;
  hd.max_iter = P_.max_refine_iter;
  hd.upright = P_.upright ? 1 : 0;
  hd.rootsift = P_.rootsift ? 1 : 0;
  hd.dsp = P_.dsp ? 1 : 0;
  hd.fp16 = P_.fp16_pyramid ? 1 : 0;
  hd.ori_peak_ratio = P_.ori_peak_ratio;
  size_t pyr = 0, bm = 0, cand = 0, ori = 0, fin = 0;
  int bmc = 0, cc = 0, M = 0;
  for (int b = 0; b < n; b++) {
    ImgDev &d = hd.img[b];
    std::memset(&d, 0, sizeof(d));
    d.src = in[b].src;
    d.H = in[b].H;
    d.W = in[b].W;
    d.spitch = in[b].pitch;
    d.src_vec_ok = ((reinterpret_cast<uintptr_t>(in[b].src) & 15) == 0 && (in[b].pitch & 3) == 0);
    d.up = magnify(in[b].H, in[b].W) ? 1 : 0;
    int hs[kMaxOct], ws[kMaxOct];
    const int no = octave_sizes(in[b].H, in[b].W, hs, ws);
    if (no == 0 || !addressable(in[b].H, in[b].W)) return SIFT_E_INVALID;
    d.n_oct = no;
    d.oct0 = b * kMaxOct;  // fixed slot: kernels locate an octave without reading ImgDev
    M = std::max(M, no);
    d.bm_begin = (long long)bm;
    long long px = 0;
    for (int o = 0; o < no; o++) {
      OctDev &od = hd.oct[d.oct0 + o];
      od.H = hs[o];
      od.W = ws[o];
      od.pitch = (int)align_up(ws[o], 32);
      od.wpr = div_up(ws[o], kBmCols);
      od.lvl = (long long)pyr;
      od.lstride = (long long)od.H * od.pitch;
      od.half = half_octave(o) ? 1 : 0;
      od.pad = 0;
      // Pitches are multiples of 32 elements, so a binary16 octave also starts
      // and keeps its rows on 64-byte boundaries.
      pyr += (size_t)(S_ + 3) * od.lstride / (od.half ? 2 : 1);
      od.bm = (long long)bm;
      bm += (size_t)S_ * od.H * od.wpr;
      px += (long long)od.H * od.W;
    }
    d.bm_words = (long long)bm - d.bm_begin;
    d.bmc0 = bmc;
    d.bmc_n = div_up(d.bm_words, kChunk);
    bmc += d.bmc_n;
    d.cand_cap = cand_capacity(px);
    d.cand_off = (long long)cand;
    cand += d.cand_cap;
    d.cc0 = cc;
    d.cc_n = d.cand_cap / kChunk;
    cc += d.cc_n;
    d.ori_cap = 2 * d.cand_cap;
    d.ori_off = (long long)ori;
    ori += d.ori_cap;
    d.kcap = P_.max_kpts;
    d.fin_off = (long long)fin;
    fin += d.kcap;
    d.ox = in[b].k.x;
    d.oy = in[b].k.y;
    d.osig = in[b].k.sigma;
    d.oang = in[b].k.angle;
    d.oresp = in[b].k.response;
    d.ooct = in[b].k.octave;
    d.olay = in[b].k.layer;
    d.odesc = in[b].desc;
    d.ocount = in[b].count;
  }
  hd.n_oct_max = M;
  hd.n_bm_chunks = bmc;
  hd.n_cc_chunks = cc;
  for (int k = 0; k < TK_COUNT; k++) {
    for (int o = 0; o < kMaxOct; o++) {
      int *pre = hd.tile_pre[k][o];
      pre[0] = 0;
      for (int b = 0; b < n; b++) {
        int t = 0;
        if (o < hd.img[b].n_oct) {
          const OctDev &od = hd.oct[hd.img[b].oct0 + o];
          if (k == TK_EXT) t = od.wpr * div_up(od.H, kExtTH);
          else t = div_up(od.W, kBlurTW) * div_up(od.H, tile_h_of(k));
        }
        pre[b + 1] = pre[b] + t;
      }
    }
  }
  // Base-blur tile queues: octave-0 tiles of the images of each mode (the
  // other mode's images contribute none).
  for (int m = 0; m < 2; m++) {
    int *pre = hd.base_pre[m];
    pre[0] = 0;
    for (int b = 0; b < n; b++)
      pre[b + 1] = pre[b] + (hd.img[b].up == m ? hd.tile_pre[TK_BLUR32][0][b + 1] -
                                                     hd.tile_pre[TK_BLUR32][0][b]
                                               : 0);
  }
  hd.bmc_pre[0] = 0;
  hd.cc_pre[0] = 0;
  for (int b = 0; b < n; b++) {
    hd.bmc_pre[b + 1] = hd.bmc_pre[b] + hd.img[b].bmc_n;
    hd.cc_pre[b + 1] = hd.cc_pre[b] + hd.img[b].cc_n;
  }
  size_t off = 0;
  auto put = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, kAlign);
    return o;
  };
  L.pyr = put(pyr * sizeof(float));
  L.bm = put(bm * sizeof(uint32_t));
  L.cand = put(cand * sizeof(int4));
  L.ref = put(cand * sizeof(RefRec));
  L.code = put(cand * sizeof(int));
  L.npk = put(cand * sizeof(int));
  L.angs = put(cand * kMaxPeaks * sizeof(float));
  L.ori = put(ori * sizeof(int2));
  L.okey = put(ori * sizeof(uint32_t));
  L.fin = put(fin * sizeof(int));
  L.cnt = put(kMaxImg * sizeof(ImgCounters));
  L.cand_flat = put((kMaxImg + 1) * sizeof(int));
  L.fin_flat = put((kMaxImg + 1) * sizeof(int));
  L.total = off;
  *max_oct = M;
  return SIFT_OK;
}

// Grows the workspace with stream-ordered allocation on the run's stream,
// which already waits for the previous run (so the old block is no longer in
// use when it is freed). Nothing here synchronises the device.
sift_status Engine::ensure_workspace(size_t bytes, cudaStream_t s) {
  if (bytes <= ws_cap_) return SIFT_OK;
  if (ws_) {
    cudaFreeAsync(ws_, s);
    ws_ = nullptr;
    ws_cap_ = 0;
  }
  const size_t want = align_up(bytes + bytes / 4, 1 << 20);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&ws_), want, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws_ = nullptr;
    err = "workspace allocation of " + std::to_string(want) + " bytes failed";
    return SIFT_E_OOM;
  }
  ws_cap_ = want;
  return SIFT_OK;
}

sift_status Engine::ensure_lb(size_t words, cudaStream_t s) {
  if (words <= lb_cap_) return SIFT_OK;
  if (lb_) {
    cudaFreeAsync(lb_, s);
    lb_ = nullptr;
    lb_cap_ = 0;
  }
  const size_t want = align_up(words + words / 4, 4096);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&lb_), want * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(lb_, 0, want * sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (lb_) cudaFreeAsync(lb_, s);
    lb_ = nullptr;
    err = "status array allocation failed";
    return SIFT_E_OOM;
  }
  lb_cap_ = want;
  return SIFT_OK;
}

sift_status Engine::upload(Desc *hd, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(ddesc_, hd, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(hevt_[ring_], s);
  if (e != cudaSuccess) {
    err = std::string("descriptor upload failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  return SIFT_OK;
}

int Engine::grid_blur(int R, int kind, int mode, int ctas) const {
  return grid_of(blur_blocks_per_sm(R, kind, mode), ctas);
}

cudaError_t Engine::enqueue_pyramid(cudaStream_t s, int M, int modes, std::vector<ProfRec> *prof) {
  cudaError_t e = cudaSuccess;
  auto rec = [&](int cls, auto &&fn) {
    if (e != cudaSuccess) return;
    ProfRec r{nullptr, nullptr, cls};
    if (prof) {
      cudaEventCreate(&r.a);
      cudaEventCreate(&r.b);
      e = cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal);
    }
    if (e == cudaSuccess) e = fn();
    if (prof && e == cudaSuccess) {
      e = cudaEventRecordWithFlags(r.b, s, cudaEventRecordExternal);
      prof->push_back(r);
    }
  };
  const Desc *d = ddesc_;
  for (int o = 0; o < M; o++) {
    if (o == 0) {
      // One base launch per mode present (bit m of modes: images with up = m).
      for (int m = 1; m >= 0; m--) {
        if (!(modes >> m & 1)) continue;
        rec(PC_BASE, [&] {
          return launch_base_blur(d, base_R_[m], base_t_[m], TK_BLUR32, m == 1,
                                  grid_blur(base_R_[m], TK_BLUR32, m == 1 ? 2 : 1), s);
        });
      }
    }
    // Octaves above 0: the level-1 launch also produces level 0 by decimating
    // level S of the previous octave (no separate decimation pass).
    for (int l = 1; l <= S_ + 2; l++) {
      const int kind = storage(o, l) ? TK_BLUR32 : tun_.lvl_kind[o][l];
      rec(PC_BLUR, [&] {
        return launch_level_blur(d, o, l, lvl_R_[l], lvl_t_[l], kind, grid_blur(lvl_R_[l], kind, 0, tun_.blur_ctas[o]), s,
                                 o > 0 && l == 1, true, storage(o, l));
      });
    }
  }
  return e;
}

cudaError_t Engine::enqueue_all(cudaStream_t s, int M, int modes, std::vector<ProfRec> *prof,
                                bool fork) {
  cudaError_t e = cudaSuccess;
  kernels_ = 0;
  auto rec_on = [&](cudaStream_t st, int cls, auto &&fn, int nk = 1) {
    if (e != cudaSuccess) return;
    kernels_ += nk;
    ProfRec r{nullptr, nullptr, cls};
    if (prof) {
      cudaEventCreate(&r.a);
      cudaEventCreate(&r.b);
      e = cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal);
    }
    if (e == cudaSuccess) e = fn();
    if (prof && e == cudaSuccess) {
      e = cudaEventRecordWithFlags(r.b, st, cudaEventRecordExternal);
      prof->push_back(r);
    }
  };
  auto rec = [&](int cls, auto &&fn, int nk = 1) { rec_on(s, cls, fn, nk); };
  // With fork, the last two levels and the extrema scan of octave o < M - 1 run
  // on a side branch (side_[o % kSides]) concurrently with octave o + 1, which
  // reads only level S of octave o, and with the other octaves' branches. The
  // branches join the main stream before the last octave's scan, which the
  // keypoint stages follow.
  fork = fork && side_[0] != nullptr && M > 1;
  const Desc *d = ddesc_;
  const int g4 = n_sm_ * 4;
  const int ext_grid = grid_of(ext_max_, tun_.ext_ctas);
  for (int o = 0; o < M; o++) {
    if (o == 0) {
      // One base launch per mode present (bit m of modes: images with up = m).
      for (int m = 1; m >= 0; m--) {
        if (!(modes >> m & 1)) continue;
        rec(PC_BASE, [&] {
          return launch_base_blur(d, base_R_[m], base_t_[m], TK_BLUR32, m == 1,
                                  grid_blur(base_R_[m], TK_BLUR32, m == 1 ? 2 : 1), s);
        });
      }
    }
    // Octaves above 0: the level-1 launch also produces level 0 by decimating
    // level S of the previous octave (no separate decimation pass).
    // With fork, levels S + 1 and S + 2 of octave o < M - 1 and its extrema scan
    // go to the side branch once level S (all the next octave reads) is done.
    const bool branch = fork && o + 1 < M;
    cudaStream_t side = side_[o % kSides];
    for (int l = 1; l <= S_ + 2; l++) {
      const int kind = storage(o, l) ? TK_BLUR32 : tun_.lvl_kind[o][l];
      const bool on_side = branch && l > S_;
      if (on_side && l == S_ + 1) {
        if (e == cudaSuccess) e = cudaEventRecord(fork_ev_[o], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork_ev_[o], 0);
      }
      rec_on(on_side ? side : s, PC_BLUR, [&] {
        return launch_level_blur(d, o, l, lvl_R_[l], lvl_t_[l], kind, grid_blur(lvl_R_[l], kind, 0, tun_.blur_ctas[o]),
                                 on_side ? side : s, o > 0 && l == 1, !(on_side && l == S_ + 1),
                                 storage(o, l));
      });
    }
    if (branch) {
      rec_on(side, PC_EXTREMA, [&] { return launch_extrema(d, o, S_, ext_grid, side, true, half_octave(o)); });
    } else if (fork) {
      for (int k = 0; k < kSides && k < M - 1; k++) {
        if (e == cudaSuccess) e = cudaEventRecord(join_ev_[k], side_[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join_ev_[k], 0);
      }
      rec(PC_EXTREMA, [&] { return launch_extrema(d, o, S_, ext_grid, s, false, half_octave(o)); });
    } else {
      rec(PC_EXTREMA, [&] { return launch_extrema(d, o, S_, ext_grid, s, true, half_octave(o)); });
    }
  }
  const int g2 = compact_grid();
  rec(PC_KEYPOINT, [&] { return launch_bm_compact(d, g2, s); });
  rec(PC_REFINE, [&] { return launch_refine(d, g4, s); });
  const bool mixed = P_.fp16_pyramid != 0;
  rec(PC_ORIENT, [&] { return launch_orientation(d, grid_of(ori_max_, tun_.ori_ctas), s, mixed); });
  rec(PC_KEYPOINT, [&] { return launch_ori_compact(d, g2, s); });
  rec(PC_KEYPOINT, [&] { return launch_select(d, n_sm_, s); });
  rec(PC_DESCRIPTOR, [&] { return launch_descriptor(d, grid_of(desc_max_, tun_.desc_ctas), s, mixed); },
      mixed ? 2 : 1);
  return e;
}

void Engine::drop_graphs() {
  for (auto &kv : graphs_) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.prof) {
      for (auto &r : *kv.second.prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
      delete kv.second.prof;
    }
  }
  graphs_.clear();
  last_prof_ = nullptr;
}

sift_status Engine::get_graph(int M, int modes, cudaGraphExec_t *out) {
  const int key = (M * 4 + modes) * 2 + (profiling_ ? 1 : 0);
  auto it = graphs_.find(key);
  if (it != graphs_.end()) {
    *out = it->second.exec;
    last_prof_ = it->second.prof;
    last_kernels_ = it->second.kernels;
    return SIFT_OK;
  }
  GraphEntry ge;
  if (profiling_) ge.prof = new std::vector<ProfRec>();
  cudaError_t e = cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal);
  // The profiled graph (an event pair around every launch) keeps every launch
  // on one stream, so that each kernel's time is its own and not shared with a
  // concurrent branch.
  cudaError_t e1 = e == cudaSuccess ? enqueue_all(cap_, M, modes, ge.prof, !profiling_) : e;
  cudaGraph_t g = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap_, &g) : e;
  cudaError_t e3 = (e1 == cudaSuccess && e2 == cudaSuccess) ? cudaGraphInstantiate(&ge.exec, g, 0)
                                                             : (e1 != cudaSuccess ? e1 : e2);
  if (g) cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    cudaGetLastError();
    err = std::string("graph capture failed: ") + cudaGetErrorString(e3);
    if (ge.prof) delete ge.prof;
    return SIFT_E_CUDA;
  }
  ge.kernels = kernels_;
  graphs_[key] = ge;
  *out = ge.exec;
  last_prof_ = ge.prof;
  last_kernels_ = ge.kernels;
  return SIFT_OK;
}

sift_status Engine::run(int n, const ImgIn *imgs, cudaStream_t s) {
  sift_status st = init();
  if (st != SIFT_OK) return st;
  if (n < 1 || n > kMaxImg) {
    err = "batch size out of range";
    return SIFT_E_INVALID;
  }
  const int slot = (ring_ + 1) % kRing;
  cudaEventSynchronize(hevt_[slot]);  // the descriptor copy that last used this buffer is done
  ring_ = slot;
  Desc *hd = hdesc_[slot];
  WsLayout lay;
  int M = 0;
  st = fill_plan(n, imgs, *hd, lay, &M);
  if (st != SIFT_OK) {
    err = "image smaller than min_octave_side";
    return st;
  }
  if (cudaStreamWaitEvent(s, done_, 0) != cudaSuccess) {
    err = "stream ordering failed";
    return SIFT_E_CUDA;
  }
  st = ensure_workspace(lay.total, s);
  if (st != SIFT_OK) return st;
  lay_ = lay;
  hd->pyr = reinterpret_cast<float *>(ws_ + lay.pyr);
  hd->bm = reinterpret_cast<uint32_t *>(ws_ + lay.bm);
  hd->cand = reinterpret_cast<int4 *>(ws_ + lay.cand);
  hd->ref = reinterpret_cast<RefRec *>(ws_ + lay.ref);
  hd->code = reinterpret_cast<int *>(ws_ + lay.code);
  hd->npk = reinterpret_cast<int *>(ws_ + lay.npk);
  hd->angs = reinterpret_cast<float *>(ws_ + lay.angs);
  hd->ori = reinterpret_cast<int2 *>(ws_ + lay.ori);
  hd->okey = reinterpret_cast<uint32_t *>(ws_ + lay.okey);
  hd->fin = reinterpret_cast<int *>(ws_ + lay.fin);
  hd->cnt = reinterpret_cast<ImgCounters *>(ws_ + lay.cnt);
  hd->cand_flat = reinterpret_cast<int *>(ws_ + lay.cand_flat);
  hd->fin_flat = reinterpret_cast<int *>(ws_ + lay.fin_flat);
  const int gc = compact_grid();
  st = ensure_lb(1 + 4 * kMaxImg + 2 * (size_t)n_sm_ * cmp_max_, s);
  if (st != SIFT_OK) return st;
  if (epoch_ >= kLbEpochMask) {  // epochs wrapped: clear every status of earlier runs
    if (cudaMemsetAsync(lb_, 0, lb_cap_ * sizeof(unsigned long long), s) != cudaSuccess) {
      err = "status clear failed";
      return SIFT_E_CUDA;
    }
    epoch_ = 0;
  }
  epoch_++;
  hd->lb_err = lb_;
  hd->lb_img = lb_ + 1;
  hd->lb_start = hd->lb_img + 2 * kMaxImg;
  hd->lb_bm = hd->lb_start + 2 * kMaxImg;
  hd->lb_cc = hd->lb_bm + gc;
  hd->lb_epoch = epoch_;
  hd->lb_spins = lb_spins_;
  hd->lb_hold = lb_hold_;
  const size_t bytes =
      offsetof(Desc, oct) + (size_t)(hd->img[n - 1].oct0 + hd->img[n - 1].n_oct) * sizeof(OctDev);
  cudaGraphExec_t exec = nullptr;
  st = get_graph(M, base_modes(*hd), &exec);
  if (st != SIFT_OK) return st;
  st = upload(hd, bytes, s);
  if (st != SIFT_OK) return st;
  cudaError_t e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(done_, s);
  if (e != cudaSuccess) {
    err = std::string("graph launch failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  ring_last_ = slot;
  last_stream = s;
  last_n = n;
  last_extract = true;
  return SIFT_OK;
}

sift_status Engine::run_pyramid(const ImgIn &img, cudaStream_t s) {
  sift_status st = init();
  if (st != SIFT_OK) return st;
  const int slot = (ring_ + 1) % kRing;
  cudaEventSynchronize(hevt_[slot]);
  ring_ = slot;
  Desc *hd = hdesc_[slot];
  WsLayout lay;
  int M = 0;
  st = fill_plan(1, &img, *hd, lay, &M);
  if (st != SIFT_OK) return st;
  if (cudaStreamWaitEvent(s, done_, 0) != cudaSuccess) {
    err = "stream ordering failed";
    return SIFT_E_CUDA;
  }
  st = ensure_workspace(lay.total, s);
  if (st != SIFT_OK) return st;
  lay_ = lay;
  hd->pyr = reinterpret_cast<float *>(ws_ + lay.pyr);
  hd->bm = reinterpret_cast<uint32_t *>(ws_ + lay.bm);
  const size_t bytes = offsetof(Desc, oct) + (size_t)hd->img[0].n_oct * sizeof(OctDev);
  cudaError_t e = cudaSuccess;
  st = upload(hd, bytes, s);
  if (e == cudaSuccess && st == SIFT_OK) e = enqueue_pyramid(s, M, base_modes(*hd), nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(done_, s);
  if (e != cudaSuccess || st != SIFT_OK) {
    err = std::string("pyramid launch failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  ring_last_ = slot;
  last_stream = s;
  last_n = 1;
  last_extract = false;  // a pyramid export: the descriptor holds no outputs
  return SIFT_OK;
}

void Engine::set_profiling(bool on) { profiling_ = on; }

sift_status Engine::kernel_times(double *ms, int *launches, int n_classes) {
  for (int c = 0; c < n_classes; c++) {
    if (ms) ms[c] = 0.0;
    if (launches) launches[c] = 0;
  }
  if (!last_prof_) {
    err = "no profiled run: enable profiling before extracting";
    return SIFT_E_INVALID;
  }
  cudaError_t e = cudaEventSynchronize(done_);
  for (auto &r : *last_prof_) {
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (r.cls < n_classes) {
      if (ms) ms[r.cls] += t;
      if (launches) launches[r.cls] += 1;
    }
  }
  if (e != cudaSuccess) {
    err = std::string("event timing failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  return SIFT_OK;
}

sift_status Engine::last_stats(int *stats, int max_images) {
  if (!ws_ || last_n == 0) {
    err = "no extraction has run";
    return SIFT_E_INVALID;
  }
  cudaError_t e = cudaEventSynchronize(done_);
  std::vector<ImgCounters> c(last_n);
  if (e == cudaSuccess)
    e = cudaMemcpy(c.data(), ws_ + lay_.cnt, last_n * sizeof(ImgCounters), cudaMemcpyDeviceToHost);
  unsigned long long gave_up = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&gave_up, lb_, sizeof gave_up, cudaMemcpyDeviceToHost);
  const Desc &hd = *hdesc_[ring_last_];
  bool trunc = false;
  for (int b = 0; b < last_n && b < max_images && e == cudaSuccess; b++) {
    std::vector<int> codes(c[b].n_cand);
    if (c[b].n_cand)
      e = cudaMemcpy(codes.data(), ws_ + lay_.code + hd.img[b].cand_off * sizeof(int),
                     c[b].n_cand * sizeof(int), cudaMemcpyDeviceToHost);
    int keep = 0;
    for (int v : codes) keep += v == RC_KEEP;
    stats[4 * b + 0] = c[b].n_cand;
    stats[4 * b + 1] = keep;
    stats[4 * b + 2] = c[b].n_ori;
    stats[4 * b + 3] = c[b].flags;
    trunc |= (c[b].flags & (TF_CAND | TF_ORI)) != 0;
  }
  if (e != cudaSuccess) {
    err = std::string("stats read failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  if (gave_up == epoch_) {
    err = "a compaction wait gave up: the counts of the last run are not valid";
    return SIFT_E_TIMEOUT;
  }
  return trunc ? SIFT_W_TRUNCATED : SIFT_OK;
}

void Engine::set_tuning(const Tuning &t) {
  tun_ = t;
  drop_graphs();
}

sift_status Engine::autotune(int H, int W, cudaStream_t s) {
  sift_status st = init();
  if (st != SIFT_OK) return st;
  float *img = nullptr;
  if (cudaMalloc(&img, (size_t)H * W * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    err = "autotune image allocation failed";
    return SIFT_E_OOM;
  }
  cudaMemsetAsync(img, 0, (size_t)H * W * sizeof(float), s);
  ImgIn in{};
  in.src = img;
  in.H = H;
  in.W = W;
  in.pitch = W;
  st = run_pyramid(in, s);
  int hs[kMaxOct], ws[kMaxOct];
  const int M = octave_sizes(H, W, hs, ws);
  const int modes = magnify(H, W) ? 2 : 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // Time the whole pyramid stage (all octaves, as the pipeline runs it), not
  // one level in isolation: a level's tile height also changes how the level
  // overlaps its neighbours and how warm L2 is for them. Coordinate descent
  // from 32-row tiles everywhere in octave 0; a level switches to 64 rows only
  // if the stage gets at least 1% faster.
  auto time_stage = [&]() -> float {
    for (int w = 0; w < 2; w++) enqueue_pyramid(s, M, modes, nullptr);
    cudaEventRecord(a, s);
    for (int r = 0; r < 5; r++) enqueue_pyramid(s, M, modes, nullptr);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  };
  if (st == SIFT_OK) {
    for (int l = 0; l < kMaxLevels; l++) tun_.lvl_kind[0][l] = TK_BLUR32;
    float best = time_stage();
    for (int l = 1; l <= S_ + 2; l++) {
      if (storage(0, l)) continue;
      tun_.lvl_kind[0][l] = TK_BLUR64;
      const float t = time_stage();
      if (t < 0.99f * best) best = t;
      else tun_.lvl_kind[0][l] = TK_BLUR32;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaStreamSynchronize(s);
  cudaFree(img);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("autotune failed: ") + cudaGetErrorString(e);
    return SIFT_E_CUDA;
  }
  drop_graphs();
  return st;
}

std::string Engine::device_key() const {
  int ma = 0, mi = 0;
  cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev_);
  cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev_);
  return "sm" + std::to_string(ma) + std::to_string(mi) + "x" + std::to_string(n_sm_);
}

float Engine::time_steps(const Tuning &t, const StepFn &step, cudaStream_t s, sift_status *st) {
  set_tuning(t);
  float best = 1e30f;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    err = "autotune event creation failed";
    *st = SIFT_E_CUDA;
  }
  // Two untimed steps (the first one captures the graph), then the best of
  // three runs of five back-to-back steps.
  for (int w = 0; w < 2 && *st == SIFT_OK; w++) *st = step();
  for (int r = 0; r < 3 && *st == SIFT_OK; r++) {
    cudaEventRecord(a, s);
    for (int k = 0; k < 5 && *st == SIFT_OK; k++) *st = step();
    cudaEventRecord(b, s);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      err = std::string("autotune timing failed: ") + cudaGetErrorString(cudaGetLastError());
      *st = SIFT_E_CUDA;
    }
    best = std::min(best, ms / 5.0f);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return best;
}

sift_status Engine::autotune_batch(int n, const ImgIn *imgs, cudaStream_t s, const StepFn &step_in) {
  const StepFn step = step_in ? step_in : StepFn([&] { return run(n, imgs, s); });
  sift_status st = init();
  if (st != SIFT_OK) return st;
  if (n < 1 || n > kMaxImg) {
    err = "autotune batch must hold 1..128 images";
    return SIFT_E_INVALID;
  }
  int M = 0;
  for (int i = 0; i < n; i++) {
    int hs[kMaxOct], ws[kMaxOct];
    M = std::max(M, octave_sizes(imgs[i].H, imgs[i].W, hs, ws));
  }
  // Coordinate descent over whole extraction steps of the caller's batch,
  // starting from the defaults (32-row tiles, occupancy-maximum grids): a
  // candidate replaces the incumbent only if the step gets at least 1% faster.
  // Searched, in order: 64-row tiles per FP32 level of the three largest
  // octaves (smaller octaves have too few tiles to fill the GPU), fewer
  // resident blur CTAs per SM for those octaves, then fewer extrema,
  // orientation and descriptor CTAs per SM (down to half the maximum).
  const Tuning t0 = default_tuning();
  Tuning best_t = t0;
  float best = time_steps(best_t, step, s, &st);
  auto try_t = [&](const Tuning &c) {
    if (st != SIFT_OK) return;
    const float t = time_steps(c, step, s, &st);
    if (st == SIFT_OK && t < 0.99f * best) {
      best = t;
      best_t = c;
    }
  };
  const int OT = std::min(M, 3);
  for (int o = 0; o < OT; o++)
    for (int l = 1; l <= S_ + 2; l++) {
      if (storage(o, l)) continue;
      Tuning c = best_t;
      c.lvl_kind[o][l] = TK_BLUR64;
      try_t(c);
    }
  int blur_max = 1;
  for (int l = 1; l <= S_ + 2; l++)
    blur_max = std::max(blur_max, blur_blocks_per_sm(lvl_R_[l], TK_BLUR32, 0));
  auto fewer = [&](int mx, auto &&field) {
    for (int c = mx - 1; c >= std::max(1, mx / 2); c--) {
      Tuning cand = best_t;
      field(cand) = c;
      try_t(cand);
    }
  };
  for (int o = 0; o < OT; o++) fewer(blur_max, [o](Tuning &t) -> int & { return t.blur_ctas[o]; });
  fewer(ext_max_, [](Tuning &t) -> int & { return t.ext_ctas; });
  fewer(ori_max_, [](Tuning &t) -> int & { return t.ori_ctas; });
  fewer(desc_max_, [](Tuning &t) -> int & { return t.desc_ctas; });
  fewer(cmp_max_, [](Tuning &t) -> int & { return t.cmp_ctas; });
  // Confirm against the defaults once more, so that a choice that won by
  // timing noise early in the search does not stay.
  if (st == SIFT_OK) {
    const float tb = time_steps(best_t, step, s, &st);
    const float td = st == SIFT_OK ? time_steps(t0, step, s, &st) : 0.f;
    if (st == SIFT_OK && !(tb < td)) best_t = t0;
  }
  if (st != SIFT_OK) return st;
  set_tuning(best_t);
  return step();  // the outputs: a run with the chosen tuning
}

}  // namespace sift
