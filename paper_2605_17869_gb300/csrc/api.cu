// C ABI of the extractor (declared in include/sift_gb300.h) and the
// continuous-batching server.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

using sift::Engine;
using sift::ImgIn;

struct sift_handle {
  Engine *eng = nullptr;
  std::string err;
  bool serving = false;
  bool split_batch = false;  // the last extraction ran as several launches
  void *match_ws = nullptr;  // matcher workspace (stream-ordered allocation)
  size_t match_cap = 0;
  cudaStream_t match_stream = nullptr;
  bool match_attr = false;
  void *magsac_ws = nullptr;  // MAGSAC++ workspace (stream-ordered allocation)
  size_t magsac_cap = 0;
  cudaStream_t magsac_stream = nullptr;
  std::string tuning_cache;  // tuning cache file ("" none)
  // A batch run as several parts (tuning batch_lanes > 1): part k holds images
  // [part_start[k], part_start[k + 1]) and runs on part_eng(k) and stream
  // lane_s[k] (part 0: eng and the caller's stream), the other streams forked
  // from and joined back into the caller's stream by events. n_parts = 0: the
  // last extraction ran on eng alone.
  Engine *lane_eng[sift::kMaxLanes] = {};  // [0] unused
  cudaStream_t lane_s[sift::kMaxLanes] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[sift::kMaxLanes] = {};
  int n_parts = 0;
  int part_start[sift::kMaxLanes + 1] = {};
  Engine *part_eng(int k) const { return k == 0 ? eng : lane_eng[k]; }
};

static sift_status fail(sift_handle *h, sift_status st, const std::string &m) {
  if (h) h->err = m;
  return st;
}

static sift_status pass(sift_handle *h, sift_status st) {
  if (st != SIFT_OK && st != SIFT_W_TRUNCATED && h) h->err = h->eng->err;
  return st;
}

static bool kpts_ok(const sift_kpts_dev &k) {
  return k.x && k.y && k.sigma && k.angle && k.response && k.octave && k.layer;
}

// Set up lane k >= 1 (its engine, stream and join event) on first use.
static sift_status ensure_lane(sift_handle *h, int k) {
  if (h->lane_eng[k]) return SIFT_OK;
  cudaError_t ce = cudaSuccess;
  if (!h->ev_fork) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess && !h->lane_s[k])
    ce = cudaStreamCreateWithFlags(&h->lane_s[k], cudaStreamNonBlocking);
  if (ce == cudaSuccess && !h->ev_join[k])
    ce = cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming);
  if (ce != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("lane set-up failed: ") + cudaGetErrorString(ce));
  Engine *e = new Engine(h->eng->params());
  const sift_status st = e->init();
  if (st != SIFT_OK) {
    h->err = e->err;
    delete e;
    return st;
  }
  h->lane_eng[k] = e;
  return SIFT_OK;
}

// Run n <= kMaxImg images on stream s: on eng alone, or (batch_lanes = k > 1,
// two or more images, not profiling) as min(k, n) contiguous parts of about
// equal pixel count on as many engines at once. Every image's output is the
// same either way (an image's results do not depend on the rest of its batch).
static sift_status run_batch(sift_handle *h, int n, const ImgIn *in, cudaStream_t s) {
  const sift::Tuning t = h->eng->tuning();
  h->n_parts = 0;
  const int K = std::min(t.batch_lanes, n);
  if (K < 2 || n > sift::kMaxImg || h->eng->profiling()) return pass(h, h->eng->run(n, in, s));
  // Part k ends at the first image whose prefix reaches (k + 1) / K of the
  // pixels, leaving at least one image for each later part.
  long long tot = 0;
  for (int i = 0; i < n; i++) tot += (long long)in[i].H * in[i].W;
  int start[sift::kMaxLanes + 1];
  start[0] = 0;
  long long acc = 0;
  int i = 0;
  for (int k = 0; k + 1 < K; k++) {
    do {
      acc += (long long)in[i].H * in[i].W;
      i++;
    } while (i < n - (K - 1 - k) && acc * K < (k + 1) * tot);
    start[k + 1] = i;
  }
  start[K] = n;
  for (int k = 1; k < K; k++) {
    const sift_status st = ensure_lane(h, k);
    if (st != SIFT_OK) return st;
    const sift::Tuning tk = h->lane_eng[k]->tuning();
    if (std::memcmp(&t, &tk, sizeof t) != 0) h->lane_eng[k]->set_tuning(t);
  }
  cudaError_t ce = cudaEventRecord(h->ev_fork, s);
  for (int k = 1; k < K && ce == cudaSuccess; k++) ce = cudaStreamWaitEvent(h->lane_s[k], h->ev_fork, 0);
  if (ce != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("fork: ") + cudaGetErrorString(ce));
  for (int k = 0; k < K; k++) {
    Engine *e = h->part_eng(k);
    const sift_status st = e->run(start[k + 1] - start[k], in + start[k], k ? h->lane_s[k] : s);
    if (st != SIFT_OK) {
      h->err = e->err;
      return st;
    }
  }
  for (int k = 1; k < K && ce == cudaSuccess; k++) {
    ce = cudaEventRecord(h->ev_join[k], h->lane_s[k]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, h->ev_join[k], 0);
  }
  if (ce != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("join: ") + cudaGetErrorString(ce));
  h->n_parts = K;
  std::memcpy(h->part_start, start, sizeof(int) * (K + 1));
  return SIFT_OK;
}

extern "C" {

sift_status sift_params_default(sift_params *p) {
  if (!p) return SIFT_E_INVALID;
  p->n_scales = 3;
  p->sigma0 = 1.6f;
  p->init_blur = 0.5f;
  p->upsample = 0;
  p->min_octave_side = 16;
  p->contrast_thr = 0.04f / 3.0f;
  p->edge_ratio = 10.0f;
  p->border = 5;
  p->max_refine_iter = 5;
  p->prefilter_ratio = 0.5f;
  p->ori_peak_ratio = 0.8f;
  p->max_kpts = 8192;
  p->upright = 0;
  p->dsp = 0;
  p->rootsift = 0;
  p->upsample_max_px = 4000000;
  p->fp16_pyramid = 0;
  return SIFT_OK;
}

sift_status sift_create(const sift_params *p, sift_handle **out) {
  if (!p || !out) return SIFT_E_INVALID;
  *out = nullptr;
  std::string why;
  if (sift::validate_params(*p, &why) != SIFT_OK) return SIFT_E_INVALID;
  sift_handle *h = new sift_handle();
  h->eng = new Engine(*p);
  const sift_status st = h->eng->init();
  if (st != SIFT_OK) {
    delete h->eng;
    delete h;
    return st;
  }
  *out = h;
  return SIFT_OK;
}

sift_status sift_destroy(sift_handle *h) {
  if (!h) return SIFT_E_INVALID;
  if (h->match_ws) {
    cudaStreamSynchronize(h->match_stream);
    cudaFree(h->match_ws);
  }
  if (h->magsac_ws) {
    cudaStreamSynchronize(h->magsac_stream);
    cudaFree(h->magsac_ws);
  }
  for (int k = 1; k < sift::kMaxLanes; k++) {
    if (h->lane_s[k]) cudaStreamSynchronize(h->lane_s[k]);
    delete h->lane_eng[k];
    if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
    if (h->lane_s[k]) cudaStreamDestroy(h->lane_s[k]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  delete h->eng;
  delete h;
  return SIFT_OK;
}

sift_status sift_match(sift_handle *h, const float *desc_a, int n_a, const float *desc_b, int n_b,
                       float ratio, void *stream, int *out_match_a) {
  if (!h) return SIFT_E_INVALID;
  if (n_a < 0 || n_b < 0 || n_a > 65536 || n_b > 65536)
    return fail(h, SIFT_E_INVALID, "set sizes must be in [0, 65536]");
  if (!(ratio > 0.f && ratio <= 1.f)) return fail(h, SIFT_E_INVALID, "ratio must be in (0, 1]");
  if ((n_a > 0 && (!desc_a || !out_match_a)) || (n_b > 0 && !desc_b))
    return fail(h, SIFT_E_INVALID, "null pointer argument");
  if (n_a == 0) return SIFT_OK;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!h->match_attr) {
    if (sift::match_set_attributes() != cudaSuccess) return fail(h, SIFT_E_CUDA, "matcher attributes");
    h->match_attr = true;
  }
  const size_t need = sift::match_workspace_bytes(n_a, n_b);
  if (need > h->match_cap) {
    if (h->match_ws) cudaFreeAsync(h->match_ws, h->match_stream ? h->match_stream : s);
    h->match_ws = nullptr;
    h->match_cap = 0;
    if (cudaMallocAsync(&h->match_ws, need, s) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SIFT_E_OOM, "matcher workspace allocation failed");
    }
    h->match_cap = need;
  }
  h->match_stream = s;
  const cudaError_t e = sift::launch_match(desc_a, n_a, desc_b, n_b, ratio, h->match_ws, out_match_a, s);
  if (e != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("matcher: ") + cudaGetErrorString(e));
  return SIFT_OK;
}

sift_status sift_pack_outputs(sift_handle *h, void *stream, void *dst_dev, size_t dst_bytes) {
  if (!h || !dst_dev) return SIFT_E_INVALID;
  if (h->serving) return fail(h, SIFT_E_INVALID, "handle is serving");
  if (!h->eng->last_extract || h->eng->last_n < 1 || !h->eng->device_desc())
    return fail(h, SIFT_E_INVALID, "the last call on this handle was not an extraction");
  if (h->split_batch)
    return fail(h, SIFT_E_INVALID, "the last batch had more than 128 images and ran as several launches");
  if (reinterpret_cast<uintptr_t>(dst_dev) & 15) return fail(h, SIFT_E_INVALID, "dst must be 16-byte aligned");
  sift::PackSrc src{};  // the batch's parts in batch order (one: it ran on eng alone)
  src.n = std::max(1, h->n_parts);
  size_t n_img = 0;
  for (int k = 0; k < src.n; k++) {
    const Engine *e = h->part_eng(k);
    if (!e->last_extract || !e->device_desc())
      return fail(h, SIFT_E_INVALID, "the last call on this handle was not an extraction");
    src.d[k] = e->device_desc();
    n_img += (size_t)e->last_n;
  }
  const size_t need = n_img * h->eng->params().max_kpts * (sift::kDescLen * sizeof(float) + 7 * 4);
  if (dst_bytes < need) return fail(h, SIFT_E_INVALID, "dst smaller than last_n * max_kpts * 540 bytes");
  const cudaError_t e = sift::launch_pack(src, dst_dev, h->eng->sm_count(),
                                          static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("pack: ") + cudaGetErrorString(e));
  return SIFT_OK;
}

sift_status sift_magsac(sift_handle *h, const float *xa, const float *xb, int n, const int *samples,
                        int n_hyp, float sigma_max, void *stream, double *H_out, int *best_out,
                        float *score_out, unsigned char *inliers_out, float *scores_out) {
  if (!h) return SIFT_E_INVALID;
  if (n < 4 || n > (1 << 24)) return fail(h, SIFT_E_INVALID, "n must be in [4, 2^24]");
  if (n_hyp < 1 || n_hyp > (1 << 20)) return fail(h, SIFT_E_INVALID, "n_hyp must be in [1, 2^20]");
  if (!(sigma_max > 0.f && sigma_max < 1e6f))
    return fail(h, SIFT_E_INVALID, "sigma_max must be in (0, 1e6)");
  if (!xa || !xb || !samples || !H_out || !best_out || !score_out || !inliers_out)
    return fail(h, SIFT_E_INVALID, "null pointer argument");
  if ((reinterpret_cast<uintptr_t>(xa) | reinterpret_cast<uintptr_t>(xb)) & 7)
    return fail(h, SIFT_E_INVALID, "point arrays must be 8-byte aligned");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t need = sift::magsac_workspace_bytes(n_hyp);
  if (need > h->magsac_cap) {
    if (h->magsac_ws) cudaFreeAsync(h->magsac_ws, h->magsac_stream ? h->magsac_stream : s);
    h->magsac_ws = nullptr;
    h->magsac_cap = 0;
    if (cudaMallocAsync(&h->magsac_ws, need, s) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SIFT_E_OOM, "MAGSAC++ workspace allocation failed");
    }
    h->magsac_cap = need;
  }
  h->magsac_stream = s;
  const cudaError_t e = sift::launch_magsac(xa, xb, n, samples, n_hyp, sigma_max, h->magsac_ws, s,
                                            H_out, best_out, score_out, inliers_out, scores_out);
  if (e != cudaSuccess) return fail(h, SIFT_E_CUDA, std::string("MAGSAC++: ") + cudaGetErrorString(e));
  return SIFT_OK;
}

const char *sift_last_error(sift_handle *h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

const char *sift_version(void) { return "gb300-sift 0.1 (sm_103a)"; }

sift_status sift_extract(sift_handle *h, const float *img_dev, int H, int W, int pitch_elems,
                         void *stream, sift_kpts_dev out_kpts, float *out_desc_dev,
                         int *out_count_dev) {
  if (!h) return SIFT_E_INVALID;
  if (h->serving) return fail(h, SIFT_E_INVALID, "handle is owned by a server");
  if (!img_dev || !out_desc_dev || !out_count_dev || !kpts_ok(out_kpts))
    return fail(h, SIFT_E_INVALID, "null pointer argument");
  const int ms = h->eng->params().min_octave_side;
  if (H < ms || W < ms || pitch_elems < W)
    return fail(h, SIFT_E_INVALID, "image smaller than min_octave_side or pitch < W");
  if (!h->eng->addressable(H, W)) return fail(h, SIFT_E_INVALID, "image too large");
  ImgIn in{img_dev, H, W, pitch_elems, out_kpts, out_desc_dev, out_count_dev};
  h->split_batch = false;
  h->n_parts = 0;
  return pass(h, h->eng->run(1, &in, (cudaStream_t)stream));
}

sift_status sift_extract_batch(sift_handle *h, int n, const float *const *imgs_dev, const int *H,
                               const int *W, const int *pitch_elems, void *stream,
                               const sift_kpts_dev *out_kpts, float *const *out_desc,
                               int *out_counts_dev) {
  if (!h) return SIFT_E_INVALID;
  if (h->serving) return fail(h, SIFT_E_INVALID, "handle is owned by a server");
  if (n < 1 || !imgs_dev || !H || !W || !out_kpts || !out_desc || !out_counts_dev)
    return fail(h, SIFT_E_INVALID, "null pointer argument or n < 1");
  const int ms = h->eng->params().min_octave_side;
  std::vector<ImgIn> in(n);
  for (int i = 0; i < n; i++) {
    const int p = pitch_elems ? pitch_elems[i] : W[i];
    if (!imgs_dev[i] || !out_desc[i] || !kpts_ok(out_kpts[i]))
      return fail(h, SIFT_E_INVALID, "null pointer in image " + std::to_string(i));
    if (H[i] < ms || W[i] < ms || p < W[i])
      return fail(h, SIFT_E_INVALID, "image " + std::to_string(i) + " smaller than min_octave_side");
    if (!h->eng->addressable(H[i], W[i]))
      return fail(h, SIFT_E_INVALID, "image " + std::to_string(i) + " too large");
    in[i] = ImgIn{imgs_dev[i], H[i], W[i], p, out_kpts[i], out_desc[i], out_counts_dev + i};
  }
  h->split_batch = n > sift::kMaxImg;
  if (!h->split_batch) return run_batch(h, n, in.data(), (cudaStream_t)stream);
  h->n_parts = 0;
  for (int b0 = 0; b0 < n; b0 += sift::kMaxImg) {
    const int m = std::min(sift::kMaxImg, n - b0);
    const sift_status st = h->eng->run(m, in.data() + b0, (cudaStream_t)stream);
    if (st != SIFT_OK) return pass(h, st);
  }
  return SIFT_OK;
}

sift_status sift_last_stats(sift_handle *h, int *stats, int max_images) {
  if (!h || !stats || max_images < 1) return SIFT_E_INVALID;
  if (h->split_batch)
    return fail(h, SIFT_E_INVALID, "the last batch had more than 128 images and ran as several launches");
  if (h->n_parts > 0) {  // the parts, in batch order
    bool trunc = false;
    for (int k = 0; k < h->n_parts && h->part_start[k] < max_images; k++) {
      Engine *e = h->part_eng(k);
      const int b0 = h->part_start[k];
      const sift_status st = e->last_stats(stats + 4 * b0, std::min(max_images, h->part_start[k + 1]) - b0);
      if (st < 0) {
        h->err = e->err;
        return st;
      }
      trunc = trunc || st == SIFT_W_TRUNCATED;
    }
    return trunc ? SIFT_W_TRUNCATED : SIFT_OK;
  }
  return pass(h, h->eng->last_stats(stats, max_images));
}

sift_status sift_pyramid_size(sift_handle *h, int H, int W, int *n_octaves, size_t *total_elems) {
  if (!h || !n_octaves || !total_elems) return SIFT_E_INVALID;
  int hs[sift::kMaxOct], ws[sift::kMaxOct];
  const int no = h->eng->octave_sizes(H, W, hs, ws);
  if (no == 0) return fail(h, SIFT_E_INVALID, "image smaller than min_octave_side");
  size_t tot = 0;
  const int L = h->eng->params().n_scales + 3;
  for (int o = 0; o < no; o++) tot += (size_t)L * hs[o] * ws[o];
  *n_octaves = no;
  *total_elems = tot;
  return SIFT_OK;
}

sift_status sift_octave_geometry(const sift_params *p, int H, int W, int *n_octaves,
                                 int *magnified, int *heights, int *widths, int cap) {
  if (!p || !n_octaves || !magnified || H < 1 || W < 1 || cap < 0) return SIFT_E_INVALID;
  if (cap > 0 && (!heights || !widths)) return SIFT_E_INVALID;
  std::string why;
  if (sift::validate_params(*p, &why) != SIFT_OK) return SIFT_E_INVALID;
  const Engine eng(*p);  // geometry only: construction touches no device state
  int hs[sift::kMaxOct], ws[sift::kMaxOct];
  const int no = eng.octave_sizes(H, W, hs, ws);
  for (int o = 0; o < no && o < cap; o++) {
    heights[o] = hs[o];
    widths[o] = ws[o];
  }
  *n_octaves = no;
  *magnified = eng.magnify(H, W) ? 1 : 0;
  return SIFT_OK;
}

sift_status sift_build_pyramid(sift_handle *h, const float *img_dev, int H, int W,
                               int pitch_elems, void *stream, float *out_dev, size_t out_elems) {
  if (!h || !img_dev || !out_dev) return SIFT_E_INVALID;
  int no = 0;
  size_t need = 0;
  sift_status st = sift_pyramid_size(h, H, W, &no, &need);
  if (st != SIFT_OK) return st;
  if (out_elems < need || pitch_elems < W) return fail(h, SIFT_E_INVALID, "output too small");
  if (!h->eng->addressable(H, W)) return fail(h, SIFT_E_INVALID, "image too large");
  ImgIn in{img_dev, H, W, pitch_elems, {}, nullptr, nullptr};
  cudaStream_t s = (cudaStream_t)stream;
  h->split_batch = false;
  h->n_parts = 0;
  st = h->eng->run_pyramid(in, s);
  if (st != SIFT_OK) return pass(h, st);
  const sift::Desc &hd = h->eng->host_desc();
  const int L = h->eng->params().n_scales + 3;
  const float *pyr = reinterpret_cast<const float *>(h->eng->workspace() + h->eng->layout().pyr);
  size_t off = 0;
  for (int o = 0; o < no; o++) {
    const sift::OctDev &od = hd.oct[o];
    for (int l = 0; l < L; l++) {
      const float *lv = od.half ? reinterpret_cast<const float *>(
                                      reinterpret_cast<const __half *>(pyr + od.lvl) + (size_t)l * od.lstride)
                                : pyr + od.lvl + (size_t)l * od.lstride;
      cudaError_t e = sift::launch_export_level(lv, od.half != 0, od.pitch, od.H, od.W,
                                                out_dev + off, s);
      if (e != cudaSuccess) return fail(h, SIFT_E_CUDA, cudaGetErrorString(e));
      off += (size_t)od.H * od.W;
    }
  }
  return SIFT_OK;
}

sift_status sift_set_profiling(sift_handle *h, int enable) {
  if (!h) return SIFT_E_INVALID;
  h->eng->set_profiling(enable != 0);
  return SIFT_OK;
}

sift_status sift_kernel_times(sift_handle *h, double *ms, int *launches, int n_classes) {
  if (!h || n_classes < 1) return SIFT_E_INVALID;
  return pass(h, h->eng->kernel_times(ms, launches, n_classes));
}

sift_status sift_last_launch_count(sift_handle *h, int *kernels) {
  if (!h || !kernels) return SIFT_E_INVALID;
  *kernels = 0;
  for (int k = 0; k < std::max(1, h->n_parts); k++) *kernels += h->part_eng(k)->last_launch_count();
  return SIFT_OK;
}

sift_status sift_autotune(sift_handle *h, int H, int W, void *stream) {
  if (!h) return SIFT_E_INVALID;
  const int ms = h->eng->params().min_octave_side;
  if (H < ms || W < ms) return fail(h, SIFT_E_INVALID, "autotune size below min_octave_side");
  return pass(h, h->eng->autotune(H, W, (cudaStream_t)stream));
}

sift_status sift_get_tuning(sift_handle *h, char *json, size_t len) {
  if (!h || !json || len == 0) return SIFT_E_INVALID;
  const std::string s = sift::tuning_json(h->eng->tuning(), h->eng->params().n_scales);
  if (s.size() + 1 > len) return fail(h, SIFT_E_INVALID, "buffer too small");
  std::memcpy(json, s.c_str(), s.size() + 1);
  return SIFT_OK;
}

sift_status sift_set_tuning(sift_handle *h, const char *json) {
  if (!h || !json) return SIFT_E_INVALID;
  sift::Tuning t;
  std::string why;
  if (!sift::parse_tuning(json, h->eng->params().n_scales, h->eng->tuning(), &t, &why))
    return fail(h, SIFT_E_INVALID, why);
  h->eng->set_tuning(t);
  return SIFT_OK;
}

sift_status sift_set_tuning_cache(sift_handle *h, const char *path) {
  if (!h) return SIFT_E_INVALID;
  h->tuning_cache = path ? path : "";
  return SIFT_OK;
}

sift_status sift_autotune_batch(sift_handle *h, int n, const float *const *imgs_dev, const int *H,
                                const int *W, const int *pitch_elems, void *stream,
                                const sift_kpts_dev *out_kpts, float *const *out_desc,
                                int *out_counts_dev, int *from_cache) {
  if (!h) return SIFT_E_INVALID;
  if (h->serving) return fail(h, SIFT_E_INVALID, "handle is owned by a server");
  if (n < 1 || n > sift::kMaxImg || !imgs_dev || !H || !W || !out_kpts || !out_desc ||
      !out_counts_dev)
    return fail(h, SIFT_E_INVALID, "null pointer argument or n outside 1..128");
  if (from_cache) *from_cache = 0;
  const int ms = h->eng->params().min_octave_side;
  std::vector<ImgIn> in(n);
  for (int i = 0; i < n; i++) {
    const int p = pitch_elems ? pitch_elems[i] : W[i];
    if (!imgs_dev[i] || !out_desc[i] || !kpts_ok(out_kpts[i]))
      return fail(h, SIFT_E_INVALID, "null pointer in image " + std::to_string(i));
    if (H[i] < ms || W[i] < ms || p < W[i])
      return fail(h, SIFT_E_INVALID, "image " + std::to_string(i) + " smaller than min_octave_side");
    if (!h->eng->addressable(H[i], W[i]))
      return fail(h, SIFT_E_INVALID, "image " + std::to_string(i) + " too large");
    in[i] = ImgIn{imgs_dev[i], H[i], W[i], p, out_kpts[i], out_desc[i], out_counts_dev + i};
  }
  h->split_batch = false;
  const cudaStream_t s = (cudaStream_t)stream;
  sift_status st = h->eng->init();
  if (st != SIFT_OK) return pass(h, st);
  const std::string sig =
      h->eng->device_key() + ";" + sift::batch_signature(h->eng->params(), n, H, W);
  if (!h->tuning_cache.empty()) {
    std::string js;
    st = sift::cache_get(h->tuning_cache.c_str(), sig.c_str(), &js);
    if (st == SIFT_OK) {
      sift::Tuning t;
      std::string why;
      if (!sift::parse_tuning(js.c_str(), h->eng->params().n_scales, sift::default_tuning(), &t,
                              &why))
        return fail(h, SIFT_E_INVALID, "tuning cache entry: " + why);
      h->eng->set_tuning(t);
      if (from_cache) *from_cache = 1;
      return run_batch(h, n, in.data(), s);
    }
    if (st != SIFT_E_NOTFOUND) return fail(h, st, "tuning cache unreadable: " + h->tuning_cache);
  }
  // Every candidate is timed as the handle runs the batch (lanes included).
  st = h->eng->autotune_batch(n, in.data(), s, [&] { return run_batch(h, n, in.data(), s); });
  if (st != SIFT_OK) return pass(h, st);
  // The number of lanes (the batch as 1 to 4 parts at once) is decided here,
  // at the handle, by timing whole steps through run_batch each way (best of
  // three runs of five steps, after two untimed ones); more lanes are kept
  // only when at least 1% faster.
  if (n >= 2) {
    sift::Tuning t = h->eng->tuning();
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaEventDestroy(a);
      return fail(h, SIFT_E_CUDA, "autotune event creation failed");
    }
    const int max_lanes = std::min(sift::kMaxLanes, n);
    float best_ms[sift::kMaxLanes] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int lanes = 1; lanes <= max_lanes && st == SIFT_OK; lanes++) {
      t.batch_lanes = lanes;
      h->eng->set_tuning(t);
      for (int w = 0; w < 2 && st == SIFT_OK; w++) st = run_batch(h, n, in.data(), s);
      for (int r = 0; r < 3 && st == SIFT_OK; r++) {
        cudaEventRecord(a, s);
        for (int k = 0; k < 5 && st == SIFT_OK; k++) st = run_batch(h, n, in.data(), s);
        cudaEventRecord(b, s);
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
          st = fail(h, SIFT_E_CUDA, "autotune timing failed");
        best_ms[lanes - 1] = std::min(best_ms[lanes - 1], ms / 5.0f);
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != SIFT_OK) return st;
    int best = 1;
    for (int lanes = 2; lanes <= max_lanes; lanes++)
      if (best_ms[lanes - 1] < 0.99f * best_ms[best - 1]) best = lanes;
    t.batch_lanes = best;
    h->eng->set_tuning(t);
    st = run_batch(h, n, in.data(), s);  // the outputs: a run with the chosen tuning
    if (st != SIFT_OK) return st;
  }
  if (!h->tuning_cache.empty()) {
    const std::string js = sift::tuning_json(h->eng->tuning(), h->eng->params().n_scales);
    st = sift::cache_put(h->tuning_cache.c_str(), sig.c_str(), js.c_str());
    if (st != SIFT_OK) return fail(h, st, "tuning cache not writable: " + h->tuning_cache);
  }
  return SIFT_OK;
}

}  // extern "C"

// ===================================================================== server

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  const float *img = nullptr;
  int H = 0, W = 0, pitch = 0;
  size_t out_bytes = 0, ws_bytes = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  sift_status status = SIFT_PENDING;
  int count = 0;
  char *buf = nullptr;
  sift_kpts_dev k{};
  float *desc = nullptr;
  int *dcount = nullptr;
};

struct Lane;

struct Server;

struct DoneMsg {
  Server *srv;
  int lane;
};

struct Lane {
  Engine *eng = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device bounds of the lane's step
  bool busy = false;
  bool finished = false;
  std::vector<uint64_t> reqs;
  int *h_counts = nullptr;                 // pinned
  sift::ImgCounters *h_flags = nullptr;    // pinned
  unsigned long long *h_gave = nullptr;    // pinned: the engine's gave-up word after the step
  unsigned epoch = 0;                      // the step's scan epoch
  Clock::time_point t_done;
  DoneMsg msg{};
};

// Device-side interval of one finished step, in ms after the server's reference event.
struct StepRec {
  int lane, n_images;
  double start_ms, end_ms;
};
constexpr size_t kStepLog = 65536;  // most recent steps kept for sift_serve_steps

struct Server {
  sift_handle *h = nullptr;
  cudaEvent_t ev_ref = nullptr;    // recorded once at creation
  std::deque<StepRec> steps;
  size_t budget = 0;
  int max_slots = 0;
  std::mutex mu;
  std::condition_variable cv;      // scheduler wake-up
  std::condition_variable cv_done; // request completion
  std::thread th;
  bool stop = false;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Lane> lanes;
  size_t held = 0;                 // output bytes of admitted / finished requests
  int in_flight = 0;
  uint64_t next_id = 1;
  std::string err;
};

size_t out_bytes_for(int K) {
  return (size_t)K * (7 * sizeof(float) + sift::kDescLen * sizeof(float)) + 256;
}

void CUDART_CB on_lane_done(void *p) {
  DoneMsg *m = static_cast<DoneMsg *>(p);
  Server *s = m->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->lanes[m->lane].finished = true;
    s->lanes[m->lane].t_done = Clock::now();
  }
  s->cv.notify_all();
}

size_t lanes_ws(Server *s) {
  size_t t = 0;
  for (auto &l : s->lanes) t += l.eng->workspace() ? l.eng->layout().total : 0;
  return t;
}

void retire(Server *s, Lane &l) {
  for (size_t i = 0; i < l.reqs.size(); i++) {
    auto it = s->reqs.find(l.reqs[i]);
    if (it == s->reqs.end()) continue;
    Request &r = it->second;
    r.state = 2;
    r.count = l.h_counts[i];
    if (*l.h_gave == l.epoch)  // a compaction wait of this step gave up
      r.status = SIFT_E_TIMEOUT;
    else
      r.status = (l.h_flags[i].flags & (sift::TF_CAND | sift::TF_ORI)) ? SIFT_W_TRUNCATED : SIFT_OK;
    r.t_done = l.t_done;
    s->in_flight--;
  }
  l.reqs.clear();
  l.busy = false;
  l.finished = false;
  s->cv_done.notify_all();
}

// One request of a step, copied out of the request table so that the CUDA
// work below runs without the server lock.
struct Job {
  uint64_t id;
  const float *img;
  int H, W, pitch;
  size_t out_bytes;
  char *buf;
  bool ok;
};

// Runs WITHOUT the server lock: the completion callback of a running step
// takes that lock, and a CUDA call made here may wait for such a step.
// Allocates missing output buffers (stream-ordered), queues the batch, the
// count / flag read-back and the completion callback. Returns the status of
// the launch; per-job allocation failures are marked in Job::ok.
sift_status launch_step(Lane &l, int K, std::vector<Job> &jobs, std::string *err) {
  std::vector<ImgIn> in;
  for (Job &j : jobs) {
    j.ok = true;
    if (!j.buf &&
        cudaMallocAsync(reinterpret_cast<void **>(&j.buf), j.out_bytes, l.stream) != cudaSuccess) {
      cudaGetLastError();
      j.buf = nullptr;
      j.ok = false;
      continue;
    }
    float *f = reinterpret_cast<float *>(j.buf);
    sift_kpts_dev k;
    k.x = f;
    k.y = f + K;
    k.sigma = f + 2 * K;
    k.angle = f + 3 * K;
    k.response = f + 4 * K;
    k.octave = reinterpret_cast<int *>(f + 5 * K);
    k.layer = reinterpret_cast<int *>(f + 6 * K);
    in.push_back(ImgIn{j.img, j.H, j.W, j.pitch, k, f + 7 * K,
                       reinterpret_cast<int *>(f + 7 * K + (size_t)K * sift::kDescLen)});
  }
  if (in.empty()) return SIFT_E_OOM;
  cudaError_t e = cudaEventRecord(l.ev_start, l.stream);
  sift_status st = e == cudaSuccess ? l.eng->run((int)in.size(), in.data(), l.stream) : SIFT_E_CUDA;
  if (st == SIFT_OK) {
    for (size_t i = 0; i < in.size() && e == cudaSuccess; i++)
      e = cudaMemcpyAsync(l.h_counts + i, in[i].count, sizeof(int), cudaMemcpyDeviceToHost, l.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(l.h_flags, l.eng->workspace() + l.eng->layout().cnt,
                          in.size() * sizeof(sift::ImgCounters), cudaMemcpyDeviceToHost, l.stream);
    l.epoch = l.eng->last_epoch();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(l.h_gave, l.eng->gave_up_word(), sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, l.stream);
    if (e == cudaSuccess) e = cudaEventRecord(l.ev_end, l.stream);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(l.stream, on_lane_done, &l.msg);
    if (e != cudaSuccess) {
      st = SIFT_E_CUDA;
      *err = cudaGetErrorString(e);
    }
  } else {
    *err = e != cudaSuccess ? cudaGetErrorString(e) : l.eng->err;
  }
  return st;
}

void set_buffers(Request &r, int K) {
  float *f = reinterpret_cast<float *>(r.buf);
  r.k.x = f;
  r.k.y = f + K;
  r.k.sigma = f + 2 * K;
  r.k.angle = f + 3 * K;
  r.k.response = f + 4 * K;
  r.k.octave = reinterpret_cast<int *>(f + 5 * K);
  r.k.layer = reinterpret_cast<int *>(f + 6 * K);
  r.desc = f + 7 * K;
  r.dcount = reinterpret_cast<int *>(f + 7 * K + (size_t)K * sift::kDescLen);
}

void scheduler(Server *s) {
  const int K = s->h->eng->params().max_kpts;
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    for (size_t i = 0; i < s->lanes.size(); i++) {
      Lane &l = s->lanes[i];
      if (!(l.busy && l.finished)) continue;
      // The step's events are complete (its completion callback ran). Their
      // times are read without the lock, like every other CUDA call here;
      // nothing else touches a finished lane meanwhile.
      lk.unlock();
      float t0 = 0.f, t1 = 0.f;
      const bool timed = cudaEventElapsedTime(&t0, s->ev_ref, l.ev_start) == cudaSuccess &&
                         cudaEventElapsedTime(&t1, s->ev_ref, l.ev_end) == cudaSuccess;
      if (!timed) cudaGetLastError();
      lk.lock();
      if (timed) {
        s->steps.push_back(StepRec{(int)i, (int)l.reqs.size(), (double)t0, (double)t1});
        if (s->steps.size() > kStepLog) s->steps.pop_front();
      }
      retire(s, l);
    }
    if (s->stop) {
      bool any = false;
      for (auto &l : s->lanes) any |= l.busy;
      if (!any) break;
    }
    // Admit queued requests into a step for the first free lane.
    int free_lane = -1;
    for (size_t i = 0; i < s->lanes.size(); i++)
      if (!s->lanes[i].busy) {
        free_lane = (int)i;
        break;
      }
    if (free_lane >= 0 && !s->queue.empty() && !s->stop) {
      Lane &lane = s->lanes[free_lane];
      Engine *eng = lane.eng;
      std::vector<Job> jobs;
      std::vector<int> hs, ws;
      size_t ws_now = lanes_ws(s) - (eng->workspace() ? eng->layout().total : 0);
      while (!s->queue.empty() && (int)jobs.size() < sift::kMaxImg &&
             s->in_flight < s->max_slots) {
        Request &r = s->reqs[s->queue.front()];
        hs.push_back(r.H);
        ws.push_back(r.W);
        const size_t need_ws = eng->workspace_bytes((int)hs.size(), hs.data(), ws.data());
        const size_t need = s->held + r.out_bytes + ws_now + need_ws + need_ws / 4;
        if (need > s->budget) {
          hs.pop_back();
          ws.pop_back();
          break;
        }
        s->held += r.out_bytes;
        s->in_flight++;
        r.state = 1;
        jobs.push_back(Job{r.id, r.img, r.H, r.W, r.pitch, r.out_bytes, r.buf, false});
        s->queue.pop_front();
      }
      if (!jobs.empty()) {
        lane.busy = true;
        lane.finished = false;
        std::string err;
        lk.unlock();
        const sift_status st = launch_step(lane, K, jobs, &err);
        lk.lock();
        const auto now = Clock::now();
        lane.reqs.clear();
        for (Job &j : jobs) {
          Request &r = s->reqs[j.id];
          r.buf = j.buf;
          if (r.buf) set_buffers(r, K);
          if (j.ok && st == SIFT_OK) {
            lane.reqs.push_back(j.id);
          } else {
            r.state = 2;
            r.status = j.ok ? st : SIFT_E_OOM;
            r.t_done = now;
            s->in_flight--;
          }
        }
        if (st != SIFT_OK) {
          s->err = err;
          lane.busy = false;
          lane.finished = false;
          lane.reqs.clear();
        }
        s->cv_done.notify_all();
        continue;
      }
    }
    s->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
}

}  // namespace

struct sift_server {
  Server s;
};

extern "C" {

sift_status sift_serve_create(sift_handle *h, size_t mem_budget_bytes, int max_slots,
                              sift_server **out) {
  if (!h || !out || max_slots < 1 || mem_budget_bytes == 0) return SIFT_E_INVALID;
  if (h->serving) return fail(h, SIFT_E_INVALID, "handle already owned by a server");
  sift_server *sv = new sift_server();
  Server &s = sv->s;
  s.h = h;
  s.budget = mem_budget_bytes;
  s.max_slots = max_slots;
  const int n_lanes = 3;
  s.lanes.resize(n_lanes);
  for (int i = 0; i < n_lanes; i++) {
    Lane &l = s.lanes[i];
    l.eng = new Engine(h->eng->params());
    l.eng->set_tuning(h->eng->tuning());
    sift_status st = l.eng->init();
    cudaError_t e = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&l.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&l.ev_end);
    if (e == cudaSuccess && i == 0) e = cudaEventCreate(&s.ev_ref);
    if (e == cudaSuccess && i == 0) e = cudaEventRecord(s.ev_ref, l.stream);
    if (e == cudaSuccess) e = cudaHostAlloc(&l.h_counts, sift::kMaxImg * sizeof(int), 0);
    if (e == cudaSuccess)
      e = cudaHostAlloc(&l.h_flags, sift::kMaxImg * sizeof(sift::ImgCounters), 0);
    if (e == cudaSuccess) e = cudaHostAlloc(&l.h_gave, sizeof(unsigned long long), 0);
    l.msg = DoneMsg{&s, i};
    if (st != SIFT_OK || e != cudaSuccess) {
      for (auto &m : s.lanes) {
        delete m.eng;
        if (m.stream) cudaStreamDestroy(m.stream);
        if (m.ev_start) cudaEventDestroy(m.ev_start);
        if (m.ev_end) cudaEventDestroy(m.ev_end);
        if (m.h_counts) cudaFreeHost(m.h_counts);
        if (m.h_flags) cudaFreeHost(m.h_flags);
        if (m.h_gave) cudaFreeHost(m.h_gave);
      }
      if (s.ev_ref) cudaEventDestroy(s.ev_ref);
      delete sv;
      return fail(h, SIFT_E_CUDA, "server lane initialisation failed");
    }
  }
  h->serving = true;
  s.th = std::thread(scheduler, &s);
  *out = sv;
  return SIFT_OK;
}

sift_status sift_serve_submit(sift_server *sv, const float *img_dev, int H, int W, int pitch_elems,
                              uint64_t *ticket) {
  if (!sv || !img_dev || !ticket) return SIFT_E_INVALID;
  Server &s = sv->s;
  const sift_params &p = s.h->eng->params();
  if (H < p.min_octave_side || W < p.min_octave_side || pitch_elems < W) return SIFT_E_INVALID;
  if (!s.h->eng->addressable(H, W)) return SIFT_E_INVALID;
  Request r;
  r.img = img_dev;
  r.H = H;
  r.W = W;
  r.pitch = pitch_elems;
  r.out_bytes = out_bytes_for(p.max_kpts);
  r.ws_bytes = s.lanes[0].eng->workspace_bytes(1, &H, &W);
  if (r.out_bytes + r.ws_bytes + r.ws_bytes / 4 > s.budget) return SIFT_E_BUDGET;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.stop) return SIFT_E_INVALID;
    r.id = s.next_id++;
    *ticket = r.id;
    s.reqs.emplace(r.id, r);
    s.queue.push_back(r.id);
  }
  s.cv.notify_all();
  return SIFT_OK;
}

static void fill_result(const Request &r, sift_result *out) {
  out->status = r.status;
  out->count = r.count;
  out->kpts = r.k;
  out->desc = r.desc;
  out->submit_to_done_ms =
      std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
}

sift_status sift_serve_poll(sift_server *sv, uint64_t ticket, sift_result *out) {
  if (!sv || !out) return SIFT_E_INVALID;
  Server &s = sv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.reqs.find(ticket);
  if (it == s.reqs.end()) return SIFT_E_NOTFOUND;
  if (it->second.state != 2) return SIFT_PENDING;
  fill_result(it->second, out);
  return it->second.status;
}

sift_status sift_serve_wait(sift_server *sv, uint64_t ticket, int timeout_ms, sift_result *out) {
  if (!sv || !out) return SIFT_E_INVALID;
  Server &s = sv->s;
  std::unique_lock<std::mutex> lk(s.mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (true) {
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return SIFT_E_NOTFOUND;
    if (it->second.state == 2) {
      fill_result(it->second, out);
      return it->second.status;
    }
    if (s.cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = s.reqs.find(ticket);
      if (it != s.reqs.end() && it->second.state == 2) {
        fill_result(it->second, out);
        return it->second.status;
      }
      return SIFT_E_TIMEOUT;
    }
  }
}

sift_status sift_serve_release(sift_server *sv, uint64_t ticket) {
  if (!sv) return SIFT_E_INVALID;
  Server &s = sv->s;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return SIFT_E_NOTFOUND;
    if (it->second.state != 2) return SIFT_PENDING;
    if (it->second.buf) cudaFreeAsync(it->second.buf, s.lanes[0].stream);
    s.held -= it->second.out_bytes;
    s.reqs.erase(it);
  }
  s.cv.notify_all();
  return SIFT_OK;
}

sift_status sift_serve_steps(sift_server *sv, int max_steps, int *lane, int *n_images,
                             double *start_ms, double *end_ms, int *n_out) {
  if (!sv || !n_out || max_steps < 0 || (max_steps > 0 && (!lane || !n_images || !start_ms || !end_ms)))
    return SIFT_E_INVALID;
  Server &s = sv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  const int n = (int)std::min<size_t>((size_t)max_steps, s.steps.size());
  const size_t first = s.steps.size() - (size_t)n;
  for (int i = 0; i < n; i++) {
    const StepRec &r = s.steps[first + i];
    lane[i] = r.lane;
    n_images[i] = r.n_images;
    start_ms[i] = r.start_ms;
    end_ms[i] = r.end_ms;
  }
  *n_out = n;
  return SIFT_OK;
}

sift_status sift_serve_destroy(sift_server *sv) {
  if (!sv) return SIFT_E_INVALID;
  Server &s = sv->s;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.stop = true;
  }
  s.cv.notify_all();
  if (s.th.joinable()) s.th.join();
  for (auto &l : s.lanes) cudaStreamSynchronize(l.stream);
  for (auto &kv : s.reqs)
    if (kv.second.buf) cudaFreeAsync(kv.second.buf, s.lanes[0].stream);
  for (auto &l : s.lanes) {
    cudaStreamSynchronize(l.stream);
    delete l.eng;
    cudaStreamDestroy(l.stream);
    cudaEventDestroy(l.ev_start);
    cudaEventDestroy(l.ev_end);
    cudaFreeHost(l.h_counts);
    cudaFreeHost(l.h_flags);
    cudaFreeHost(l.h_gave);
  }
  cudaEventDestroy(s.ev_ref);
  s.h->serving = false;
  delete sv;
  return SIFT_OK;
}

}  // extern "C"
